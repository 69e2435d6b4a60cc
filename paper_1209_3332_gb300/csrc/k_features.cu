// K6: per-object features (Sec. II: pixel statistics, gradient statistics,
// Haralick texture, morphometry; Sec. V-A: gradient among the feature-stage
// transforms).  Features of object l over its pixel set O (N pixels):
//   0 area N, 1 perimeter = number of (p in O, 4-neighbour n) with n outside O
//   or outside the image, 2/3 mean and population std of hem8, 4/5 min/max,
//   6..9 mean, population std, min, max of |Sobel(hem8)| with replicated
//   border, 10..14 contrast, energy, homogeneity, entropy, correlation of the
//   8-level co-occurrence matrix of same-object pairs (p, p+(dx,dy)),
//   averaged over the offsets (1,0),(0,1),(1,1),(1,-1) that have pairs.
//
// GB300 design: labels are raster-numbered, so a bounding box per object
// (warp-aggregated atomics over a single pass of the label plane, or
// produced directly by the relabel pass in the batched form) lets one CTA
// own one object and walk only its box.  Pixel sums are integers (exact,
// order-free); the gradient sums are FP64 in a fixed thread order; the
// co-occurrence counts are shared-memory histograms.  The FP64 finishing
// math runs once per object, never per pixel.
#include "internal.cuh"

namespace nucseg {

constexpr int FT = 128;  // threads per object CTA
constexpr unsigned FULLF = 0xffffffffu;

__global__ void k_fbbox_init(int4* bbox, int K) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < K) bbox[i] = make_int4(0x7fffffff, 0x7fffffff, -1, -1);
}

// one warp per 32 consecutive pixels of a row
__global__ void __launch_bounds__(256) k_fbbox(const int32_t* __restrict__ labels, int W, int H, int K,
                                               int4* bbox) {
    const int lane = threadIdx.x & 31;
    const int spr = (W + 31) >> 5;
    long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (long long)spr * H) return;
    int y = (int)(gw / spr), x = (int)(gw - (long long)y * spr) * 32 + lane;
    int lab = x < W ? __ldcs(labels + (size_t)y * W + x) : 0;
    if (lab < 1 || lab > K) lab = 0;
    if (__ballot_sync(FULLF, lab != 0) == 0) return;
    unsigned grp = __match_any_sync(FULLF, lab);
    if (lab == 0) return;
    int mn = __reduce_min_sync(grp, (unsigned)x), mx = __reduce_max_sync(grp, (unsigned)x);
    if (lane == __ffs(grp) - 1) {
        int4* b = bbox + (lab - 1);
        atomicMin(&b->x, mn);
        atomicMax(&b->z, mx);
        atomicMin(&b->y, y);
        atomicMax(&b->w, y);
    }
}

struct ObjJob {
    const uint8_t* hem8;
    const int32_t* labels;
    int W, H;
    const int4* bbox;
    float* feats;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int sobel_m2(const uint8_t* I, int W, int H, int y, int x) {
    int ym = max(y - 1, 0), yp = min(y + 1, H - 1), xm = max(x - 1, 0), xp = min(x + 1, W - 1);
    const uint8_t* rm = I + (size_t)ym * W;
    const uint8_t* r0 = I + (size_t)y * W;
    const uint8_t* rp = I + (size_t)yp * W;
    int a = rm[xm], b = rm[x], c = rm[xp], d = r0[xm], f = r0[xp], g = rp[xm], h = rp[x], i = rp[xp];
    int gx = (c + 2 * f + i) - (a + 2 * d + g);
    int gy = (g + 2 * h + i) - (a + 2 * b + c);
    return gx * gx + gy * gy;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLF, v, o);
    return v;
}

// block reduction of a sum in fixed order: lanes (xor tree), then warps in index order
template <typename T>
__device__ T block_sum(T v, T* tmp) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) tmp[warp] = v;
    __syncthreads();
    T s = 0;
    for (int i = 0; i < FT / 32; i++) s += tmp[i];
    __syncthreads();
    return s;
}
__device__ int block_min(int v, int* tmp) {
    v = __reduce_min_sync(FULLF, v);
    if ((threadIdx.x & 31) == 0) tmp[threadIdx.x >> 5] = v;
    __syncthreads();
    int s = tmp[0];
    for (int i = 1; i < FT / 32; i++) s = min(s, tmp[i]);
    __syncthreads();
    return s;
}
__device__ int block_max(int v, int* tmp) {
    v = __reduce_max_sync(FULLF, v);
    if ((threadIdx.x & 31) == 0) tmp[threadIdx.x >> 5] = v;
    __syncthreads();
    int s = tmp[0];
    for (int i = 1; i < FT / 32; i++) s = max(s, tmp[i]);
    __syncthreads();
    return s;
}

__device__ void object_features(const ObjJob& J, int obj, int* glcm, long long* tl, double* td,
                                int* ti, double* ostat) {
    const int l = obj + 1;
    const int4 box = J.bbox[obj];
    float* out = J.feats + (size_t)obj * NFEAT;
    const int W = J.W, H = J.H;
    // a box outside the image (no pixel carries this label) yields zeros
    if (box.x < 0 || box.y < 0 || box.z >= W || box.w >= H || box.x > box.z || box.y > box.w) {
        if (threadIdx.x < NFEAT) out[threadIdx.x] = 0.f;
        return;
    }
    const int bw = box.z - box.x + 1, bh = box.w - box.y + 1;
    const long long npx = (long long)bw * bh;
    for (int i = threadIdx.x; i < 4 * 64; i += FT) glcm[i] = 0;
    __syncthreads();
    int cnt = 0, per = 0, mn = 255, mx = 0, gmn = 0x7fffffff, gmx = 0;
    long long S = 0, Q = 0;
    double gs = 0.0;
    const int odx[4] = {1, 0, 1, 1}, ody[4] = {0, 1, 1, -1};
    for (long long idx = threadIdx.x; idx < npx; idx += FT) {
        int y = box.y + (int)(idx / bw), x = box.x + (int)(idx % bw);
        size_t p = (size_t)y * W + x;
        if (J.labels[p] != l) continue;
        int v = J.hem8[p];
        cnt++;
        S += v;
        Q += v * v;
        mn = min(mn, v);
        mx = max(mx, v);
        per += (y == 0 || J.labels[p - W] != l);
        per += (y == H - 1 || J.labels[p + W] != l);
        per += (x == 0 || J.labels[p - 1] != l);
        per += (x == W - 1 || J.labels[p + 1] != l);
        int m2 = sobel_m2(J.hem8, W, H, y, x);
        gs += sqrt((double)m2);
        gmn = min(gmn, m2);
        gmx = max(gmx, m2);
#pragma unroll
        for (int o = 0; o < 4; o++) {
            int yy = y + ody[o], xx = x + odx[o];
            if (yy < 0 || yy >= H || xx >= W) continue;
            size_t q = (size_t)yy * W + xx;
            if (J.labels[q] != l) continue;
            atomicAdd(&glcm[o * 64 + (v >> 5) * 8 + (J.hem8[q] >> 5)], 1);
        }
    }
    const long long N = block_sum<long long>(cnt, tl);
    const long long Ssum = block_sum<long long>(S, tl);
    const long long Qsum = block_sum<long long>(Q, tl);
    const long long Per = block_sum<long long>(per, tl);
    const int Mn = block_min(mn, ti), Mx = block_max(mx, ti);
    const int Gmn = block_min(gmn, ti), Gmx = block_max(gmx, ti);
    const double Gs = block_sum<double>(gs, td);
    if (N == 0) {
        if (threadIdx.x < NFEAT) out[threadIdx.x] = 0.f;
        __syncthreads();
        return;
    }
    const double gmean = Gs / (double)N;
    double gss = 0.0;
    for (long long idx = threadIdx.x; idx < npx; idx += FT) {
        int y = box.y + (int)(idx / bw), x = box.x + (int)(idx % bw);
        if (J.labels[(size_t)y * W + x] != l) continue;
        double d = sqrt((double)sobel_m2(J.hem8, W, H, y, x)) - gmean;
        gss += d * d;
    }
    const double Gss = block_sum<double>(gss, td);
    // co-occurrence statistics: warp o handles offset o (bins lane, lane+32)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
        const int* c = glcm + warp * 64;
        long long T = 0, si = 0, sj = 0, sii = 0, sjj = 0, sij = 0;
        for (int b = lane; b < 64; b += 32) {
            long long v = c[b];
            int i = b >> 3, j = b & 7;
            T += v; si += i * v; sj += j * v; sii += i * i * v; sjj += j * j * v; sij += i * j * v;
        }
        T = warp_sum(T); si = warp_sum(si); sj = warp_sum(sj);
        sii = warp_sum(sii); sjj = warp_sum(sjj); sij = warp_sum(sij);
        double con = 0, ene = 0, hom = 0, ent = 0;
        if (T > 0) {
            for (int b = lane; b < 64; b += 32) {
                int v = c[b];
                if (!v) continue;
                int i = b >> 3, j = b & 7;
                double P = (double)v / (double)T;
                con += (double)((i - j) * (i - j)) * P;
                ene += P * P;
                hom += P / (1.0 + (double)((i - j) * (i - j)));
                ent -= P * log(P);
            }
        }
        con = warp_sum(con); ene = warp_sum(ene); hom = warp_sum(hom); ent = warp_sum(ent);
        if (lane == 0) {
            long long vi = T * sii - si * si, vj = T * sjj - sj * sj, cv = T * sij - si * sj;
            double cor = (vi == 0 || vj == 0) ? 0.0 : (double)cv / sqrt((double)vi * (double)vj);
            double* os = ostat + warp * 6;
            os[0] = T > 0 ? 1.0 : 0.0;
            os[1] = con; os[2] = ene; os[3] = hom; os[4] = ent; os[5] = cor;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double n = (double)N;
        __int128 var_num = (__int128)N * Qsum - (__int128)Ssum * Ssum;
        double f[NFEAT];
        f[0] = n;
        f[1] = (double)Per;
        f[2] = (double)Ssum / n;
        f[3] = sqrt((double)var_num) / n;
        f[4] = Mn;
        f[5] = Mx;
        f[6] = gmean;
        f[7] = sqrt(Gss / n);
        f[8] = sqrt((double)Gmn);
        f[9] = sqrt((double)Gmx);
        double acc[5] = {0, 0, 0, 0, 0};
        int used = 0;
        for (int o = 0; o < 4; o++) {
            const double* os = ostat + o * 6;
            if (os[0] == 0.0) continue;
            used++;
            for (int k = 0; k < 5; k++) acc[k] += os[1 + k];
        }
        for (int k = 0; k < 5; k++) f[10 + k] = used ? acc[k] / used : 0.0;
        for (int k = 0; k < NFEAT; k++) out[k] = (float)f[k];
    }
    __syncthreads();
}

// Object CTAs.  Plain form: one tile, objects [0, K).  Batched form: the
// objects of all tiles, item -> (tile, object) through obj_base prefixes.
__global__ void __launch_bounds__(FT) k_fobj_plain(ObjJob J, int K) {
    __shared__ int glcm[4 * 64];
    __shared__ long long tl[FT / 32];
    __shared__ double td[FT / 32];
    __shared__ int ti[FT / 32];
    __shared__ double ostat[4 * 6];
    for (int obj = blockIdx.x; obj < K; obj += gridDim.x) object_features(J, obj, glcm, tl, td, ti, ostat);
}

__global__ void k_obj_prefix(Launch L) {
    if (threadIdx.x != 0) return;
    int run = 0;
    for (int t = 0; t < L.ntiles; t++) {
        TileDev& T = L.tiles[t];
        int K = *T.n_objects;
        int m = min(K, T.feats_cap);
        if (K > T.feats_cap) L.tile_status[t] = ST_OVERFLOW;
        T.obj_base = run;
        run += m;
    }
    L.sh->nobj = run;
}

__global__ void __launch_bounds__(FT) k_fobj_batched(Launch L) {
    __shared__ int glcm[4 * 64];
    __shared__ long long tl[FT / 32];
    __shared__ double td[FT / 32];
    __shared__ int tis[FT / 32];
    __shared__ double ostat[4 * 6];
    const int total = L.sh->nobj;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int t = find_tile(L.tiles, L.ntiles, item, &TileDev::obj_base);
        // skip tiles that contribute no object (equal bases): take the last with base <= item
        const TileDev& T = L.tiles[t];
        ObjJob J{T.hem8, T.labels, T.W, T.H, T.bbox, T.feats};
        object_features(J, item - T.obj_base, glcm, tl, td, tis, ostat);
    }
}

void launch_features_plain(const uint8_t* hem8, const int32_t* labels, int W, int H, int K, float* feats,
                           int4* bbox, int sms, cudaStream_t s, Profiler* pf) {
    if (K <= 0) return;
    pf->begin("feat_bbox_init", s);
    k_fbbox_init<<<(K + 255) / 256, 256, 0, s>>>(bbox, K);
    pf->end("feat_bbox_init", s);
    pf->begin("feat_bbox", s);
    long long warps = (long long)((W + 31) / 32) * H;
    k_fbbox<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(labels, W, H, K, bbox);
    pf->end("feat_bbox", s);
    ObjJob J{hem8, labels, W, H, bbox, feats};
    int grid = K < sms * 16 ? K : sms * 16;
    pf->begin("feat_objects", s);
    k_fobj_plain<<<grid, FT, 0, s>>>(J, K);
    pf->end("feat_objects", s);
}

void launch_features_batched(const Launch& L, int sms, cudaStream_t s, Profiler* pf) {
    pf->begin("feat_prefix", s);
    k_obj_prefix<<<1, 32, 0, s>>>(L);
    pf->end("feat_prefix", s);
    pf->begin("feat_objects", s);
    k_fobj_batched<<<sms * 16, FT, 0, s>>>(L);
    pf->end("feat_objects", s);
}

}  // namespace nucseg
