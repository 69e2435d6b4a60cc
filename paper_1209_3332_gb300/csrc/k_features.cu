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
// order-free); the co-occurrence counts are shared-memory histograms.  FP64
// throughput is scarce on this part (about 2 FMA per cycle per SM), so the
// finishing math is FP32 arranged so that no step cancels: every
// co-occurrence statistic is a ratio of exact integers, entropy is a sum of
// non-negative terms, and the gradient mean and variance come from one pass
// of Welford updates per lane, the lanes combined pairwise (a sum of
// non-negative terms).
#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace nucseg {

constexpr unsigned FULLF = 0xffffffffu;

__global__ void k_fbbox_init(int4* bbox, int K) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < K) bbox[i] = make_int4(0x7fffffff, 0x7fffffff, -1, -1);
}

// One warp per row segment of 32*4*FB_STEPS pixels: each lane reads 4 labels
// at a time; the lanes holding the same label (one __match_any_sync group per
// label value) combine their column range and one lane updates the box.
__global__ void __launch_bounds__(256) k_fbbox(const int32_t* __restrict__ labels, int W, int H, int K,
                                               int4* bbox) {
    const int lane = threadIdx.x & 31;
    const int spr = (W + FB_SEG - 1) / FB_SEG;
    long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (long long)spr * H) return;
    const int y = (int)(gw / spr), xs = (int)(gw - (long long)y * spr) * FB_SEG;
    bbox_segment(labels + (size_t)y * W, W, K, y, xs, bbox, lane);
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

constexpr int STAGE_PX = 5120;  // staged region (box + 1-px margin) capacity per warp

// Features of object `obj` by one warp; glcm: this warp's 4x64 counters;
// spx: this warp's staging buffer.  When the object's box plus a
// 1-pixel margin (clipped to the image) fits, it is staged once with
// coalesced row loads as one 16-bit word per pixel (hem8 and an in-object
// bit), and every neighbourhood read comes from shared memory; larger boxes read global
// memory directly.  Sobel neighbours (clamped to the image), 4-neighbours and
// co-occurrence partners of box pixels all lie inside that region.
template <bool STAGED>
__device__ __forceinline__ void object_features_impl(const ObjJob& J, int obj, int* glcm, uint16_t* spx) {
    const int lane = threadIdx.x & 31;
    const int l = obj + 1;
    const int4 box = J.bbox[obj];
    float* out = J.feats + (size_t)obj * NFEAT;
    const int W = J.W, H = J.H;
    // a box outside the image (no pixel carries this label) yields zeros
    if (box.x < 0 || box.y < 0 || box.z >= W || box.w >= H || box.x > box.z || box.y > box.w) {
        if (lane < NFEAT) out[lane] = 0.f;
        return;
    }
    const int bw = box.z - box.x + 1, bh = box.w - box.y + 1;
    const long long npx = (long long)bw * bh;
    const int rx0 = max(box.x - 1, 0), ry0 = max(box.y - 1, 0);
    const int rw = min(box.z + 1, W - 1) - rx0 + 1, rh = min(box.w + 1, H - 1) - ry0 + 1;
    constexpr bool staged = STAGED;
    for (int i = lane; i < 4 * 64; i += 32) glcm[i] = 0;
    if (staged) {
        // the region as one index space, four pixels per lane per step with
        // all their loads issued before the stores, so their latencies overlap
        const int nreg = rh * rw;
        int sy = lane / rw, sx = lane - sy * rw;
        for (int base = lane; base < nreg; base += 4 * 32) {
            int lab[4], hv[4], at[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                at[u] = base + 32 * u < nreg ? sy * rw + sx : -1;
                const size_t g = (size_t)(ry0 + sy) * W + rx0 + sx;
                lab[u] = at[u] >= 0 ? J.labels[g] : 0;
                hv[u] = at[u] >= 0 ? J.hem8[g] : 0;
                sx += 32;
                while (sx >= rw) { sx -= rw; sy++; }
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (at[u] >= 0) spx[at[u]] = (uint16_t)(hv[u] | (lab[u] == l ? 0x100 : 0));
        }
    }
    __syncwarp();
    // pixel (y, x) of the region as hem8 | (in object) << 8: the 3x3
    // neighbourhood of a pixel serves its Sobel sums, its perimeter test and
    // its co-occurrence partners
    auto PX = [&](int y, int x) -> uint32_t {
        if (staged) return spx[(y - ry0) * rw + (x - rx0)];
        const size_t o = (size_t)y * W + x;
        return (uint32_t)J.hem8[o] | (J.labels[o] == l ? 0x100u : 0u);
    };
    int cnt = 0, per = 0, mn = 255, mx = 0, gmn = 0x7fffffff, gmx = 0;
    long long S = 0, Q = 0;
    float wm = 0.f, wq = 0.f;  // this lane's running mean and sum of squared deviations of |Sobel|
    // lane walks the box row-major with stride 32, advancing (y, x) without divisions
    int y = box.y + lane / bw, x = box.x + lane % bw;
    for (long long idx = lane; idx < npx; idx += 32) {
        const int cy = y, cx = x;
        x += 32;
        while (x > box.z) { x -= bw; y++; }
        const uint32_t pc = PX(cy, cx);
        if (!(pc >> 8)) continue;
        const int v = (int)(pc & 0xffu);
        cnt++;
        S += v;
        Q += v * v;
        mn = min(mn, v);
        mx = max(mx, v);
        // the 8 neighbours, clamped to the image (the replicated border of the Sobel sums)
        const int ym = max(cy - 1, 0), yp = min(cy + 1, H - 1), xm = max(cx - 1, 0), xp = min(cx + 1, W - 1);
        const uint32_t a = PX(ym, xm), b = PX(ym, cx), c = PX(ym, xp), d = PX(cy, xm), f = PX(cy, xp);
        const uint32_t g = PX(yp, xm), h = PX(yp, cx), i = PX(yp, xp);
        per += (cy == 0 || !(b >> 8));
        per += (cy == H - 1 || !(h >> 8));
        per += (cx == 0 || !(d >> 8));
        per += (cx == W - 1 || !(f >> 8));
        const int gx = (int)((c & 0xffu) + 2 * (f & 0xffu) + (i & 0xffu)) - (int)((a & 0xffu) + 2 * (d & 0xffu) + (g & 0xffu));
        const int gy = (int)((g & 0xffu) + 2 * (h & 0xffu) + (i & 0xffu)) - (int)((a & 0xffu) + 2 * (b & 0xffu) + (c & 0xffu));
        const int m2 = gx * gx + gy * gy;
        {  // Welford's update
            const float gv = sqrtf((float)m2), dv = __fsub_rn(gv, wm);
            wm = __fadd_rn(wm, __fdiv_rn(dv, (float)cnt));
            wq = __fmaf_rn(dv, __fsub_rn(gv, wm), wq);
        }
        gmn = min(gmn, m2);
        gmx = max(gmx, m2);
        // co-occurrence partners (x + 1, y), (x, y + 1), (x + 1, y + 1), (x + 1, y - 1) inside the image
        const int vb = (v >> 5) * 8;
        if (cx + 1 < W && (f >> 8)) atomicAdd(&glcm[0 * 64 + vb + ((f & 0xffu) >> 5)], 1);
        if (cy + 1 < H && (h >> 8)) atomicAdd(&glcm[1 * 64 + vb + ((h & 0xffu) >> 5)], 1);
        if (cy + 1 < H && cx + 1 < W && (i >> 8)) atomicAdd(&glcm[2 * 64 + vb + ((i & 0xffu) >> 5)], 1);
        if (cy > 0 && cx + 1 < W && (c >> 8)) atomicAdd(&glcm[3 * 64 + vb + ((c & 0xffu) >> 5)], 1);
    }
    const long long N = warp_sum<long long>(cnt);
    const long long Ssum = warp_sum<long long>(S), Qsum = warp_sum<long long>(Q);
    const long long Per = warp_sum<long long>(per);
    const int Mn = __reduce_min_sync(FULLF, mn), Mx = __reduce_max_sync(FULLF, mx);
    const int Gmn = __reduce_min_sync(FULLF, gmn), Gmx = __reduce_max_sync(FULLF, gmx);
    // the lanes' (count, mean, squared deviations) combined pairwise (Chan,
    // Golub, LeVeque): every term of the combined sum is non-negative
    float gn = (float)cnt, gm = wm, gq = wq;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float nb = __shfl_xor_sync(FULLF, gn, o), mb = __shfl_xor_sync(FULLF, gm, o);
        const float qb = __shfl_xor_sync(FULLF, gq, o);
        // both lanes of a pair form the same sum: the lower lane's part first
        const bool lo = (lane & o) == 0;
        const float na = lo ? gn : nb, ma = lo ? gm : mb, qa = lo ? gq : qb;
        const float n2 = lo ? nb : gn, m2v = lo ? mb : gm, q2 = lo ? qb : gq;
        const float n = __fadd_rn(na, n2);
        if (n > 0.f) {
            const float f = __fdiv_rn(n2, n), d = __fsub_rn(m2v, ma);
            gm = __fmaf_rn(d, f, ma);
            gq = __fadd_rn(__fadd_rn(qa, q2), __fmul_rn(__fmul_rn(d, d), __fmul_rn(na, f)));
        } else {
            gm = 0.f;
            gq = 0.f;
        }
        gn = n;
    }
    if (N == 0) {
        if (lane < NFEAT) out[lane] = 0.f;
        __syncwarp();
        return;
    }
    __syncwarp();
    // co-occurrence statistics per offset: lanes hold bins lane and lane+32.
    // With counts C_ij and T = sum C_ij: contrast = sum (i-j)^2 C / T, energy =
    // sum C^2 / T^2, homogeneity = sum C/(1+(i-j)^2) / T (integer numerator over
    // the common multiple 408850 of the denominators 1+(i-j)^2), correlation
    // from exact integer moments, each one FP32 division of exact integers;
    // entropy = sum (C/T) ln(T/C) with ln(T/C) = log1p((T-C)/C), a sum of
    // non-negative terms, equal to ln T - sum C ln C / T.
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int used = 0;
    const int i0 = lane >> 3, j0 = lane & 7, i1 = i0 + 4, j1 = j0;
    const int d0 = (i0 - j0) * (i0 - j0), d1 = (i1 - j1) * (i1 - j1);
    const long long HL = 408850;  // lcm of 1+d^2 for d = 0..7
    auto ent = [](long long C, long long T) -> float {
        return C > 0 ? __fmul_rn(__fdiv_rn((float)C, (float)T), log1pf(__fdiv_rn((float)(T - C), (float)C))) : 0.f;
    };
#pragma unroll
    for (int o = 0; o < 4; o++) {
        const int* cc = glcm + o * 64;
        const long long v0 = cc[lane], v1 = cc[lane + 32];
        const long long T = warp_sum<long long>(v0 + v1);
        if (T == 0) continue;
        used++;
        const long long si = warp_sum<long long>(i0 * v0 + i1 * v1);
        const long long sj = warp_sum<long long>(j0 * v0 + j1 * v1);
        const long long sii = warp_sum<long long>(i0 * i0 * v0 + i1 * i1 * v1);
        const long long sjj = warp_sum<long long>(j0 * j0 * v0 + j1 * j1 * v1);
        const long long sij = warp_sum<long long>(i0 * j0 * v0 + i1 * j1 * v1);
        const long long scon = warp_sum<long long>(d0 * v0 + d1 * v1);
        const long long sene = warp_sum<long long>(v0 * v0 + v1 * v1);
        const long long shom = warp_sum<long long>((HL / (1 + d0)) * v0 + (HL / (1 + d1)) * v1);
        const float sent = warp_sum<float>(__fadd_rn(ent(v0, T), ent(v1, T)));
        const float Tf = (float)T;
        const long long vi = T * sii - si * si, vj = T * sjj - sj * sj, cv = T * sij - si * sj;
        acc[0] = __fadd_rn(acc[0], __fdiv_rn((float)scon, Tf));
        acc[1] = __fadd_rn(acc[1], __fdiv_rn((float)sene, __fmul_rn(Tf, Tf)));
        acc[2] = __fadd_rn(acc[2], __fdiv_rn((float)shom, __fmul_rn((float)HL, Tf)));
        acc[3] = __fadd_rn(acc[3], sent);
        acc[4] = __fadd_rn(acc[4], (vi == 0 || vj == 0) ? 0.f
                                   : __fdiv_rn((float)cv, sqrtf(__fmul_rn((float)vi, (float)vj))));
    }
    if (lane == 0) {
        const double n = (double)N;
        __int128 var_num = (__int128)N * Qsum - (__int128)Ssum * Ssum;
        double f[NFEAT];
        f[0] = n;
        f[1] = (double)Per;
        f[2] = (double)Ssum / n;
        f[3] = sqrt((double)var_num) / n;
        f[4] = Mn;
        f[5] = Mx;
        f[6] = (double)gm;
        f[7] = sqrt(__ddiv_rn((double)gq, n));
        f[8] = sqrt((double)Gmn);
        f[9] = sqrt((double)Gmx);
        for (int k = 0; k < 5; k++) f[10 + k] = used ? __fdiv_rn(acc[k], (float)used) : 0.f;
        for (int k = 0; k < NFEAT; k++) out[k] = (float)f[k];
    }
    __syncwarp();
}

// boxes larger than the stage read global memory; that rare path is kept out
// of line so the common one stays small in the instruction cache
__device__ __noinline__ void object_features_global(const ObjJob& J, int obj, int* glcm) {
    object_features_impl<false>(J, obj, glcm, nullptr);
}

__device__ __forceinline__ void object_features(const ObjJob& J, int obj, int* glcm, uint16_t* spx) {
    const int4 box = J.bbox[obj];
    const int rx0 = max(box.x - 1, 0), ry0 = max(box.y - 1, 0);
    const long long rw = (long long)min(box.z + 1, J.W - 1) - rx0 + 1, rh = (long long)min(box.w + 1, J.H - 1) - ry0 + 1;
    if (rw > 0 && rh > 0 && rw * rh <= STAGE_PX)
        object_features_impl<true>(J, obj, glcm, spx);
    else
        object_features_global(J, obj, glcm);
}

constexpr int FW = 4;  // object warps per CTA

// Plain form: objects [0, K) of one tile, one warp each.
struct ObjSmem {
    int glcm[4 * 64];
    uint16_t px[STAGE_PX];  // hem8 | (in object) << 8
};

__global__ void __launch_bounds__(FW * 32) k_fobj_plain(ObjJob J, int K) {
    __shared__ ObjSmem sm[FW];
    const int warp = threadIdx.x >> 5;
    ObjSmem& S = sm[warp];
    for (int obj = blockIdx.x * FW + warp; obj < K; obj += gridDim.x * FW)
        object_features(J, obj, S.glcm, S.px);
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
    L.sh->next_obj = 0;
}

// Batched form: the objects of all tiles, item -> (tile, object) through the
// obj_base prefixes (the last tile whose base is <= item owns it).
__global__ void __launch_bounds__(FW * 32) k_fobj_batched(Launch L) {
    __shared__ ObjSmem sm[FW];
    const int warp = threadIdx.x >> 5;
    ObjSmem& S = sm[warp];
    const int total = L.sh->nobj;
    const int lane = threadIdx.x & 31;
    // objects are drawn one at a time from a counter, so a warp that drew
    // large boxes does not hold back the end of the pass
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&L.sh->next_obj, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        const int t = find_tile(L.tiles, L.ntiles, item, &TileDev::obj_base);
        const TileDev& T = L.tiles[t];
        ObjJob J{T.hem8, T.labels, T.W, T.H, T.bbox, T.feats};
        object_features(J, item - T.obj_base, S.glcm, S.px);
    }
}

void launch_object_boxes(const int32_t* labels, int W, int H, int K, int4* bbox, cudaStream_t s, Profiler* pf) {
    pf->begin("feat_bbox_init", s);
    k_fbbox_init<<<(K + 255) / 256, 256, 0, s>>>(bbox, K);
    pf->end("feat_bbox_init", s);
    pf->begin("feat_bbox", s);
    long long warps = (long long)((W + FB_SEG - 1) / FB_SEG) * H;
    k_fbbox<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(labels, W, H, K, bbox);
    pf->end("feat_bbox", s);
}

void launch_features_plain(const uint8_t* hem8, const int32_t* labels, int W, int H, int K, float* feats,
                           int4* bbox, int sms, cudaStream_t s, Profiler* pf) {
    if (K <= 0) return;
    launch_object_boxes(labels, W, H, K, bbox, s, pf);
    ObjJob J{hem8, labels, W, H, bbox, feats};
    int grid = (K + FW - 1) / FW < sms * 16 ? (K + FW - 1) / FW : sms * 16;
    pf->begin("feat_objects", s);
    k_fobj_plain<<<grid, FW * 32, 0, s>>>(J, K);
    pf->end("feat_objects", s);
}

void launch_features_batched(const Launch& L, int grid, cudaStream_t s, Profiler* pf) {
    pf->begin("feat_prefix", s);
    k_obj_prefix<<<1, 32, 0, s>>>(L);
    pf->end("feat_prefix", s);
    pf->begin("feat_objects", s);
    k_fobj_batched<<<grid, FW * 32, 0, s>>>(L);
    pf->end("feat_objects", s);
}

}  // namespace nucseg
