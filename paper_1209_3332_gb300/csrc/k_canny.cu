// Canny edges of a uint8 plane (Sec. V-A lists Canny among the
// feature-stage transforms applied to the deconvolved image; Table I
// "Features comp.") and the per-object edge counts (Sec. II "edge"
// features).  Definition (the paper gives no parameter):
//   gx, gy = 3x3 Sobel with replicated border; m = |gx| + |gy|;
//   sector: horizontal if (ax + ay)^2 < 2 ax^2 (ay < ax tan 22.5 deg),
//     vertical if ay > ax and (ay - ax)^2 > 2 ax^2 (ay > ax tan 67.5 deg),
//     else the diagonal along (+x,+y) when gx gy > 0, (+x,-y) otherwise;
//   neighbours a, b along the sector (a on the previous row, or the left
//     one for the horizontal sector); m outside the image is 0;
//   p survives iff m(p) > m(a) and m(p) >= m(b); candidate iff it survives
//     with m > low, strong iff it survives with m > high;
//   edges = candidates 8-connected through candidates to a strong pixel.
// Every kernel takes an array of tile descriptors, so one launch covers any
// number of tiles (the plain form is the batched form of one tile), a CTA
// finding its tile by binary search over the tiles' first blocks.
// k_canny_nms writes the strong pixels (the marker) and the candidates (the
// mask) as 0/1 planes from one 32x32 block per CTA staged with a 2-px halo,
// and flags the 64x64 work tiles the strong pixels touch; the hysteresis is
// then the reconstruction by dilation of the marker under the mask, run by
// the reconstruction kernel of the segmentation from the flagged work tiles
// only.  The counts are a stencil pass over the same blocks: each edge pixel
// adds one to every object with a pixel within its disk -- the same count
// as the edge pixels within each object's disk dilation, with the labels
// and edges read once, coalesced.
#include "internal.cuh"

namespace nucseg {

constexpr int CT = 32;                 // block of the counts pass: CT x CT pixels

// the tile of launch item b, by binary search over the tiles' first items
__device__ __forceinline__ int find_desc(const CannyDesc* __restrict__ D, int n, int b, int CannyDesc::*base) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (D[mid].*base <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---- suppression: one warp streams a strip of 128 columns (4 per lane) down
// a segment of 64 rows (one work-tile row), keeping the last three image rows,
// the magnitudes of the last three rows and the Sobel pair of the current row
// in registers ------------------------------------------------------------------
constexpr int NS_COLS = 128, NS_ROWS = 64;
constexpr int NS_WARPS = 4;          // warps per CTA

struct Row8 {                        // image row, columns cx0 - 2 .. cx0 + 5 (replicated border), as
    uint32_t p[4];                   // four pairs of 16-bit lanes: (-2,-1), (0,1), (2,3), (4,5)
};

// the global reads of one row for one lane: its own 4 pixels, and on the
// strip's edge lanes the two pixels beyond the strip
struct RowFetch {
    uint32_t w;
    int e0, e1;
};

__device__ __forceinline__ RowFetch ns_fetch(const uint8_t* __restrict__ I, int W, int H, int y, int cx0, bool vec,
                                             int lane) {
    const uint8_t* row = I + (size_t)min(max(y, 0), H - 1) * W;
    RowFetch f;
    if (vec && cx0 < W) {
        f.w = __ldg(reinterpret_cast<const uint32_t*>(row + cx0));
    } else {
        f.w = 0;
#pragma unroll
        for (int k = 3; k >= 0; k--) f.w = (f.w << 8) | __ldg(row + min(cx0 + k, W - 1));
    }
    f.e0 = f.e1 = 0;
    if (lane == 0) {
        f.e0 = __ldg(row + max(cx0 - 2, 0));
        f.e1 = __ldg(row + max(cx0 - 1, 0));
    } else if (lane == 31) {
        f.e0 = __ldg(row + min(cx0 + 4, W - 1));
        f.e1 = __ldg(row + min(cx0 + 5, W - 1));
    }
    return f;
}

// columns cx0 - 2 .. cx0 + 5 of a fetched row: the neighbours' pixels by shuffle
__device__ __forceinline__ Row8 ns_row(const RowFetch& f, int lane) {
    uint32_t wl = __shfl_up_sync(0xffffffffu, f.w, 1), wr = __shfl_down_sync(0xffffffffu, f.w, 1);
    if (lane == 0) wl = ((uint32_t)f.e0 << 16) | ((uint32_t)f.e1 << 24);   // bytes 2, 3: columns -2, -1
    if (lane == 31) wr = (uint32_t)f.e0 | ((uint32_t)f.e1 << 8);            // bytes 0, 1: columns 4, 5
    Row8 r;
    r.p[0] = __byte_perm(wl, 0u, 0x4342);
    r.p[1] = __byte_perm(f.w, 0u, 0x4140);
    r.p[2] = __byte_perm(f.w, 0u, 0x4342);
    r.p[3] = __byte_perm(wr, 0u, 0x4140);
    return r;
}

__device__ __forceinline__ Row8 ns_load_row(const uint8_t* __restrict__ I, int W, int H, int y, int cx0, bool vec,
                                            int lane) {
    return ns_row(ns_fetch(I, W, H, y, cx0, vec, lane), lane);
}

struct Sob6 {                        // columns cx0 - 1 .. cx0 + 4 of one row (index j = column - cx0 + 1)
    int m[6];                        // L1 magnitude, 0 off the image
    int ax[4], ay[4], same[4];       // |gx|, |gy| and whether gx, gy have one sign, columns cx0 .. cx0 + 3
};

__device__ __forceinline__ uint32_t max2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t min2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Sobel of the row between A and C (rows r - 1, r, r + 1, replicated) in
// 16x2-bit lanes, for the column pairs (-1, 0), (1, 2), (3, 4): with
// vs = A + 2B + C and vd = C - A per column, gx(c) = vs(c+1) - vs(c-1) and
// gy(c) = vd(c-1) + 2 vd(c) + vd(c+1).  Signed values carry a bias (256 on
// vd, 1024 on gx and gy) so that every lane stays in [0, 2^16) and packed
// adds never borrow across lanes.  colmask: per pair, 0xffff on the lanes of
// columns inside the image; m is 0 elsewhere and on a row off the image.
__device__ __forceinline__ Sob6 ns_sobel(const Row8& A, const Row8& B, const Row8& C, const uint32_t colmask[3],
                                         bool row_in) {
    constexpr uint32_t B256 = 0x01000100u, B1024 = 0x04000400u;
    uint32_t V[4], Dv[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        V[k] = A.p[k] + (B.p[k] << 1) + C.p[k];
        Dv[k] = C.p[k] + B256 - A.p[k];
    }
    const uint32_t rm = row_in ? 0xffffffffu : 0u;
    uint32_t SX[3], SY[3], AX[3], AY[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        SX[k] = V[k + 1] + B1024 - V[k];
        SY[k] = Dv[k] + (__byte_perm(Dv[k], Dv[k + 1], 0x5432) << 1) + Dv[k + 1];
        AX[k] = max2(SX[k], B1024) - min2(SX[k], B1024);
        AY[k] = max2(SY[k], B1024) - min2(SY[k], B1024);
    }
    Sob6 o;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const uint32_t M = (AX[k] + AY[k]) & colmask[k] & rm;
        o.m[2 * k] = (int)(M & 0xffffu);
        o.m[2 * k + 1] = (int)(M >> 16);
    }
    // columns 0..3 are the high lane of pair 0, both lanes of pair 1, the low lane of pair 2
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int k = (c + 1) >> 1, sh = (c & 1) ? 0 : 16;
        o.ax[c] = (int)((AX[k] >> sh) & 0xffffu);
        o.ay[c] = (int)((AY[k] >> sh) & 0xffffu);
        o.same[c] = (((SX[k] >> sh) & 0xffffu) > 1024u) == (((SY[k] >> sh) & 0xffffu) > 1024u);
    }
    return o;
}

__global__ void __launch_bounds__(32 * NS_WARPS, 4) k_canny_nms(const CannyDesc* __restrict__ D, int n, int n_warps,
                                                            int low, int high, int* __restrict__ flags) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * NS_WARPS + (threadIdx.x >> 5);
    if (gw >= n_warps) return;
    const CannyDesc& d = D[find_desc(D, n, gw, &CannyDesc::nms_base)];
    const uint8_t* __restrict__ I = d.img;
    const int W = d.W, H = d.H, wi = gw - d.nms_base;
    const int strips = (W + NS_COLS - 1) / NS_COLS, nw = strips * ((H + NS_ROWS - 1) / NS_ROWS);
    const int seg = wi / strips, strip = wi - seg * strips;
    const int cx0 = strip * NS_COLS + 4 * lane, ya = seg * NS_ROWS, yb = min(ya + NS_ROWS, H);
    // this warp's share of the counts to zero
    for (long long i = (long long)wi * 32 + lane; i < d.K; i += (long long)nw * 32) d.counts[i] = 0;
    const bool vec = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(I) & 3) == 0;
    const bool out_vec = vec && (reinterpret_cast<uintptr_t>(d.edges) & 3) == 0 &&
                         (reinterpret_cast<uintptr_t>(d.cand) & 3) == 0;
    uint32_t colmask[3];  // pair k holds columns cx0 + 2k - 1 and cx0 + 2k
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int x = cx0 + 2 * k - 1;
        colmask[k] = ((x >= 0 && x < W) ? 0xffffu : 0u) | ((x + 1 >= 0 && x + 1 < W) ? 0xffff0000u : 0u);
    }
    Row8 P = ns_load_row(I, W, H, ya - 1, cx0, vec, lane);
    Row8 Q = ns_load_row(I, W, H, ya, cx0, vec, lane);
    Sob6 prev = ns_sobel(ns_load_row(I, W, H, ya - 2, cx0, vec, lane), P, Q, colmask, ya - 1 >= 0);
    Sob6 cur = ns_sobel(P, Q, ns_load_row(I, W, H, ya + 1, cx0, vec, lane), colmask, true);
    P = Q;
    Q = ns_load_row(I, W, H, ya + 1, cx0, vec, lane);
    const int rtx = (W + RT - 1) / RT, rty = (H + RT - 1) / RT;
    unsigned seed = 0u;
    RowFetch fn = ns_fetch(I, W, H, ya + 2, cx0, vec, lane);  // one row ahead of its use
#pragma unroll 1
    for (int y = ya; y < yb; y++) {
        const Row8 N = ns_row(fn, lane);
        fn = ns_fetch(I, W, H, y + 3, cx0, vec, lane);
        const Sob6 next = ns_sobel(P, Q, N, colmask, y + 1 < H);
        uint32_t ws = 0, wc = 0;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int j = c + 1;
            const int ax = cur.ax[c], ay = cur.ay[c], m = cur.m[j];
            int ma, mb;
            if ((ax + ay) * (ax + ay) < 2 * ax * ax) {                  // horizontal
                ma = cur.m[j - 1]; mb = cur.m[j + 1];
            } else if (ay > ax && (ay - ax) * (ay - ax) > 2 * ax * ax) {  // vertical
                ma = prev.m[j]; mb = next.m[j];
            } else if (cur.same[c]) {                                   // along (+x, +y)
                ma = prev.m[j - 1]; mb = next.m[j + 1];
            } else {                                                    // along (+x, -y)
                ma = prev.m[j + 1]; mb = next.m[j - 1];
            }
            const bool keep = m > ma && m >= mb;
            ws |= (uint32_t)(keep && m > high) << (8 * c);
            wc |= (uint32_t)(keep && m > low) << (8 * c);
        }
        if (cx0 < W) {
            const size_t o = (size_t)y * W + cx0;
            if (out_vec) {
                *reinterpret_cast<uint32_t*>(d.edges + o) = ws;
                *reinterpret_cast<uint32_t*>(d.cand + o) = wc;
            } else {
                for (int c = 0; c < 4 && cx0 + c < W; c++) {
                    d.edges[o + c] = (uint8_t)(ws >> (8 * c));
                    d.cand[o + c] = (uint8_t)(wc >> (8 * c));
                }
            }
            if (ws) {
#pragma unroll
                for (int c = 0; c < 4; c++)
                    if ((ws >> (8 * c)) & 1u) seed |= seed_bits_px(rtx, rty, cx0 + c, y);
            }
        }
        prev = cur;
        cur = next;
        P = Q;
        Q = N;
    }
    // lanes 0-15 and 16-31 each lie in one work tile: one flag store per touched work tile
    const unsigned lo = __reduce_or_sync(0xffffffffu, lane < 16 ? seed : 0u);
    const unsigned hi = __reduce_or_sync(0xffffffffu, lane >= 16 ? seed : 0u);
    if ((lane == 0 || lane == 16) && cx0 < W) {
        const unsigned m9 = lane == 0 ? lo : hi;
        const int tx = cx0 / RT, ty = ya / RT;
        for (int b = 0; b < 9; b++)
            if ((m9 >> b) & 1u) flags[d.rt_base + (ty + b / 3 - 1) * rtx + (tx + b % 3 - 1)] = 1;
    }
}

constexpr int CR_MAX = 4;                 // largest disk radius of the counts
constexpr int CC_S = CT + 2 * CR_MAX;     // staged labels: the block and a CR_MAX-pixel halo (40 x 40)

// Edge counts, one 32x32 block per CTA: the edge bytes of the block, then
// (for a block with an edge pixel) the labels of the block and a 4-pixel
// halo (0 off the image, and for labels outside 1..K), staged in shared
// memory with 16-byte loads where the rows allow; each edge pixel adds one
// to every distinct object in its disk (the first four remembered in
// registers, beyond that an object is new iff no earlier disk offset holds
// it).
__global__ void __launch_bounds__(256) k_canny_counts(const CannyDesc* __restrict__ D, int n, int r) {
    __shared__ __align__(16) int32_t sl[CC_S][CC_S];
    __shared__ __align__(16) uint8_t se[CT][CT];
    const int t = threadIdx.x;
    const CannyDesc& d = D[find_desc(D, n, blockIdx.x, &CannyDesc::blk_base)];
    const int K = d.K;
    if (K <= 0) return;
    const int W = d.W, H = d.H, bl = blockIdx.x - d.blk_base;
    const int by = bl / d.bx, x0 = (bl - by * d.bx) * CT, y0 = by * CT;
    int any = 0;
    if (t < 64) {  // the block's edge bytes: one 16-byte row half per thread
        const int ly = t >> 1, lx = (t & 1) * 16, gy = y0 + ly, gx = x0 + lx;
        uint4 v = make_uint4(0, 0, 0, 0);
        const uint8_t* src = d.edges + (size_t)gy * W + gx;
        if (gy < H) {
            if (gx + 16 <= W && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                v = *reinterpret_cast<const uint4*>(src);
            } else {
                uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
                for (int k = 0; k < 16; k++)
                    if (gx + k < W) w[k >> 2] |= (uint32_t)src[k] << (8 * (k & 3));
                v = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        *reinterpret_cast<uint4*>(&se[ly][lx]) = v;
        any = (v.x | v.y | v.z | v.w) != 0;
    }
    if (!__syncthreads_or(any)) return;       // no edge pixel: no label is needed
    const bool vec = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(d.labels) & 15) == 0;
    // 400 four-label groups over 256 threads: both of a thread's loads are
    // issued before either is stored, so their latencies overlap
    constexpr int NQ = CC_S * (CC_S / 4);
    int4 v[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int i = t + 256 * u;
        const int ly = i / (CC_S / 4), q = i - ly * (CC_S / 4);
        const int gy = y0 - CR_MAX + ly, gx = x0 - CR_MAX + 4 * q;
        v[u] = make_int4(0, 0, 0, 0);
        if (i < NQ && (unsigned)gy < (unsigned)H) {
            const int32_t* src = d.labels + (size_t)gy * W + gx;
            if (vec && gx >= 0 && gx + 4 <= W) {
                v[u] = __ldg(reinterpret_cast<const int4*>(src));
            } else {
                int e[4];
#pragma unroll
                for (int k = 0; k < 4; k++) e[k] = (unsigned)(gx + k) < (unsigned)W ? __ldg(src + k) : 0;
                v[u] = make_int4(e[0], e[1], e[2], e[3]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int i = t + 256 * u;
        if (i >= NQ) break;
        const int ly = i / (CC_S / 4), q = i - ly * (CC_S / 4);
        int4 w = v[u];
        w.x = (w.x >= 1 && w.x <= K) ? w.x : 0;
        w.y = (w.y >= 1 && w.y <= K) ? w.y : 0;
        w.z = (w.z >= 1 && w.z <= K) ? w.z : 0;
        w.w = (w.w >= 1 && w.w <= K) ? w.w : 0;
        *reinterpret_cast<int4*>(&sl[ly][4 * q]) = w;
    }
    __syncthreads();
    const int r2 = r * r;
    for (int i = t; i < CT * CT; i += 256) {
        const int ly = i / CT, lx = i - ly * CT;
        if (!se[ly][lx]) continue;
        int seen0 = 0, seen1 = 0, seen2 = 0, seen3 = 0, nseen = 0;
        for (int dy = -r; dy <= r; dy++)
            for (int dx = -r; dx <= r; dx++) {
                if (dx * dx + dy * dy > r2) continue;
                const int v = sl[ly + CR_MAX + dy][lx + CR_MAX + dx];
                if (!v || v == seen0 || v == seen1 || v == seen2 || v == seen3) continue;
                bool fresh = true;
                if (nseen >= 4) {  // look for v at an earlier disk offset
                    for (int ey = -r; ey <= dy && fresh; ey++)
                        for (int ex = -r; ex <= r; ex++) {
                            if (ey == dy && ex >= dx) break;
                            if (ex * ex + ey * ey <= r2 && sl[ly + CR_MAX + ey][lx + CR_MAX + ex] == v) {
                                fresh = false;
                                break;
                            }
                        }
                }
                if (!fresh) continue;
                atomicAdd(&d.counts[v - 1], 1);
                if (nseen == 0) seen0 = v; else if (nseen == 1) seen1 = v; else if (nseen == 2) seen2 = v;
                else if (nseen == 3) seen3 = v;
                nseen++;
            }
    }
}

int canny_blocks(int W, int H) { return ((W + CT - 1) / CT) * ((H + CT - 1) / CT); }

// descriptors reach the device through kernel parameters (no host staging
// buffer has to outlive the call)
constexpr int CANNY_DESC_PACK = 8;
struct CannyDescPack {
    CannyDesc d[CANNY_DESC_PACK];
    int n, first;
};
__global__ void k_set_canny_desc(CannyDesc* dst, CannyDescPack p) {
    if (threadIdx.x < p.n) dst[p.first + threadIdx.x] = p.d[threadIdx.x];
}
void upload_canny_descs(CannyDesc* dst, const std::vector<CannyDesc>& v, cudaStream_t s) {
    for (int i = 0; i < (int)v.size(); i += CANNY_DESC_PACK) {
        CannyDescPack pk;
        pk.first = i;
        pk.n = (int)v.size() - i < CANNY_DESC_PACK ? (int)v.size() - i : CANNY_DESC_PACK;
        for (int k = 0; k < pk.n; k++) pk.d[k] = v[i + k];
        k_set_canny_desc<<<1, 32, 0, s>>>(dst, pk);
    }
}

int canny_nms_warps(int W, int H) { return ((W + NS_COLS - 1) / NS_COLS) * ((H + NS_ROWS - 1) / NS_ROWS); }

void launch_canny_nms(const std::vector<CannyDesc>& descs, CannyDesc* d_descs, int low, int high, int* flags,
                      cudaStream_t s, Profiler* pf) {
    int warps = 0;
    for (auto& d : descs) warps += canny_nms_warps(d.W, d.H);
    if (!warps) return;
    pf->begin("canny_nms", s);
    k_canny_nms<<<(warps + NS_WARPS - 1) / NS_WARPS, 32 * NS_WARPS, 0, s>>>(d_descs, (int)descs.size(), warps, low,
                                                                          high, flags);
    pf->end("canny_nms", s);
}

void launch_canny_counts(const std::vector<CannyDesc>& descs, CannyDesc* d_descs, int r, cudaStream_t s,
                         Profiler* pf) {
    int blocks = 0, K = 0;
    for (auto& d : descs) {
        blocks += canny_blocks(d.W, d.H);
        K += d.K;
    }
    if (!blocks || !K) return;
    pf->begin("canny_counts", s);
    k_canny_counts<<<blocks, 256, 0, s>>>(d_descs, (int)descs.size(), r);
    pf->end("canny_counts", s);
}

}  // namespace nucseg
