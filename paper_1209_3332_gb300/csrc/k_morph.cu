// Next step before the path: grayscale opening by a disk (Table I, "Morph.
// Open", by a 19x19 disk).  The disk of radius r is the set of integer
// offsets (dx, dy) with dx^2 + dy^2 <= r^2; pixels outside the image take no
// part.  Opening = dilation of the erosion, each by that disk.
//
// Design: one CTA per 64x64 output block.  The input block with a 2r halo is
// staged in shared memory (outside the image: 255, neutral for the min).
// The disk is a stack of 2r + 1 row chords, chord dy spanning
// [x - w(dy), x + w(dy)] with w(dy) = floor(sqrt(r^2 - dy^2)); each chord's
// minimum is two lookups into a per-row table of minima over windows of
// 1, 2, 4, 8 and 16 pixels (two windows of length 2^k <= 2w + 1 < 2^(k+1)
// cover the chord), so the erosion costs 2 (2r + 1) lookups per pixel
// whatever r is.  The erosion is taken over the block plus an r halo and
// kept in shared memory (outside the image: 0, neutral for the max); the
// same tables with max then give the dilation on the block.
#include "internal.cuh"

namespace nucseg {

constexpr int MB = 64;           // output block side
constexpr int MLEV = 5;          // table levels: windows 1, 2, 4, 8, 16

// chord half-widths and table levels for dy = -r..r, index dy + r
struct Chords {
    int r;
    unsigned char w[2 * MORPH_RMAX + 1];
    unsigned char k[2 * MORPH_RMAX + 1];
};

// Builds levels 1..4 of the window table over an n x n plane at T (level 0
// given; level k holds minima (or maxima) over [x, x + 2^k), valid for x <=
// n - 2^k).
template <bool MAX>
__device__ __forceinline__ void build_levels(uint8_t* T, int n) {
    const int plane = n * n;
    for (int k = 1; k < MLEV; k++) {
        const uint8_t* a = T + (size_t)(k - 1) * plane;
        uint8_t* b = T + (size_t)k * plane;
        const int h = 1 << (k - 1), valid = n - (1 << k) + 1;
        for (int i = threadIdx.x; i < n * valid; i += blockDim.x) {
            const int y = i / valid, x = i - y * valid;
            const int u = a[y * n + x], v = a[y * n + x + h];
            b[y * n + x] = (uint8_t)(MAX ? max(u, v) : min(u, v));
        }
        __syncthreads();
    }
}

// min (max) over the disk of radius r centred at (cy, cx) of an n x n plane
// with tables; wk[i] = w | k << 8 for dy = i - r
template <bool MAX>
__device__ __forceinline__ int disk_extreme(const uint8_t* T, int n, const int* wk, int r, int cy, int cx) {
    const int plane = n * n;
    int v = MAX ? 0 : 255;
    for (int i = 0; i <= 2 * r; i++) {
        const int w = wk[i] & 0xff, k = wk[i] >> 8;
        const uint8_t* row = T + (size_t)k * plane + (size_t)(cy + i - r) * n;
        const int a = row[cx - w], b = row[cx + w + 1 - (1 << k)];
        v = MAX ? max(v, max(a, b)) : min(v, min(a, b));
    }
    return v;
}

__global__ void __launch_bounds__(256) k_morph_open(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst,
                                                    int W, int H, Chords C) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ int wk[2 * MORPH_RMAX + 1];
    const int r = C.r, n = MB + 4 * r, e = MB + 2 * r;
    if (threadIdx.x <= 2 * r) wk[threadIdx.x] = C.w[threadIdx.x] | (C.k[threadIdx.x] << 8);
    uint8_t* T = sm;                           // MLEV planes of n x n (input tables, then erosion tables)
    uint8_t* E = sm + (size_t)MLEV * n * n;    // erosion over the block plus an r halo, e x e
    const int x0 = blockIdx.x * MB, y0 = blockIdx.y * MB;
    // stage the input with a 2r halo
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        const int y = i / n, x = i - y * n;
        const int gy = y0 - 2 * r + y, gx = x0 - 2 * r + x;
        T[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? __ldg(src + (size_t)gy * W + gx) : (uint8_t)255;
    }
    __syncthreads();
    build_levels<false>(T, n);
    // erosion at staged (y + r, x + r) for the e x e region
    for (int i = threadIdx.x; i < e * e; i += blockDim.x) {
        const int y = i / e, x = i - y * e;
        const int gy = y0 - r + y, gx = x0 - r + x;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        E[i] = in ? (uint8_t)disk_extreme<false>(T, n, wk, r, y + r, x + r) : (uint8_t)0;
    }
    __syncthreads();
    // the erosion plane becomes level 0 of the max tables (in T's space)
    for (int i = threadIdx.x; i < e * e; i += blockDim.x) T[i] = E[i];
    __syncthreads();
    build_levels<true>(T, e);
    for (int i = threadIdx.x; i < MB * MB; i += blockDim.x) {
        const int y = i / MB, x = i - y * MB;
        const int gy = y0 + y, gx = x0 + x;
        if (gy < H && gx < W) dst[(size_t)gy * W + gx] = (uint8_t)disk_extreme<true>(T, e, wk, r, y + r, x + r);
    }
}

// ---- streaming form for a compile-time radius -----------------------------------
// One pass is one erosion (MAX = false) or one dilation (MAX = true); the
// opening runs an erosion into a scratch plane and a dilation from it.  One
// warp per strip of 64 output columns and a segment of rows; lane l holds the
// output columns xs + 2l and + 1 as one pair of 16-bit lanes.  The warp
// streams the input rows down the strip:
//  * a row arrives as one aligned 32-bit word per lane (rows are 4-byte
//    aligned: W % 4 == 0) and enters a per-warp buffer of 16-bit pixels kept
//    in two copies, the second shifted by one pixel, so every pixel pair is
//    one aligned 32-bit load; the chords of half-widths 0..R around a pair are nested,
//    C_w = min(C_{w-1}, pair at -w, pair at +w), one 3-input SIMD min each;
//  * instead of keeping rows, each lane keeps 2R + 1 accumulators, one per
//    output row that the entering row reaches: row t lowers (raises) the
//    accumulator of row t - dy by C_{w(dy)} for every dy, and the
//    accumulator of row t - R is then complete.  The step loop is unrolled
//    2R + 1 times so that every accumulator index is a constant, and input
//    rows are fetched two loop trips ahead.
// Pixels outside the image take no part: they enter as 255 for a min and 0
// for a max.
constexpr int MS_WARPS = 4, MS_SW = 64, MS_SEG = 128;

__device__ __forceinline__ uint32_t smin2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t smax2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// the pixel pair (i, i + 1) of a row kept as ev[] and od[] = ev[] shifted by one
__device__ __forceinline__ uint32_t row_pair(const uint16_t* ev, const uint16_t* od, int i) {
    return (i & 1) ? *reinterpret_cast<const uint32_t*>(od + i - 1) : *reinterpret_cast<const uint32_t*>(ev + i);
}

template <int R, bool MAX>
__global__ void __launch_bounds__(MS_WARPS * 32) k_morph_stream(const uint8_t* __restrict__ src,
                                                                uint8_t* __restrict__ dst, int W, int H,
                                                                int nstrip, int nseg) {
    constexpr int K = 2 * R + 1;
    constexpr int A = (R + 3) & ~3;           // the row segment starts at xs - A, a multiple of 4
    constexpr int NWORD = (MS_SW + A + R + 3) / 4;  // 32-bit words that cover columns xs - R .. xs + 63 + R
    constexpr int BL = 4 * NWORD + 4;
    static_assert(NWORD <= 32, "one word per lane");
    constexpr uint32_t NEUTRAL = MAX ? 0u : 0x00ff00ffu;
    constexpr uint32_t NEUTRAL_WORD = MAX ? 0u : 0xffffffffu;
    __shared__ __align__(16) uint16_t buf[MS_WARPS][2][BL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * MS_WARPS + warp;
    if (gw >= nstrip * nseg) return;  // whole warps only
    uint16_t* ev = buf[warp][0];
    uint16_t* od = buf[warp][1];
    const int strip = gw % nstrip, seg = gw / nstrip;
    const int xs = strip * MS_SW, ys = seg * MS_SEG, ye = min(H, ys + MS_SEG);
    const int ox = xs + 2 * lane;
    const int t0 = ys - R, t1 = ye + R;  // input rows that reach the segment
    // this lane's word: columns cw .. cw + 3 (in the image or not at all, as W % 4 == 0)
    const int cw = xs - A + 4 * lane;
    const bool wok = lane < NWORD && cw >= 0 && cw < W;
    auto fetch = [&](int t) -> uint32_t {
        return (wok && t >= 0 && t < H && t < t1)
                   ? __ldg(reinterpret_cast<const unsigned int*>(src + (size_t)t * W + cw))
                   : NEUTRAL_WORD;
    };
    // slot u of the unrolled step loop holds the row that step u consumes
    // (pf) and the one after it (pf2): a row is fetched two loop trips
    // (4R + 2 rows) ahead and moves from pf2 to pf after one trip, when its
    // load has long completed (one trip ahead left loads exposed)
    uint32_t pf[K], pf2[K];
#pragma unroll
    for (int q = 0; q < K; q++) { pf[q] = fetch(t0 + q); pf2[q] = fetch(t0 + K + q); }
    uint32_t acc[K];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = NEUTRAL;
    for (int tb = t0; tb < t1; tb += K) {
#pragma unroll
        for (int u = 0; u < K; u++) {
            const int t = tb + u;
            if (t >= t1) break;
            const uint32_t w = pf[u];
            pf[u] = pf2[u];
            pf2[u] = fetch(t + 2 * K);
            // the row's 16-bit pixels: ev[j] = column xs - A + j, od[j] = ev[j + 1]
            const uint32_t e0 = __byte_perm(w, 0u, 0x4140), e1 = __byte_perm(w, 0u, 0x4342);
            const uint32_t ne0 = __shfl_down_sync(0xffffffffu, e0, 1);
            if (lane < NWORD) {
                *reinterpret_cast<uint32_t*>(ev + 4 * lane) = e0;
                *reinterpret_cast<uint32_t*>(ev + 4 * lane + 2) = e1;
                *reinterpret_cast<uint32_t*>(od + 4 * lane) = __byte_perm(w, 0u, 0x4241);
                *reinterpret_cast<uint32_t*>(od + 4 * lane + 2) = __byte_perm(e1, ne0, 0x5432);
            }
            __syncwarp();
            // chords of half-widths 0..R around this lane's pair (buffer index 2l + A)
            const int b0 = 2 * lane + A;
            uint32_t C[R + 1];
            C[0] = row_pair(ev, od, b0);
#pragma unroll
            for (int wd = 1; wd <= R; wd++) {
                const uint32_t l = row_pair(ev, od, b0 - wd), r = row_pair(ev, od, b0 + wd);
                C[wd] = MAX ? __vimax3_u16x2(C[wd - 1], l, r) : __vimin3_u16x2(C[wd - 1], l, r);
            }
            __syncwarp();  // every lane has read the row buffers
            // row t reaches row t - dy through the chord of half-width w(dy): slot (u - dy) mod K
#pragma unroll
            for (int dy = -R; dy <= R; dy++) {
                int wd = 0;
                while ((wd + 1) * (wd + 1) + dy * dy <= R * R) wd++;
                const int k = ((u - dy) % K + K) % K;
                acc[k] = MAX ? smax2(acc[k], C[wd]) : smin2(acc[k], C[wd]);
            }
            // row y = t - R is complete
            const int y = t - R, ky = ((u - R) % K + K) % K;
            if (y >= ys && y < ye && ox < W)
                *reinterpret_cast<uint16_t*>(dst + (size_t)y * W + ox) = (uint16_t)__byte_perm(acc[ky], 0u, 0x4420);
            acc[ky] = NEUTRAL;
        }
    }
}

size_t morph_open_smem(int r) {
    const size_t n = MB + 4 * r, e = MB + 2 * r;
    return (size_t)MLEV * n * n + e * e;
}

void launch_morph_open(const uint8_t* src, uint8_t* dst, uint8_t* tmp, int W, int H, int r, cudaStream_t s,
                       Profiler* pf) {
    const bool aligned4 = (W & 3) == 0 && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) |
                                            reinterpret_cast<uintptr_t>(tmp)) & 3) == 0;
    if (r == 9 && tmp && aligned4) {  // the paper's 19x19 disk: two streaming passes through tmp
        constexpr int R = 9;
        const int nstrip = (W + MS_SW - 1) / MS_SW, nseg = (H + MS_SEG - 1) / MS_SEG;
        const int blocks = (nstrip * nseg + MS_WARPS - 1) / MS_WARPS;
        pf->begin("morph_erode", s);
        k_morph_stream<R, false><<<blocks, MS_WARPS * 32, 0, s>>>(src, tmp, W, H, nstrip, nseg);
        pf->end("morph_erode", s);
        pf->begin("morph_dilate", s);
        k_morph_stream<R, true><<<blocks, MS_WARPS * 32, 0, s>>>(tmp, dst, W, H, nstrip, nseg);
        pf->end("morph_dilate", s);
        return;
    }
    Chords C{};
    C.r = r;
    for (int dy = -r; dy <= r; dy++) {
        int w = 0;
        while ((w + 1) * (w + 1) + dy * dy <= r * r) w++;
        int k = 0;
        while ((2 << k) <= 2 * w + 1) k++;
        C.w[dy + r] = (unsigned char)w;
        C.k[dy + r] = (unsigned char)k;
    }
    const size_t smem = morph_open_smem(r);
    cudaFuncSetAttribute(k_morph_open, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const dim3 grid((W + MB - 1) / MB, (H + MB - 1) / MB);
    pf->begin("morph_open", s);
    k_morph_open<<<grid, 256, smem, s>>>(src, dst, W, H, C);
    pf->end("morph_open", s);
}

}  // namespace nucseg
