// K5: exact squared Euclidean distance transform to the nearest label-0
// pixel (Table I, the distance transform of "Pre-Watershed").
//
// Separable form (as in Meijster, Roerdink, Hesselink 2000): g(y,x) is the
// distance along column x to the nearest background pixel, and
// D(y,x) = min_q (x-q)^2 + g(y,q)^2 along row y.
//
// GB300 layout: the relabel pass leaves the kept-pixel bitmap (2 MB for a
// 4K tile) and, per 32-row chunk and column, the first and last background
// row.  k_edt_carry turns those into, per chunk, the nearest background row
// above and below the chunk (a short sequential scan per column).  k_edt_rows
// then handles a band of rows per CTA: it rebuilds g for the band from the
// bitmap (a 32x32 bit transpose by warp shuffles) and the carries, keeps the
// band's g rows in shared memory and solves every row there, so the only
// full-plane traffic is the single int32 write of D.  Rows whose g stays
// within WMAX use an exact windowed search (a candidate at distance r costs
// at least r^2, so the search stops once r^2 >= the best value); other rows
// run Meijster's lower-envelope scan on one thread.
#include "internal.cuh"

namespace nucseg {

constexpr int INFG = 32767;       // "no background in this column"
constexpr int WMAX = 128;
constexpr unsigned FULLE = 0xffffffffu;

// per column: carryL[c] <- last background row above chunk c (or -1),
//             carryF[c] <- first background row below chunk c (or -1)
__global__ void __launch_bounds__(256) k_edt_carry(Launch L) {
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= L.n_cols) return;
    int ti = find_tile(L.tiles, L.ntiles, gid, &TileDev::col_base);
    const TileDev& T = L.tiles[ti];
    if (!T.edt) return;
    int x = gid - T.col_base;
    int above = -1;
    for (int c = 0; c < T.cby; c++) {
        size_t o = (size_t)c * T.W + x;
        int lb = T.edtL[o];
        T.edtL[o] = above;
        if (lb >= 0) above = lb;
    }
    int below = -1;
    for (int c = T.cby - 1; c >= 0; c--) {
        size_t o = (size_t)c * T.W + x;
        int fb = T.edtF[o];
        T.edtF[o] = below;
        if (fb >= 0) below = fb;
    }
}

__device__ __forceinline__ int sq(int v) { return v * v; }

__device__ void meijster_row(const uint16_t* g, int W, int16_t* s, int16_t* t, int32_t* out) {
    // lower envelope of f_i(u) = (u-i)^2 + g_i^2
    auto F = [&](int u, int i) -> long long { return (long long)(u - i) * (u - i) + (long long)g[i] * g[i]; };
    int q = 0;
    s[0] = 0;
    t[0] = 0;
    for (int u = 1; u < W; u++) {
        while (q >= 0 && F(t[q], s[q]) > F(t[q], u)) q--;
        if (q < 0) {
            q = 0;
            s[0] = (int16_t)u;
        } else {
            int i = s[q];
            long long num = (long long)u * u - (long long)i * i + (long long)g[u] * g[u] - (long long)g[i] * g[i];
            long long den = 2LL * (u - i);
            long long fl = num / den;
            if ((num % den != 0) && (num < 0)) fl--;
            long long w = 1 + fl;
            if (w < W) {
                q++;
                s[q] = (int16_t)u;
                t[q] = (int16_t)w;
            }
        }
    }
    for (int u = W - 1; u >= 0; u--) {
        long long d = F(u, s[q]);
        out[u] = d >= (long long)INFG * INFG ? 0x7fffffff : (int32_t)d;
        if (u == t[q]) q--;
    }
}

__global__ void __launch_bounds__(256) k_edt_rows(Launch L, int RB, int Wmax) {
    extern __shared__ __align__(16) unsigned char smraw[];
    uint16_t* gs = reinterpret_cast<uint16_t*>(smraw);                 // [RB][Wmax]
    int16_t* ms = reinterpret_cast<int16_t*>(gs + (size_t)RB * Wmax);  // [Wmax]
    int16_t* mt = ms + Wmax;                                           // [Wmax]
    __shared__ int rowmax[32];
    const int gbnd = blockIdx.x;
    const int ti = find_tile(L.tiles, L.ntiles, gbnd, &TileDev::row_base);
    const TileDev& T = L.tiles[ti];
    if (!T.edt) return;
    const int W = T.W, H = T.H;
    const int y0 = (gbnd - T.row_base) * RB;
    const int c = y0 / CB, r0 = c * CB;
    const int nrow = min(RB, H - y0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int kmax = min(CB, H - r0);  // valid rows in this chunk
    const uint32_t rowvalid = kmax >= 32 ? FULLE : ((1u << kmax) - 1u);
    // g for the band: one warp per 32-column strip
    for (int sidx = warp; sidx < T.wpr; sidx += nw) {
        uint32_t word = lane < kmax ? T.keptbits[(size_t)(r0 + lane) * T.wpr + sidx] : 0xffffffffu;
        uint32_t col = 0;  // bit k: row r0+k of column (32*sidx+lane) is kept (foreground)
#pragma unroll
        for (int k = 0; k < 32; k++) {
            uint32_t w = __shfl_sync(FULLE, word, k);
            col |= ((w >> lane) & 1u) << k;
        }
        const int x = sidx * 32 + lane;
        if (x >= W) continue;
        const uint32_t bg = ~col & rowvalid;
        const int above = T.edtL[(size_t)c * W + x], below = T.edtF[(size_t)c * W + x];
        for (int j = 0; j < nrow; j++) {
            int y = y0 + j, k = y - r0;
            uint32_t mu = bg & ((2u << k) - 1u);
            int du = mu ? k - (31 - __clz(mu)) : (above >= 0 ? y - above : INFG);
            uint32_t md = bg & ~((1u << k) - 1u);
            int dd = md ? (__ffs(md) - 1) - k : (below >= 0 ? below - y : INFG);
            int gv = min(min(du, dd), INFG);
            gs[(size_t)j * Wmax + x] = (uint16_t)gv;
        }
    }
    __syncthreads();
    for (int j = 0; j < nrow; j++) {
        const uint16_t* g = gs + (size_t)j * Wmax;
        int m = 0;
        for (int x = threadIdx.x; x < W; x += blockDim.x) m = max(m, (int)g[x]);
        m = __reduce_max_sync(FULLE, m);
        if (lane == 0) rowmax[warp] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            int mm = 0;
            for (int i = 0; i < nw; i++) mm = max(mm, rowmax[i]);
            rowmax[31] = mm;
        }
        __syncthreads();
        const int mm = rowmax[31];
        int32_t* out = T.edt + (size_t)(y0 + j) * W;
        if (mm <= WMAX) {
            for (int x = threadIdx.x; x < W; x += blockDim.x) {
                int g0 = g[x];
                int D = sq(g0);
                for (int r = 1; r * r < D; r++) {
                    int rr = r * r;
                    if (x - r >= 0) D = min(D, rr + sq(g[x - r]));
                    if (x + r < W) D = min(D, rr + sq(g[x + r]));
                }
                out[x] = D;
            }
        } else if (threadIdx.x == 0) {
            meijster_row(g, W, ms, mt, out);
        }
        __syncthreads();
    }
}

size_t edt_rows_smem(int RB, int Wmax) { return (size_t)RB * Wmax * 2 + (size_t)2 * Wmax * 2; }

void launch_edt(const Launch& L, int RB, int Wmax, cudaStream_t s, Profiler* pf) {
    if (L.n_rows == 0) return;
    pf->begin("edt_carry", s);
    k_edt_carry<<<(L.n_cols + 255) / 256, 256, 0, s>>>(L);
    pf->end("edt_carry", s);
    size_t smem = edt_rows_smem(RB, Wmax);
    cudaFuncSetAttribute(k_edt_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pf->begin("edt_rows", s);
    k_edt_rows<<<L.n_rows, 256, smem, s>>>(L, RB, Wmax);
    pf->end("edt_rows", s);
}

}  // namespace nucseg
