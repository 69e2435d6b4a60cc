// K5: exact squared Euclidean distance transform to the nearest label-0
// pixel (Table I, the distance transform of "Pre-Watershed").
//
// Separable form (as in Meijster, Roerdink, Hesselink 2000): g(y,x) is the
// distance along column x to the nearest background pixel, and
// D(y,x) = min_q (x-q)^2 + g(y,q)^2 along row y.
//
// GB300 layout: the relabel pass leaves, per 32-row chunk and column, one
// word with the chunk's 32 kept bits of that column (2 MB for a 4K tile).
// k_edt_rows handles a band of rows per CTA: for each column it finds the
// nearest background row within the chunk with bit scans, and above/below
// the chunk by walking to the nearest chunk that has background (almost
// always the adjacent one), keeps the band's g rows in shared memory and
// solves every row there, so the only full-plane traffic is the single
// int32 write of D.  Rows whose g stays
// within WMAX use an exact windowed search (a candidate at distance r costs
// at least r^2, so the search stops once r^2 >= the best value); other rows
// run Meijster's lower-envelope scan on one thread.  Shared memory holds
// only the band (4 rows of u16 for a 4096-wide tile, each padded with WMAX
// "no background" entries on both sides so that the search needs no bounds
// test), so several CTAs fit on an SM.
#include "internal.cuh"

namespace nucseg {

constexpr int INFG = 32767;       // "no background in this column"
constexpr int WMAX = 128;
constexpr unsigned FULLE = 0xffffffffu;

__device__ __forceinline__ int sq(int v) { return v * v; }
__device__ __forceinline__ uint32_t below_or_at(int k) { return (2u << k) - 1u; }  // bits 0..k

// Meijster's row pass for rows whose column distances exceed WMAX (rare:
// long stretches of foreground).  The stack of (site s, start t) pairs lives
// in the output row itself, packed as (s << 16) | t: in the backward pass the
// live stack index q satisfies q <= t[q] <= u, and entry q is read before
// out[u] is written, so no scratch memory is needed.
__device__ void meijster_row(const uint16_t* g, int W, int32_t* out) {
    auto F = [&](int u, int i) -> long long { return (long long)(u - i) * (u - i) + (long long)g[i] * g[i]; };
    auto S = [&](int k) -> int { return (int)((uint32_t)out[k] >> 16); };
    auto Tt = [&](int k) -> int { return (int)(out[k] & 0xffff); };
    int q = 0;
    out[0] = 0;
    for (int u = 1; u < W; u++) {
        while (q >= 0 && F(Tt(q), S(q)) > F(Tt(q), u)) q--;
        if (q < 0) {
            q = 0;
            out[0] = (int32_t)((uint32_t)u << 16);
        } else {
            int i = S(q);
            long long num = (long long)u * u - (long long)i * i + (long long)g[u] * g[u] - (long long)g[i] * g[i];
            long long den = 2LL * (u - i);
            long long fl = num / den;
            if ((num % den != 0) && (num < 0)) fl--;
            long long w = 1 + fl;
            if (w < W) {
                q++;
                out[q] = (int32_t)(((uint32_t)u << 16) | (uint32_t)w);
            }
        }
    }
    for (int u = W - 1; u >= 0; u--) {
        const int su = S(q), tu = Tt(q);
        long long d = F(u, su);
        out[u] = d >= (long long)INFG * INFG ? 0x7fffffff : (int32_t)d;
        if (u == tu) q--;
    }
}

__global__ void __launch_bounds__(256) k_edt_rows(Launch L, int RB, int Wmax) {
    extern __shared__ __align__(16) unsigned char smraw[];
    uint16_t* gs = reinterpret_cast<uint16_t*>(smraw);  // [RB][WMAX + Wmax + WMAX]
    const int Wp = Wmax + 2 * WMAX;
    __shared__ int rowslow[32];
    const int gbnd = blockIdx.x;
    const int ti = find_tile(L.tiles, L.ntiles, gbnd, &TileDev::row_base);
    const TileDev T = L.tiles[ti];
    if (!T.edt) return;
    const int W = T.W, H = T.H;
    const int y0 = (gbnd - T.row_base) * RB;
    const int c = y0 / CB, r0 = c * CB;
    const int nrow = min(RB, H - y0);
    const int nchunk = T.cby;
    if (threadIdx.x < 32) rowslow[threadIdx.x] = 0;
    for (int i = threadIdx.x; i < nrow * 2 * WMAX; i += blockDim.x) {
        const int j = i / (2 * WMAX), k = i - j * 2 * WMAX;
        gs[(size_t)j * Wp + (k < WMAX ? k : W + k)] = (uint16_t)INFG;
    }
    __syncthreads();
    auto rows_valid = [&](int cc) -> uint32_t {
        int k = min(CB, H - cc * CB);
        return k >= 32 ? FULLE : ((1u << k) - 1u);
    };
    const uint32_t rv = rows_valid(c);
    const uint32_t* const colbits = T.colbits;
    // g for the band, one column per thread; the column words of four columns
    // are loaded before any is used, so their latencies overlap
    constexpr int CU = 4;
    for (int xb = threadIdx.x; xb < W; xb += CU * blockDim.x) {
    uint32_t wv[CU];
#pragma unroll
    for (int u = 0; u < CU; u++) {
        const int x = xb + u * blockDim.x;
        wv[u] = x < W ? __ldg(colbits + (size_t)c * W + x) : 0u;
    }
#pragma unroll
    for (int u = 0; u < CU; u++) {
        const int x = xb + u * blockDim.x;
        if (x >= W) break;
        const uint32_t bg = ~wv[u] & rv;
        const int k0 = y0 - r0, k1 = y0 + nrow - 1 - r0;
        const uint32_t band = below_or_at(k1) & ~((1u << k0) - 1u);
        if ((bg & band) == band) {  // background on every row of the band: g = 0
            for (int j = 0; j < nrow; j++) gs[(size_t)j * Wp + WMAX + x] = 0;
            continue;
        }
        int above = -1, below = -1;  // nearest background row above / below this chunk
        if (!(bg & below_or_at(k0)))
            for (int cc = c - 1; cc >= 0; cc--) {
                uint32_t b2 = ~colbits[(size_t)cc * W + x] & rows_valid(cc);
                if (b2) { above = cc * CB + 31 - __clz(b2); break; }
            }
        if (!(bg & ~((1u << k1) - 1u)))
            for (int cc = c + 1; cc < nchunk; cc++) {
                uint32_t b2 = ~colbits[(size_t)cc * W + x] & rows_valid(cc);
                if (b2) { below = cc * CB + __ffs(b2) - 1; break; }
            }
        for (int j = 0; j < nrow; j++) {
            const int y = y0 + j, k = y - r0;
            const uint32_t mu = bg & below_or_at(k);
            const int du = mu ? k - (31 - __clz(mu)) : (above >= 0 ? y - above : INFG);
            const uint32_t md = bg & ~((1u << k) - 1u);
            const int dd = md ? (__ffs(md) - 1) - k : (below >= 0 ? below - y : INFG);
            const int gv = min(min(du, dd), INFG);
            gs[(size_t)j * Wp + WMAX + x] = (uint16_t)gv;
            if (gv > WMAX) rowslow[j] = 1;
        }
    }
    }
    __syncthreads();
    for (int j = 0; j < nrow; j++) {
        const uint16_t* g = gs + (size_t)j * Wp + WMAX;
        int32_t* out = T.edt + (size_t)(y0 + j) * W;
        if (!rowslow[j]) {
            // g <= WMAX on this row, so r < WMAX stays within the padding,
            // whose entries cost INFG^2 and never win
            auto solve = [&](int x) -> int {
                int D = sq(g[x]);
                for (int r = 1, rr = 1; rr < D; rr += 2 * r + 1, r++) {
                    D = __viaddmin_s32(sq(g[x - r]), rr, D);
                    D = __viaddmin_s32(sq(g[x + r]), rr, D);
                }
                return D;
            };
            if ((W & 3) == 0 && (Wp & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
                // four pixels per thread: one 8-byte read of g (8-byte aligned:
                // WMAX, x and the row stride Wp are multiples of 4), one 16-byte
                // store; a run of four background pixels needs no search at all
                for (int x = 4 * threadIdx.x; x < W; x += 4 * blockDim.x) {
                    const uint2 gq = *reinterpret_cast<const uint2*>(g + x);
                    int4 D = make_int4(0, 0, 0, 0);
                    if (gq.x | gq.y) D = make_int4(solve(x), solve(x + 1), solve(x + 2), solve(x + 3));
                    *reinterpret_cast<int4*>(out + x) = D;
                }
            } else {
                for (int x = threadIdx.x; x < W; x += blockDim.x) out[x] = solve(x);
            }
        } else if (threadIdx.x == 0) {
            meijster_row(g, W, out);
        }
    }
}

size_t edt_rows_smem(int RB, int Wmax) { return (size_t)RB * (Wmax + 2 * WMAX) * 2; }

void launch_edt(const Launch& L, int RB, int Wmax, cudaStream_t s, Profiler* pf) {
    if (L.n_rows == 0) return;
    size_t smem = edt_rows_smem(RB, Wmax);
    cudaFuncSetAttribute(k_edt_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pf->begin("edt_rows", s);
    k_edt_rows<<<L.n_rows, 256, smem, s>>>(L, RB, Wmax);
    pf->end("edt_rows", s);
}

}  // namespace nucseg
