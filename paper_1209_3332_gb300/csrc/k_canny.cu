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

constexpr int CT = 32;                 // output tile of one CTA: CT x CT pixels
constexpr int CT_THREADS = 256;
constexpr int CT_S = CT + 4;           // staged plane, 2-px halo
constexpr int CT_M = CT + 2;           // magnitudes, 1-px halo

__device__ __forceinline__ int find_block_tile(const CannyDesc* __restrict__ D, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (D[mid].blk_base <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(CT_THREADS) k_canny_nms(const CannyDesc* __restrict__ D, int n, int low, int high,
                                                          int* __restrict__ flags) {
    __shared__ uint8_t si[CT_S][CT_S + 4];
    __shared__ int16_t sm[CT_M][CT_M + 2];
    __shared__ unsigned seeds;
    const int t = threadIdx.x;
    const CannyDesc& d = D[find_block_tile(D, n, blockIdx.x)];
    const uint8_t* __restrict__ I = d.img;
    const int W = d.W, H = d.H, bl = blockIdx.x - d.blk_base;
    const int by = bl / d.bx, x0 = (bl - by * d.bx) * CT, y0 = by * CT;
    if (t == 0) seeds = 0u;
    // this block's share of the counts to zero (strided over the tile's blocks)
    const int nblk = d.bx * ((H + CT - 1) / CT);
    for (long long i = (long long)bl * CT_THREADS + t; i < d.K; i += (long long)nblk * CT_THREADS) d.counts[i] = 0;
    for (int i = t; i < CT_S * CT_S; i += CT_THREADS) {  // replicated border: clamped coordinates
        const int ly = i / CT_S, lx = i - ly * CT_S;
        const int gy = min(max(y0 - 2 + ly, 0), H - 1), gx = min(max(x0 - 2 + lx, 0), W - 1);
        si[ly][lx] = I[(size_t)gy * W + gx];
    }
    __syncthreads();
    for (int i = t; i < CT_M * CT_M; i += CT_THREADS) {  // m at (y0 - 1 + ly, x0 - 1 + lx); 0 off the image
        const int ly = i / CT_M, lx = i - ly * CT_M;
        const int gy = y0 - 1 + ly, gx = x0 - 1 + lx;
        int m = 0;
        if ((unsigned)gy < (unsigned)H && (unsigned)gx < (unsigned)W) {
            const int a = si[ly][lx], b = si[ly][lx + 1], c = si[ly][lx + 2];
            const int e = si[ly + 1][lx], f = si[ly + 1][lx + 2];
            const int g = si[ly + 2][lx], hh = si[ly + 2][lx + 1], k = si[ly + 2][lx + 2];
            const int sx = (c + 2 * f + k) - (a + 2 * e + g);
            const int sy = (g + 2 * hh + k) - (a + 2 * b + c);
            m = abs(sx) + abs(sy);
        }
        sm[ly][lx] = (int16_t)m;
    }
    __syncthreads();
    const int rtx = (W + RT - 1) / RT, rty = (H + RT - 1) / RT;
    unsigned seed = 0u;
    for (int i = t; i < CT * CT; i += CT_THREADS) {
        const int ly = i / CT, lx = i - ly * CT;
        const int gy = y0 + ly, gx = x0 + lx;
        if (gy >= H || gx >= W) continue;
        const int a = si[ly + 1][lx + 1], b = si[ly + 1][lx + 2], c = si[ly + 1][lx + 3];
        const int e = si[ly + 2][lx + 1], f = si[ly + 2][lx + 3];
        const int g = si[ly + 3][lx + 1], hh = si[ly + 3][lx + 2], k = si[ly + 3][lx + 3];
        const int sx = (c + 2 * f + k) - (a + 2 * e + g);
        const int sy = (g + 2 * hh + k) - (a + 2 * b + c);
        const int ax = abs(sx), ay = abs(sy);
        int ady, adx, bdy, bdx;
        if ((ax + ay) * (ax + ay) < 2 * ax * ax) {           // |gx| <= 1020 per term: no overflow
            ady = 0; adx = -1; bdy = 0; bdx = 1;
        } else if (ay > ax && (ay - ax) * (ay - ax) > 2 * ax * ax) {
            ady = -1; adx = 0; bdy = 1; bdx = 0;
        } else if ((sx > 0) == (sy > 0)) {                   // sx sy > 0 (both nonzero here)
            ady = -1; adx = -1; bdy = 1; bdx = 1;
        } else {
            ady = -1; adx = 1; bdy = 1; bdx = -1;
        }
        const int m = sm[ly + 1][lx + 1];
        const bool keep = m > sm[ly + 1 + ady][lx + 1 + adx] && m >= sm[ly + 1 + bdy][lx + 1 + bdx];
        const size_t o = (size_t)gy * W + gx;
        const bool strong = keep && m > high;
        d.edges[o] = (uint8_t)strong;
        d.cand[o] = (uint8_t)(keep && m > low);
        if (strong) seed |= seed_bits_px(rtx, rty, gx, gy);
    }
    // the block lies in one work tile: one flag store per touched work tile
    if (seed) atomicOr(&seeds, seed);
    __syncthreads();
    if (t < 9 && ((seeds >> t) & 1u)) {
        const int dy = t / 3 - 1, dx = t % 3 - 1;
        flags[d.rt_base + (y0 / RT + dy) * rtx + (x0 / RT + dx)] = 1;
    }
}

constexpr int CR_MAX = 4;                 // largest disk radius of the counts
constexpr int CC_S = CT + 2 * CR_MAX;     // staged labels: the block and an r-pixel halo

// Edge counts, one 32x32 block per CTA: the labels of the block and its
// r-pixel halo (0 off the image, and for labels outside 1..K) and the edge
// bytes of the block staged in shared memory; each edge pixel adds one to
// every distinct object in its disk (the first four remembered in registers,
// beyond that an object is new iff no earlier disk offset holds it).
__global__ void __launch_bounds__(256) k_canny_counts(const CannyDesc* __restrict__ D, int n, int r) {
    __shared__ int32_t sl[CC_S][CC_S + 1];
    __shared__ uint8_t se[CT][CT];
    const int t = threadIdx.x;
    const CannyDesc& d = D[find_block_tile(D, n, blockIdx.x)];
    const int K = d.K;
    if (K <= 0) return;
    const int W = d.W, H = d.H, bl = blockIdx.x - d.blk_base;
    const int by = bl / d.bx, x0 = (bl - by * d.bx) * CT, y0 = by * CT;
    const int S = CT + 2 * r;
    for (int i = t; i < CT * CT; i += 256) {
        const int ly = i / CT, lx = i - ly * CT, gy = y0 + ly, gx = x0 + lx;
        se[ly][lx] = (gy < H && gx < W) ? d.edges[(size_t)gy * W + gx] : (uint8_t)0;
    }
    __syncthreads();
    // skip the labels of a block without edge pixels
    int any = 0;
    for (int i = t; i < CT * CT; i += 256) any |= se[i / CT][i % CT];
    if (!__syncthreads_or(any)) return;
    for (int i = t; i < S * S; i += 256) {
        const int ly = i / S, lx = i - ly * S, gy = y0 - r + ly, gx = x0 - r + lx;
        int v = 0;
        if ((unsigned)gy < (unsigned)H && (unsigned)gx < (unsigned)W) v = d.labels[(size_t)gy * W + gx];
        sl[ly][lx] = (v >= 1 && v <= K) ? v : 0;
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
                const int v = sl[ly + r + dy][lx + r + dx];
                if (!v || v == seen0 || v == seen1 || v == seen2 || v == seen3) continue;
                bool fresh = true;
                if (nseen >= 4) {  // look for v at an earlier disk offset
                    for (int ey = -r; ey <= dy && fresh; ey++)
                        for (int ex = -r; ex <= r; ex++) {
                            if (ey == dy && ex >= dx) break;
                            if (ex * ex + ey * ey <= r2 && sl[ly + r + ey][lx + r + ex] == v) {
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

void launch_canny_nms(const std::vector<CannyDesc>& descs, CannyDesc* d_descs, int low, int high, int* flags,
                      cudaStream_t s, Profiler* pf) {
    int blocks = 0;
    for (auto& d : descs) blocks += canny_blocks(d.W, d.H);
    if (!blocks) return;
    pf->begin("canny_nms", s);
    k_canny_nms<<<blocks, CT_THREADS, 0, s>>>(d_descs, (int)descs.size(), low, high, flags);
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
