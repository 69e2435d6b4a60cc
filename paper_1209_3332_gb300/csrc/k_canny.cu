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
// k_canny_nms writes the strong pixels (the marker) and the candidates (the
// mask) as 0/1 planes from one 32x32 tile per CTA staged with a 2-px halo;
// the hysteresis is then the reconstruction by dilation of the marker under
// the mask, run by the reconstruction kernel of the segmentation; the counts
// take one warp per object over its box grown by the disk radius.
#include "internal.cuh"

namespace nucseg {

constexpr int CT = 32;                 // output tile of one CTA: CT x CT pixels
constexpr int CT_THREADS = 256;
constexpr int CT_S = CT + 4;           // staged plane, 2-px halo
constexpr int CT_M = CT + 2;           // magnitudes, 1-px halo

__global__ void __launch_bounds__(CT_THREADS) k_canny_nms(const uint8_t* __restrict__ I, int W, int H, int low,
                                                          int high, uint8_t* __restrict__ strong,
                                                          uint8_t* __restrict__ cand) {
    __shared__ uint8_t si[CT_S][CT_S + 4];
    __shared__ int16_t sm[CT_M][CT_M + 2];
    const int x0 = blockIdx.x * CT, y0 = blockIdx.y * CT, t = threadIdx.x;
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
            const int d = si[ly + 1][lx], f = si[ly + 1][lx + 2];
            const int g = si[ly + 2][lx], hh = si[ly + 2][lx + 1], k = si[ly + 2][lx + 2];
            const int sx = (c + 2 * f + k) - (a + 2 * d + g);
            const int sy = (g + 2 * hh + k) - (a + 2 * b + c);
            m = abs(sx) + abs(sy);
        }
        sm[ly][lx] = (int16_t)m;
    }
    __syncthreads();
    for (int i = t; i < CT * CT; i += CT_THREADS) {
        const int ly = i / CT, lx = i - ly * CT;
        const int gy = y0 + ly, gx = x0 + lx;
        if (gy >= H || gx >= W) continue;
        const int a = si[ly + 1][lx + 1], b = si[ly + 1][lx + 2], c = si[ly + 1][lx + 3];
        const int d = si[ly + 2][lx + 1], f = si[ly + 2][lx + 3];
        const int g = si[ly + 3][lx + 1], hh = si[ly + 3][lx + 2], k = si[ly + 3][lx + 3];
        const int sx = (c + 2 * f + k) - (a + 2 * d + g);
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
        strong[o] = (uint8_t)(keep && m > high);
        cand[o] = (uint8_t)(keep && m > low);
    }
}

// One warp per object: the edge pixels of the object's box grown by r (the
// disk's reach) that have a pixel of the object within the disk.
__global__ void __launch_bounds__(256) k_canny_counts(const uint8_t* __restrict__ edges,
                                                      const int32_t* __restrict__ labels, int W, int H, int K,
                                                      int r, const int4* __restrict__ bbox, int32_t* counts) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int obj = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); obj < K; obj += nw) {
        const int4 bx = bbox[obj];
        int c = 0;
        if (bx.z >= bx.x) {
            const int x0 = max(bx.x - r, 0), y0 = max(bx.y - r, 0);
            const int x1 = min(bx.z + r, W - 1), y1 = min(bx.w + r, H - 1);
            const int bw = x1 - x0 + 1, n = bw * (y1 - y0 + 1);
            for (int f = lane; f < n; f += 32) {
                const int ly = f / bw, y = y0 + ly, x = x0 + (f - ly * bw);
                if (!edges[(size_t)y * W + x]) continue;
                bool hit = false;
                for (int dy = -r; dy <= r && !hit; dy++) {
                    const int yy = y + dy;
                    if ((unsigned)yy >= (unsigned)H) continue;
                    for (int dx = -r; dx <= r; dx++) {
                        const int xx = x + dx;
                        if (dx * dx + dy * dy > r * r || (unsigned)xx >= (unsigned)W) continue;
                        if (labels[(size_t)yy * W + xx] == obj + 1) {
                            hit = true;
                            break;
                        }
                    }
                }
                c += hit;
            }
            c = (int)__reduce_add_sync(0xffffffffu, (unsigned)c);
        }
        if (lane == 0) counts[obj] = c;
    }
}

void launch_canny_nms(const uint8_t* img, int W, int H, int low, int high, uint8_t* strong, uint8_t* cand,
                      cudaStream_t s, Profiler* pf) {
    dim3 grid((W + CT - 1) / CT, (H + CT - 1) / CT);
    pf->begin("canny_nms", s);
    k_canny_nms<<<grid, CT_THREADS, 0, s>>>(img, W, H, low, high, strong, cand);
    pf->end("canny_nms", s);
}

void launch_canny_counts(const uint8_t* edges, const int32_t* labels, int W, int H, int K, int r, int4* bbox,
                         int32_t* counts, int sms, cudaStream_t s, Profiler* pf) {
    if (K <= 0) return;
    launch_object_boxes(labels, W, H, K, bbox, s, pf);
    const int ctas = (K + 7) / 8;
    pf->begin("canny_counts", s);
    k_canny_counts<<<ctas < sms * 8 ? ctas : sms * 8, 256, 0, s>>>(edges, labels, W, H, K, r, bbox, counts);
    pf->end("canny_counts", s);
}

}  // namespace nucseg
