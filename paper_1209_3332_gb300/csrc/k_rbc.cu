// RBC detection (Table I "RBC detection": OpenCV colour operations and
// Vincent's MR; the paper gives no definition).  The reading computed here:
//   d = R - max(G, B) per pixel (red dominance);
//   marker = d >= t_hi, mask = d >= t_lo (0 <= t_lo <= t_hi <= 255);
//   RBC = the binary reconstruction by dilation, 8-connected, of the marker
//         under the mask: the mask components that hold a marker pixel.
// k_rbc_planes writes the marker (into the caller's output plane, where the
// reconstruction then grows it in place) and the mask as 0/1 planes, and
// flags the 64x64 work tiles that a marker pixel touches (the tile holding
// it and the neighbours whose one-pixel halo holds it), so that the
// reconstruction starts from those tiles only: a tile with no marker pixel
// in it or in its halo is already at a fixed point.  One thread converts 16
// consecutive pixels of a row (three 16-byte loads of interleaved RGB, one
// 16-byte store to each plane when the rows allow it).  HBM-bound: 3 B read
// and 2 B written per pixel.
#include "internal.cuh"

namespace nucseg {

// marker and mask bytes (0/1) of one pixel, and whether it is a marker
struct RbcPx {
    uint32_t mk, ms;
};
__device__ __forceinline__ RbcPx rbc_px(uint32_t r, uint32_t g, uint32_t b, int t_lo, int t_hi) {
    const int d = (int)r - (int)max(g, b);
    return RbcPx{d >= t_hi ? 1u : 0u, d >= t_lo ? 1u : 0u};
}

__global__ void __launch_bounds__(256) k_rbc_planes(const uint8_t* __restrict__ rgb, size_t pitch, int W, int H,
                                                    int t_lo, int t_hi, uint8_t* __restrict__ marker,
                                                    uint8_t* __restrict__ mask, int* __restrict__ flags, int rtx,
                                                    int rty, long long n_items) {
    const int cpr = (W + 15) >> 4;  // 16-pixel chunks per row
    for (long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x; gid < n_items;
         gid += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(gid / cpr), x0 = (int)(gid - (long long)y * cpr) * 16;
        const uint8_t* src = rgb + (size_t)y * pitch + (size_t)x0 * 3;
        uint8_t* dk = marker + (size_t)y * W + x0;
        uint8_t* ds = mask + (size_t)y * W + x0;
        unsigned bits = 0;  // bit p: pixel x0 + p is a marker pixel
        if (x0 + 16 <= W && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            const uint4 a = __ldcs(reinterpret_cast<const uint4*>(src));
            const uint4 b = __ldcs(reinterpret_cast<const uint4*>(src) + 1);
            const uint4 c = __ldcs(reinterpret_cast<const uint4*>(src) + 2);
            const uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
            auto byte_at = [&](int k) -> uint32_t { return __byte_perm(w[k >> 2], 0u, 0x4440 | (k & 3)); };
            uint32_t kv[4] = {0, 0, 0, 0}, sv[4] = {0, 0, 0, 0};
#pragma unroll
            for (int p = 0; p < 16; p++) {
                const RbcPx q = rbc_px(byte_at(3 * p), byte_at(3 * p + 1), byte_at(3 * p + 2), t_lo, t_hi);
                kv[p >> 2] |= q.mk << (8 * (p & 3));
                sv[p >> 2] |= q.ms << (8 * (p & 3));
                bits |= q.mk << p;
            }
            if (((reinterpret_cast<uintptr_t>(dk) | reinterpret_cast<uintptr_t>(ds)) & 15) == 0) {
                *reinterpret_cast<uint4*>(dk) = make_uint4(kv[0], kv[1], kv[2], kv[3]);
                *reinterpret_cast<uint4*>(ds) = make_uint4(sv[0], sv[1], sv[2], sv[3]);
            } else {
#pragma unroll
                for (int p = 0; p < 16; p++) {
                    dk[p] = (uint8_t)(kv[p >> 2] >> (8 * (p & 3)));
                    ds[p] = (uint8_t)(sv[p >> 2] >> (8 * (p & 3)));
                }
            }
        } else {
            const int n = min(16, W - x0);
            for (int p = 0; p < n; p++) {
                const RbcPx q = rbc_px(src[3 * p], src[3 * p + 1], src[3 * p + 2], t_lo, t_hi);
                dk[p] = (uint8_t)q.mk;
                ds[p] = (uint8_t)q.ms;
                bits |= q.mk << p;
            }
        }
        flag_seed_tiles(flags, rtx, rty, x0, y, bits);
    }
}

void launch_rbc_planes(const uint8_t* rgb, size_t pitch, int W, int H, int t_lo, int t_hi, uint8_t* marker,
                       uint8_t* mask, int* flags, cudaStream_t s, Profiler* pf) {
    const long long n_items = (long long)H * ((W + 15) >> 4);
    if (n_items == 0) return;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (n_items + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    const int rtx = (W + RT - 1) / RT, rty = (H + RT - 1) / RT;
    pf->begin("rbc_planes", s);
    k_rbc_planes<<<(int)blocks, 256, 0, s>>>(rgb, pitch, W, H, t_lo, t_hi, marker, mask, flags, rtx, rty, n_items);
    pf->end("rbc_planes", s);
}

}  // namespace nucseg
