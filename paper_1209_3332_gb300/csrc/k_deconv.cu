// K1: colour deconvolution RGB -> hematoxylin plane (Sec. V-A, "Color
// deconvolution" among the feature-stage transforms), fused with the h-dome
// marker: R0 = max(hem8 - h, 0) seeds the reconstruction plane (Table I,
// ReconToNuclei).
//
// hem8 = clamp((sum_c T_c[rgb_c] + 2^18) >> 19, 0, 255) with the premultiplied
// integer tables T_c[v] = wq_c * od_lut[v] built on the host at pipe creation.
// One thread converts 16 consecutive pixels of a row: three 16-byte loads of
// interleaved RGB, one 16-byte store to each output plane, when the row is
// 16-byte aligned; byte accesses otherwise.  HBM-bound: 3 B read + 2 B
// written per pixel.
#include "internal.cuh"

namespace nucseg {

__constant__ int32_t c_tab[3 * 256];

void upload_deconv_tables(const int32_t* lut3x256) {
    cudaMemcpyToSymbol(c_tab, lut3x256, sizeof(int32_t) * 3 * 256);
}

__device__ __forceinline__ uint32_t hem_of(const int32_t* T, uint32_t r, uint32_t g, uint32_t b) {
    int32_t acc = T[r] + T[256 + g] + T[512 + b];
    int32_t v = acc < 0 ? 0 : (acc + (1 << 18)) >> 19;
    return (uint32_t)(v > 255 ? 255 : v);
}

__global__ void __launch_bounds__(256) k_deconv(const TileDev* __restrict__ tiles, int ntiles,
                                                int n_items, int h) {
    __shared__ int32_t T[3 * 256];
    for (int i = threadIdx.x; i < 3 * 256; i += blockDim.x) T[i] = c_tab[i];
    __syncthreads();
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n_items) return;
    int ti = find_tile(tiles, ntiles, gid, &TileDev::px_base);
    const TileDev& t = tiles[ti];
    int item = gid - t.px_base;
    int cpr = (t.W + 15) >> 4;  // 16-pixel chunks per row
    int y = item / cpr, cx = item - y * cpr;
    int x0 = cx * 16;
    const uint8_t* src = t.rgb + (size_t)y * t.pitch + (size_t)x0 * 3;
    uint8_t* dh = t.hem8 + (size_t)y * t.W + x0;
    uint8_t* dr = t.R + (size_t)y * t.W + x0;
    bool full = x0 + 16 <= t.W;
    if (full && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
        uint4 a = __ldcs(reinterpret_cast<const uint4*>(src));
        uint4 b = __ldcs(reinterpret_cast<const uint4*>(src) + 1);
        uint4 c = __ldcs(reinterpret_cast<const uint4*>(src) + 2);
        uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
        uint32_t hv[4] = {0, 0, 0, 0}, rv[4] = {0, 0, 0, 0};
#pragma unroll
        for (int p = 0; p < 16; p++) {
            int o = p * 3;
            uint32_t r = (w[o >> 2] >> ((o & 3) * 8)) & 255;
            uint32_t g = (w[(o + 1) >> 2] >> (((o + 1) & 3) * 8)) & 255;
            uint32_t bb = (w[(o + 2) >> 2] >> (((o + 2) & 3) * 8)) & 255;
            uint32_t hm = hem_of(T, r, g, bb);
            uint32_t mk = hm > (uint32_t)h ? hm - h : 0;
            hv[p >> 2] |= hm << ((p & 3) * 8);
            rv[p >> 2] |= mk << ((p & 3) * 8);
        }
        if ((reinterpret_cast<uintptr_t>(dh) & 15) == 0 && (reinterpret_cast<uintptr_t>(dr) & 15) == 0) {
            *reinterpret_cast<uint4*>(dh) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
            *reinterpret_cast<uint4*>(dr) = make_uint4(rv[0], rv[1], rv[2], rv[3]);
        } else {
#pragma unroll
            for (int p = 0; p < 16; p++) {
                dh[p] = (uint8_t)(hv[p >> 2] >> ((p & 3) * 8));
                dr[p] = (uint8_t)(rv[p >> 2] >> ((p & 3) * 8));
            }
        }
    } else {
        int n = min(16, t.W - x0);
        for (int p = 0; p < n; p++) {
            uint32_t hm = hem_of(T, src[3 * p], src[3 * p + 1], src[3 * p + 2]);
            dh[p] = (uint8_t)hm;
            dr[p] = (uint8_t)(hm > (uint32_t)h ? hm - h : 0);
        }
    }
}

void launch_deconv(const Launch& L, cudaStream_t s, Profiler* pf) {
    if (L.n_px == 0) return;
    pf->begin("deconv", s);
    k_deconv<<<(L.n_px + 255) / 256, 256, 0, s>>>(L.tiles, L.ntiles, L.n_px, L.h);
    pf->end("deconv", s);
}

}  // namespace nucseg
