// K1: colour deconvolution RGB -> hematoxylin plane (Sec. V-A, "Color
// deconvolution" among the feature-stage transforms), fused with the h-dome
// marker: R0 = max(hem8 - h, 0) seeds the reconstruction plane (Table I,
// ReconToNuclei).
//
// hem8 = clamp((sum_c wq_c * od_lut[rgb_c] + 2^18) >> 19, 0, 255) with the
// integer tables built on the host at pipe creation.  The 256-entry od_lut
// is replicated once per lane in shared memory as 32-bit words, entry v of
// lane l at v*32 + l, so 32 data-dependent lookups always hit 32 different
// banks.  One thread converts 16 consecutive pixels of a row: three 16-byte
// loads of interleaved RGB, one 16-byte store to each output plane, when the
// row is 16-byte aligned; byte accesses otherwise.  Clamping and the marker
// are one DPX instruction each and the output bytes are packed with integer
// multiply-adds, which keeps the integer ALU pipe below the memory bound.
// HBM-bound: 3 B read + 2 B written per pixel.
#include "internal.cuh"

namespace nucseg {

__constant__ int32_t c_lut[256];  // od_lut
__constant__ int32_t c_wq[3];     // channel weights

void upload_deconv_tables(const int32_t* lut256, const int32_t* wq3) {
    cudaMemcpyToSymbol(c_lut, lut256, sizeof(int32_t) * 256);
    cudaMemcpyToSymbol(c_wq, wq3, sizeof(int32_t) * 3);
}

struct DeconvLut {
    const int32_t* t;  // this lane's column: entry v at t[v * 32]
    int w0, w1, w2;
    // clamp((acc + 2^18) >> 19, 0, 255) for acc >= 0 and 0 for acc < 0: the
    // shifted value is <= 0 exactly when acc < 2^18, so one min-with-relu
    // covers both ends
    __device__ __forceinline__ uint32_t hem(uint32_t r, uint32_t g, uint32_t b) const {
        const int32_t acc = w0 * t[r * 32] + (w1 * t[g * 32] + (w2 * t[b * 32] + (1 << 18)));
        return (uint32_t)__vimin_s32_relu(acc >> 19, 255);
    }
};

__device__ __forceinline__ void deconv_item(const TileDev* __restrict__ tiles, int ntiles, int gid, int h,
                                            const DeconvLut& lut, int* __restrict__ rt_src);

// marker values from which a work tile counts as holding a source (nuclei
// reach about 140, stroma 22 and the background about 10)
constexpr uint32_t SRC_MARKER = 40;

__global__ void __launch_bounds__(256) k_deconv(const TileDev* __restrict__ tiles, int ntiles,
                                                int n_items, int h, int* __restrict__ rt_src) {
    __shared__ int32_t T[256 * 32];
    for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) T[i] = c_lut[i >> 5];
    __syncthreads();
    const DeconvLut lut{T + (threadIdx.x & 31), c_wq[0], c_wq[1], c_wq[2]};
    for (int gid = blockIdx.x * blockDim.x + threadIdx.x; gid < n_items; gid += gridDim.x * blockDim.x)
        deconv_item(tiles, ntiles, gid, h, lut, rt_src);
}

__device__ __forceinline__ void deconv_item(const TileDev* __restrict__ tiles, int ntiles, int gid, int h,
                                            const DeconvLut& lut, int* __restrict__ rt_src) {
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
        uint32_t hv[4] = {0, 0, 0, 0}, rv[4] = {0, 0, 0, 0}, mkmax = 0;
        // byte k of the 48 loaded bytes, zero-extended
        auto byte_at = [&](int k) -> uint32_t { return __byte_perm(w[k >> 2], 0u, 0x4440 | (k & 3)); };
#pragma unroll
        for (int p = 15; p >= 0; p--) {  // high pixel first: each word is built by multiply-adds
            const uint32_t hm = lut.hem(byte_at(3 * p), byte_at(3 * p + 1), byte_at(3 * p + 2));
            const uint32_t mk = (uint32_t)__viaddmax_s32((int)hm, -h, 0);
            hv[p >> 2] = hv[p >> 2] * 256u + hm;
            rv[p >> 2] = rv[p >> 2] * 256u + mk;
            mkmax = max(mkmax, mk);
        }
        if (rt_src && mkmax >= SRC_MARKER) rt_src[t.rt_base + (y / RT) * t.rtx + x0 / RT] = 1;
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
        uint32_t mkmax = 0;
        for (int p = 0; p < n; p++) {
            const uint32_t hm = lut.hem(src[3 * p], src[3 * p + 1], src[3 * p + 2]);
            dh[p] = (uint8_t)hm;
            const uint32_t mk = (uint32_t)__viaddmax_s32((int)hm, -h, 0);
            dr[p] = (uint8_t)mk;
            mkmax = max(mkmax, mk);
        }
        if (rt_src && mkmax >= SRC_MARKER) rt_src[t.rt_base + (y / RT) * t.rtx + x0 / RT] = 1;
    }
}

void launch_deconv(const Launch& L, cudaStream_t s, Profiler* pf) {
    if (L.n_px == 0) return;
    pf->begin("deconv", s);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one wave of resident CTAs (the 32 KB table limits them to about six per
    // SM); the per-CTA table setup is amortised over a grid-stride loop
    static int per_sm = 0;
    if (per_sm == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deconv, 256, 0) != cudaSuccess ||
                        per_sm < 1))
        per_sm = 1;
    int blocks = (L.n_px + 255) / 256;
    if (blocks > sms * per_sm) blocks = sms * per_sm;
    cudaMemsetAsync(L.rt_src, 0, sizeof(int) * (size_t)L.n_rt, s);
    k_deconv<<<blocks, 256, 0, s>>>(L.tiles, L.ntiles, L.n_px, L.h, L.rt_src);
    pf->end("deconv", s);
}

}  // namespace nucseg
