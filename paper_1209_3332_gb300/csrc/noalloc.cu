// features_tile_noalloc: the per-object feature pass for callers that cannot
// allocate device memory (see include/pipe.h).  The only scratch it needs --
// one bounding box per object -- lives in the file-scope array below, which
// every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pipe.h"
#include "internal.cuh"

using namespace nucseg;

namespace {

static __device__ __align__(256) int4 g_noalloc_bbox[PIPE_NOALLOC_MAX_OBJECTS];

// Device address of g_noalloc_bbox, per device.  In host code the symbol name
// is only a host-side stand-in, so the address is looked up once per device
// with that device current.
constexpr int MAX_DEVICES = 64;
int4* g_addr[MAX_DEVICES] = {nullptr};
int g_sms[MAX_DEVICES] = {0};
std::mutex g_mu;

struct NoEventProfiler : Profiler {
    void begin(const char*, cudaStream_t) override {}
    void end(const char*, cudaStream_t) override {}
};

int setup(int dev, int4** addr, int* sms) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_bbox) != cudaSuccess || !p) return PIPE_ECUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PIPE_ECUDA;
        g_sms[dev] = n;
        g_addr[dev] = static_cast<int4*>(p);
    }
    *addr = g_addr[dev];
    *sms = g_sms[dev];
    return PIPE_OK;
}

}  // namespace

extern "C" int features_tile_noalloc(const uint8_t* hem8_dev, const int32_t* labels_dev, int W, int H,
                                     int n_objects, float* feats_dev, pipe_stream_t stream) {
    if (!hem8_dev || !labels_dev || W < 1 || H < 1 || W > 16384 || H > 16384 || n_objects < 0 ||
        (n_objects > 0 && !feats_dev))
        return PIPE_EINVAL;
    if (n_objects > PIPE_NOALLOC_MAX_OBJECTS) return PIPE_EINVAL;
    if (n_objects == 0) return PIPE_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return PIPE_ECUDA;
    int4* bbox = nullptr;
    int sms = 0;
    int rc = setup(dev, &bbox, &sms);
    if (rc != PIPE_OK) return rc;
    NoEventProfiler pf;
    // the box pass starts by resetting the n_objects boxes it uses, so stale
    // contents of earlier calls are never read
    launch_features_plain(hem8_dev, labels_dev, W, H, n_objects, feats_dev, bbox, sms, (cudaStream_t)stream, &pf);
    return cudaGetLastError() == cudaSuccess ? PIPE_OK : PIPE_ECUDA;
}
