// Host side of libpipe: the C ABI of include/pipe.h.
//
// A pipe owns one plain-form workspace (used by seg_tile / features_tile in
// stream order), a batched-form arena with a cache of captured CUDA graphs
// keyed by batch shape, and the serving slots of the served form.  Every
// device pass of the path is one of the kernels in k_*.cu; this file only
// sizes buffers, fills per-tile descriptors and enqueues launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pipe.h"
#include "internal.cuh"

using namespace nucseg;

namespace {

#define CK(x)                                 \
    do {                                      \
        cudaError_t e__ = (x);                \
        if (e__ != cudaSuccess) return PIPE_ECUDA; \
    } while (0)

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

// ---- colour deconvolution constants, rebuilt from their formulas ------------------
// Stain OD vectors of Ruifrok & Johnston (2001); hematoxylin weight per
// channel = first column of the inverse of the stain matrix [H; E; H x E].
void deconv_tables(int32_t lut[256], int32_t wq[3]) {
    double Hs[3] = {0.650, 0.704, 0.286}, Es[3] = {0.072, 0.990, 0.105};
    auto nrm = [](double* v) {
        double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int i = 0; i < 3; i++) v[i] /= n;
    };
    nrm(Hs);
    nrm(Es);
    double Rs[3] = {Hs[1] * Es[2] - Hs[2] * Es[1], Hs[2] * Es[0] - Hs[0] * Es[2], Hs[0] * Es[1] - Hs[1] * Es[0]};
    nrm(Rs);
    const double* M[3] = {Hs, Es, Rs};  // rows
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                 M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                 M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    // c = od * M^-1, so channel k weighs (M^-1)[k][0] = cofactor(0,k) / det
    for (int k = 0; k < 3; k++) {
        int c1 = k == 0 ? 1 : 0, c2 = k == 2 ? 1 : 2;
        double minor = M[1][c1] * M[2][c2] - M[1][c2] * M[2][c1];
        double w = ((k & 1) ? -minor : minor) / det;
        wq[k] = (int32_t)std::llround(100.0 * w * 2048.0);
    }
    for (int v = 0; v < 256; v++) lut[v] = (int32_t)std::floor(-std::log((v + 1) / 256.0) * 256.0 + 0.5);
}

// ---- profiler ---------------------------------------------------------------------
struct EventProfiler : Profiler {
    bool enabled = false;
    long long launches = 0;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec { std::string name; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::map<std::string, std::pair<long long, double>> totals;
    std::map<std::string, int> open;
    cudaEvent_t pending_begin = nullptr;
    std::string pending_name;

    cudaEvent_t get() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void begin(const char* name, cudaStream_t s) override {
        launches++;
        if (!enabled) return;
        pending_begin = get();
        pending_name = name;
        cudaEventRecord(pending_begin, s);
    }
    void end(const char* name, cudaStream_t s) override {
        if (!enabled || !pending_begin) return;
        cudaEvent_t b = get();
        cudaEventRecord(b, s);
        recs.push_back({pending_name, pending_begin, b});
        pending_begin = nullptr;
        if (used > 8192) flush();
    }
    void flush() {
        cudaDeviceSynchronize();
        for (auto& r : recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                auto& t = totals[r.name];
                t.first++;
                t.second += ms;
            }
        }
        recs.clear();
        used = 0;
    }
    ~EventProfiler() {
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// a profiler that only counts (used while capturing graphs)
struct CountingProfiler : Profiler {
    long long* counter;
    void begin(const char*, cudaStream_t) override { (*counter)++; }
    void end(const char*, cudaStream_t) override {}
};

// CUDA graphs of the launch sequence, keyed by batch shape.  Descriptors live
// in device memory (uploaded before each replay), so a graph replays for any
// buffers of its shape on the context it was captured for.
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
};
using GraphCache = std::map<std::string, GraphEntry>;

void clear_graphs(GraphCache& g) {
    for (auto& kv : g) cudaGraphExecDestroy(kv.second.exec);
    g.clear();
}

// ---- device buffers -----------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    int ensure(size_t bytes) {
        if (bytes <= n) return PIPE_OK;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return PIPE_ENOMEM;
        n = bytes;
        return PIPE_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

// Geometry and workspace sizes of one image.
struct Geo {
    int W, H, wpr, rtx, rty, cbx, cby, nchunks;
    size_t N, ws_bytes;
};

int bands_rows(int Wmax) { return Wmax <= 4096 ? 4 : (Wmax <= 8192 ? 2 : 1); }

// Launch shapes of one batch.  None of them changes any result: they set how
// many persistent reconstruction workers run, how many rows one EDT block
// solves (a divisor of the 32-row chunk), and how many blocks the feature
// pass spreads the objects over.
struct Tune {
    int recon_grid, edt_rb, feat_grid;
};
std::string tune_str(const Tune& t) {
    return std::to_string(t.recon_grid) + " " + std::to_string(t.edt_rb) + " " + std::to_string(t.feat_grid);
}

Geo geometry(int W, int H, int feats_cap) {
    Geo g;
    g.W = W;
    g.H = H;
    g.N = (size_t)W * H;
    g.wpr = (W + 31) / 32;
    g.rtx = (W + RT - 1) / RT;
    g.rty = (H + RT - 1) / RT;
    g.cbx = (W + CB - 1) / CB;
    g.cby = (H + CB - 1) / CB;
    size_t words = (size_t)H * g.wpr;
    g.nchunks = (int)((words + SCAN_CHUNK - 1) / SCAN_CHUNK);
    size_t b = 0;
    b += al256(g.N);                              // R
    b += 2 * al256(g.N * 4);                      // P, A
    b += al256((size_t)g.cbx * g.cby * RL_CAP * 4);  // per-block root lists
    b += al256((size_t)g.cbx * g.cby * 4);        // per-block root counts
    const size_t bwords = (size_t)g.cbx * g.cby * CB;  // block-major bitmaps: CB words per block
    b += 2 * al256(bwords * 4);                   // fg, filled bitmaps (block-major)
    b += al256(words * 4);                        // root bitmap (row-major)
    b += al256(words * 4);                        // word prefix
    b += al256((size_t)g.nchunks * 4);            // chunk sums
    b += al256((size_t)g.cbx * g.cby * 4 * CB * 4);  // block edges
    b += al256((size_t)g.cby * W * 4);            // EDT column bits per chunk
    b += al256((size_t)std::max(feats_cap, 1) * 16);  // object boxes
    g.ws_bytes = b;
    return g;
}

// Carve the workspace of one image at `base` into a descriptor.
void carve(TileDev& t, const Geo& g, char* base) {
    size_t words = (size_t)g.H * g.wpr;
    char* p = base;
    auto take = [&](size_t n) { char* r = p; p += al256(n); return r; };
    t.R = (uint8_t*)take(g.N);
    t.P = (int32_t*)take(g.N * 4);
    t.A = (int32_t*)take(g.N * 4);
    t.rootlist = (int32_t*)take((size_t)g.cbx * g.cby * RL_CAP * 4);
    t.blkroots = (int32_t*)take((size_t)g.cbx * g.cby * 4);
    const size_t bwords = (size_t)g.cbx * g.cby * CB;
    t.fgbits = (uint32_t*)take(bwords * 4);
    t.filledbits = (uint32_t*)take(bwords * 4);
    t.rootbits = (uint32_t*)take(words * 4);
    t.wordprefix = (int32_t*)take(words * 4);
    t.chunksum = (int32_t*)take((size_t)g.nchunks * 4);
    t.border = (int32_t*)take((size_t)g.cbx * g.cby * 4 * CB * 4);
    t.colbits = (uint32_t*)take((size_t)g.cby * g.W * 4);
    t.bbox = (int4*)take((size_t)std::max(t.feats_cap, 1) * 16);
    t.W = g.W;
    t.H = g.H;
    t.wpr = g.wpr;
    t.rtx = g.rtx;
    t.rty = g.rty;
    t.cbx = g.cbx;
    t.cby = g.cby;
    t.nchunks = g.nchunks;
}

// descriptors are written by a kernel that receives them as parameters, so
// no host staging buffer must outlive the call and graph capture works
constexpr int DESC_PER_LAUNCH = 8;
struct DescPack {
    TileDev d[DESC_PER_LAUNCH];
    int n, first;
};
__global__ void k_set_desc(TileDev* dst, DescPack p) {
    if (threadIdx.x < p.n) dst[p.first + threadIdx.x] = p.d[threadIdx.x];
}

// Everything one launch sequence needs besides the descriptors.
struct LaunchCtx {
    DevBuf tiles, wl, shared;  // TileDev[], slots+state, Shared + statuses
    DevBuf arena;
    int ntiles_cap = 0;
};

}  // namespace

// ---- the pipe ---------------------------------------------------------------------------

// One served-form context: buffers for a group of tiles submitted together,
// processed as one batched launch on the context's own stream.
struct Ctx {
    cudaStream_t stream = nullptr;  // this context's uploads
    cudaEvent_t uploaded = nullptr;
    cudaEvent_t done = nullptr;
    LaunchCtx lc;
    DevBuf dev;                    // rgb, hem8, labels, edt, n_objects, feats of all tiles
    void* h_in = nullptr;          // pinned RGB staging (pageable inputs)
    size_t h_in_n = 0;
    void* h_out = nullptr;         // pinned results
    size_t h_out_n = 0;
    size_t bytes = 0;              // device bytes held (budget accounting)
    bool busy = false;
    GraphCache graphs;            // compute part of a group, per shape
};

struct TicketTile {
    int W, H, want;
    int cap;                       // feature rows the result buffer holds
    size_t out_off, nobj_off, st_off;
};

struct Ticket {
    int ctx = -1;
    std::vector<TicketTile> tiles;
    double t_submit = 0;
    bool done = false;
    double t_done_ms = 0;
    std::vector<std::vector<float>> feats;
    std::vector<std::vector<uint8_t>> hem8;
    std::vector<std::vector<int32_t>> labels, edt;
};

struct pipe_s {
    int device = 0;
    pipe_params prm;
    int sms = 0;
    int recon_cap = 1;
    EventProfiler prof;
    // plain form
    LaunchCtx plain;
    TileDev last_plain{};
    bool have_last = false;
    DevBuf fbbox;
    DevBuf morph_tmp;  // scratch plane of morph_open_tile
    DevBuf ws_obj;      // watershed_tile: per-object boxes and basin counts
    DevBuf ws_scratch;  // watershed_tile: planes for boxes larger than the shared-memory stage
    DevBuf ws_status;   // watershed_tile: device status word
    DevBuf ws_desc;     // watershed_batch: tile descriptors
    cudaStream_t ws_side = nullptr;        // watershed_tile: large boxes overlap the small ones here
    LaunchCtx rbc;      // rbc_tile: the reconstruction of the RBC markers runs on this context
    DevBuf rbc_mask;    // rbc_tile: the mask plane
    DevBuf rbc_flags;   // rbc_tile: seed flags, one int per work tile
    LaunchCtx canny;    // canny_tile: the hysteresis runs the reconstruction on this context
    DevBuf canny_cand;  // canny_tile / canny_batch: candidate planes (the reconstruction's masks)
    DevBuf canny_flags; // canny_tile / canny_batch: seed flags, one int per work tile
    DevBuf canny_desc;  // canny_tile / canny_batch: tile descriptors
    cudaEvent_t ws_fork = nullptr, ws_join = nullptr;
    // batched form
    LaunchCtx batch;
    GraphCache graphs;
    int batch_ntiles = 0;
    // served form
    std::mutex mu;
    std::vector<std::unique_ptr<Ctx>> ctxs;
    std::map<uint64_t, std::unique_ptr<Ticket>> tickets;
    uint64_t next_ticket = 1;
    EventProfiler serve_prof;      // launches of the served form (counted, not timed)
    cudaStream_t serve_compute = nullptr;  // all groups compute in submission order
    cudaEvent_t serve_ref = nullptr;       // recorded at serve_ref_ms (host clock)
    double serve_ref_ms = 0;
    size_t peak_io = 0, peak_ws = 0;       // largest served group so far
    int peak_rt = 0, peak_n = 0;
    // launch shapes per batch shape: tuned by the batched form on first sight
    // of a shape, or read from the autotune cache file
    std::map<std::string, Tune> tuned;
    std::string tune_file;
    long long tune_runs = 0;
    Tune last_tune{0, 0, 0};
};

namespace {

// Reconstruction queue per launch: a 64-bit slot, a state word and a source
// flag per work tile.
size_t wl_bytes(int n_rt) { return sizeof(int) * 4 * (size_t)std::max(n_rt, 1); }

int ensure_ctx(LaunchCtx& c, int ntiles, int n_rt, size_t arena_bytes) {
    int rc;
    if ((rc = c.tiles.ensure(sizeof(TileDev) * std::max(ntiles, 1)))) return rc;
    if ((rc = c.wl.ensure(wl_bytes(n_rt)))) return rc;
    if ((rc = c.shared.ensure(sizeof(Shared) + sizeof(int) * (2 + std::max(ntiles, 1))))) return rc;
    if ((rc = c.arena.ensure(std::max(arena_bytes, (size_t)256)))) return rc;
    return PIPE_OK;
}

// Device bytes of a served context's buffers, and what they become when the
// context is made ready for a group of n tiles (io: caller-visible buffers,
// ws: workspace arena, n_rt: reconstruction work tiles).  ensure() only
// grows a buffer, so each part becomes the larger of the two.

size_t tiles_bytes(int n) { return sizeof(TileDev) * (size_t)std::max(n, 1); }
size_t shared_bytes(int n) { return sizeof(Shared) + sizeof(int) * (2 + (size_t)std::max(n, 1)); }
size_t ctx_need(size_t io, size_t ws, int n, int n_rt) {
    return io + std::max(ws, (size_t)256) + tiles_bytes(n) + wl_bytes(n_rt) + shared_bytes(n);
}
bool ctx_fits(const Ctx& c, size_t io, size_t ws, int n, int n_rt) {
    return c.dev.n >= io && c.lc.arena.n >= ws && c.lc.wl.n >= wl_bytes(n_rt) && c.lc.tiles.n >= tiles_bytes(n) &&
           c.lc.shared.n >= shared_bytes(n);
}
size_t ctx_bytes(const Ctx& c) { return c.dev.n + c.lc.arena.n + c.lc.tiles.n + c.lc.wl.n + c.lc.shared.n; }
size_t ctx_bytes_after(const Ctx& c, size_t io, size_t ws, int n, int n_rt) {
    return std::max(c.dev.n, io) + std::max(c.lc.arena.n, std::max(ws, (size_t)256)) +
           std::max(c.lc.tiles.n, tiles_bytes(n)) + std::max(c.lc.wl.n, wl_bytes(n_rt)) +
           std::max(c.lc.shared.n, shared_bytes(n));
}
// Frees an idle context's device buffers (its graphs refer to them).  Idle
// means batch_poll has seen its last group complete, so no GPU work still
// uses them.
void ctx_release_device(Ctx& c) {
    clear_graphs(c.graphs);
    c.dev.release();
    c.lc.tiles.release();
    c.lc.wl.release();
    c.lc.shared.release();
    c.lc.arena.release();
    c.bytes = 0;
}
// Device bytes held by all served contexts, busy or idle.
size_t serve_allocated(pipe_t p) {
    size_t s = 0;
    for (auto& c : p->ctxs) s += c->bytes;
    return s;
}

// Fill launch-wide bases of the descriptors and the Launch totals.
Launch make_launch(pipe_t p, LaunchCtx& c, std::vector<TileDev>& td, int n_rt_total, int RB) {
    Launch L{};
    L.tiles = (TileDev*)c.tiles.p;
    L.ntiles = (int)td.size();
    L.wl_slots = (unsigned long long*)c.wl.p;
    L.wl_state = (int*)c.wl.p + 2 * std::max(n_rt_total, 1);
    L.rt_src = L.wl_state + std::max(n_rt_total, 1);
    L.sh = (Shared*)c.shared.p;
    L.status = (int*)((char*)c.shared.p + sizeof(Shared));
    L.tile_status = L.status + 2;
    int rt = 0, cb = 0, ch = 0, col = 0, row = 0, px = 0;
    for (auto& t : td) {
        t.rt_base = rt;
        t.cb_base = cb;
        t.chunk_base = ch;
        t.col_base = col;
        t.row_base = row;
        t.px_base = px;
        t.obj_base = 0;
        rt += t.rtx * t.rty;
        cb += t.cbx * t.cby;
        ch += t.nchunks;
        col += t.W;
        row += (t.H + RB - 1) / RB;
        px += t.H * ((t.W + 15) / 16);
    }
    for (int i = 0; i < (int)td.size() && i < LAUNCH_TAB; i++) L.cb_first[i] = td[i].cb_base;
    L.n_rt = rt;
    L.n_cb = cb;
    L.n_chunks = ch;
    L.n_cols = col;
    L.n_rows = row;
    L.n_px = px;
    L.wait_budget = p->prm.wait_budget_cycles;
    L.h = p->prm.h;
    L.thr = p->prm.dome_thresh;
    L.amin = p->prm.area_min;
    L.amax = p->prm.area_max;
    return L;
}

int upload_desc(const Launch& L, const std::vector<TileDev>& td, cudaStream_t s) {
    for (int i = 0; i < (int)td.size(); i += DESC_PER_LAUNCH) {
        DescPack pk;
        pk.first = i;
        pk.n = std::min(DESC_PER_LAUNCH, (int)td.size() - i);
        for (int k = 0; k < pk.n; k++) pk.d[k] = td[i + k];
        k_set_desc<<<1, 32, 0, s>>>(L.tiles, pk);
    }
    CK(cudaGetLastError());
    return PIPE_OK;
}

int max_width(const std::vector<TileDev>& td) {
    int w = 1;
    for (auto& t : td) w = std::max(w, t.W);
    return w;
}

// The whole path over the descriptors of L (segmentation, and features when
// `features` is set: boxes come from the relabel pass).
void run_path(pipe_t p, const Launch& L, int Wmax, bool features, int max_objects, const Tune& tu,
              cudaStream_t s, Profiler* pf) {
    launch_deconv(L, s, pf);
    launch_recon(L, tu.recon_grid, s, pf);
    launch_label(L, features ? 1 : 0, max_objects, p->sms, s, pf);
    launch_edt(L, tu.edt_rb, Wmax, s, pf);
    if (features) launch_features_batched(L, tu.feat_grid, s, pf);
}

int run_path_graph(pipe_t p, GraphCache& cache, const std::string& shape_key, const Launch& L, int Wmax,
                   int max_obj, const Tune& tu, cudaStream_t s, long long* launches) {
    const std::string key = shape_key + "|" + tune_str(tu);
    auto it = cache.find(key);
    if (it == cache.end()) {
        cudaStream_t cs;
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        long long nk = 0;
        CountingProfiler cp;
        cp.counter = &nk;
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaStreamDestroy(cs);
            return PIPE_ECUDA;
        }
        run_path(p, L, Wmax, true, max_obj, tu, cs, &cp);
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return PIPE_ECUDA;
        GraphEntry ge;
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return PIPE_ECUDA;
        ge.kernels = nk;
        it = cache.emplace(key, ge).first;
    }
    CK(cudaGraphLaunch(it->second.exec, s));
    *launches += it->second.kernels;
    return PIPE_OK;
}

Tune default_tune(pipe_t p, int Wmax) { return Tune{p->recon_cap, bands_rows(Wmax), p->sms * 16}; }

constexpr size_t EDT_SMEM_MAX = 96 * 1024;

bool tune_ok(pipe_t p, const Tune& t, int Wmax) {
    return t.recon_grid >= 1 && t.recon_grid <= p->recon_cap && (t.edt_rb == 1 || t.edt_rb == 2 || t.edt_rb == 4 ||
           t.edt_rb == 8) && edt_rows_smem(t.edt_rb, Wmax) <= EDT_SMEM_MAX && t.feat_grid >= 1 &&
           t.feat_grid <= p->sms * 64;
}

// Tuning key: the device's SM count and the tile sizes, in batch order.
std::string tune_key(pipe_t p, const std::vector<Geo>& geos) {
    std::string k = std::to_string(p->sms) + "sm:";
    for (const Geo& g : geos) k += std::to_string(g.W) + "x" + std::to_string(g.H) + ";";
    return k;
}

// The cache file holds one line per key: "<key> <recon_grid> <edt_rb> <feat_grid>".
void load_tune_file(pipe_t p) {
    FILE* f = std::fopen(p->tune_file.c_str(), "r");
    if (!f) return;
    std::vector<char> line(1 << 20);
    while (std::fgets(line.data(), (int)line.size(), f)) {
        char* sp = std::strchr(line.data(), ' ');
        if (!sp) continue;
        Tune t;
        if (std::sscanf(sp + 1, "%d %d %d", &t.recon_grid, &t.edt_rb, &t.feat_grid) != 3) continue;
        p->tuned[std::string(line.data(), sp)] = t;
    }
    std::fclose(f);
}

void save_tune(pipe_t p, const std::string& key, const Tune& t) {
    if (p->tune_file.empty()) return;
    FILE* f = std::fopen(p->tune_file.c_str(), "a");
    if (!f) return;
    std::fprintf(f, "%s %s\n", key.c_str(), tune_str(t).c_str());
    std::fclose(f);
}

// Picks the launch shapes of a batch by timing the whole batched path on the
// batch itself, one parameter at a time (coordinate descent from the
// defaults); each candidate runs once to warm and is timed as the fastest of
// two runs with CUDA events.  Every candidate computes the same results, so
// the runs only rewrite the caller's outputs with identical values.  A
// candidate replaces the current choice only if it is 2% faster.
int autotune(pipe_t p, LaunchCtx& c, std::vector<TileDev>& td, int n_rt, int Wmax, int max_obj, cudaStream_t s,
             Tune* out) {
    Tune best = default_tune(p, Wmax);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PIPE_ECUDA;
    }
    CountingProfiler cp;
    cp.counter = &p->prof.launches;
    int rc = PIPE_OK;
    auto timeit = [&](const Tune& tu, float* ms) -> int {
        Launch L = make_launch(p, c, td, n_rt, tu.edt_rb);
        int r = upload_desc(L, td, s);
        if (r) return r;
        float b = 1e30f;
        for (int k = 0; k < 3; k++) {
            if (cudaEventRecord(e0, s) != cudaSuccess) return PIPE_ECUDA;
            run_path(p, L, Wmax, true, max_obj, tu, s, &cp);
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return PIPE_ECUDA;
            float t = 0;
            if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return PIPE_ECUDA;
            if (k > 0) b = std::min(b, t);
        }
        p->tune_runs += 3;
        *ms = b;
        return PIPE_OK;
    };
    float cur = 0;
    auto consider = [&](Tune t) -> int {
        if (!tune_ok(p, t, Wmax)) return PIPE_OK;
        float ms = 0;
        int r = timeit(t, &ms);
        if (r) return r;
        if (ms < 0.98f * cur) {
            best = t;
            cur = ms;
        }
        return PIPE_OK;
    };
    if ((rc = timeit(best, &cur))) goto done;
    {
        const int per = std::max(1, p->recon_cap / std::max(p->sms, 1));
        const int fr[3] = {per / 4, per / 2, (3 * per) / 4};
        Tune base = best;
        for (int f : fr)
            if (f >= 1 && f < per) {
                Tune t = base;
                t.recon_grid = f * p->sms;
                if ((rc = consider(t))) goto done;
            }
        base = best;
        for (int rb : {1, 2, 8})
            if (rb != base.edt_rb) {
                Tune t = base;
                t.edt_rb = rb;
                if ((rc = consider(t))) goto done;
            }
        base = best;
        for (int fg : {4, 8, 32})
            if (fg * p->sms != base.feat_grid) {
                Tune t = base;
                t.feat_grid = fg * p->sms;
                if ((rc = consider(t))) goto done;
            }
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == PIPE_OK) *out = best;
    return rc;
}

bool valid_size(int W, int H) { return W >= 1 && H >= 1 && W <= 16384 && H <= 16384; }

// where one tile's results go in mapped host memory
struct ResultSlot {
    int32_t* head;   // [0] K, [1] tile status, [2] launch status
    float* feats;    // [cap][15]
};
constexpr int RESULTS_PER_LAUNCH = 64;
struct ResultPack {
    ResultSlot r[RESULTS_PER_LAUNCH];
    int n, first;
};
// one CTA per tile: count, status words and exactly min(K, cap) feature rows
__global__ void k_results(Launch L, ResultPack pk) {
    const int i = blockIdx.x;
    if (i >= pk.n) return;
    const TileDev& T = L.tiles[pk.first + i];
    const int K = *T.n_objects;
    const int rows = K < T.feats_cap ? K : T.feats_cap;
    if (threadIdx.x == 0) {
        pk.r[i].head[0] = K;
        pk.r[i].head[1] = L.tile_status[pk.first + i];
        pk.r[i].head[2] = L.sh->err;
    }
    const int n = rows * NFEAT;
    for (int j = threadIdx.x; j < n; j += blockDim.x) pk.r[i].feats[j] = T.feats[j];
}

int launch_results(const Launch& L, const ResultSlot* rs, int n, cudaStream_t s, Profiler* pf) {
    for (int i = 0; i < n; i += RESULTS_PER_LAUNCH) {
        ResultPack pk;
        pk.first = i;
        pk.n = std::min(RESULTS_PER_LAUNCH, n - i);
        for (int k = 0; k < pk.n; k++) pk.r[k] = rs[i + k];
        pf->begin("results", s);
        k_results<<<pk.n, 256, 0, s>>>(L, pk);
        pf->end("results", s);
    }
    CK(cudaGetLastError());
    return PIPE_OK;
}

}  // namespace

// ======================================================================================
extern "C" {

void pipe_default_params(pipe_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->h = 20;
    p->dome_thresh = 10;
    p->area_min = 20;
    p->area_max = 1500;
    p->glcm_levels = 8;
    p->n_offsets = 4;
    int off[4][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}};
    std::memcpy(p->offsets, off, sizeof(off));
    p->hbm_budget_bytes = (size_t)40 << 30;
    p->max_slots = 16;
    p->wait_budget_cycles = 1LL << 32;
    p->autotune_cache = nullptr;
    p->autotune = 1;
}

int pipe_create(const pipe_params* params, int device, pipe_t* out) {
    if (!out) return PIPE_EINVAL;
    *out = nullptr;
    pipe_params prm;
    if (params) prm = *params; else pipe_default_params(&prm);
    int off[4][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}};
    if (prm.glcm_levels != 8 || prm.n_offsets != 4 || std::memcmp(prm.offsets, off, sizeof(off)) != 0 ||
        prm.h < 0 || prm.h > 255 || prm.dome_thresh < 0 || prm.area_min < 0 || prm.area_max < prm.area_min ||
        prm.max_slots < 1 || prm.wait_budget_cycles <= 0)
        return PIPE_EINVAL;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return PIPE_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return PIPE_ECUDA;
    pipe_t p = new pipe_s();
    p->device = device;
    p->prm = prm;
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, device);
    int32_t lut[256], wq[3];
    deconv_tables(lut, wq);
    upload_deconv_tables(lut, wq);
    p->recon_cap = std::max(1, recon_grid(device));
    if (prm.autotune_cache) {
        p->tune_file = prm.autotune_cache;
        load_tune_file(p);
    }
    if (cudaGetLastError() != cudaSuccess) {
        delete p;
        return PIPE_ECUDA;
    }
    *out = p;
    return PIPE_OK;
}

void pipe_destroy(pipe_t p) {
    if (!p) return;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    clear_graphs(p->graphs);
    auto rel = [](LaunchCtx& c) { c.tiles.release(); c.wl.release(); c.shared.release(); c.arena.release(); };
    rel(p->plain);
    rel(p->batch);
    p->fbbox.release();
    p->morph_tmp.release();
    p->ws_obj.release();
    rel(p->rbc);
    p->rbc_mask.release();
    p->rbc_flags.release();
    rel(p->canny);
    p->canny_cand.release();
    p->canny_flags.release();
    p->canny_desc.release();
    p->ws_scratch.release();
    p->ws_status.release();
    p->ws_desc.release();
    if (p->ws_side) cudaStreamDestroy(p->ws_side);
    if (p->ws_fork) cudaEventDestroy(p->ws_fork);
    if (p->ws_join) cudaEventDestroy(p->ws_join);
    for (auto& c : p->ctxs) {
        rel(c->lc);
        c->dev.release();
        if (c->h_in) cudaFreeHost(c->h_in);
        if (c->h_out) cudaFreeHost(c->h_out);
        clear_graphs(c->graphs);
        if (c->uploaded) cudaEventDestroy(c->uploaded);
        if (c->done) cudaEventDestroy(c->done);
        if (c->stream) cudaStreamDestroy(c->stream);
    }
    if (p->serve_ref) cudaEventDestroy(p->serve_ref);
    if (p->serve_compute) cudaStreamDestroy(p->serve_compute);
    delete p;
}

int seg_tile(pipe_t p, const uint8_t* rgb_dev, int W, int H, size_t pitch_bytes, uint8_t* hem8_dev,
             int32_t* labels_dev, int32_t* edt_dev, int32_t* n_objects_dev, pipe_stream_t stream) {
    if (!p || !rgb_dev || !hem8_dev || !labels_dev || !n_objects_dev) return PIPE_EINVAL;
    if (!valid_size(W, H) || pitch_bytes < (size_t)W * 3) return PIPE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(p->device));
    Geo g = geometry(W, H, 1);
    int n_rt = g.rtx * g.rty;
    if (p->plain.arena.n < g.ws_bytes || p->plain.wl.n < wl_bytes(n_rt)) CK(cudaStreamSynchronize(s));
    int rc = ensure_ctx(p->plain, 1, n_rt, g.ws_bytes);
    if (rc) return rc;
    std::vector<TileDev> td(1);
    TileDev& t = td[0];
    std::memset(&t, 0, sizeof(t));
    t.feats_cap = 1;
    carve(t, g, (char*)p->plain.arena.p);
    t.pitch = pitch_bytes;
    t.rgb = rgb_dev;
    t.hem8 = hem8_dev;
    t.labels = labels_dev;
    t.edt = edt_dev;
    t.n_objects = n_objects_dev;
    t.feats = nullptr;
    const Tune tu = default_tune(p, W);
    Launch L = make_launch(p, p->plain, td, n_rt, tu.edt_rb);
    if ((rc = upload_desc(L, td, s))) return rc;
    run_path(p, L, W, false, 0, tu, s, &p->prof);
    CK(cudaGetLastError());
    p->last_plain = td[0];
    p->have_last = true;
    return PIPE_OK;
}

int features_tile(pipe_t p, const uint8_t* hem8_dev, const int32_t* labels_dev, int W, int H, int n_objects,
                  float* feats_dev, pipe_stream_t stream) {
    if (!p || !hem8_dev || !labels_dev || n_objects < 0 || (n_objects > 0 && !feats_dev)) return PIPE_EINVAL;
    if (!valid_size(W, H)) return PIPE_EINVAL;
    if (n_objects == 0) return PIPE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(p->device));
    size_t need = (size_t)n_objects * sizeof(int4);
    if (p->fbbox.n < need) {
        CK(cudaStreamSynchronize(s));
        int rc = p->fbbox.ensure(need);
        if (rc) return rc;
    }
    launch_features_plain(hem8_dev, labels_dev, W, H, n_objects, feats_dev, (int4*)p->fbbox.p, p->sms, s,
                          &p->prof);
    CK(cudaGetLastError());
    return PIPE_OK;
}

int morph_open_tile(pipe_t p, const uint8_t* src_dev, int W, int H, int radius, uint8_t* dst_dev,
                    pipe_stream_t stream) {
    if (!p || !src_dev || !dst_dev || radius < 0 || radius > MORPH_RMAX) return PIPE_EINVAL;
    if (!valid_size(W, H)) return PIPE_EINVAL;
    const size_t N = (size_t)W * H;
    if (src_dev < dst_dev + N && dst_dev < src_dev + N) return PIPE_EINVAL;  // the planes overlap
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(p->device));
    if (p->morph_tmp.n < N) {  // the scratch plane of the two-pass form grows to the largest plane seen
        CK(cudaStreamSynchronize(s));
        const int rc = p->morph_tmp.ensure(N);
        if (rc) return rc;
    }
    launch_morph_open(src_dev, dst_dev, (uint8_t*)p->morph_tmp.p, W, H, radius, s, &p->prof);
    CK(cudaGetLastError());
    return PIPE_OK;
}

int watershed_tile(pipe_t p, const int32_t* labels_dev, const int32_t* edt_dev, int W, int H, int n_objects,
                   int h, int32_t* out_dev, int32_t* n_basins_dev, pipe_stream_t stream) {
    if (!p || !labels_dev || !edt_dev || !out_dev || !n_basins_dev || n_objects < 0 || h < 0 || h > 255)
        return PIPE_EINVAL;
    if (!valid_size(W, H)) return PIPE_EINVAL;
    const size_t N = (size_t)W * H;
    auto overlap = [N](const void* a, const void* b) {
        const char *x = (const char*)a, *y = (const char*)b;
        return x < y + N * 4 && y < x + N * 4;
    };
    if (overlap(out_dev, labels_dev) || overlap(out_dev, edt_dev)) return PIPE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(p->device));
    const size_t need_obj = (size_t)std::max(n_objects, 1) * (sizeof(int4) + 2 * sizeof(int)) + 3 * sizeof(int);
    const size_t need_scr = watershed_scratch_bytes(W, H);
    if (p->ws_obj.n < need_obj || p->ws_scratch.n < need_scr || !p->ws_status.p) {
        CK(cudaStreamSynchronize(s));
        int rc;
        if ((rc = p->ws_obj.ensure(need_obj)) || (rc = p->ws_scratch.ensure(need_scr))) return rc;
        if (!p->ws_status.p) {
            if ((rc = p->ws_status.ensure(sizeof(int)))) return rc;
            CK(cudaMemset(p->ws_status.p, 0, sizeof(int)));
        }
    }
    if (!p->ws_side) {
        int lo_pri = 0, hi_pri = 0;  // the large boxes go first when SM room frees up
        CK(cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri));
        CK(cudaStreamCreateWithPriority(&p->ws_side, cudaStreamNonBlocking, hi_pri));
        CK(cudaEventCreateWithFlags(&p->ws_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&p->ws_join, cudaEventDisableTiming));
    }
    int4* bbox = (int4*)p->ws_obj.p;
    int* cnt = (int*)(bbox + std::max(n_objects, 1));
    int* next = cnt + std::max(n_objects, 1);
    launch_watershed(labels_dev, edt_dev, W, H, n_objects, h, out_dev, n_basins_dev, bbox, cnt, next, p->ws_scratch.p,
                     (int*)p->ws_status.p, p->sms, s, p->ws_side, p->ws_fork, p->ws_join, &p->prof);
    CK(cudaGetLastError());
    return PIPE_OK;
}

int watershed_batch(pipe_t p, const ws_tile* tiles, int n, int h, pipe_stream_t stream) {
    if (!p || !tiles || n < 1 || n > 4096 || h < 0 || h > 255) return PIPE_EINVAL;
    std::vector<WsDesc> d(n);
    size_t objs = 0, px = 0;
    for (int i = 0; i < n; i++) {
        const ws_tile& t = tiles[i];
        if (!t.labels || !t.edt || !t.out || !t.n_basins || t.n_objects < 0 || !valid_size(t.W, t.H))
            return PIPE_EINVAL;
        const size_t N = (size_t)t.W * t.H;
        const char *o = (const char*)t.out, *l = (const char*)t.labels, *e = (const char*)t.edt;
        if ((o < l + N * 4 && l < o + N * 4) || (o < e + N * 4 && e < o + N * 4)) return PIPE_EINVAL;
        d[i].labels = t.labels;
        d[i].edt = t.edt;
        d[i].out = t.out;
        d[i].n_basins = t.n_basins;
        d[i].px_base = (long long)px;
        d[i].W = t.W;
        d[i].H = t.H;
        d[i].K = t.n_objects;
        d[i].obj_base = (int)objs;
        d[i].seg_base = 0;
        objs += (size_t)t.n_objects;
        px += N;
    }
    if (objs > (size_t)INT32_MAX / 32) return PIPE_EINVAL;
    long long segs = 0;
    for (auto& x : d) {
        x.seg_base = (int)segs;
        segs += (long long)(x.W + FB_SEG - 1) / FB_SEG * x.H;
    }
    if (segs * 32 > INT32_MAX) return PIPE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(p->device));
    const size_t need_obj = std::max(objs, (size_t)1) * (sizeof(int4) + 2 * sizeof(int)) + 3 * sizeof(int);
    const size_t need_scr = px * (sizeof(unsigned long long) + sizeof(uint16_t));
    const size_t need_desc = sizeof(WsDesc) * (size_t)n;
    if (p->ws_obj.n < need_obj || p->ws_scratch.n < need_scr || p->ws_desc.n < need_desc || !p->ws_status.p) {
        CK(cudaStreamSynchronize(s));
        int rc;
        if ((rc = p->ws_obj.ensure(need_obj)) || (rc = p->ws_scratch.ensure(need_scr)) ||
            (rc = p->ws_desc.ensure(need_desc)))
            return rc;
        if (!p->ws_status.p) {
            if ((rc = p->ws_status.ensure(sizeof(int)))) return rc;
            CK(cudaMemset(p->ws_status.p, 0, sizeof(int)));
        }
    }
    if (!p->ws_side) {
        int lo_pri = 0, hi_pri = 0;  // the large boxes go first when SM room frees up
        CK(cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri));
        CK(cudaStreamCreateWithPriority(&p->ws_side, cudaStreamNonBlocking, hi_pri));
        CK(cudaEventCreateWithFlags(&p->ws_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&p->ws_join, cudaEventDisableTiming));
    }
    int4* bbox = (int4*)p->ws_obj.p;
    int* cnt = (int*)(bbox + std::max(objs, (size_t)1));
    int* next = cnt + std::max(objs, (size_t)1);
    launch_watershed_batch(d, (WsDesc*)p->ws_desc.p, h, bbox, cnt, next, p->ws_scratch.p, px, (int*)p->ws_status.p, p->sms,
                           s, p->ws_side, p->ws_fork, p->ws_join, &p->prof);
    CK(cudaGetLastError());
    return PIPE_OK;
}

int rbc_tile(pipe_t p, const uint8_t* rgb_dev, int W, int H, size_t pitch_bytes, int t_lo, int t_hi, uint8_t* out_dev,
             pipe_stream_t stream) {
    if (!p || !rgb_dev || !out_dev || t_lo < 0 || t_hi < t_lo || t_hi > 255) return PIPE_EINVAL;
    if (!valid_size(W, H) || pitch_bytes < (size_t)W * 3) return PIPE_EINVAL;
    const size_t N = (size_t)W * H;
    const uint8_t* rgb_end = rgb_dev + (size_t)(H - 1) * pitch_bytes + (size_t)W * 3;
    if (rgb_dev < out_dev + N && out_dev < rgb_end) return PIPE_EINVAL;  // the planes overlap
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(p->device));
    const int rtx = (W + RT - 1) / RT, rty = (H + RT - 1) / RT, n_rt = rtx * rty;
    if (p->rbc_mask.n < N || p->rbc_flags.n < sizeof(int) * (size_t)n_rt || p->rbc.wl.n < wl_bytes(n_rt) ||
        !p->rbc.shared.p) {
        CK(cudaStreamSynchronize(s));
        const bool fresh = !p->rbc.shared.p;
        int rc;
        if ((rc = p->rbc_mask.ensure(N)) || (rc = p->rbc_flags.ensure(sizeof(int) * (size_t)n_rt)) ||
            (rc = ensure_ctx(p->rbc, 1, n_rt, 0)))
            return rc;
        if (fresh) CK(cudaMemset(p->rbc.shared.p, 0, p->rbc.shared.n));
    }
    std::vector<TileDev> td(1);
    std::memset(&td[0], 0, sizeof(TileDev));
    td[0].W = W;
    td[0].H = H;
    td[0].R = out_dev;
    td[0].hem8 = (uint8_t*)p->rbc_mask.p;
    td[0].rtx = rtx;
    td[0].rty = rty;
    Launch L = make_launch(p, p->rbc, td, n_rt, 4);
    int* flags = (int*)p->rbc_flags.p;
    // 1. red dominance: the marker into out_dev, the mask into the pipe's
    //    plane, and the work tiles the marker touches
    CK(cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)n_rt, s));
    CK(cudaMemsetAsync(&L.sh->nseed, 0, sizeof(int), s));
    launch_rbc_planes(rgb_dev, pitch_bytes, W, H, t_lo, t_hi, out_dev, (uint8_t*)p->rbc_mask.p, flags, s, &p->prof);
    // 2. reconstruction by dilation of the marker under the mask, started from
    //    the flagged work tiles only
    int rc;
    if ((rc = upload_desc(L, td, s))) return rc;
    launch_recon_seeded(L, flags, p->recon_cap, s, &p->prof);
    CK(cudaGetLastError());
    return PIPE_OK;
}

namespace {

// Canny of n tiles: one NMS launch over all of them, one reconstruction
// queue for every tile's hysteresis (seeded from the work tiles that hold a
// strong pixel), one counts launch.  Arguments already checked.
int canny_run(pipe_t p, const edge_tile* tiles, int n, int low, int high, int radius, cudaStream_t s) {
    size_t cand_bytes = 0;
    int n_rt = 0;
    for (int i = 0; i < n; i++) {
        cand_bytes += al256((size_t)tiles[i].W * tiles[i].H);
        n_rt += ((tiles[i].W + RT - 1) / RT) * ((tiles[i].H + RT - 1) / RT);
    }
    const size_t desc_bytes = sizeof(CannyDesc) * (size_t)n, flag_bytes = sizeof(int) * (size_t)n_rt;
    if (p->canny_cand.n < cand_bytes || p->canny_flags.n < flag_bytes || p->canny_desc.n < desc_bytes ||
        p->canny.wl.n < wl_bytes(n_rt) || p->canny.tiles.n < tiles_bytes(n) || p->canny.shared.n < shared_bytes(n) ||
        !p->canny.shared.p) {
        CK(cudaStreamSynchronize(s));
        int rc;
        if ((rc = p->canny_cand.ensure(cand_bytes)) || (rc = p->canny_flags.ensure(flag_bytes)) ||
            (rc = p->canny_desc.ensure(desc_bytes)) || (rc = ensure_ctx(p->canny, n, n_rt, 0)))
            return rc;
        CK(cudaMemset(p->canny.shared.p, 0, p->canny.shared.n));
    }
    std::vector<CannyDesc> cd(n);
    std::vector<TileDev> td(n);
    char* cand = (char*)p->canny_cand.p;
    int blk = 0, nw = 0, rt = 0;
    for (int i = 0; i < n; i++) {
        const edge_tile& t = tiles[i];
        CannyDesc& c = cd[i];
        c.img = t.img;
        c.labels = t.labels;
        c.edges = t.edges;
        c.cand = (uint8_t*)cand;
        c.counts = t.counts;
        c.W = t.W;
        c.H = t.H;
        c.K = t.n_objects;
        c.bx = (t.W + 31) / 32;
        c.blk_base = blk;
        c.nms_base = nw;
        c.rt_base = rt;
        blk += canny_blocks(t.W, t.H);
        nw += canny_nms_warps(t.W, t.H);
        cand += al256((size_t)t.W * t.H);
        TileDev& d = td[i];
        std::memset(&d, 0, sizeof(TileDev));
        d.W = t.W;
        d.H = t.H;
        d.R = t.edges;
        d.hem8 = c.cand;
        d.rtx = (t.W + RT - 1) / RT;
        d.rty = (t.H + RT - 1) / RT;
        rt += d.rtx * d.rty;
    }
    CannyDesc* dcd = (CannyDesc*)p->canny_desc.p;
    int* flags = (int*)p->canny_flags.p;
    Launch L = make_launch(p, p->canny, td, n_rt, 4);  // rt_base in the same order as above
    upload_canny_descs(dcd, cd, s);
    CK(cudaMemsetAsync(flags, 0, flag_bytes, s));
    CK(cudaMemsetAsync(&L.sh->nseed, 0, sizeof(int), s));
    // 1. gradient and non-maximum suppression: strong pixels into the edge
    //    planes, candidates into the pipe's planes, counts zeroed, seed flags
    launch_canny_nms(cd, dcd, low, high, flags, s, &p->prof);
    // 2. hysteresis: reconstruction by dilation of the strong pixels under the candidates
    int rc;
    if ((rc = upload_desc(L, td, s))) return rc;
    launch_recon_seeded(L, flags, p->recon_cap, s, &p->prof);
    // 3. edge pixels within each object's disk dilation
    launch_canny_counts(cd, dcd, radius, s, &p->prof);
    CK(cudaGetLastError());
    return PIPE_OK;
}

bool canny_args_ok(const edge_tile& t) {
    if (!t.img || !t.edges || t.n_objects < 0 || !valid_size(t.W, t.H)) return false;
    if (t.n_objects > 0 && (!t.labels || !t.counts)) return false;
    const size_t N = (size_t)t.W * t.H;
    return !(t.img < t.edges + N && t.edges < t.img + N);  // the planes must not overlap
}

}  // namespace

int canny_tile(pipe_t p, const uint8_t* img_dev, const int32_t* labels_dev, int W, int H, int n_objects, int low,
               int high, int radius, uint8_t* edges_dev, int32_t* counts_dev, pipe_stream_t stream) {
    if (!p || low < 0 || high < low || radius < 0 || radius > 4) return PIPE_EINVAL;
    edge_tile t{img_dev, labels_dev, W, H, n_objects, edges_dev, counts_dev};
    if (!canny_args_ok(t)) return PIPE_EINVAL;
    CK(cudaSetDevice(p->device));
    return canny_run(p, &t, 1, low, high, radius, (cudaStream_t)stream);
}

int canny_batch(pipe_t p, const edge_tile* tiles, int n, int low, int high, int radius, pipe_stream_t stream) {
    if (!p || !tiles || n < 1 || n > 4096 || low < 0 || high < low || radius < 0 || radius > 4) return PIPE_EINVAL;
    for (int i = 0; i < n; i++)
        if (!canny_args_ok(tiles[i])) return PIPE_EINVAL;
    CK(cudaSetDevice(p->device));
    return canny_run(p, tiles, n, low, high, radius, (cudaStream_t)stream);
}

int seg_features_batch(pipe_t p, const tile_dev* tiles, int n, pipe_stream_t stream) {
    if (!p || !tiles || n < 1 || n > 4096) return PIPE_EINVAL;
    for (int i = 0; i < n; i++) {
        const tile_dev& d = tiles[i];
        if (!d.rgb || !d.hem8 || !d.labels || !d.n_objects || !valid_size(d.W, d.H) || d.pitch < (size_t)d.W * 3 ||
            d.feats_cap < 0 || (d.feats_cap > 0 && !d.feats))
            return PIPE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(p->device));
    int Wmax = 1;
    for (int i = 0; i < n; i++) Wmax = std::max(Wmax, tiles[i].W);
    std::vector<Geo> geos(n);
    std::vector<size_t> off(n);
    size_t total = 0;
    int n_rt = 0;
    std::string key;
    for (int i = 0; i < n; i++) {
        geos[i] = geometry(tiles[i].W, tiles[i].H, tiles[i].feats_cap);
        off[i] = total;
        total += geos[i].ws_bytes;
        n_rt += geos[i].rtx * geos[i].rty;
        key += std::to_string(tiles[i].W) + "x" + std::to_string(tiles[i].H) + "c" +
               std::to_string(tiles[i].feats_cap) + (tiles[i].edt ? "e" : "n") + ";";
    }
    bool grow = p->batch.arena.n < total || p->batch.wl.n < wl_bytes(n_rt) ||
                p->batch.tiles.n < sizeof(TileDev) * n || p->batch.shared.n < sizeof(Shared) + sizeof(int) * (2 + n);
    if (grow) {
        CK(cudaStreamSynchronize(s));
        clear_graphs(p->graphs);
        int rc = ensure_ctx(p->batch, n, n_rt, total);
        if (rc) return rc;
    }
    std::vector<TileDev> td(n);
    int max_obj = 1;
    for (int i = 0; i < n; i++) {
        TileDev& t = td[i];
        std::memset(&t, 0, sizeof(t));
        t.feats_cap = tiles[i].feats_cap;
        carve(t, geos[i], (char*)p->batch.arena.p + off[i]);
        t.pitch = tiles[i].pitch;
        t.rgb = tiles[i].rgb;
        t.hem8 = tiles[i].hem8;
        t.labels = tiles[i].labels;
        t.edt = tiles[i].edt;
        t.n_objects = tiles[i].n_objects;
        t.feats = tiles[i].feats;
        max_obj = std::max(max_obj, t.feats_cap);
    }
    p->batch_ntiles = n;
    int rc;
    Tune tu = default_tune(p, Wmax);
    {
        const std::string tk = tune_key(p, geos);
        auto it = p->tuned.find(tk);
        if (it != p->tuned.end() && tune_ok(p, it->second, Wmax)) {
            tu = it->second;
        } else if (p->prm.autotune) {
            if ((rc = autotune(p, p->batch, td, n_rt, Wmax, max_obj, s, &tu))) return rc;
            p->tuned[tk] = tu;
            save_tune(p, tk, tu);
        }
    }
    p->last_tune = tu;
    Launch L = make_launch(p, p->batch, td, n_rt, tu.edt_rb);
    if ((rc = upload_desc(L, td, s))) return rc;
    if (p->prof.enabled) {
        // profiled runs launch eagerly so that each kernel is bracketed by events
        run_path(p, L, Wmax, true, max_obj, tu, s, &p->prof);
    } else if ((rc = run_path_graph(p, p->graphs, key, L, Wmax, max_obj, tu, s, &p->prof.launches))) {
        return rc;
    }
    CK(cudaGetLastError());
    return PIPE_OK;
}

int pipe_status_read(pipe_t p) {
    if (!p) return PIPE_EINVAL;
    CK(cudaSetDevice(p->device));
    CK(cudaDeviceSynchronize());
    int result = PIPE_OK;
    auto check = [&](LaunchCtx& c, int ntiles) {
        if (!c.shared.p) return;
        Shared sh;
        if (cudaMemcpy(&sh, c.shared.p, sizeof(sh), cudaMemcpyDeviceToHost) != cudaSuccess) {
            result = PIPE_ECUDA;
            return;
        }
        if (sh.err && result == PIPE_OK) result = sh.err;
        std::vector<int> st(2 + ntiles);
        cudaMemcpy(st.data(), (char*)c.shared.p + sizeof(Shared), sizeof(int) * st.size(), cudaMemcpyDeviceToHost);
        for (int i = 2; i < (int)st.size(); i++)
            if (st[i] && result == PIPE_OK) result = st[i];
        int zero = 0;
        cudaMemcpy((char*)c.shared.p + offsetof(Shared, err), &zero, sizeof(int), cudaMemcpyHostToDevice);
        cudaMemset((char*)c.shared.p + sizeof(Shared), 0, sizeof(int) * st.size());
    };
    check(p->plain, 1);
    check(p->batch, p->batch_ntiles);
    check(p->canny, 1);
    check(p->rbc, 1);
    if (p->ws_status.p) {
        int st = 0;
        if (cudaMemcpy(&st, p->ws_status.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PIPE_ECUDA;
        if (st && result == PIPE_OK) result = st;
        cudaMemset(p->ws_status.p, 0, sizeof(int));
    }
    return result;
}

int pipe_debug_plane(pipe_t p, int which, void* dst_dev, pipe_stream_t stream) {
    if (!p || !dst_dev || !p->have_last || which < 0 || which > 2) return PIPE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const TileDev& t = p->last_plain;
    if (which == 0) {
        CK(cudaMemcpyAsync(dst_dev, t.R, (size_t)t.W * t.H, cudaMemcpyDeviceToDevice, s));
    } else {
        launch_unpack_bits(which == 1 ? t.fgbits : t.filledbits, t.W, t.H, t.cbx, (uint8_t*)dst_dev, s, &p->prof);
        CK(cudaGetLastError());
    }
    return PIPE_OK;
}

int pipe_profile_enable(pipe_t p, int enable) {
    if (!p) return PIPE_EINVAL;
    if (!enable && p->prof.enabled) p->prof.flush();
    p->prof.enabled = enable != 0;
    return PIPE_OK;
}

int pipe_profile_read(pipe_t p, const char** names, long long* launches, double* total_ms, int cap) {
    if (!p) return -1;
    cudaSetDevice(p->device);
    p->prof.flush();
    static thread_local std::vector<std::string> keep;
    keep.clear();
    int i = 0;
    for (auto& kv : p->prof.totals) {
        if (i < cap) {
            keep.push_back(kv.first);
            if (launches) launches[i] = kv.second.first;
            if (total_ms) total_ms[i] = kv.second.second;
        }
        i++;
    }
    for (int k = 0; k < (int)keep.size() && names; k++) names[k] = keep[k].c_str();
    p->prof.totals.clear();
    return i;
}

long long pipe_launch_count(pipe_t p) { return p ? p->prof.launches + p->serve_prof.launches : -1; }

int pipe_autotune_info(pipe_t p, int* recon_grid, int* edt_rows, int* feat_grid, long long* tune_runs) {
    if (!p) return PIPE_EINVAL;
    if (recon_grid) *recon_grid = p->last_tune.recon_grid;
    if (edt_rows) *edt_rows = p->last_tune.edt_rb;
    if (feat_grid) *feat_grid = p->last_tune.feat_grid;
    if (tune_runs) *tune_runs = p->tune_runs;
    return PIPE_OK;
}

long long pipe_recon_visits(pipe_t p) {
    if (!p || !p->plain.shared.p) return -1;
    if (cudaSetDevice(p->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return -1;
    Shared sh;
    if (cudaMemcpy(&sh, p->plain.shared.p, sizeof(sh), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return sh.processed;
}

int batch_submit(pipe_t p, const tile_desc* tiles, int n, uint64_t* ticket) {
    if (!p || !tiles || n < 1 || n > 1024 || !ticket) return PIPE_EINVAL;
    for (int i = 0; i < n; i++)
        if (!tiles[i].rgb_host || !valid_size(tiles[i].W, tiles[i].H) || tiles[i].pitch < (size_t)tiles[i].W * 3)
            return PIPE_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    CK(cudaSetDevice(p->device));
    const double t_submit = now_ms();
    // sizes of this group
    int Wmax = 1;
    for (int i = 0; i < n; i++) Wmax = std::max(Wmax, tiles[i].W);
    std::vector<Geo> geos(n);
    std::vector<int> caps(n);
    size_t ws = 0, io = 0, hin = 0, hout = 0;
    int n_rt = 0;
    std::vector<char> pinned(n);
    for (int i = 0; i < n; i++) {
        size_t N = (size_t)tiles[i].W * tiles[i].H;
        caps[i] = (int)std::min<size_t>(N / 20 + 1, 65536);
        geos[i] = geometry(tiles[i].W, tiles[i].H, caps[i]);
        ws += geos[i].ws_bytes;
        io += al256(3 * N) + al256(N) + 2 * al256(4 * N) + al256(16) + al256((size_t)caps[i] * NFEAT * 4);
        // pinned inputs are copied directly; pageable ones through a pinned staging buffer
        cudaPointerAttributes pa;
        pinned[i] = cudaPointerGetAttributes(&pa, tiles[i].rgb_host) == cudaSuccess && pa.type == cudaMemoryTypeHost;
        cudaGetLastError();
        if (!pinned[i]) hin += al256(3 * N);
        hout += al256(16) + al256((size_t)caps[i] * NFEAT * 4) +
                (tiles[i].want_planes ? al256(N) + 2 * al256(4 * N) : 0);
        n_rt += geos[i].rtx * geos[i].rty;
    }
    // admission: a free context (reused if large enough) within the HBM budget.
    // The budget counts the device memory of every context, busy or idle: an
    // idle context keeps its buffers for the next group, so growing one (or
    // starting a new one) first frees idle contexts when the total would
    // pass the budget.
    const size_t need = ctx_need(io, ws, n, n_rt);
    if (need > p->prm.hbm_budget_bytes) return PIPE_ENOMEM;  // never admissible as one group
    int ci = -1;
    for (int k = 0; k < (int)p->ctxs.size(); k++) {
        Ctx& c = *p->ctxs[k];
        if (!c.busy && ctx_fits(c, io, ws, n, n_rt) && c.h_in_n >= hin && c.h_out_n >= hout) {
            ci = k;
            break;
        }
    }
    const bool reuse = ci >= 0;
    if (!reuse) {
        for (int k = 0; k < (int)p->ctxs.size() && ci < 0; k++)
            if (!p->ctxs[k]->busy) ci = k;  // a free context to grow
        if (ci < 0 && (int)p->ctxs.size() >= p->prm.max_slots) return PIPE_EBUSY;
    }
    size_t g_io = io, g_ws = ws;
    int g_rt = n_rt, g_n = n;
    // A context that has to grow grows to the largest group seen so far (when
    // the budget allows), so that contexts converge to one size instead of
    // each growing -- a synchronising allocation -- as group sizes vary.
    p->peak_io = std::max(p->peak_io, io);
    p->peak_ws = std::max(p->peak_ws, ws);
    p->peak_rt = std::max(p->peak_rt, n_rt);
    p->peak_n = std::max(p->peak_n, n);
    if (!reuse) {
        const size_t cur = ci >= 0 ? p->ctxs[ci]->bytes : 0;
        const size_t others = serve_allocated(p) - cur;
        size_t idle_others = 0;
        for (int k = 0; k < (int)p->ctxs.size(); k++)
            if (k != ci && !p->ctxs[k]->busy) idle_others += p->ctxs[k]->bytes;
        auto after = [&](size_t a_io, size_t a_ws, int a_n, int a_rt) {
            return ci >= 0 ? ctx_bytes_after(*p->ctxs[ci], a_io, a_ws, a_n, a_rt) : ctx_need(a_io, a_ws, a_n, a_rt);
        };
        const size_t at_peak = after(p->peak_io, p->peak_ws, p->peak_n, p->peak_rt);
        const size_t at_need = after(io, ws, n, n_rt);
        const size_t budget = p->prm.hbm_budget_bytes;
        size_t target;
        if (others + at_peak <= budget) {
            target = at_peak;
            g_io = p->peak_io; g_ws = p->peak_ws; g_n = p->peak_n; g_rt = p->peak_rt;
        } else if (others + at_need <= budget) {
            target = at_need;
        } else if (others - idle_others + at_need <= budget) {
            target = at_need;  // fits once idle contexts give their memory back
        } else {
            return PIPE_EBUSY;
        }
        // free idle contexts, largest first, until the grown context fits
        while (serve_allocated(p) - cur + target > budget) {
            int big = -1;
            for (int k = 0; k < (int)p->ctxs.size(); k++)
                if (k != ci && !p->ctxs[k]->busy && p->ctxs[k]->bytes > 0 &&
                    (big < 0 || p->ctxs[k]->bytes > p->ctxs[big]->bytes))
                    big = k;
            if (big < 0) return PIPE_EBUSY;
            ctx_release_device(*p->ctxs[big]);
        }
        if (ci < 0) {
            p->ctxs.emplace_back(new Ctx());
            ci = (int)p->ctxs.size() - 1;
            Ctx& c = *p->ctxs[ci];
            CK(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&c.uploaded, cudaEventDisableTiming));
            CK(cudaEventCreate(&c.done));  // timed: its GPU timestamp gives the completion time
        }
    }
    Ctx& c = *p->ctxs[ci];
    int rc;
    if (!ctx_fits(c, io, ws, n, n_rt)) {
        clear_graphs(c.graphs);
        rc = c.dev.ensure(g_io);
        if (!rc) rc = ensure_ctx(c.lc, g_n, g_rt, g_ws);
        c.bytes = ctx_bytes(c);
        if (rc) return rc;
    }
    c.bytes = ctx_bytes(c);
    if (c.h_in_n < hin) {
        if (c.h_in) cudaFreeHost(c.h_in);
        c.h_in = nullptr;
        c.h_in_n = 0;
        CK(cudaHostAlloc(&c.h_in, hin, cudaHostAllocDefault));
        c.h_in_n = hin;
    }
    if (c.h_out_n < hout) {
        if (c.h_out) cudaFreeHost(c.h_out);
        c.h_out = nullptr;
        c.h_out_n = 0;
        CK(cudaHostAlloc(&c.h_out, hout, cudaHostAllocMapped));
        c.h_out_n = hout;
    }
    // carve device buffers and fill descriptors
    std::unique_ptr<Ticket> tk(new Ticket());
    tk->ctx = ci;
    tk->t_submit = t_submit;
    std::vector<TileDev> td(n);
    char* d = (char*)c.dev.p;
    char* hi = (char*)c.h_in;
    size_t wsoff = 0, hoff = 0;
    for (int i = 0; i < n; i++) {
        const tile_desc& t = tiles[i];
        size_t N = (size_t)t.W * t.H;
        TileDev& x = td[i];
        std::memset(&x, 0, sizeof(x));
        x.feats_cap = caps[i];
        carve(x, geos[i], (char*)c.lc.arena.p + wsoff);
        wsoff += geos[i].ws_bytes;
        uint8_t* rgb = (uint8_t*)d; d += al256(3 * N);
        x.hem8 = (uint8_t*)d; d += al256(N);
        x.labels = (int32_t*)d; d += al256(4 * N);
        x.edt = (int32_t*)d; d += al256(4 * N);
        x.n_objects = (int32_t*)d; d += al256(16);
        x.feats = (float*)d; d += al256((size_t)caps[i] * NFEAT * 4);
        x.rgb = rgb;
        x.pitch = (size_t)t.W * 3;
        // upload: pinned source directly, pageable through the staging buffer
        const void* src = t.rgb_host;
        size_t spitch = t.pitch;
        if (!pinned[i]) {
            for (int y = 0; y < t.H; y++) std::memcpy(hi + (size_t)y * t.W * 3, t.rgb_host + (size_t)y * t.pitch, (size_t)t.W * 3);
            src = hi;
            spitch = (size_t)t.W * 3;
            hi += al256(3 * N);
        }
        if (spitch == (size_t)t.W * 3)  // dense rows: one contiguous copy, not H row copies
            CK(cudaMemcpyAsync(rgb, src, (size_t)t.W * 3 * t.H, cudaMemcpyHostToDevice, c.stream));
        else
            CK(cudaMemcpy2DAsync(rgb, (size_t)t.W * 3, src, spitch, (size_t)t.W * 3, t.H, cudaMemcpyHostToDevice,
                                 c.stream));
        TicketTile tt{t.W, t.H, t.want_planes, caps[i], 0, 0, 0};
        tt.nobj_off = hoff; hoff += al256(16);
        tt.out_off = hoff; hoff += al256((size_t)caps[i] * NFEAT * 4);
        if (t.want_planes) hoff += al256(N) + 2 * al256(4 * N);
        tk->tiles.push_back(tt);
    }
    // three phases (Sec. IV-D): this group's upload runs on the context's copy
    // stream, overlapping the compute of groups submitted before it; compute and
    // download run on the shared compute stream, in submission order
    if (!p->serve_compute) {
        CK(cudaStreamCreateWithFlags(&p->serve_compute, cudaStreamNonBlocking));
        // reference point mapping GPU event time to the host clock
        CK(cudaEventCreate(&p->serve_ref));
        CK(cudaEventRecord(p->serve_ref, p->serve_compute));
        CK(cudaEventSynchronize(p->serve_ref));
        p->serve_ref_ms = now_ms();
    }
    CK(cudaEventRecord(c.uploaded, c.stream));
    cudaStream_t cs = p->serve_compute;
    CK(cudaStreamWaitEvent(cs, c.uploaded, 0));
    // launch shapes: those tuned for this shape by the batched form, if any
    // (the served form never blocks to tune)
    Tune tu = default_tune(p, Wmax);
    {
        auto it = p->tuned.find(tune_key(p, geos));
        if (it != p->tuned.end() && tune_ok(p, it->second, Wmax)) tu = it->second;
    }
    Launch L = make_launch(p, c.lc, td, n_rt, tu.edt_rb);
    if ((rc = upload_desc(L, td, cs))) return rc;
    {
        std::string key;
        for (int i = 0; i < n; i++)
            key += std::to_string(tiles[i].W) + "x" + std::to_string(tiles[i].H) + (tiles[i].want_planes ? "p;" : ";");
        rc = run_path_graph(p, c.graphs, key, L, Wmax, *std::max_element(caps.begin(), caps.end()), tu, cs,
                            &p->serve_prof.launches);
        if (rc) return rc;
    }
    // download: a kernel writes count, status and exactly min(K, cap) feature
    // rows of every tile into the mapped pinned result buffer; planes by copy
    char* ho = (char*)c.h_out;
    char* ho_dev = nullptr;
    CK(cudaHostGetDevicePointer((void**)&ho_dev, c.h_out, 0));
    {
        std::vector<ResultSlot> rs(n);
        for (int i = 0; i < n; i++) {
            rs[i].head = (int32_t*)(ho_dev + tk->tiles[i].nobj_off);
            rs[i].feats = (float*)(ho_dev + tk->tiles[i].out_off);
        }
        if ((rc = launch_results(L, rs.data(), n, cs, &p->serve_prof))) return rc;
    }
    for (int i = 0; i < n; i++) {
        const TicketTile& tt = tk->tiles[i];
        size_t N = (size_t)tt.W * tt.H;
        if (tt.want) {
            char* q = ho + tt.out_off + al256((size_t)caps[i] * NFEAT * 4);
            CK(cudaMemcpyAsync(q, td[i].hem8, N, cudaMemcpyDeviceToHost, cs));
            CK(cudaMemcpyAsync(q + al256(N), td[i].labels, 4 * N, cudaMemcpyDeviceToHost, cs));
            CK(cudaMemcpyAsync(q + al256(N) + al256(4 * N), td[i].edt, 4 * N, cudaMemcpyDeviceToHost, cs));
        }
    }
    CK(cudaEventRecord(c.done, cs));
    // No device-side wait orders this context's next upload after this group:
    // a context takes new work only after batch_poll has seen its done event
    // complete, so nothing of this group still reads the context's buffers.
    CK(cudaGetLastError());
    c.busy = true;
    p->prof.launches += 0;
    uint64_t id = p->next_ticket++;
    p->tickets[id] = std::move(tk);
    *ticket = id;
    return PIPE_OK;
}

int batch_poll(pipe_t p, uint64_t ticket, int* n_done, tile_result* out) {
    if (!p || !n_done) return PIPE_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    auto it = p->tickets.find(ticket);
    if (it == p->tickets.end()) return PIPE_EINVAL;
    Ticket& tk = *it->second;
    const int n = (int)tk.tiles.size();
    if (!tk.done) {
        Ctx& c = *p->ctxs[tk.ctx];
        cudaError_t q = cudaEventQuery(c.done);
        if (q == cudaErrorNotReady) {
            *n_done = 0;
            return PIPE_EAGAIN;
        }
        if (q != cudaSuccess) return PIPE_ECUDA;
        // copy results out of the context so that it can take new work
        const char* ho = (const char*)c.h_out;
        tk.feats.resize(n);
        tk.hem8.resize(n);
        tk.labels.resize(n);
        tk.edt.resize(n);
        std::vector<int> st(n), K(n);
        for (int i = 0; i < n; i++) {
            const TicketTile& tt = tk.tiles[i];
            int vals[3];
            std::memcpy(vals, ho + tt.nobj_off, sizeof(vals));
            K[i] = vals[0];
            st[i] = vals[1] ? vals[1] : vals[2];
            const int rows = std::max(0, std::min(K[i], tt.cap));
            const float* f = (const float*)(ho + tt.out_off);
            tk.feats[i].assign(f, f + (size_t)rows * NFEAT);
            if (tt.want) {
                size_t N = (size_t)tt.W * tt.H;
                const char* q = ho + tt.out_off + al256((size_t)tt.cap * NFEAT * 4);
                tk.hem8[i].assign((const uint8_t*)q, (const uint8_t*)q + N);
                tk.labels[i].assign((const int32_t*)(q + al256(N)), (const int32_t*)(q + al256(N)) + N);
                tk.edt[i].assign((const int32_t*)(q + al256(N) + al256(4 * N)), (const int32_t*)(q + al256(N) + al256(4 * N)) + N);
            }
            tk.tiles[i].st_off = (size_t)st[i];
            tk.tiles[i].nobj_off = (size_t)K[i];  // reuse the fields for the host copies
        }
        tk.done = true;
        float el = 0.f;
        double td = now_ms();
        if (cudaEventElapsedTime(&el, p->serve_ref, c.done) == cudaSuccess) td = p->serve_ref_ms + el;
        c.busy = false;
        for (int i = 0; i < n; i++) tk.tiles[i].out_off = 0;
        tk.t_submit = tk.t_submit;
        tk.ctx = -1;
        tk.feats.shrink_to_fit();
        // completion time of the whole group
        tk.tiles.shrink_to_fit();
        tk.done = true;
        tk.t_done_ms = td;
    }
    if (out) {
        for (int i = 0; i < n; i++) {
            tile_result& r = out[i];
            r.status = (int)tk.tiles[i].st_off;
            r.n_objects = (int)tk.tiles[i].nobj_off;
            r.n_feats = (int)(tk.feats[i].size() / NFEAT);
            if (r.status == PIPE_OK && r.n_objects > r.n_feats) r.status = PIPE_EOVERFLOW;
            r.feats = tk.feats[i].empty() ? nullptr : tk.feats[i].data();
            r.hem8 = tk.hem8[i].empty() ? nullptr : tk.hem8[i].data();
            r.labels = tk.labels[i].empty() ? nullptr : tk.labels[i].data();
            r.edt = tk.edt[i].empty() ? nullptr : tk.edt[i].data();
            r.t_arrive_ms = tk.t_submit;
            r.t_done_ms = tk.t_done_ms;
        }
    }
    *n_done = n;
    return PIPE_OK;
}

int batch_release(pipe_t p, uint64_t ticket) {
    if (!p) return PIPE_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    auto it = p->tickets.find(ticket);
    if (it == p->tickets.end()) return PIPE_EINVAL;
    if (!it->second->done) return PIPE_EAGAIN;  // its group still uses a context
    p->tickets.erase(it);
    return PIPE_OK;
}

int pipe_serve_memory(pipe_t p, size_t* allocated, size_t* in_flight, int* contexts) {
    if (!p) return PIPE_EINVAL;
    std::lock_guard<std::mutex> lk(p->mu);
    size_t a = 0, f = 0;
    for (auto& c : p->ctxs) {
        a += c->bytes;
        if (c->busy) f += c->bytes;
    }
    if (allocated) *allocated = a;
    if (in_flight) *in_flight = f;
    if (contexts) *contexts = (int)p->ctxs.size();
    return PIPE_OK;
}

}  // extern "C"
