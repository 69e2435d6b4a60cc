// Internal declarations shared by the CUDA translation units of libpipe.
// Nothing here is part of the C ABI (include/pipe.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <vector>

namespace nucseg {

// ---- geometry ---------------------------------------------------------------
constexpr int RT = 64;            // reconstruction work tile: RT x RT pixels, one warp
constexpr int RECON_MIN_BLOCKS = 16;  // resident reconstruction workers (one-warp CTAs) per SM the register budget must allow
constexpr int CB = 32;            // labelling block: CB x CB pixels (one bitmap word per row)
constexpr int CB_THREADS = 256;
constexpr int CCL_WARPS = 4;      // labelling blocks (one per warp) per CTA
constexpr int RL_CAP = 512;       // root-list slots per labelling block
constexpr int NFEAT = 15;
constexpr int MORPH_RMAX = 15;   // largest disk radius of the opening (chords of up to 31 pixels)

// worklist tile states
constexpr int WL_IDLE = 0, WL_QUEUED = 1, WL_RUNNING = 2, WL_DIRTY = 3;

// device status codes (same values as pipe_status)
constexpr int ST_OK = 0, ST_TIMEOUT = 5, ST_OVERFLOW = 6;

// One image of a launch: pointers into caller buffers and the pipe's arena.
struct TileDev {
    int W, H;
    size_t pitch;                 // RGB row pitch in bytes
    const uint8_t* rgb;
    uint8_t* hem8;                // H*W
    uint8_t* R;                   // H*W reconstruction (workspace)
    int32_t* labels;              // H*W
    int32_t* edt;                 // H*W (may be null: EDT skipped)
    int32_t* n_objects;           // [1]
    float* feats;                 // [feats_cap][15] (batched form)
    int feats_cap;
    uint32_t* fgbits;             // bitmaps, block-major: CB words (rows) per labelling block
    uint32_t* filledbits;
    uint32_t* rootbits;           // kept component roots, row-major: H rows of wpr words
    int32_t* wordprefix;          // exclusive popcount prefix of rootbits words
    int32_t* chunksum;            // per scan chunk
    int32_t* P;                   // union-find parents (sparse, H*W)
    int32_t* A;                   // per-root payload (sparse, H*W)
    int32_t* border;              // per labelling block: 4*CB local roots
    int32_t* rootlist;            // local roots, RL_CAP per labelling block
    int32_t* blkroots;            // local roots recorded per labelling block
    int4* bbox;                   // per object: xmin, ymin, xmax, ymax
    uint32_t* colbits;            // per 32-row chunk and column: kept bits of the 32 rows
    int wpr;                      // bitmap words per row = ceil(W/32)
    int rtx, rty, rt_base;        // reconstruction tiles and global base id
    int cbx, cby, cb_base;        // labelling blocks and global base id
    int nchunks, chunk_base;      // scan chunks (of SCAN_CHUNK words)
    int col_base;                 // EDT column strips base
    int row_base;                 // EDT rows base
    int px_base;                  // deconvolution work items base
    int obj_base;                 // first object item of this tile (batched features)
    int cls[8], cls_pos[8];       // reconstruction queue order: work tiles per class, and placed so far
};

constexpr int SCAN_THREADS = 1024;           // threads of a scan CTA, four bitmap words each
constexpr int SCAN_CHUNK = 4 * SCAN_THREADS;  // bitmap words per scan chunk
constexpr int LAUNCH_TAB = 64;    // tiles whose block bases travel in the launch parameters

// Shared state of one launch sequence (device memory).
struct Shared {
    unsigned long long tp;              // reconstruction worklist: tail << 32 | pending
    int head, err;                      // worklist head; first device-side error
    int processed;                      // tile processings (diagnostic)
    int nobj;                           // object items of a batched feature pass
    int next_obj;                       // the batched feature pass draws its objects from this counter
    int nseed;                          // work tiles of a seeded reconstruction queued at the start
};

struct Launch {
    TileDev* tiles;        // device array [ntiles]
    int ntiles;
    unsigned long long* wl_slots;  // [n_rt] queue ring: sequence << 32 | item
    int* wl_state;         // [n_rt] per-tile state
    int* rt_src;           // [n_rt] work tiles holding a strong marker (queued first)
    Shared* sh;
    int* tile_status;      // [ntiles]
    int* status;           // global status word
    // totals (host-computed) for grid sizing
    int n_rt, n_cb, n_chunks, n_cols, n_rows, n_px;
    long long wait_budget;
    int h, thr, amin, amax;
    // first labelling block of each of the first LAUNCH_TAB tiles (kernel
    // parameters live in the constant bank, so a search over them is cheap)
    int cb_first[LAUNCH_TAB];
};

// ---- small device helpers ----------------------------------------------------
__device__ __forceinline__ int find_tile(const TileDev* t, int n, int gid, int TileDev::*base) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (t[mid].*base <= gid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void set_status(int* status, int code) {
    atomicCAS(status, 0, code);
}

// Object boxes from one row segment of FB_SEG labels, one warp: each lane
// reads 4 labels at a time; the lanes holding the same label (one
// __match_any_sync group per label value) combine their column range and
// one lane updates the box with atomics.  Labels outside 1..K are ignored.
constexpr int FB_STEPS = 8;
constexpr int FB_SEG = 32 * 4 * FB_STEPS;
__device__ __forceinline__ void bbox_segment(const int32_t* __restrict__ row, int W, int K, int y, int xs,
                                             int4* bbox, int lane) {
    const unsigned full = 0xffffffffu;
    const bool vec = (W & 3) == 0;
    for (int step = 0; step < FB_STEPS; step++) {
        const int x0 = xs + (step * 32 + lane) * 4;
        int v[4] = {0, 0, 0, 0};
        if (vec && x0 + 3 < W) {
            int4 q = __ldcs(reinterpret_cast<const int4*>(row + x0));
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
            for (int k = 0; k < 4; k++) v[k] = x0 + k < W ? __ldcs(row + x0 + k) : 0;
        }
        if (__ballot_sync(full, (v[0] | v[1] | v[2] | v[3]) != 0) == 0) continue;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            int lab = (v[k] >= 1 && v[k] <= K) ? v[k] : 0;
            // the other pixels of this lane with the same label join this update
            int mn = 0x7fffffff, mx = -1;
            if (lab) {
                for (int j = k; j < 4; j++)
                    if (v[j] == lab) { mn = min(mn, x0 + j); mx = max(mx, x0 + j); v[j] = 0; }
            }
            unsigned grp = __match_any_sync(full, lab);
            if (lab) {
                int gmn = __reduce_min_sync(grp, (unsigned)mn), gmx = __reduce_max_sync(grp, (unsigned)mx);
                if (lane == __ffs(grp) - 1) {
                    int4* b = bbox + (lab - 1);
                    atomicMin(&b->x, gmn);
                    atomicMax(&b->z, gmx);
                    atomicMin(&b->y, y);
                    atomicMax(&b->w, y);
                }
            }
        }
    }
}

// ---- launchers (one per translation unit) -----------------------------------
// Profiler hook: every kernel launch is bracketed by begin/end with its name;
// the pipe counts launches and, when enabled, records CUDA events.
struct Profiler {
    virtual void begin(const char* name, cudaStream_t s) = 0;
    virtual void end(const char* name, cudaStream_t s) = 0;
    virtual ~Profiler() {}
};

void upload_deconv_tables(const int32_t* lut256, const int32_t* wq3);
void launch_deconv(const Launch& L, cudaStream_t s, Profiler* pf);
int recon_grid(int device);
void launch_recon(const Launch& L, int grid_cap, cudaStream_t s, Profiler* pf);
// The reconstruction started from a sparse marker: only the work tiles whose
// flag is set (a marker pixel in the tile or its one-pixel halo) are queued
// at the start; the others are at a fixed point and wait to be requested.
// flags: one int per work tile of the launch, set by the kernel that wrote the
// marker and zeroed by the caller before it; L.sh->nseed must be zeroed too.
void launch_recon_seeded(const Launch& L, const int* flags, int grid_cap, cudaStream_t s, Profiler* pf);

// Sets the seed flags of a 16-pixel chunk at (x0, y) of an image with rtx x
// rty work tiles (x0 a multiple of 16, so the chunk lies in one work tile):
// the tile holding it, and the neighbours whose one-pixel halo holds one of
// its marker pixels (bit p of m: pixel x0 + p is a marker pixel).
// The work tiles (RT x RT, rtx x rty of them) whose tile or one-pixel halo
// holds pixel (x, y), as bits of a 3 x 3 neighbourhood: bit (dy + 1) * 3 +
// (dx + 1) for the tile at offset (dx, dy) from the pixel's own.
__device__ __forceinline__ unsigned seed_bits_px(int rtx, int rty, int x, int y) {
    const int tx = x / RT, ty = y / RT, xr = x - tx * RT, yr = y - ty * RT;
    const int dxl = (xr == 0 && tx > 0) ? -1 : 0, dxh = (xr == RT - 1 && tx + 1 < rtx) ? 1 : 0;
    const int dyl = (yr == 0 && ty > 0) ? -1 : 0, dyh = (yr == RT - 1 && ty + 1 < rty) ? 1 : 0;
    unsigned m = 0;
    for (int dy = dyl; dy <= dyh; dy++)
        for (int dx = dxl; dx <= dxh; dx++) m |= 1u << ((dy + 1) * 3 + dx + 1);
    return m;
}

__device__ __forceinline__ void flag_seed_tiles(int* flags, int rtx, int rty, int x0, int y, unsigned m) {
    if (!m) return;
    const int tx = x0 / RT, ty = y / RT, yr = y - ty * RT;
    const int ylo = (yr == 0 && ty > 0) ? ty - 1 : ty, yhi = (yr == RT - 1 && ty + 1 < rty) ? ty + 1 : ty;
    const int xlo = ((x0 & (RT - 1)) == 0 && (m & 1u) && tx > 0) ? tx - 1 : tx;
    const int xhi = (((x0 + 15) & (RT - 1)) == RT - 1 && (m & 0x8000u) && tx + 1 < rtx) ? tx + 1 : tx;
    for (int yy = ylo; yy <= yhi; yy++)
        for (int xx = xlo; xx <= xhi; xx++) flags[yy * rtx + xx] = 1;
}
void launch_label(const Launch& L, int want_bbox, int max_objects, int sms, cudaStream_t s, Profiler* pf);
size_t edt_rows_smem(int RB, int Wmax);
void launch_edt(const Launch& L, int RB, int Wmax, cudaStream_t s, Profiler* pf);
size_t morph_open_smem(int r);
// tmp: a W x H scratch plane (the radius-9 form runs two passes through it); may be null
void launch_morph_open(const uint8_t* src, uint8_t* dst, uint8_t* tmp, int W, int H, int r, cudaStream_t s,
                       Profiler* pf);
void launch_features_plain(const uint8_t* hem8, const int32_t* labels, int W, int H, int K, float* feats,
                           int4* bbox, int sms, cudaStream_t s, Profiler* pf);
void launch_features_batched(const Launch& L, int grid, cudaStream_t s, Profiler* pf);
// per object 1..K of a label plane: its box (xmin, ymin, xmax, ymax); empty (xmax < xmin) if absent
void launch_object_boxes(const int32_t* labels, int W, int H, int K, int4* bbox, cudaStream_t s, Profiler* pf);
// One tile of a Canny launch (plain: one tile; batched: many).
struct CannyDesc {
    const uint8_t* img;      // W x H plane
    const int32_t* labels;   // W x H labels (may be null when K == 0)
    uint8_t* edges;          // strong pixels (0/1), grown into the edge map by the hysteresis
    uint8_t* cand;           // candidates (0/1): the hysteresis mask
    int32_t* counts;         // K edge counts
    int W, H, K;
    int bx;                  // 32-pixel blocks per row
    int blk_base;            // first 32x32 block of this tile in the counts launch
    int nms_base;            // first warp of this tile in the suppression launch
    int rt_base;             // first work tile of this tile in the reconstruction launch
};
// Blocks of a tile in the Canny launches (32 x 32 pixels each).
int canny_blocks(int W, int H);
int canny_nms_warps(int W, int H);
void upload_canny_descs(CannyDesc* dst, const std::vector<CannyDesc>& v, cudaStream_t s);
// descs: host copy; d_descs: device array of the same length.  Zeroes the
// counts, writes strong pixels into edges and candidates into cand, and sets
// the seed flags (indexed by rt_base + work tile) of the work tiles the
// strong pixels touch.
void launch_canny_nms(const std::vector<CannyDesc>& descs, CannyDesc* d_descs, int low, int high, int* flags,
                      cudaStream_t s, Profiler* pf);
// Edge counts of every tile: each edge pixel adds one to every object 1..K
// with a pixel within its disk of radius r (the disk dilation of the object).
void launch_canny_counts(const std::vector<CannyDesc>& descs, CannyDesc* d_descs, int r, cudaStream_t s,
                         Profiler* pf);
// One tile of a batched watershed split.
struct WsDesc {
    const int32_t* labels;
    const int32_t* edt;
    int32_t* out;
    int32_t* n_basins;
    long long px_base;    // first pixel of this tile in the scratch planes
    int W, H, K;
    int obj_base;         // first object item of this tile
    int seg_base;         // first box row segment of this tile
};
// descs: host copy; d_descs: device array of the same length
void launch_watershed_batch(const std::vector<WsDesc>& descs, WsDesc* d_descs, int h, int4* bbox, int* cnt,
                            int* next, void* scratch, size_t scratch_px, int* status, int sms, cudaStream_t s,
                            cudaStream_t side, cudaEvent_t fork, cudaEvent_t join, Profiler* pf);
// scratch of the watershed's out-of-stage boxes: a 64-bit and a 16-bit word per pixel
size_t watershed_scratch_bytes(int W, int H);
// cnt: K ints (per-object basin counts, then their exclusive prefix); next: 3 + K device ints (the
// large-box draw counter, the large-box list length and the small-box draw counter, zeroed by the
// launcher, then the large-box list); status: a device int
// side: a second stream for the large boxes (fork/join through the two events)
void launch_watershed(const int32_t* labels, const int32_t* edt, int W, int H, int K, int h, int32_t* out,
                      int32_t* n_basins, int4* bbox, int* cnt, int* next, void* scratch, int* status, int sms,
                      cudaStream_t s, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join, Profiler* pf);
// RBC detection planes: d = R - max(G, B); marker (0/1) = d >= t_hi into
// marker, mask (0/1) = d >= t_lo into mask, and the seed flags of the work
// tiles (RT x RT) that the marker pixels touch.
void launch_rbc_planes(const uint8_t* rgb, size_t pitch, int W, int H, int t_lo, int t_hi, uint8_t* marker,
                       uint8_t* mask, int* flags, cudaStream_t s, Profiler* pf);
void launch_unpack_bits(const uint32_t* bits, int W, int H, int cbx, uint8_t* out, cudaStream_t s,
                        Profiler* pf);

}  // namespace nucseg
