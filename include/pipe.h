/*
 * pipe.h -- C ABI of the GB300 per-tile nucleus segmentation + feature path.
 *
 * Paper: G. Teodoro, T. Pan, T. Kurc, J. Kong, L. Cooper, J. Saltz,
 * "High-throughput Execution of Hierarchical Analysis Pipelines on Hybrid
 * Cluster Platforms".  The input of the pipeline is an image tile and its
 * output is a feature vector per segmented nucleus (Sec. II, caption of
 * Fig. 1); tiles are processed independently as a bag of tasks (Sec. II);
 * the operations are those of Table I (ReconToNuclei, FillHoles, BWLabel,
 * AreaThreshold, the distance transform of Pre-Watershed) and the
 * feature-stage transforms of Sec. V-A (colour deconvolution, gradient).
 *
 * Conventions for every entry point:
 *  - Returns a pipe_status; no entry point aborts, traps or prints.
 *  - Device pointers are caller-owned, must be on the pipe's device and
 *    must stay valid until the work enqueued on `stream` has finished.
 *  - Calls taking a stream are asynchronous on that stream.  Device-side
 *    failures (a wait budget exhausted, a capacity exceeded) are written to
 *    a status word in device memory; pipe_status_read() returns it.
 *  - Image planes are row-major with a row pitch of W elements unless a
 *    pitch argument says otherwise.
 *  - A pipe_t may be used from one host thread at a time, except
 *    batch_submit / batch_poll, which are safe to call concurrently.
 *  - The stream-taking calls of one pipe share its scratch buffers: calls
 *    on different streams must not overlap on the GPU (order the streams
 *    with events, or use one stream per pipe).
 */
#ifndef GB300_NUCSEG_PIPE_H
#define GB300_NUCSEG_PIPE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pipe_s* pipe_t;
typedef struct CUstream_st* pipe_stream_t; /* a cudaStream_t; NULL = legacy default */

typedef enum {
    PIPE_OK = 0,
    PIPE_EINVAL = 1,     /* bad argument (size, pointer, parameter) */
    PIPE_ENOMEM = 2,     /* device or pinned-host allocation failed */
    PIPE_EBUSY = 3,      /* admission refused: HBM budget or slots exhausted */
    PIPE_EAGAIN = 4,     /* ticket not finished yet */
    PIPE_ETIMEOUT = 5,   /* a device-side wait hit its cycle budget */
    PIPE_EOVERFLOW = 6,  /* a caller-sized output was too small */
    PIPE_ECUDA = 7       /* a CUDA runtime call failed */
} pipe_status;

#define PIPE_NFEAT 15

/* Parameters.  Defaults (pipe_default_params): h = 20, dome_thresh = 10,
 * area [20, 1500], 8 GLCM levels, offsets (dx,dy) = (1,0),(0,1),(1,1),(1,-1),
 * hbm_budget_bytes = 40 GiB, max_slots = 16, wait_budget_cycles = 2^32,
 * autotune_cache = NULL, autotune = 1. */
typedef struct {
    int h;               /* h-dome height (ReconToNuclei, Table I) */
    int dome_thresh;     /* foreground iff hem8 - R >= dome_thresh */
    int area_min;        /* AreaThreshold (Table I): keep areas in [min, max] */
    int area_max;
    int glcm_levels;     /* must be 8 (hem8 >> 5) */
    int n_offsets;       /* must be 4 */
    int offsets[4][2];   /* (dx, dy); must be the four defaults */
    size_t hbm_budget_bytes;  /* device memory the served form may hold */
    int max_slots;            /* tiles in flight in the served form */
    long long wait_budget_cycles; /* bound on every device-side spin wait */
    const char* autotune_cache;   /* path of the launch-shape cache file, or NULL */
    int autotune;                 /* 1: tune the launch shapes of new batch shapes */
} pipe_params;

void pipe_default_params(pipe_params* p);

/* Creates a pipe on CUDA device `device`.  The pipe owns all workspaces;
 * it grows them on demand (a synchronising allocation) when a larger tile
 * than any seen before arrives. */
int pipe_create(const pipe_params* params, int device, pipe_t* out);

/* Drains all outstanding work and frees everything the pipe owns. */
void pipe_destroy(pipe_t p);

/* Segmentation of one RGB tile (Sec. II segmentation stage; Table I):
 *   hem8   = colour deconvolution, hematoxylin plane, uint8 (Sec. V-A)
 *   R      = reconstruction by dilation of max(hem8-h,0) under hem8, 8-conn
 *   fg     = hem8 - R >= dome_thresh                      (ReconToNuclei)
 *   filled = fg with background holes not 4-connected to the border filled
 *   labels = 8-connected components of filled with area in [area_min,
 *            area_max], numbered 1..K by first pixel in row-major order,
 *            0 elsewhere                                  (BWLabel, AreaThreshold)
 *   edt    = exact squared Euclidean distance to the nearest label-0 pixel,
 *            INT32_MAX everywhere if there is none        (Pre-Watershed)
 * rgb_dev: H rows of 3*W bytes (R,G,B) at pitch_bytes >= 3*W.
 * hem8_dev [H*W] uint8, labels_dev [H*W] int32, edt_dev [H*W] int32 (may be
 * NULL to skip the EDT), n_objects_dev [1] int32 receives K.
 * Errors: PIPE_EINVAL for W,H < 1, W*H >= 2^31 or NULL required pointers. */
int seg_tile(pipe_t p, const uint8_t* rgb_dev, int W, int H, size_t pitch_bytes,
             uint8_t* hem8_dev, int32_t* labels_dev, int32_t* edt_dev, int32_t* n_objects_dev,
             pipe_stream_t stream);

/* Per-object features (Sec. II feature families; Sec. V-A gradient) of
 * labels 1..n_objects, written as float32 rows feats_dev[n_objects][15]:
 *  0 area, 1 perimeter (4-neighbour crack count, image outside counts),
 *  2 mean, 3 population std, 4 min, 5 max of hem8,
 *  6 mean, 7 population std, 8 min, 9 max of the Sobel magnitude of hem8
 *    (replicated border),
 *  10 contrast, 11 energy, 12 homogeneity, 13 entropy, 14 correlation of the
 *    8-level (hem8 >> 5) co-occurrence matrix of same-object pixel pairs,
 *    averaged over the offsets that have pairs (0 if none; correlation 0
 *    when a marginal is constant).
 * n_objects may be 0 (nothing is launched).  Errors: PIPE_EINVAL. */
int features_tile(pipe_t p, const uint8_t* hem8_dev, const int32_t* labels_dev, int W, int H,
                  int n_objects, float* feats_dev, pipe_stream_t stream);

/* features_tile without a pipe and without any device allocation.  The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code that runs under a framework's own caching allocator
 * (where a raw allocation would bypass its accounting or fail because the
 * pool already holds the memory), or a serving loop that must not take the
 * implicit device synchronisation an allocation can cause.  Inputs, outputs
 * and results are exactly those of features_tile.  Its only scratch, one
 * box per object, is a static device array of PIPE_NOALLOC_MAX_OBJECTS
 * entries (1 MiB) that every GPU loading this library holds until exit.
 *  - Uses the current CUDA device.  The first call on a device looks up the
 *    array's device address (cudaGetSymbolAddress); make that first call
 *    before any stream capture.  The address is kept for the life of the
 *    process: after a cudaDeviceReset of that device it is stale, so the
 *    entry point must not be called on a device this process has reset.
 *  - n_objects > PIPE_NOALLOC_MAX_OBJECTS: PIPE_EINVAL, nothing launched.
 *  - All calls share the one array (each call first resets the entries it
 *    uses): calls that overlap on the GPU -- on different streams, or from
 *    different threads -- race and must be serialised by the caller. */
#define PIPE_NOALLOC_MAX_OBJECTS 65536
int features_tile_noalloc(const uint8_t* hem8_dev, const int32_t* labels_dev, int W, int H,
                          int n_objects, float* feats_dev, pipe_stream_t stream);

/* Batched form, device-resident: segmentation + features of n tiles of any
 * sizes, one launch per pass over all tiles (the reconstruction pass is one
 * persistent launch with a work queue spanning every tile), replayed from a
 * CUDA graph when the same batch shape recurs.  Bag of tasks over tiles,
 * Sec. II; demand-driven assignment, Sec. III-B.  Results are identical to
 * seg_tile + features_tile on each tile alone.  feats receives up to
 * feats_cap rows; if K > feats_cap, n_objects still reports K and the
 * tile's status (pipe_status_read) becomes PIPE_EOVERFLOW. */
typedef struct {
    const uint8_t* rgb; int W, H; size_t pitch;
    uint8_t* hem8; int32_t* labels; int32_t* edt; int32_t* n_objects;
    float* feats; int feats_cap;
} tile_dev;
/* Launch shapes (the number of persistent reconstruction workers, the rows
 * one distance-transform block solves, the blocks of the feature pass)
 * never change a result.  With params.autotune set, the first call with a
 * new list of tile sizes synchronises `stream` and picks them by timing the
 * whole path on this batch (about 30 extra passes; the outputs are
 * rewritten with identical values); the choice is kept per tile-size list
 * for the pipe's lifetime and, if params.autotune_cache names a file,
 * appended to it ("<key> <workers> <rows> <blocks>" per line) and read back
 * by later pipes.  Such a first call cannot be captured into a CUDA graph.
 * The served form uses a shape's tuned values when it has them and the
 * defaults otherwise; it never tunes. */
int seg_features_batch(pipe_t p, const tile_dev* tiles, int n, pipe_stream_t stream);

/* Grayscale opening by a disk (Table I "Morph. Open", which uses a 19x19
 * disk: radius = 9).  The disk of radius r is the set of integer offsets
 * (dx, dy) with dx^2 + dy^2 <= r^2.  dst = the dilation of the erosion of
 * src, each the maximum / minimum over the disk around a pixel, taken over
 * in-image pixels only.
 *  src_dev, dst_dev: W x H uint8 planes, row pitch W, caller-owned device
 *    memory; they must not overlap.
 *  0 <= radius <= 15; W, H as for seg_tile.
 * Returns PIPE_EINVAL on a bad argument (nothing is launched); otherwise
 * the work is asynchronous on `stream`. */
int morph_open_tile(pipe_t p, const uint8_t* src_dev, int W, int H, int radius, uint8_t* dst_dev,
                    pipe_stream_t stream);

/* Watershed split of the labelled objects on the distance transform (Table I
 * "Pre-Watershed": distance transform and markers; "Watershed").  The paper
 * names the operations only (and notes that its CPU and GPU versions give
 * different results); the definition computed here, per object k of the
 * label plane, is:
 *   d = min(255, floor(sqrt(edt))) on the object, 0 elsewhere;
 *   R = reconstruction by dilation, 8-connected, of max(d - h, 0) under d
 *       (the h-maxima of d);
 *   markers = maximal 8-connected plateaus of equal R with no 8-neighbour of
 *       larger R, each named by its first pixel in row-major order;
 *   flooding in synchronous waves: with F the unnamed object pixels having
 *       a named 8-neighbour and L = max d over F, every pixel of F with
 *       d >= L takes, in one wave, the name of its named neighbour of largest
 *       edt (ties: smallest name); waves repeat at L while any pixel is
 *       named, then L is taken again from the new F;
 *   out = basins numbered 1..n_basins object by object in label order, and
 *       within an object by the row-major order of each basin's first pixel;
 *       0 where labels is 0 or above n_objects.
 *  labels_dev, edt_dev: W x H int32 planes as written by seg_tile (edt must
 *    be the exact squared distance transform of labels: > 0 on every object
 *    pixel); n_objects = K of seg_tile; 0 <= h <= 255 (the marker height).
 *  out_dev: W x H int32, caller-owned, must not overlap labels or edt;
 *  n_basins_dev: one int32 receiving the number of basins.
 *  Objects whose bounding box with a 1-pixel margin exceeds 1024 pixels run
 *  on a pipe-owned side stream (forked from and joined back to `stream`, so
 *  the call stays in `stream` order); boxes beyond 7021 pixels are processed
 *  from image-sized scratch planes the pipe owns (10 bytes per pixel,
 *  allocated on the first call of a larger size, which synchronises
 *  `stream`).  A flood that would exceed its wave bound (box pixels + 300)
 *  leaves that object 0 and sets PIPE_EOVERFLOW in the status word.
 * Returns PIPE_EINVAL on a bad argument (nothing is launched); otherwise
 * the work is asynchronous on `stream`. */
int watershed_tile(pipe_t p, const int32_t* labels_dev, const int32_t* edt_dev, int W, int H, int n_objects,
                   int h, int32_t* out_dev, int32_t* n_basins_dev, pipe_stream_t stream);

/* Batched form of watershed_tile: the split of n tiles of any sizes, one
 * launch per pass over the objects of all tiles (so that many tiles'
 * objects share the GPU instead of each call waiting for its slowest
 * object).  Results are identical to watershed_tile on each tile alone.
 *  tiles[i]: labels, edt, out (W x H int32, out not overlapping the
 *    inputs), n_objects = K of the tile (host int), n_basins (one device
 *    int32); 1 <= n <= 4096; 0 <= h <= 255.
 *  The pipe's scratch covers all tiles at once: boxes, basin counts and the
 *  list of large boxes (24 bytes per object) and the planes for boxes
 *  beyond the shared-memory stage (10 bytes per pixel of all tiles),
 *  allocated on the first call of a larger size, which synchronises
 *  `stream`.
 * Returns PIPE_EINVAL on a bad argument (nothing is launched); otherwise
 * the work is asynchronous on `stream`. */
typedef struct {
    const int32_t* labels; const int32_t* edt; int W, H;
    int n_objects;
    int32_t* out; int32_t* n_basins;
} ws_tile;
int watershed_batch(pipe_t p, const ws_tile* tiles, int n, int h, pipe_stream_t stream);

/* Red blood cell detection (Table I "RBC detection", which the paper lists
 * with its CPU sources, OpenCV and Vincent's morphological reconstruction,
 * and no definition).  The definition computed here:
 *   d = R - max(G, B) per pixel (red dominance, an integer in [-255, 255]);
 *   marker = d >= t_hi; mask = d >= t_lo;
 *   out_dev = 1 on the 8-connected components of the mask that hold a
 *     marker pixel (the binary reconstruction by dilation of the marker
 *     under the mask), 0 elsewhere.
 *  rgb_dev: H rows of 3*W bytes (R,G,B) at pitch_bytes >= 3*W; out_dev: a
 *  W x H uint8 plane, caller-owned, not overlapping the input;
 *  0 <= t_lo <= t_hi <= 255 (the workload uses 40 and 100).  The pipe owns
 *  the scratch (a W x H mask plane, one seed flag per 64x64 work tile and a
 *  work queue), allocated on the first call of a larger size, which
 *  synchronises `stream`.
 * Returns PIPE_EINVAL on a bad argument (nothing is launched); otherwise
 * the work is asynchronous on `stream`. */
int rbc_tile(pipe_t p, const uint8_t* rgb_dev, int W, int H, size_t pitch_bytes, int t_lo, int t_hi,
             uint8_t* out_dev, pipe_stream_t stream);

/* Canny edges of a uint8 plane and the per-object edge counts (Sec. V-A
 * lists Canny among the feature-stage transforms applied to the
 * deconvolved image; Sec. II names "edge" among the feature families;
 * Table I "Features comp." uses OpenCV's Canny).  The paper gives no
 * parameter; the definition computed here:
 *   gx, gy = 3x3 Sobel with replicated border; m = |gx| + |gy|;
 *   gradient sector, ax = |gx|, ay = |gy|: horizontal if
 *     (ax + ay)^2 < 2 ax^2, vertical if ay > ax and (ay - ax)^2 > 2 ax^2,
 *     else diagonal along (+x,+y) if gx gy > 0, along (+x,-y) otherwise;
 *   a pixel survives non-maximum suppression iff m > m(a) and m >= m(b),
 *     a and b its neighbours along the sector (a on the previous row, or
 *     the left one for the horizontal sector; m off the image is 0);
 *   candidates: survivors with m > low; strong: survivors with m > high;
 *   edges_dev = 1 on candidates 8-connected through candidates to a strong
 *     pixel, 0 elsewhere;
 *   counts_dev[k-1] = edge pixels within the disk dilation of object k of
 *     labels_dev (offsets dx^2 + dy^2 <= radius^2 from one of its pixels;
 *     a pixel near two objects counts for both), k = 1..n_objects.
 *  img_dev, edges_dev: W x H uint8 planes, caller-owned, not overlapping;
 *  labels_dev: W x H int32 (may be NULL when n_objects = 0); counts_dev:
 *  n_objects int32.  0 <= low <= high; 0 <= radius <= 4.  The hysteresis
 *  runs the segmentation's reconstruction kernel, started from the 64x64
 *  work tiles that hold a strong pixel, on pipe-owned scratch (a W x H
 *  candidate plane, one seed flag per work tile and a work queue), allocated
 *  on the first call of a larger size, which synchronises `stream`.
 * Returns PIPE_EINVAL on a bad argument (nothing is launched); otherwise
 * the work is asynchronous on `stream`. */
int canny_tile(pipe_t p, const uint8_t* img_dev, const int32_t* labels_dev, int W, int H, int n_objects, int low,
               int high, int radius, uint8_t* edges_dev, int32_t* counts_dev, pipe_stream_t stream);

/* Batched form of canny_tile: the edges and edge counts of n tiles of any
 * sizes in one launch per pass (one suppression launch over all tiles, one
 * reconstruction queue for every tile's hysteresis, one counts launch), so
 * that many tiles share the GPU.  Results are identical to canny_tile on
 * each tile alone.
 *  tiles[i]: img (W x H uint8), edges (W x H uint8, not overlapping img),
 *    labels (W x H int32; may be NULL when n_objects = 0), n_objects (host
 *    int), counts (n_objects int32); 1 <= n <= 4096; low, high, radius as
 *    for canny_tile.  The pipe's scratch covers all tiles at once (a
 *    candidate byte per pixel, a seed flag per work tile, the queue),
 *    allocated on the first call of a larger size, which synchronises
 *    `stream`.
 * Returns PIPE_EINVAL on a bad argument (nothing is launched); otherwise
 * the work is asynchronous on `stream`. */
typedef struct {
    const uint8_t* img; const int32_t* labels; int W, H;
    int n_objects;
    uint8_t* edges; int32_t* counts;
} edge_tile;
int canny_batch(pipe_t p, const edge_tile* tiles, int n, int low, int high, int radius, pipe_stream_t stream);

/* Served form (Sec. IV-D prefetching and asynchronous copy): tiles in host
 * memory are admitted as slots and HBM budget allow, uploaded on copy
 * streams overlapped with compute, processed, and their results downloaded.
 * batch_submit never blocks on the GPU; PIPE_EBUSY if the tiles cannot be
 * admitted now.  Host buffers must stay valid until batch_poll reports the
 * tile done. */
typedef struct {
    const uint8_t* rgb_host;  /* pinned or pageable */
    int W, H; size_t pitch;
    int want_planes;          /* 1: also download hem8, labels and edt */
} tile_desc;
typedef struct {
    int status, n_objects;
    int n_feats;              /* feature rows in feats: min(n_objects, the tile's capacity) */
    float* feats;             /* pipe-owned [n_feats][15] */
    uint8_t* hem8; int32_t* labels; int32_t* edt; /* pipe-owned, if want_planes */
    double t_arrive_ms, t_done_ms;  /* submit and completion times, ms of CLOCK_MONOTONIC */
} tile_result;
/* Admits the n tiles as one group: they are uploaded and processed together
 * as one batched launch on a context of their own, concurrently with the
 * groups already in flight.  Contexts keep their device buffers between
 * groups, and hbm_budget_bytes bounds the device memory of all contexts,
 * busy or idle: to grow a context, or start a new one, idle contexts are
 * freed first when the total would pass the budget.  PIPE_EBUSY (nothing
 * enqueued) when max_slots contexts are busy or the group does not fit
 * beside the busy ones; PIPE_ENOMEM when the group alone exceeds the
 * budget. */
int batch_submit(pipe_t p, const tile_desc* tiles, int n, uint64_t* ticket);
/* PIPE_EAGAIN (n_done = 0) until every tile of the ticket is done; then
 * fills out[0..n) and sets n_done = n (a done ticket may be polled again).
 * The pipe-owned result arrays of a completed ticket stay valid until
 * batch_release is called for that ticket or the pipe is destroyed; polls
 * of other tickets, from any thread, never touch them.  A tile whose object
 * count exceeds its feature capacity (min(W*H/20+1, 65536) rows) reports
 * PIPE_EOVERFLOW with n_objects = K and n_feats = the capacity.
 * PIPE_EINVAL for an unknown or released ticket. */
int batch_poll(pipe_t p, uint64_t ticket, int* n_done, tile_result* out);
/* Frees the results of a completed ticket; the ticket is unknown afterwards.
 * The caller must not read them (from any thread) after this call.
 * PIPE_EAGAIN if the ticket is not done yet, PIPE_EINVAL if unknown. */
int batch_release(pipe_t p, uint64_t ticket);

/* ---- introspection used by tests and the benchmark ---------------------- */

/* Synchronises the pipe's streams and returns (then clears) the device
 * status word: PIPE_OK or the first device-side error since the last read. */
int pipe_status_read(pipe_t p);

/* Copies an internal plane of the most recent seg_tile call into dst_dev
 * (device memory), enqueued on `stream`:
 *   0: R, the reconstruction (uint8 H*W)
 *   1: fg (uint8 0/1, H*W)      2: filled (uint8 0/1, H*W) */
int pipe_debug_plane(pipe_t p, int which, void* dst_dev, pipe_stream_t stream);

/* Per-kernel CUDA-event timing.  While enabled, every kernel launch of the
 * pipe is bracketed by events on its stream; pipe_profile_read synchronises
 * and returns, for up to `cap` kernels, their names, launch counts and total
 * milliseconds, then resets the totals.  Returns the number of kernels. */
int pipe_profile_enable(pipe_t p, int enable);
int pipe_profile_read(pipe_t p, const char** names, long long* launches, double* total_ms,
                      int cap);

/* Launch shapes used by the most recent seg_features_batch call, and the
 * number of timed passes the autotuner has run since creation. */
int pipe_autotune_info(pipe_t p, int* recon_workers, int* edt_rows, int* feat_blocks, long long* tune_runs);

/* Device memory of the served form: bytes held by all its contexts (never
 * above hbm_budget_bytes), bytes of the contexts with a group in flight,
 * and the number of contexts; any pointer may be NULL. */
int pipe_serve_memory(pipe_t p, size_t* allocated, size_t* in_flight, int* contexts);

/* Number of kernels the pipe has launched since creation. */
long long pipe_launch_count(pipe_t p);

/* Synchronises the device and returns how many 64x64 work tiles the
 * reconstruction of the most recent seg_tile call processed (a tile that is
 * re-queued counts again), or -1 before any call.  Diagnostic only. */
long long pipe_recon_visits(pipe_t p);

/* ---- Demand-driven tile dispatch (host only; no GPU needed) ----------------
 * The paper's Manager assigns stage instances on demand: a Worker requests
 * work as it finishes earlier work and holds at most `window` instances at a
 * time (Sec. III-B); its PATS scheduler keeps queued instances sorted by an
 * estimate and gives an idle GPU the one at the top of that order (Sec.
 * IV-B).  With GPU-only workers the estimate is a tile's processing cost:
 * a requesting worker gets the most expensive pending tile (longest
 * processing time first); equal costs keep their order of arrival.  All
 * calls on one sched_t are thread-safe. */
typedef struct sched_s* sched_t;
/* n_workers in [1, 4096], window >= 1.  PIPE_EINVAL / PIPE_ENOMEM. */
int sched_create(int n_workers, int window, sched_t* out);
void sched_destroy(sched_t s);
/* Queues task (an id the caller chooses, unique among queued and held
 * tasks) with its cost (finite, >= 0).  PIPE_EINVAL otherwise. */
int sched_push(sched_t s, uint64_t task, double cost);
/* Grants worker the most expensive queued task: PIPE_OK with *task set;
 * PIPE_EBUSY if the worker already holds `window` tasks; PIPE_EAGAIN if
 * nothing is queued; PIPE_EINVAL for a bad worker. */
int sched_request(sched_t s, int worker, uint64_t* task);
/* The worker finished task (frees one window slot).  PIPE_EINVAL if the
 * worker does not hold it. */
int sched_done(sched_t s, int worker, uint64_t task);
/* Failure recovery (the Manager re-serves work): every task the worker
 * holds goes back to the queue with its cost, and its window empties; a
 * later sched_done from it for those tasks returns PIPE_EINVAL.
 * *requeued (may be NULL) receives the number of tasks returned. */
int sched_release(sched_t s, int worker, long long* requeued);
/* Queued, held (all workers) and completed task counts; any may be NULL. */
int sched_counts(sched_t s, long long* queued, long long* in_flight, long long* completed);
/* Cost estimate of an RGB tile for the queue: W * H * (1 + 8 f), f the
 * fraction of dark pixels (R + G + B < 450: nuclei, not background or
 * stroma) on a 1-in-64 sample grid.  -1 on bad arguments. */
double tile_cost(const uint8_t* rgb, int W, int H, size_t pitch);

#ifdef __cplusplus
}
#endif
#endif
