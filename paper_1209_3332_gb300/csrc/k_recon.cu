// K2: grayscale reconstruction by dilation, 8-connected, of the h-dome
// marker under hem8 (Table I, "ReconToNuclei"; the paper's GPU version is a
// queue-based wave propagation, Sec. V-A).  R = lim R_k with
// R_{k+1} = min(dilate8(R_k), hem8), R_0 = max(hem8 - h, 0) (written by K1).
//
// Design (GB300): a persistent kernel whose warps are independent workers.
// The image is cut into 64x64 work tiles; a device-wide queue holds the
// tiles that may still change.  A warp pops a tile, stages R and hem8 (M) of
// the tile and a one-pixel halo in its own shared memory, and runs rounds of
// four directional sweeps over the whole tile (down, up, right, left), each
// an exact sequential sweep along one axis:
//  * the tile is stored as 2x2-pixel blocks, one 32-bit word of R and one of
//    M per block, so that two pixels of a row and two pixels of a column are
//    equally one byte permute away from a pair of 16-bit lanes;
//  * a row sweep gives each lane two adjacent columns, a column sweep two
//    adjacent rows; the pair is updated with 16x2-bit SIMD max/min
//    (new = min(max(R, max of the three pixels of the line before), M)),
//    the two outer neighbours come from the adjacent lanes by shuffle, and
//    the halo reaches the edge lanes as a third operand of the max (the
//    other lanes read zeros there), so no lane needs a branch or a select;
//  * a sweep reads each block once per two lines and never reads what
//    another lane stored during it.
// After each round an exact, chain-free test decides whether another is
// needed.  The warp then writes the tile back and queues each neighbouring
// tile that one of the changed border pixels can still raise.  Values only
// grow and are bounded by hem8, so any order of tile processings reaches the
// same unique fixed point; a per-tile state machine (idle / queued / running
// / running+dirty) makes sure a tile is never processed by two workers at
// once and never misses a raise of its halo.  Every spin wait is bounded by
// the pipe's cycle budget, after which the worker records ST_TIMEOUT and
// returns.
#include "internal.cuh"

namespace nucseg {

constexpr int NB = RT / 2;        // blocks per tile side
constexpr int BS = NB + 1;        // block row stride: 33 8-byte blocks (odd: column sweeps are conflict-free)
constexpr int HL = RT + 2;        // halo line length: index = coordinate + 1, coordinates -1..RT
constexpr int MAX_ROUNDS = 256;   // sweep rounds before a tile re-queues itself
constexpr unsigned FULL = 0xffffffffu;

// A worker's staged tile.  Block (j, i) covers pixels (2j + a, 2i + b),
// a, b in {0, 1}: B[j * BS + i].x holds their R bytes and .y their M bytes,
// byte 2a + b.  The halo lines keep R as one 32-bit word per pixel: the
// first line of each pair (row -1, column -1) in bits 0-7, the second
// (row RT, column RT) in bits 16-23, which is where a pixel pair of the
// neighbouring edge lane needs it; the corners appear in a row and in a
// column line.  Z is a line of zeros, the halo operand of the inner lanes.
// B0 keeps the four border lines as they were when neighbours were last
// queued for them (top, bottom, left, right).
struct WarpTile {
    uint2 B[NB * BS];
    uint32_t HRow[2][HL];
    uint32_t HC[2][HL];
    uint32_t Z[HL];
    uint8_t HMr[2][HL + 2];  // M of the halo rows
    uint8_t HMc[2][HL + 2];  // M of the halo columns
    uint8_t B0[4][RT];
    int flags[9];            // neighbours to queue: up, down, left, right, UL, UR, DL, DR, self
};

// R / M byte of interior pixel (y, x)
__device__ __forceinline__ uint8_t& rpx(WarpTile& S, int y, int x) {
    return reinterpret_cast<uint8_t*>(&S.B[(y >> 1) * BS + (x >> 1)].x)[((y & 1) << 1) | (x & 1)];
}
__device__ __forceinline__ uint8_t mpx(const WarpTile& S, int y, int x) {
    return reinterpret_cast<const uint8_t*>(&S.B[(y >> 1) * BS + (x >> 1)].y)[((y & 1) << 1) | (x & 1)];
}
// R and M of halo pixel (hy, hx)
__device__ __forceinline__ int halo_r(const WarpTile& S, int hy, int hx) {
    if (hy == -1) return (int)(S.HRow[0][hx + 1] & 0xffu);
    if (hy == RT) return (int)(S.HRow[1][hx + 1] >> 16);
    if (hx == -1) return (int)(S.HC[0][hy + 1] & 0xffu);
    return (int)(S.HC[1][hy + 1] >> 16);
}
__device__ __forceinline__ int halo_m(const WarpTile& S, int hy, int hx) {
    if (hy == -1) return S.HMr[0][hx + 1];
    if (hy == RT) return S.HMr[1][hx + 1];
    if (hx == -1) return S.HMc[0][hy + 1];
    return S.HMc[1][hy + 1];
}
__device__ __forceinline__ void set_halo_r(WarpTile& S, int hy, int hx, uint32_t r) {
    if (hy == -1) S.HRow[0][hx + 1] = r;
    if (hy == RT) S.HRow[1][hx + 1] = r << 16;
    if (hx == -1) S.HC[0][hy + 1] = r;
    if (hx == RT) S.HC[1][hy + 1] = r << 16;
}
__device__ __forceinline__ void set_halo_m(WarpTile& S, int hy, int hx, uint8_t m) {
    if (hy == -1) S.HMr[0][hx + 1] = m;
    if (hy == RT) S.HMr[1][hx + 1] = m;
    if (hx == -1) S.HMc[0][hy + 1] = m;
    if (hx == RT) S.HMc[1][hy + 1] = m;
}

// 16x2-bit SIMD helpers (values are bytes zero-extended to 16-bit lanes)
__device__ __forceinline__ uint32_t max2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t min2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// byte permutes: a block word -> the pixel pair of row a (ROW0/ROW1) or of
// column b (COL0/COL1) as two 16-bit lanes; two row or column pairs -> a block word
constexpr uint32_t ROW0 = 0x4140, ROW1 = 0x4342, COL0 = 0x4240, COL1 = 0x4341;
constexpr uint32_t PACK_ROWS = 0x6420, PACK_COLS = 0x6240;
// (left neighbour's high lane, own low lane) and (own high lane, right neighbour's low lane)
constexpr uint32_t FROM_LEFT = 0x1076, FROM_RIGHT = 0x5432;
// two halo-line words -> a pixel pair (first line: bits 0-7; second line: bits 16-23)
constexpr uint32_t LINE0_PAIR = 0x5410, LINE1_PAIR = 0x7632;

__device__ __forceinline__ int ld_vol(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ bool budget_over(long long t0, long long budget) {
    return clock64() - t0 > budget;
}

// ---- worklist -----------------------------------------------------------------
// A ticket queue: producers and consumers take indices with atomicAdd (no
// compare-and-swap retries under contention).  Slot k is one 64-bit word,
// sequence << 32 | item: sequence i means "free for producer index i",
// i + 1 means "holds the item of index i"; the consumer of index i hands the
// slot to producer index i + cap.  One word per slot, so an item and its
// sequence number become visible together.  An item is the image index
// << ITEM_BITS | the work tile's index within its image, with bit 31 set on
// the tile's first visit (queued by k_wl_init).  The tail and the
// count of queued-or-running tiles (pending) share one 64-bit word, so a push
// moves both with one atomic.  A consumer holding a ticket waits until its
// item arrives or until no tile is queued or running any more.

constexpr int ITEM_BITS = 18;  // work tiles per image <= (16384 / 64)^2 = 2^16 < 2^18
constexpr unsigned ITEM_MASK = (1u << ITEM_BITS) - 1;
constexpr unsigned ITEM_FIRST = 1u << 31;
constexpr unsigned ITEM_IMAGE_MASK = (1u << (31 - ITEM_BITS)) - 1;  // up to 8192 images

__device__ __forceinline__ unsigned long long ld_vol64(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}
__device__ __forceinline__ void st_vol64(unsigned long long* p, unsigned long long v) {
    *(volatile unsigned long long*)p = v;
}

__device__ void wl_push(const Launch& L, unsigned item) {
    const unsigned cap = (unsigned)L.n_rt;
    const unsigned i = (unsigned)(atomicAdd(&L.sh->tp, (1ull << 32) | 1ull) >> 32);
    unsigned long long* slot = L.wl_slots + i % cap;
    long long t0 = clock64();
    while ((unsigned)(ld_vol64(slot) >> 32) != i) {
        if (budget_over(t0, L.wait_budget)) { atomicCAS(&L.sh->err, 0, ST_TIMEOUT); return; }
        __nanosleep(32);
    }
    st_vol64(slot, ((unsigned long long)(i + 1) << 32) | item);
}

// work tile k of image ti, whose first work tile has global index base
__device__ void wl_request(const Launch& L, int ti, int base, int k) {
    const int t = base + k;
    for (int it = 0; it < 1024; it++) {
        int s = atomicCAS(&L.wl_state[t], WL_IDLE, WL_QUEUED);
        if (s == WL_IDLE) {
            wl_push(L, ((unsigned)ti << ITEM_BITS) | (unsigned)k);
            return;
        }
        if (s == WL_QUEUED || s == WL_DIRTY) return;
        if (atomicCAS(&L.wl_state[t], WL_RUNNING, WL_DIRTY) == WL_RUNNING) return;
    }
    atomicCAS(&L.sh->err, 0, ST_TIMEOUT);
}

// takes the next item; false when the queue is drained (or on error)
__device__ bool wl_pop(const Launch& L, unsigned* item) {
    const unsigned cap = (unsigned)L.n_rt;
    const unsigned h = (unsigned)atomicAdd(&L.sh->head, 1);
    unsigned long long* slot = L.wl_slots + h % cap;
    long long t0 = clock64();
    for (;;) {
        const unsigned long long v = ld_vol64(slot);
        if ((unsigned)(v >> 32) == h + 1) {
            st_vol64(slot, (unsigned long long)(h + cap) << 32);
            *item = (unsigned)v;
            return true;
        }
        if ((unsigned)ld_vol64(&L.sh->tp) == 0u || ld_vol(&L.sh->err)) return false;
        if (budget_over(t0, L.wait_budget)) { atomicCAS(&L.sh->err, 0, ST_TIMEOUT); return false; }
        __nanosleep(64);
    }
}

// ---- initial queue, by groups of ORDER_GROUP images: within a group the
// work tiles that hold a strong marker first (a nucleus: its first visit
// raises the background around it, so that the tiles without one start from
// raised halos), and within each of the two classes four colours by the
// parities of tx and ty -- (even, even), (odd, odd), (odd, even), (even,
// odd) -- so that no two tiles of a colour touch, not even at a corner, and a
// tile of the last colour starts with all eight neighbours visited (3136
// tiles/s per batched step against 3101 for a checkerboard of two).  The later the tiles without
// a source come, the fewer visits (per image: 3.04 ms per 16 tiles of 4096^2,
// one group of 16: 2.45 ms); groups of four keep the time of one group with a
// fifth less DRAM traffic, since fewer images' planes are in use at once.  Places within a class are taken by atomics: the
// order inside a class is not fixed, and the result does not depend on it.
// The per-image class counters live in the tile descriptors and are zeroed
// by k_wl_reset at the start of every launch. --------------------------------------
constexpr int ORDER_GROUP = 4;   // images per ordering group: all their sources before their other tiles

__device__ __forceinline__ int order_class(const Launch& L, int i, int* ti_out, int* k_out) {
    const int ti = find_tile(L.tiles, L.ntiles, i, &TileDev::rt_base);
    const TileDev& T = L.tiles[ti];
    const int k = i - T.rt_base, ty = k / T.rtx, tx = k - ty * T.rtx;
    *ti_out = ti;
    *k_out = k;
    // four colours: (even, even), (odd, odd), (odd, even), (even, odd) -- no two
    // tiles of one colour touch, not even at a corner
    const int col = ((tx & 1) == (ty & 1)) ? (tx & 1) : 2 + (tx & 1);
    return (L.rt_src[i] ? 0 : 4) + col;
}

__global__ void k_wl_reset(Launch L) {
    for (int t = threadIdx.x; t < L.ntiles; t += blockDim.x)
#pragma unroll
        for (int j = 0; j < 8; j++) L.tiles[t].cls[j] = L.tiles[t].cls_pos[j] = 0;
}

// Counts and places are taken once per group of lanes with the same image
// and class, so the counters see one atomic per group instead of one per
// work tile.
__global__ void k_wl_count(Launch L) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    int ti = -1, k = 0, c = 0;
    if (i < L.n_rt) c = order_class(L, i, &ti, &k);
    const int g0 = ti < 0 ? -1 : (ti / ORDER_GROUP) * ORDER_GROUP;  // the group's first image keeps its counters
    const unsigned grp = __match_any_sync(FULL, g0 * 8 + c);
    if (ti >= 0 && lane == __ffs(grp) - 1) atomicAdd(&L.tiles[g0].cls[c], __popc(grp));
}

__global__ void k_wl_init(Launch L) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    if (i == 0) {
        L.sh->head = 0;
        L.sh->tp = ((unsigned long long)(unsigned)L.n_rt << 32) | (unsigned)L.n_rt;
        L.sh->err = 0;
        L.sh->processed = 0;
    }
    int ti = -1, k = 0, c = 0;
    if (i < L.n_rt) c = order_class(L, i, &ti, &k);
    const int g0 = ti < 0 ? -1 : (ti / ORDER_GROUP) * ORDER_GROUP;
    const unsigned grp = __match_any_sync(FULL, g0 * 8 + c);
    const int leader = __ffs(grp) - 1;
    int first = 0;
    if (ti >= 0 && lane == leader) {
        TileDev& T = L.tiles[g0];
        int base = T.rt_base;
        for (int q = 0; q < c; q++) base += T.cls[q];
        first = base + atomicAdd(&T.cls_pos[c], __popc(grp));
    }
    first = __shfl_sync(FULL, first, leader);
    if (ti < 0) return;
    const int pos = first + __popc(grp & ((1u << lane) - 1u));
    L.wl_slots[pos] = ((unsigned long long)(unsigned)(pos + 1) << 32) |
                      (ITEM_FIRST | ((unsigned)ti << ITEM_BITS) | (unsigned)k);
    L.wl_state[i] = WL_QUEUED;
}


// ---- staging ----------------------------------------------------------------------
// Halo pixel q (0..8) of a lane: q 0-1 top row (-1, 2l + q), q 2-3 bottom row
// (RT, 2l + q - 2), q 4-5 left column (2l + q - 4, -1), q 6-7 right column
// (2l + q - 6, RT), q 8 the corners, one each on lanes 0-3.
__device__ __forceinline__ void halo_coord(int q, int lane, int& hy, int& hx) {
    if (q < 2) { hy = -1; hx = 2 * lane + q; }
    else if (q < 4) { hy = RT; hx = 2 * lane + q - 2; }
    else if (q < 6) { hy = 2 * lane + q - 4; hx = -1; }
    else if (q < 8) { hy = 2 * lane + q - 6; hx = RT; }
    else { hy = (lane & 2) ? RT : -1; hx = (lane & 1) ? RT : -1; }
}
__device__ __forceinline__ bool halo_lane(int q, int lane) { return q < 8 || lane < 4; }

// R (and M) of this lane's halo pixels, 0 outside the image
__device__ __forceinline__ void load_halo(uint8_t hr[9], uint8_t* hm, const uint8_t* Rg, const uint8_t* Mg, int W,
                                          int H, int x0, int y0, int lane) {
#pragma unroll
    for (int q = 0; q < 9; q++) {
        int hy, hx;
        halo_coord(q, lane, hy, hx);
        const int gy = y0 + hy, gx = x0 + hx;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W && halo_lane(q, lane);
        const size_t o = (size_t)gy * W + gx;
        hr[q] = in ? __ldcg(Rg + o) : (uint8_t)0;
        if (hm) hm[q] = in ? __ldg(Mg + o) : (uint8_t)0;
    }
}

__device__ __forceinline__ bool fast_rows(const uint8_t* p, const uint8_t* q, int W, int x0) {
    return (W & 15) == 0 && x0 + RT <= W && ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15) == 0;
}

__device__ __forceinline__ void load_tile(WarpTile& S, const uint8_t* Rg, const uint8_t* Mg, int W, int H, int x0,
                                          int y0, int lane) {
    uint8_t hr[9], hm[9];
    load_halo(hr, hm, Rg, Mg, W, H, x0, y0, lane);
    if (fast_rows(Rg, Mg, W, x0)) {
        // lane: block row jj of a group of 8, 16-pixel segment seg; rows 2j and
        // 2j + 1 of R and M with 16-byte loads, eight blocks built from them
        const int jj = lane >> 2, seg = lane & 3;
#pragma unroll 2
        for (int g = 0; g < NB / 8; g++) {
            const int j = g * 8 + jj, gy = y0 + 2 * j;
            const size_t o = (size_t)gy * W + x0 + seg * 16;
            const uint4 z = make_uint4(0, 0, 0, 0);
            const uint4 rt = gy < H ? __ldcg(reinterpret_cast<const uint4*>(Rg + o)) : z;
            const uint4 rb = gy + 1 < H ? __ldcg(reinterpret_cast<const uint4*>(Rg + o + W)) : z;
            const uint4 mt = gy < H ? __ldg(reinterpret_cast<const uint4*>(Mg + o)) : z;
            const uint4 mb = gy + 1 < H ? __ldg(reinterpret_cast<const uint4*>(Mg + o + W)) : z;
            const uint32_t rtw[4] = {rt.x, rt.y, rt.z, rt.w}, rbw[4] = {rb.x, rb.y, rb.z, rb.w};
            const uint32_t mtw[4] = {mt.x, mt.y, mt.z, mt.w}, mbw[4] = {mb.x, mb.y, mb.z, mb.w};
#pragma unroll
            for (int u = 0; u < 4; u++) {
                uint2* d = &S.B[j * BS + seg * 8 + 2 * u];
                d[0] = make_uint2(__byte_perm(rtw[u], rbw[u], 0x5410), __byte_perm(mtw[u], mbw[u], 0x5410));
                d[1] = make_uint2(__byte_perm(rtw[u], rbw[u], 0x7632), __byte_perm(mtw[u], mbw[u], 0x7632));
            }
        }
    } else {
        for (int j = 0; j < NB; j++) {
            uint32_t rw = 0, mw = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int gy = y0 + 2 * j + (q >> 1), gx = x0 + 2 * lane + (q & 1);
                const bool in = gy < H && gx < W;
                const size_t o = (size_t)gy * W + gx;
                rw |= (in ? (uint32_t)__ldcg(Rg + o) : 0u) << (8 * q);
                mw |= (in ? (uint32_t)__ldg(Mg + o) : 0u) << (8 * q);
            }
            S.B[j * BS + lane] = make_uint2(rw, mw);
        }
    }
#pragma unroll
    for (int q = 0; q < 9; q++) {
        if (!halo_lane(q, lane)) continue;
        int hy, hx;
        halo_coord(q, lane, hy, hx);
        set_halo_r(S, hy, hx, hr[q]);
        set_halo_m(S, hy, hx, hm[q]);
    }
}

// Writes the tile's R back: 16-byte stores where rows are 16-byte aligned.
__device__ __forceinline__ void store_tile(WarpTile& S, uint8_t* Rg, int W, int H, int x0, int y0, int lane) {
    if (fast_rows(Rg, Rg, W, x0)) {
        const int jj = lane >> 2, seg = lane & 3;
#pragma unroll 1
        for (int g = 0; g < NB / 8; g++) {
            const int j = g * 8 + jj, gy = y0 + 2 * j;
            uint32_t top[4], bot[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const uint2* s = &S.B[j * BS + seg * 8 + 2 * u];
                const uint32_t a = s[0].x, b = s[1].x;
                top[u] = __byte_perm(a, b, 0x5410);
                bot[u] = __byte_perm(a, b, 0x7632);
            }
            const size_t o = (size_t)gy * W + x0 + seg * 16;
            if (gy < H) __stcg(reinterpret_cast<uint4*>(Rg + o), make_uint4(top[0], top[1], top[2], top[3]));
            if (gy + 1 < H) __stcg(reinterpret_cast<uint4*>(Rg + o + W), make_uint4(bot[0], bot[1], bot[2], bot[3]));
        }
    } else {
        for (int j = 0; j < NB; j++) {
            const uint32_t rw = S.B[j * BS + lane].x;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int gy = y0 + 2 * j + (q >> 1), gx = x0 + 2 * lane + (q & 1);
                if (gy < H && gx < W) __stcg(Rg + (size_t)gy * W + gx, (uint8_t)(rw >> (8 * q)));
            }
        }
    }
}

// Raises the staged halo pixels to the values just read; true if any grew.
__device__ __forceinline__ bool merge_halo(WarpTile& S, const uint8_t hr[9], int lane) {
    bool grew = false;
#pragma unroll
    for (int q = 0; q < 9; q++) {
        if (!halo_lane(q, lane)) continue;
        int hy, hx;
        halo_coord(q, lane, hy, hx);
        if (hr[q] > halo_r(S, hy, hx)) {
            set_halo_r(S, hy, hx, hr[q]);
            grew = true;
        }
    }
    return grew;
}

// ---- sweeps -------------------------------------------------------------------------
// With R <= M everywhere, max(R, min(m, M)) = min(max(R, m), M).

// A row sweep pair: the down sweep (rows 0 -> RT-1) and the up sweep
// (rows RT-1 -> 0) run at once as two independent chains, one block row of
// each per step, so the warp always has two dependent chains in flight.
// Lane l owns block column l in both chains, so every store to a block comes
// from the one thread that also loads it: in the first half of the steps the
// chains work on disjoint halves of the tile; at the middle each chain loads
// its next block row only after the other chain has stored it, and in the
// second half each chain runs over rows the other has already swept.  Each
// chain is still one full directional sweep (every row after the line
// before it), so a round of the two pairs propagates as the four sweeps do,
// and values only grow towards the unique fixed point whatever the order.
// P is the pixel pair of the line before (columns 2l, 2l + 1); its outer
// neighbours come from lanes l - 1 and l + 1 (the edge lanes get their own
// pair back, harmlessly, and the halo column through E).
__device__ __forceinline__ uint32_t line_step(uint32_t& P, uint32_t R, uint32_t M, uint32_t e) {
    const uint32_t L = __shfl_up_sync(FULL, P, 1), Rt = __shfl_down_sync(FULL, P, 1);
    const uint32_t w = __vimax3_u16x2(__byte_perm(P, L, FROM_LEFT), P, __byte_perm(P, Rt, FROM_RIGHT));
    P = min2(__vimax3_u16x2(R, w, e), M);
    return P;
}

__device__ __forceinline__ void row_sweeps(WarpTile& S, int lane) {
    const uint32_t* E = lane == 0 ? S.HC[0] : lane == 31 ? S.HC[1] : S.Z;
    uint32_t Pd = __byte_perm(S.HRow[0][2 * lane + 1], S.HRow[0][2 * lane + 2], LINE0_PAIR);
    uint32_t Pu = __byte_perm(S.HRow[1][2 * lane + 1], S.HRow[1][2 * lane + 2], LINE1_PAIR);
    // down: block row k, rows 2k then 2k + 1; up: block row NB-1-k, rows 2(NB-1-k) + 1 then 2(NB-1-k)
    auto step = [&](uint2 bd, uint2 bu, int k) {
        const int jd = k, ju = NB - 1 - k;
        const uint32_t d0 = line_step(Pd, __byte_perm(bd.x, 0u, ROW0), __byte_perm(bd.y, 0u, ROW0), E[2 * jd]);
        const uint32_t u1 = line_step(Pu, __byte_perm(bu.x, 0u, ROW1), __byte_perm(bu.y, 0u, ROW1), E[2 * ju + 3]);
        const uint32_t d1 = line_step(Pd, __byte_perm(bd.x, 0u, ROW1), __byte_perm(bd.y, 0u, ROW1), E[2 * jd + 1]);
        const uint32_t u0 = line_step(Pu, __byte_perm(bu.x, 0u, ROW0), __byte_perm(bu.y, 0u, ROW0), E[2 * ju + 2]);
        S.B[jd * BS + lane].x = __byte_perm(d0, d1, PACK_ROWS);
        S.B[ju * BS + lane].x = __byte_perm(u0, u1, PACK_ROWS);
    };
    uint2 bd = S.B[lane], bu = S.B[(NB - 1) * BS + lane];
#pragma unroll 3
    for (int k = 0; k < NB / 2 - 1; k++) {  // first half: disjoint rows, next blocks loaded one step ahead
        const uint2 nd = S.B[(k + 1) * BS + lane], nu = S.B[(NB - 2 - k) * BS + lane];
        step(bd, bu, k);
        bd = nd;
        bu = nu;
    }
    step(bd, bu, NB / 2 - 1);
    // the middle: each chain's next block row is the one the other chain just stored
    bd = S.B[(NB / 2) * BS + lane];
    bu = S.B[(NB / 2 - 1) * BS + lane];
#pragma unroll 3
    for (int k = NB / 2; k < NB - 1; k++) {
        const uint2 nd = S.B[(k + 1) * BS + lane], nu = S.B[(NB - 2 - k) * BS + lane];
        step(bd, bu, k);
        bd = nd;
        bu = nu;
    }
    step(bd, bu, NB - 1);
}

// The column sweep pair: right (columns 0 -> RT-1) and left (RT-1 -> 0) at
// once, lane l owning block row l (rows 2l, 2l + 1) in both chains; the halo
// rows reach the edge lanes through E.
__device__ __forceinline__ void col_sweeps(WarpTile& S, int lane) {
    const uint32_t* E = lane == 0 ? S.HRow[0] : lane == 31 ? S.HRow[1] : S.Z;
    uint32_t Cr = __byte_perm(S.HC[0][2 * lane + 1], S.HC[0][2 * lane + 2], LINE0_PAIR);
    uint32_t Cl = __byte_perm(S.HC[1][2 * lane + 1], S.HC[1][2 * lane + 2], LINE1_PAIR);
    auto step = [&](uint2 br, uint2 bl, int k) {
        const int ir = k, il = NB - 1 - k;
        const uint32_t r0 = line_step(Cr, __byte_perm(br.x, 0u, COL0), __byte_perm(br.y, 0u, COL0), E[2 * ir]);
        const uint32_t l1 = line_step(Cl, __byte_perm(bl.x, 0u, COL1), __byte_perm(bl.y, 0u, COL1), E[2 * il + 3]);
        const uint32_t r1 = line_step(Cr, __byte_perm(br.x, 0u, COL1), __byte_perm(br.y, 0u, COL1), E[2 * ir + 1]);
        const uint32_t l0 = line_step(Cl, __byte_perm(bl.x, 0u, COL0), __byte_perm(bl.y, 0u, COL0), E[2 * il + 2]);
        S.B[lane * BS + ir].x = __byte_perm(r0, r1, PACK_COLS);
        S.B[lane * BS + il].x = __byte_perm(l0, l1, PACK_COLS);
    };
    uint2 br = S.B[lane * BS], bl = S.B[lane * BS + NB - 1];
#pragma unroll 3
    for (int k = 0; k < NB / 2 - 1; k++) {
        const uint2 nr = S.B[lane * BS + k + 1], nl = S.B[lane * BS + NB - 2 - k];
        step(br, bl, k);
        br = nr;
        bl = nl;
    }
    step(br, bl, NB / 2 - 1);
    br = S.B[lane * BS + NB / 2];
    bl = S.B[lane * BS + NB / 2 - 1];
#pragma unroll 3
    for (int k = NB / 2; k < NB - 1; k++) {
        const uint2 nr = S.B[lane * BS + k + 1], nl = S.B[lane * BS + NB - 2 - k];
        step(br, bl, k);
        br = nr;
        bl = nl;
    }
    step(br, bl, NB - 1);
}

// One round: the row sweep pair, then the column sweep pair.  __syncwarp
// orders each pair's stores before the next pair's loads (the pairs map
// lanes to blocks differently).
__device__ __forceinline__ void sweep_round(WarpTile& S, int lane) {
    row_sweeps(S, lane);
    __syncwarp();
    col_sweeps(S, lane);
    __syncwarp();
}

// Whether some pixel of the tile can still be raised by one of its 8
// neighbours: the exact convergence test, two pixels per lane and row, with
// no dependent chain; it stops at the first 16-row group that has one.
__device__ __forceinline__ bool can_raise(const WarpTile& S, int lane) {
    const uint32_t* E = lane == 0 ? S.HC[0] : lane == 31 ? S.HC[1] : S.Z;
    // maximum of R over the three columns around each pixel of a pair in row y
    auto hmax = [&](uint32_t R, int y) -> uint32_t {
        const uint32_t L = __shfl_up_sync(FULL, R, 1), Rt = __shfl_down_sync(FULL, R, 1);
        return __vimax3_u16x2(__byte_perm(R, L, FROM_LEFT), __byte_perm(R, Rt, FROM_RIGHT), max2(R, E[y + 1]));
    };
    uint32_t hp = hmax(__byte_perm(S.HRow[0][2 * lane + 1], S.HRow[0][2 * lane + 2], LINE0_PAIR), -1);
    uint2 b = S.B[lane];
    uint32_t R0 = __byte_perm(b.x, 0u, ROW0), M0 = __byte_perm(b.y, 0u, ROW0);
    uint32_t h0 = hmax(R0, 0);
    bool v = false;
    // block row j: rows 2j (R0, M0, h0) and 2j + 1; R2 is row 2j + 2
    auto block_row = [&](uint32_t R2, uint32_t M2, int j) {
        const uint32_t R1 = __byte_perm(b.x, 0u, ROW1), M1 = __byte_perm(b.y, 0u, ROW1);
        const uint32_t h1 = hmax(R1, 2 * j + 1), h2 = hmax(R2, 2 * j + 2);
        v |= min2(__vimax3_u16x2(hp, h0, h1), M0) != R0;
        v |= min2(__vimax3_u16x2(h0, h1, h2), M1) != R1;
        hp = h1;
        h0 = h2;
        R0 = R2;
        M0 = M2;
    };
#pragma unroll 1
    for (int g = 0; g < NB / 8; g++) {
#pragma unroll
        for (int jj = 0; jj < 8; jj++) {
            const int j = g * 8 + jj;
            if (j + 1 < NB) {
                const uint2 nb = S.B[(j + 1) * BS + lane];
                block_row(__byte_perm(nb.x, 0u, ROW0), __byte_perm(nb.y, 0u, ROW0), j);
                b = nb;
            } else {
                block_row(__byte_perm(S.HRow[1][2 * lane + 1], S.HRow[1][2 * lane + 2], LINE1_PAIR), 0u, j);
            }
        }
        if (__any_sync(FULL, v)) return true;
    }
    return false;
}

// Whether a halo pixel can raise a pixel of the tile border.  When the
// tile's interior was at a fixed point before the halo grew, only border
// pixels can have become raisable, so this is the exact test in that case.
__device__ __forceinline__ bool border_can_raise(WarpTile& S, int lane) {
    // lane l: border pixels 2l and 2l + 1 of each side from one block word of
    // R and one of M, and the four halo pixels around them (the halo lines
    // hold the corners too, with the same values as the halo rows)
    const uint2 bt = S.B[lane], bb = S.B[(NB - 1) * BS + lane];
    const uint2 bl = S.B[lane * BS], br = S.B[lane * BS + NB - 1];
    const int i = 2 * lane;
    auto raisable = [](int h0, int h1, int h2, uint32_t r, uint32_t m, int sh) -> bool {
        const int mh = max(max(h0, h1), h2);
        return min(mh, (int)((m >> sh) & 0xffu)) > (int)((r >> sh) & 0xffu);
    };
    bool v = false;
    {
        const int a = S.HRow[0][i] & 0xff, b = S.HRow[0][i + 1] & 0xff, c = S.HRow[0][i + 2] & 0xff,
                  d = S.HRow[0][i + 3] & 0xff;
        v |= raisable(a, b, c, bt.x, bt.y, 0) | raisable(b, c, d, bt.x, bt.y, 8);  // top row
    }
    {
        const int a = S.HRow[1][i] >> 16, b = S.HRow[1][i + 1] >> 16, c = S.HRow[1][i + 2] >> 16,
                  d = S.HRow[1][i + 3] >> 16;
        v |= raisable(a, b, c, bb.x, bb.y, 16) | raisable(b, c, d, bb.x, bb.y, 24);  // bottom row
    }
    {
        const int a = S.HC[0][i] & 0xff, b = S.HC[0][i + 1] & 0xff, c = S.HC[0][i + 2] & 0xff,
                  d = S.HC[0][i + 3] & 0xff;
        v |= raisable(a, b, c, bl.x, bl.y, 0) | raisable(b, c, d, bl.x, bl.y, 16);  // left column
    }
    {
        const int a = S.HC[1][i] >> 16, b = S.HC[1][i + 1] >> 16, c = S.HC[1][i + 2] >> 16,
                  d = S.HC[1][i + 3] >> 16;
        v |= raisable(a, b, c, br.x, br.y, 8) | raisable(b, c, d, br.x, br.y, 24);  // right column
    }
    return __any_sync(FULL, v);
}

// ---- neighbour requests ---------------------------------------------------------------
// Side s (0 top, 1 bottom, 2 left, 3 right) of the tile, after the tile is at
// a fixed point: halo pixel h of the side (h = -1..RT along it) needs its
// tile queued when a border pixel changed since the last requests and next
// to h can raise it.  h = -1 and h = RT are the halo corners, which belong
// to the diagonal neighbours.  The side's border then becomes the reference
// for the next requests.
__device__ __forceinline__ void side_requests(WarpTile& S, int lane) {
    // lane l holds border pixels 2l and 2l + 1 of every side: one block word
    // of R (top: block (0, l) bytes 0, 1; bottom: block (NB-1, l) bytes 2, 3;
    // left: block (l, 0) bytes 0, 2; right: block (l, NB-1) bytes 1, 3); the
    // changed values of the pixels beyond its pair come from the next lanes
    const uint32_t wt = S.B[lane].x, wb = S.B[(NB - 1) * BS + lane].x;
    const uint32_t wl = S.B[lane * BS].x, wr = S.B[lane * BS + NB - 1].x;
    const int p0 = 2 * lane, p1 = 2 * lane + 1;
#pragma unroll
    for (int s = 0; s < 4; s++) {
        const uint32_t w = s == 0 ? wt : s == 1 ? wb : s == 2 ? wl : wr;
        const int sh0 = s == 0 ? 0 : s == 1 ? 16 : s == 2 ? 0 : 8;
        const int sh1 = s == 0 ? 8 : s == 1 ? 24 : s == 2 ? 16 : 24;
        const int v0 = (int)((w >> sh0) & 0xffu), v1 = (int)((w >> sh1) & 0xffu);
        // border values changed since the last requests (else 0)
        const int c0 = v0 != (int)S.B0[s][p0] ? v0 : 0, c1 = v1 != (int)S.B0[s][p1] ? v1 : 0;
        int cl = __shfl_up_sync(FULL, c1, 1), cr = __shfl_down_sync(FULL, c0, 1);
        if (lane == 0) cl = 0;
        if (lane == 31) cr = 0;
        const int m0 = max(max(cl, c0), c1), m1 = max(max(c0, c1), cr);
        // the halo pixels facing p0, p1: R and M
        int hr0, hr1, hm0, hm1;
        if (s == 0) {
            hr0 = (int)(S.HRow[0][p0 + 1] & 0xffu); hr1 = (int)(S.HRow[0][p1 + 1] & 0xffu);
            hm0 = S.HMr[0][p0 + 1]; hm1 = S.HMr[0][p1 + 1];
        } else if (s == 1) {
            hr0 = (int)(S.HRow[1][p0 + 1] >> 16); hr1 = (int)(S.HRow[1][p1 + 1] >> 16);
            hm0 = S.HMr[1][p0 + 1]; hm1 = S.HMr[1][p1 + 1];
        } else if (s == 2) {
            hr0 = (int)(S.HC[0][p0 + 1] & 0xffu); hr1 = (int)(S.HC[0][p1 + 1] & 0xffu);
            hm0 = S.HMc[0][p0 + 1]; hm1 = S.HMc[0][p1 + 1];
        } else {
            hr0 = (int)(S.HC[1][p0 + 1] >> 16); hr1 = (int)(S.HC[1][p1 + 1] >> 16);
            hm0 = S.HMc[1][p0 + 1]; hm1 = S.HMc[1][p1 + 1];
        }
        const bool line = min(m0, hm0) > hr0 || min(m1, hm1) > hr1;
        // the corners (-1 and RT along the side) belong to the diagonal
        // neighbours; corner pixels are read from the halo rows
        const int kl = s == 1 ? 1 : 0, kh = s == 0 ? 0 : 1;        // halo row of the low / high corner
        const int il = s == 3 ? RT + 1 : 0, ih = s == 2 ? 0 : RT + 1;  // its index in that row
        bool lo = false, hi = false;
        if (lane == 0) {
            const int r = kl ? (int)(S.HRow[1][il] >> 16) : (int)(S.HRow[0][il] & 0xffu);
            lo = min(c0, (int)S.HMr[kl][il]) > r;
        }
        if (lane == 31) {
            const int r = kh ? (int)(S.HRow[1][ih] >> 16) : (int)(S.HRow[0][ih] & 0xffu);
            hi = min(c1, (int)S.HMr[kh][ih]) > r;
        }
        const bool anyl = __any_sync(FULL, line), anylo = __any_sync(FULL, lo), anyhi = __any_sync(FULL, hi);
        if (lane == 0) {
            // corners: top -> UL, UR; bottom -> DL, DR; left -> UL, DL; right -> UR, DR
            const int fl = s == 0 ? 4 : s == 1 ? 6 : s == 2 ? 4 : 5;
            const int fh = s == 0 ? 5 : s == 1 ? 7 : s == 2 ? 6 : 7;
            if (anyl) S.flags[s] = 1;
            if (anylo) S.flags[fl] = 1;
            if (anyhi) S.flags[fh] = 1;
        }
        // the side's border becomes the reference for the next requests
        S.B0[s][p0] = (uint8_t)v0;
        S.B0[s][p1] = (uint8_t)v1;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32, RECON_MIN_BLOCKS) k_recon(Launch L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    WarpTile& S = *reinterpret_cast<WarpTile*>(smraw);
    const int lane = threadIdx.x;
    int visits = 0;  // tile processings of this worker (diagnostic), added once at exit
    if (lane < 9) S.flags[lane] = 0;
    for (int i = lane; i < HL; i += 32) S.Z[i] = 0u;
    __syncwarp();
    for (;;) {
        unsigned item = 0;
        int ok = 0;
        if (lane == 0) ok = wl_pop(L, &item) ? 1 : 0;
        ok = __shfl_sync(FULL, ok, 0);
        if (!ok) break;
        item = __shfl_sync(FULL, item, 0);
        const int ti = (int)((item >> ITEM_BITS) & ITEM_IMAGE_MASK), k = (int)(item & ITEM_MASK);
        // a tile released by a visit was at a fixed point, so on later visits
        // only its border can have become raisable; its first visit starts
        // from the marker and sweeps at once
        bool sweep_now = (item & ITEM_FIRST) != 0, full_check = false;
        const TileDev& T = L.tiles[ti];
        const int W = T.W, H = T.H, rx = T.rtx, ry = T.rty, base = T.rt_base;
        uint8_t* const Rg = T.R;
        const uint8_t* const Mg = T.hem8;
        const int t = base + k, ty = k / rx, tx = k - ty * rx;
        const int x0 = tx * RT, y0 = ty * RT;
        if (lane == 0) atomicExch(&L.wl_state[t], WL_RUNNING);
        visits++;
        __threadfence();
        __syncwarp();
        load_tile(S, Rg, Mg, W, H, x0, y0, lane);
        __syncwarp();
        // the border as loaded is the reference for the first requests (lane l:
        // border pixels 2l, 2l + 1 of each side, from one block word per side)
        {
            const uint32_t wt = S.B[lane].x, wb = S.B[(NB - 1) * BS + lane].x;
            const uint32_t wl = S.B[lane * BS].x, wr = S.B[lane * BS + NB - 1].x;
            S.B0[0][2 * lane] = (uint8_t)wt;
            S.B0[0][2 * lane + 1] = (uint8_t)(wt >> 8);
            S.B0[1][2 * lane] = (uint8_t)(wb >> 16);
            S.B0[1][2 * lane + 1] = (uint8_t)(wb >> 24);
            S.B0[2][2 * lane] = (uint8_t)wl;
            S.B0[2][2 * lane + 1] = (uint8_t)(wl >> 16);
            S.B0[3][2 * lane] = (uint8_t)(wr >> 8);
            S.B0[3][2 * lane + 1] = (uint8_t)(wr >> 24);
        }
        __syncwarp();
        for (;;) {
            int nr = 0;
            bool more = false;
            bool go = sweep_now || (full_check ? can_raise(S, lane) : border_can_raise(S, lane));
            sweep_now = false;
            while (go) {
                if (nr >= MAX_ROUNDS) { more = true; break; }
                sweep_round(S, lane);
                nr++;
                go = can_raise(S, lane);
            }
            full_check = more;  // otherwise the interior is at a fixed point now
            bool grew = false;
            if (nr > 0) {
                // the halo read only decides which neighbours to queue; it is
                // issued before the write-back so that the two overlap (a stale
                // value can only cause a needless request)
                uint8_t hr[9];
                load_halo(hr, nullptr, Rg, Mg, W, H, x0, y0, lane);
                store_tile(S, Rg, W, H, x0, y0, lane);
                // the stores drain while the requests are worked out in shared memory
                grew = __any_sync(FULL, merge_halo(S, hr, lane));
                __syncwarp();
                side_requests(S, lane);
                if (more && lane == 0) S.flags[8] = 1;  // not converged within MAX_ROUNDS: run again
                __threadfence();  // this tile's pixels before any request
                __syncwarp();
                if (lane < 9 && S.flags[lane]) {
                    int target = -1;
                    switch (lane) {
                        case 0: if (ty > 0) target = k - rx; break;
                        case 1: if (ty + 1 < ry) target = k + rx; break;
                        case 2: if (tx > 0) target = k - 1; break;
                        case 3: if (tx + 1 < rx) target = k + 1; break;
                        case 4: if (ty > 0 && tx > 0) target = k - rx - 1; break;
                        case 5: if (ty > 0 && tx + 1 < rx) target = k - rx + 1; break;
                        case 6: if (ty + 1 < ry && tx > 0) target = k + rx - 1; break;
                        case 7: if (ty + 1 < ry && tx + 1 < rx) target = k + rx + 1; break;
                        default: target = k; break;
                    }
                    S.flags[lane] = 0;
                    if (target >= 0) wl_request(L, ti, base, target);
                }
            }
            // every request (and the pending count it adds) comes before this
            // tile stops counting as running
            __syncwarp();
            if (grew) continue;  // the fresher halo may raise pixels: check again
            int again = 0;
            if (lane == 0) {
                // no fence needed here: every write-back above was followed by
                // one, and the requests' pending counts precede this update in
                // the counter's order through the warp barrier
                const int st = atomicCAS(&L.wl_state[t], WL_RUNNING, WL_IDLE);
                if (st == WL_RUNNING) {
                    atomicAdd(&L.sh->tp, ~0ull);  // pending - 1
                } else {
                    // a neighbour raised the halo meanwhile: take the tile again
                    atomicExch(&L.wl_state[t], WL_RUNNING);
                    again = 1;
                }
            }
            if (!__shfl_sync(FULL, again, 0)) break;
            visits++;
            __threadfence();
            if (__any_sync(FULL, ld_vol(&L.sh->err) != 0)) break;
            // only the halo can have changed: the interior belongs to this worker
            uint8_t hr[9];
            load_halo(hr, nullptr, Rg, Mg, W, H, x0, y0, lane);
            merge_halo(S, hr, lane);
            __syncwarp();
        }
        __syncwarp();
    }
    if (lane == 0 && visits) atomicAdd(&L.sh->processed, visits);
}

// ---- seeded start: only the flagged work tiles are queued (any order: the
// fixed point does not depend on it); the others start idle ------------------------
__global__ void k_wl_seed(Launch L, const int* __restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n_rt) return;
    if (flags[i]) {
        const int ti = find_tile(L.tiles, L.ntiles, i, &TileDev::rt_base);
        const unsigned pos = (unsigned)atomicAdd(&L.sh->nseed, 1);
        L.wl_slots[pos] = ((unsigned long long)(pos + 1) << 32) |
                          (ITEM_FIRST | ((unsigned)ti << ITEM_BITS) | (unsigned)(i - L.tiles[ti].rt_base));
        L.wl_state[i] = WL_QUEUED;
    } else {
        L.wl_state[i] = WL_IDLE;
    }
}

// the slots past the seeds are free for their producer index; the queue
// counters start at the seeds
__global__ void k_wl_seed_finish(Launch L) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = L.sh->nseed;
    if (i == 0) {
        L.sh->head = 0;
        L.sh->tp = ((unsigned long long)(unsigned)n << 32) | (unsigned)n;
        L.sh->err = 0;
        L.sh->processed = 0;
    }
    if (i >= n && i < L.n_rt) L.wl_slots[i] = (unsigned long long)(unsigned)i << 32;
}

void launch_recon_seeded(const Launch& L, const int* flags, int grid_cap, cudaStream_t s, Profiler* pf) {
    if (L.n_rt == 0) return;
    pf->begin("recon_seed", s);
    k_wl_seed<<<(L.n_rt + 255) / 256, 256, 0, s>>>(L, flags);
    pf->end("recon_seed", s);
    pf->begin("recon_seed_finish", s);
    k_wl_seed_finish<<<(L.n_rt + 255) / 256, 256, 0, s>>>(L);
    pf->end("recon_seed_finish", s);
    const int grid = L.n_rt < grid_cap ? L.n_rt : grid_cap;
    pf->begin("recon", s);
    k_recon<<<grid, 32, sizeof(WarpTile), s>>>(L);
    pf->end("recon", s);
}

// resident workers (one warp each) of the reconstruction kernel
int recon_grid(int device) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const size_t smem = sizeof(WarpTile);
    cudaFuncSetAttribute(k_recon, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_recon, 32, smem);
    return sms * (per < 1 ? 1 : per);
}

void launch_recon(const Launch& L, int grid_cap, cudaStream_t s, Profiler* pf) {
    if (L.n_rt == 0) return;
    pf->begin("recon_init", s);
    k_wl_reset<<<1, 256, 0, s>>>(L);
    k_wl_count<<<(L.n_rt + 255) / 256, 256, 0, s>>>(L);
    k_wl_init<<<(L.n_rt + 255) / 256, 256, 0, s>>>(L);
    pf->end("recon_init", s);
    const int grid = L.n_rt < grid_cap ? L.n_rt : grid_cap;  // one work tile per worker at a time
    pf->begin("recon", s);
    k_recon<<<grid, 32, sizeof(WarpTile), s>>>(L);
    pf->end("recon", s);
}

}  // namespace nucseg
