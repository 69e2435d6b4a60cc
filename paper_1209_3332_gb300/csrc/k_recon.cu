// K2: grayscale reconstruction by dilation, 8-connected, of the h-dome
// marker under hem8 (Table I, "ReconToNuclei"; the paper's GPU version is a
// queue-based wave propagation, Sec. V-A).  R = lim R_k with
// R_{k+1} = min(dilate8(R_k), hem8), R_0 = max(hem8 - h, 0) (written by K1).
//
// Design (GB300): a persistent kernel whose warps are independent workers.
// The image is cut into 32x32 work tiles; a device-wide queue holds the
// tiles that may still change.  A worker pops a tile, stages R and hem8 of
// the tile plus a one-pixel halo in shared memory (bytes, 2.4 KB per warp,
// so that many workers fit on an SM and hide the queue and L2 latencies),
// and while an exact, chain-free test says some pixel can still be raised it
// runs four directional sweeps (down, up, right, left) -- each an exact
// sequential sweep along one axis with the 32 lanes moving in lockstep along
// the other axis, neighbours exchanged by shuffles.  It writes the tile back
// and queues each neighbouring tile that one of the changed border pixels
// can still raise.  Values only grow and are bounded by hem8, so any order
// of tile processings reaches the same unique fixed point; a per-tile state
// machine (idle / queued / running / running+dirty) makes sure a tile is
// never processed by two workers at once and never misses a raise of its
// halo.  Every spin wait is bounded by the pipe's cycle budget, after which
// the worker records ST_TIMEOUT and returns.
#include "internal.cuh"

namespace nucseg {

constexpr int HS = 46;            // shared row stride in pixels: 23 words (odd: column sweeps are conflict-free)
constexpr int MAX_ROUNDS = 256;   // sweep rounds before a tile re-queues itself
constexpr unsigned FULL = 0xffffffffu;

// One warp's staged tile: pixel (y, x), y and x in [-1, RT], is the 16-bit
// word P[pidx(y, x)] holding R in its low byte and M (hem8) in its high byte,
// so that one load yields both.  The interior column 0 sits on a 4-byte
// boundary.
struct WarpTile {
    uint16_t P[(RT + 2) * HS];
};
__device__ __forceinline__ int pidx(int y, int x) { return (y + 1) * HS + x + 4; }

#define SR(y, x) reinterpret_cast<uint8_t*>(S.P)[2 * pidx(y, x)]
#define SM(y, x) reinterpret_cast<uint8_t*>(S.P)[2 * pidx(y, x) + 1]

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

constexpr int ITEM_BITS = 18;  // work tiles per image <= (16384 / 32)^2 = 2^18
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

// ---- initial queue: per image, checkerboard order (all tiles with even
// tx+ty first) so that the first wave of workers does not process adjacent
// tiles at the same time ----------------------------------------------------------
__global__ void k_wl_init(Launch L) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        L.sh->head = 0;
        L.sh->tp = ((unsigned long long)(unsigned)L.n_rt << 32) | (unsigned)L.n_rt;
        L.sh->err = 0;
        L.sh->processed = 0;
    }
    if (i >= L.n_rt) return;
    int ti = find_tile(L.tiles, L.ntiles, i, &TileDev::rt_base);
    const TileDev& T = L.tiles[ti];
    int k = i - T.rt_base, ty = k / T.rtx, tx = k - ty * T.rtx;
    int rx = T.rtx, ry = T.rty;
    int evens = ((rx + 1) / 2) * ((ry + 1) / 2) + (rx / 2) * (ry / 2);
    int before = ((ty + 1) / 2) * ((rx + 1) / 2) + (ty / 2) * (rx / 2);  // evens in rows < ty
    before += (ty & 1) ? tx / 2 : (tx + 1) / 2;                       // evens in row ty, x < tx
    int pos = T.rt_base + (((tx + ty) & 1) ? evens + (k - before) : before);
    L.wl_slots[pos] = ((unsigned long long)(unsigned)(pos + 1) << 32) |
                      (ITEM_FIRST | ((unsigned)ti << ITEM_BITS) | (unsigned)k);
    L.wl_state[i] = WL_QUEUED;
}

// ---- tile processing --------------------------------------------------------------

// halo pixel q of this lane: q=0 row -1 and q=1 row RT (columns lane-1), q=2
// column -1 and q=3 column RT (rows lane), q=4 the halo-row pixels of columns
// RT-1 and RT (lanes 0..3)
__device__ __forceinline__ void halo_coord(int q, int lane, int x0, int y0, int& gy, int& gx) {
    if (q < 2) { gy = q == 0 ? y0 - 1 : y0 + RT; gx = x0 + lane - 1; }
    else if (q < 4) { gy = y0 + lane; gx = q == 2 ? x0 - 1 : x0 + RT; }
    else { gy = (lane & 1) ? y0 + RT : y0 - 1; gx = x0 + RT - 1 + ((lane >> 1) & 1); }
}
__device__ __forceinline__ uint8_t& halo_ref(WarpTile& S, int q, int lane, bool mask) {
    uint8_t* A = reinterpret_cast<uint8_t*>(S.P) + (mask ? 1 : 0);
#define AX(y, x) A[2 * pidx(y, x)]
    if (q == 0) return AX(-1, lane - 1);
    if (q == 1) return AX(RT, lane - 1);
    if (q == 2) return AX(lane, -1);
    if (q == 3) return AX(lane, RT);
    return AX((lane & 1) ? RT : -1, RT - 1 + ((lane >> 1) & 1));
#undef AX
}

// R of the halo pixels of this lane (see halo_coord), 0 outside the image
__device__ __forceinline__ void load_halo(uint8_t hr[5], const uint8_t* Rg, int W, int H, int x0, int y0,
                                          int lane) {
#pragma unroll
    for (int q = 0; q < 5; q++) {
        int gy, gx;
        halo_coord(q, lane, x0, y0, gy, gx);
        bool in = gy >= 0 && gy < H && gx >= 0 && gx < W && (q < 4 || lane < 4);
        hr[q] = in ? __ldcg(Rg + (size_t)gy * W + gx) : (uint8_t)0;
    }
}

__device__ __forceinline__ void load_tile(WarpTile& S, const uint8_t* Rg, const uint8_t* Mg, int W, int H,
                                          int x0, int y0, int lane) {
    uint8_t hr[5], hm[5];
#pragma unroll
    for (int q = 0; q < 5; q++) {
        int gy, gx;
        halo_coord(q, lane, x0, y0, gy, gx);
        bool in = gy >= 0 && gy < H && gx >= 0 && gx < W && (q < 4 || lane < 4);
        size_t o = (size_t)gy * W + gx;
        hr[q] = in ? __ldcg(Rg + o) : (uint8_t)0;
        hm[q] = in ? __ldg(Mg + o) : (uint8_t)0;
    }
    if ((W & 3) == 0 && x0 + RT <= W) {
        // interior: 8 lanes x 4 bytes per row, 4 rows per step, all loads issued first
        const int r4 = lane >> 3, c4 = (lane & 7) * 4;
        uint32_t rv[RT / 4], mv[RT / 4];
#pragma unroll
        for (int j = 0; j < RT / 4; j++) {
            int gy = y0 + j * 4 + r4;
            bool in = gy < H;
            size_t o = (size_t)gy * W + x0 + c4;
            rv[j] = in ? __ldcg(reinterpret_cast<const unsigned int*>(Rg + o)) : 0u;
            mv[j] = in ? __ldg(reinterpret_cast<const unsigned int*>(Mg + o)) : 0u;
        }
#pragma unroll
        for (int j = 0; j < RT / 4; j++) {
            // four pixels: (R0 M0 R1 M1) and (R2 M2 R3 M3)
            uint32_t* d = reinterpret_cast<uint32_t*>(&S.P[pidx(j * 4 + r4, c4)]);
            d[0] = __byte_perm(rv[j], mv[j], 0x5140);
            d[1] = __byte_perm(rv[j], mv[j], 0x7362);
        }
    } else {
        for (int yy = 0; yy < RT; yy++) {
            int gy = y0 + yy, gx = x0 + lane;
            bool in = gy < H && gx < W;
            size_t o = (size_t)gy * W + gx;
            SR(yy, lane) = in ? __ldcg(Rg + o) : (uint8_t)0;
            SM(yy, lane) = in ? __ldg(Mg + o) : (uint8_t)0;
        }
    }
#pragma unroll
    for (int q = 0; q < 5; q++) {
        if (q == 4 && lane >= 4) continue;
        halo_ref(S, q, lane, false) = hr[q];
        halo_ref(S, q, lane, true) = hm[q];
    }
    __syncwarp();
}

// Writes the tile's R back: 4-byte stores where rows are word aligned.
__device__ __forceinline__ void store_tile(WarpTile& S, uint8_t* Rg, int W, int H, int x0, int y0, int lane) {
    if ((W & 3) == 0 && x0 + RT <= W) {
        const int r4 = lane >> 3, c4 = (lane & 7) * 4;
#pragma unroll
        for (int j = 0; j < RT / 4; j++) {
            int yy = j * 4 + r4, gy = y0 + yy;
            if (gy < H) {
                const uint32_t* d = reinterpret_cast<const uint32_t*>(&S.P[pidx(yy, c4)]);
                __stcg(reinterpret_cast<unsigned int*>(Rg + (size_t)gy * W + x0 + c4), __byte_perm(d[0], d[1], 0x6420));
            }
        }
    } else {
        const int gx = x0 + lane;
        for (int y = 0; y < RT; y++) {
            int gy = y0 + y;
            if (gy < H && gx < W) __stcg(Rg + (size_t)gy * W + gx, SR(y, lane));
        }
    }
}

// Raises the staged halo to the values just read; true if any grew.
__device__ __forceinline__ bool merge_halo(WarpTile& S, const uint8_t hr[5], int lane) {
    bool grew = false;
#pragma unroll
    for (int q = 0; q < 5; q++) {
        if (q == 4 && lane >= 4) continue;
        uint8_t& h = halo_ref(S, q, lane, false);
        if (hr[q] > h) {
            h = hr[q];
            grew = true;
        }
    }
    __syncwarp();
    return __any_sync(FULL, grew);
}

// One sweep: RT steps, each updating one line of the tile (a row, lanes =
// columns; or a column, lanes = rows) from the three pixels of the line
// before it, which the previous step stored.  A lane's pixel at step i sits
// at byte offset o + i*ds of the staged planes; its two diagonal neighbours
// on the previous line are at offset +/- dl from the previous pixel, where
// the edge lanes find the halo, so no lane needs a special case.  With
// R <= M everywhere, max(R, min(m, M)) = min(max(R, m), M).  __syncwarp
// orders each step's stores before the next step's loads.  One body serves
// the four directions, which keeps the unrolled code small.
__device__ __forceinline__ void sweep(uint16_t* P, int o, int ds, int dl) {
    uint8_t* R = reinterpret_cast<uint8_t*>(P);  // R of pixel i is byte 2 i
    int prev = R[2 * (o - ds)];
#pragma unroll 8
    for (int i = 0; i < RT; i++, o += ds) {
        const int a = R[2 * (o - ds - dl)], b = R[2 * (o - ds + dl)];
        const uint32_t rm = P[o];
        const int nv = min(max((int)(rm & 0xffu), __vimax3_s32(prev, a, b)), (int)(rm >> 8));
        R[2 * o] = (uint8_t)nv;
        prev = nv;
        __syncwarp();
    }
}

// One round of the four sweeps: down, up, right, left.
__device__ __forceinline__ void sweep_round(WarpTile& S, int lane) {
    const int c = lane + 4, r = (lane + 1) * HS;  // this lane's column / row offset
    sweep(S.P, HS + c, HS, 1);               // down: rows 0..31
    sweep(S.P, RT * HS + c, -HS, 1);         // up: rows 31..0
    sweep(S.P, r + 4, 1, HS);                // right: columns 0..31
    sweep(S.P, r + RT + 3, -1, HS);          // left: columns 31..0
}

// Whether some pixel of the tile can still be raised by one of its 8
// neighbours: the exact convergence test, evaluated for all pixels in
// parallel (lane = column), so it has no dependent chain.
__device__ __forceinline__ bool can_raise(WarpTile& S, int lane) {
    bool v = false;
    int a = __vimax3_s32(SR(-1, lane - 1), SR(-1, lane), SR(-1, lane + 1));
    int b = __vimax3_s32(SR(0, lane - 1), SR(0, lane), SR(0, lane + 1));
#pragma unroll 4
    for (int y = 0; y < RT; y++) {
        int c = __vimax3_s32(SR(y + 1, lane - 1), SR(y + 1, lane), SR(y + 1, lane + 1));
        const uint32_t rm = S.P[pidx(y, lane)];
        v |= min(__vimax3_s32(a, b, c), (int)(rm >> 8)) > (int)(rm & 0xffu);
        a = b;
        b = c;
    }
    return __any_sync(FULL, v);
}

// Whether a halo pixel can raise one of the tile's border pixels.  When the
// interior was at a fixed point before the halo grew, only border pixels
// can have become raisable, so this is the exact test in that case.
__device__ __forceinline__ bool border_can_raise(WarpTile& S, int lane) {
    const int ht = __vimax3_s32(SR(-1, lane - 1), SR(-1, lane), SR(-1, lane + 1));
    const int hb = __vimax3_s32(SR(RT, lane - 1), SR(RT, lane), SR(RT, lane + 1));
    const int hl = __vimax3_s32(SR(lane - 1, -1), SR(lane, -1), SR(lane + 1, -1));
    const int hr = __vimax3_s32(SR(lane - 1, RT), SR(lane, RT), SR(lane + 1, RT));
    const bool v = min(ht, (int)SM(0, lane)) > (int)SR(0, lane) ||
                   min(hb, (int)SM(RT - 1, lane)) > (int)SR(RT - 1, lane) ||
                   min(hl, (int)SM(lane, 0)) > (int)SR(lane, 0) ||
                   min(hr, (int)SM(lane, RT - 1)) > (int)SR(lane, RT - 1);
    return __any_sync(FULL, v);
}

// Whether a changed border line of this tile can raise the facing halo line.
__device__ __forceinline__ bool line_need(int own, bool changed, int halo_r, int halo_m, int lane) {
    int cv = changed ? own : 0;
    int a = __shfl_up_sync(FULL, cv, 1), b = __shfl_down_sync(FULL, cv, 1);
    if (lane == 0) a = 0;
    if (lane == 31) b = 0;
    return __any_sync(FULL, min(halo_m, __vimax3_s32(cv, a, b)) > halo_r);
}

__global__ void __launch_bounds__(RT_WARPS * 32, RECON_MIN_BLOCKS) k_recon(Launch L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTile& S = reinterpret_cast<WarpTile*>(smraw)[warp];
    int visits = 0;  // tile processings of this warp (diagnostic), added once at exit
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
        // border values as last written (or as loaded): a request is due
        // only for border pixels changed since
        int top0 = SR(0, lane), bot0 = SR(RT - 1, lane);
        int lef0 = SR(lane, 0), rig0 = SR(lane, RT - 1);
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
            int rel = -1;  // lane 31: the state the release found
            if (nr > 0) {
                // the halo read only decides which neighbours to queue; it is
                // issued before the write-back so that the two overlap (a stale
                // value can only cause a needless request)
                uint8_t hr[5];
                load_halo(hr, Rg, W, H, x0, y0, lane);
                store_tile(S, Rg, W, H, x0, y0, lane);
                __threadfence();  // this tile's pixels before any request
                grew = merge_halo(S, hr, lane);
                // the release overlaps the requests below; only the pending
                // decrement has to wait for them
                if (!grew && lane == 31) rel = atomicCAS(&L.wl_state[t], WL_RUNNING, WL_IDLE);
                const int top = SR(0, lane), bot = SR(RT - 1, lane);
                const int lef = SR(lane, 0), rig = SR(lane, RT - 1);
                const bool nU = line_need(top, top != top0, SR(-1, lane), SM(-1, lane), lane);
                const bool nD = line_need(bot, bot != bot0, SR(RT, lane), SM(RT, lane), lane);
                const bool nL = line_need(lef, lef != lef0, SR(lane, -1), SM(lane, -1), lane);
                const bool nR = line_need(rig, rig != rig0, SR(lane, RT), SM(lane, RT), lane);
                // corner halo pixels face a single tile pixel
                const int t00 = __shfl_sync(FULL, top0, 0), t31 = __shfl_sync(FULL, top0, 31);
                const int b00 = __shfl_sync(FULL, bot0, 0), b31 = __shfl_sync(FULL, bot0, 31);
                int v;
                const bool nUL = (v = SR(0, 0)) != t00 && min((int)SM(-1, -1), v) > SR(-1, -1);
                const bool nUR = (v = SR(0, RT - 1)) != t31 && min((int)SM(-1, RT), v) > SR(-1, RT);
                const bool nDL = (v = SR(RT - 1, 0)) != b00 && min((int)SM(RT, -1), v) > SR(RT, -1);
                const bool nDR = (v = SR(RT - 1, RT - 1)) != b31 && min((int)SM(RT, RT), v) > SR(RT, RT);
                // lane j issues request j, so the requests overlap instead of queueing
                int target = -1;
                switch (lane) {
                    case 0: if (nU && ty > 0) target = k - rx; break;
                    case 1: if (nD && ty + 1 < ry) target = k + rx; break;
                    case 2: if (nL && tx > 0) target = k - 1; break;
                    case 3: if (nR && tx + 1 < rx) target = k + 1; break;
                    case 4: if (nUL && ty > 0 && tx > 0) target = k - rx - 1; break;
                    case 5: if (nUR && ty > 0 && tx + 1 < rx) target = k - rx + 1; break;
                    case 6: if (nDL && ty + 1 < ry && tx > 0) target = k + rx - 1; break;
                    case 7: if (nDR && ty + 1 < ry && tx + 1 < rx) target = k + rx + 1; break;
                    case 8: if (more) target = k; break;  // not converged within MAX_ROUNDS: run again
                    default: break;
                }
                if (target >= 0) wl_request(L, ti, base, target);
                top0 = top;
                bot0 = bot;
                lef0 = lef;
                rig0 = rig;
            }
            // every lane's requests (and the pending counts they add) come
            // before this tile stops counting as running
            __syncwarp();
            if (grew) continue;  // the fresher halo may raise pixels: check again
            // No fence is needed before releasing: every write-back above was
            // followed by one, and the requests' pending counts precede the
            // decrement in the counter's order through the __syncwarp.
            if (nr == 0 && lane == 31) rel = atomicCAS(&L.wl_state[t], WL_RUNNING, WL_IDLE);
            int again = 0;
            if (lane == 31) {
                if (rel == WL_RUNNING) {
                    atomicAdd(&L.sh->tp, ~0ull);  // pending - 1
                } else {
                    // a neighbour raised the halo meanwhile: take the tile again
                    atomicExch(&L.wl_state[t], WL_RUNNING);
                    again = 1;
                }
            }
            again = __shfl_sync(FULL, again, 31);
            if (!again) break;
            visits++;
            __threadfence();
            if (ld_vol(&L.sh->err)) break;
            // only the halo can have changed: the interior belongs to this worker
            uint8_t hr[5];
            load_halo(hr, Rg, W, H, x0, y0, lane);
            merge_halo(S, hr, lane);
        }
    }
    if (lane == 0 && visits) atomicAdd(&L.sh->processed, visits);
}

// resident CTAs of the reconstruction kernel
int recon_grid(int device) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    size_t smem = sizeof(WarpTile) * RT_WARPS;
    cudaFuncSetAttribute(k_recon, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_recon, RT_WARPS * 32, smem);
    return sms * (per < 1 ? 1 : per);
}

void launch_recon(const Launch& L, int grid_cap, cudaStream_t s, Profiler* pf) {
    if (L.n_rt == 0) return;
    pf->begin("recon_init", s);
    k_wl_init<<<(L.n_rt + 255) / 256, 256, 0, s>>>(L);
    pf->end("recon_init", s);
    const int want = (L.n_rt + RT_WARPS - 1) / RT_WARPS;
    const int grid = want < grid_cap ? want : grid_cap;
    pf->begin("recon", s);
    k_recon<<<grid, RT_WARPS * 32, sizeof(WarpTile) * RT_WARPS, s>>>(L);
    pf->end("recon", s);
}

}  // namespace nucseg
