// K2: grayscale reconstruction by dilation, 8-connected, of the h-dome
// marker under hem8 (Table I, "ReconToNuclei"; the paper's GPU version is a
// queue-based wave propagation, Sec. V-A).  R = lim R_k with
// R_{k+1} = min(dilate8(R_k), hem8), R_0 = max(hem8 - h, 0) (written by K1).
//
// Design (GB300): a persistent kernel whose CTAs are independent workers.
// The image is cut into 64x64 work tiles; a device-wide queue holds the
// tiles that may still change.  A CTA pops a tile and stages R and hem8 of
// the tile plus a one-pixel halo in shared memory, interleaved as one 16-bit
// word per pixel.  Each of its four warps owns a 32x32 quadrant and runs four
// directional sweeps over it (down, up, right, left) -- each an exact
// sequential sweep along one axis with the 32 lanes moving in lockstep along
// the other -- reading its neighbour quadrants' edge pixels straight from
// shared memory; after each round an exact, chain-free test per quadrant
// decides, through the CTA barrier, whether another round is needed.  The CTA
// then writes the tile back and queues each neighbouring tile that one of the
// changed border pixels can still raise.  A visit thus pays the queue's
// round trips (pop, state change, load, write-back, requests, release) once
// per 4096 pixels.  Values only grow and are bounded by hem8, so any order of
// tile processings reaches the same unique fixed point; a per-tile state
// machine (idle / queued / running / running+dirty) makes sure a tile is
// never processed by two workers at once and never misses a raise of its
// halo.  Every spin wait is bounded by the pipe's cycle budget, after which
// the worker records ST_TIMEOUT and returns.
#include "internal.cuh"

namespace nucseg {

constexpr int QT = 32;            // quadrant side: one warp per quadrant
static_assert(RT == 2 * QT && RT_WARPS == 4, "a work tile is four 32x32 quadrants, one warp each");
constexpr int HS = 70;            // staged row stride in pixels: 35 words (odd: column sweeps are conflict-free)
constexpr int MAX_ROUNDS = 256;   // sweep rounds before a tile re-queues itself
constexpr unsigned FULL = 0xffffffffu;

// The CTA's staged tile: pixel (y, x), y and x in [-1, RT], is the 16-bit
// word P[pidx(y, x)] holding R in its low byte and M (hem8) in its high byte,
// so one load yields both.  Interior columns 0 and 32 sit on 4-byte
// boundaries.  B0 keeps the four border lines as they were when neighbours
// were last queued for them (top, bottom, left, right).
struct CtaTile {
    uint16_t P[(RT + 2) * HS];
    uint8_t B0[4][RT];
    int flags[9];      // neighbours to queue: up, down, left, right, UL, UR, DL, DR, self
    unsigned item;
    int ok, again;
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

// ---- staging ----------------------------------------------------------------------
// A warp's part of the tile halo: line A is the halo row next to its quadrant
// (row -1 for the top quadrants, row RT for the bottom ones) over its 32
// columns, line B the halo column (-1 or RT) over its 32 rows, and lane 0
// adds the corner between them.  The four warps together cover the halo.
__device__ __forceinline__ void halo_coord(int q, int lane, int qy, int qx, int& hy, int& hx) {
    const int ay = qy == 0 ? -1 : RT, bx = qx == 0 ? -1 : RT;
    if (q == 0) { hy = ay; hx = qx + lane; }
    else if (q == 1) { hy = qy + lane; hx = bx; }
    else { hy = ay; hx = bx; }
}

// R (and M) of this warp's halo pixels, 0 outside the image
__device__ __forceinline__ void load_halo(uint8_t hr[3], uint8_t* hm, const uint8_t* Rg, const uint8_t* Mg, int W,
                                          int H, int x0, int y0, int qy, int qx, int lane) {
#pragma unroll
    for (int q = 0; q < 3; q++) {
        int hy, hx;
        halo_coord(q, lane, qy, qx, hy, hx);
        const int gy = y0 + hy, gx = x0 + hx;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W && (q < 2 || lane == 0);
        const size_t o = (size_t)gy * W + gx;
        hr[q] = in ? __ldcg(Rg + o) : (uint8_t)0;
        if (hm) hm[q] = in ? __ldg(Mg + o) : (uint8_t)0;
    }
}

__device__ __forceinline__ void load_quadrant(CtaTile& S, const uint8_t* Rg, const uint8_t* Mg, int W, int H,
                                              int x0, int y0, int qy, int qx, int lane) {
    uint8_t hr[3], hm[3];
    load_halo(hr, hm, Rg, Mg, W, H, x0, y0, qy, qx, lane);
    const int gx0 = x0 + qx, gy0 = y0 + qy;
    if ((W & 3) == 0 && gx0 + QT <= W) {
        // 8 lanes x 4 bytes per row, 4 rows per step, all loads issued first
        const int r4 = lane >> 3, c4 = (lane & 7) * 4;
        uint32_t rv[QT / 4], mv[QT / 4];
#pragma unroll
        for (int j = 0; j < QT / 4; j++) {
            const int gy = gy0 + j * 4 + r4;
            const bool in = gy < H;
            const size_t o = (size_t)gy * W + gx0 + c4;
            rv[j] = in ? __ldcg(reinterpret_cast<const unsigned int*>(Rg + o)) : 0u;
            mv[j] = in ? __ldg(reinterpret_cast<const unsigned int*>(Mg + o)) : 0u;
        }
#pragma unroll
        for (int j = 0; j < QT / 4; j++) {
            // four pixels: (R0 M0 R1 M1) and (R2 M2 R3 M3)
            uint32_t* d = reinterpret_cast<uint32_t*>(&S.P[pidx(qy + j * 4 + r4, qx + c4)]);
            d[0] = __byte_perm(rv[j], mv[j], 0x5140);
            d[1] = __byte_perm(rv[j], mv[j], 0x7362);
        }
    } else {
        const int gx = gx0 + lane;
        for (int y = 0; y < QT; y++) {
            const int gy = gy0 + y;
            const bool in = gy < H && gx < W;
            const size_t o = (size_t)gy * W + gx;
            S.P[pidx(qy + y, qx + lane)] =
                (uint16_t)((in ? __ldcg(Rg + o) : 0) | ((in ? __ldg(Mg + o) : 0) << 8));
        }
    }
#pragma unroll
    for (int q = 0; q < 3; q++) {
        if (q == 2 && lane != 0) continue;
        int hy, hx;
        halo_coord(q, lane, qy, qx, hy, hx);
        S.P[pidx(hy, hx)] = (uint16_t)(hr[q] | (hm[q] << 8));
    }
}

// Writes this warp's quadrant of R back: 4-byte stores where rows are word aligned.
__device__ __forceinline__ void store_quadrant(CtaTile& S, uint8_t* Rg, int W, int H, int x0, int y0, int qy,
                                               int qx, int lane) {
    const int gx0 = x0 + qx, gy0 = y0 + qy;
    if ((W & 3) == 0 && gx0 + QT <= W) {
        const int r4 = lane >> 3, c4 = (lane & 7) * 4;
#pragma unroll
        for (int j = 0; j < QT / 4; j++) {
            const int yy = j * 4 + r4, gy = gy0 + yy;
            if (gy < H) {
                const uint32_t* d = reinterpret_cast<const uint32_t*>(&S.P[pidx(qy + yy, qx + c4)]);
                __stcg(reinterpret_cast<unsigned int*>(Rg + (size_t)gy * W + gx0 + c4), __byte_perm(d[0], d[1], 0x6420));
            }
        }
    } else {
        const int gx = gx0 + lane;
        for (int y = 0; y < QT; y++) {
            const int gy = gy0 + y;
            if (gy < H && gx < W) __stcg(Rg + (size_t)gy * W + gx, SR(qy + y, qx + lane));
        }
    }
}

// Raises this warp's staged halo pixels to the values just read; true if any grew.
__device__ __forceinline__ bool merge_halo(CtaTile& S, const uint8_t hr[3], int qy, int qx, int lane) {
    bool grew = false;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        if (q == 2 && lane != 0) continue;
        int hy, hx;
        halo_coord(q, lane, qy, qx, hy, hx);
        uint8_t& h = SR(hy, hx);
        if (hr[q] > h) {
            h = hr[q];
            grew = true;
        }
    }
    return grew;
}

// ---- sweeps -------------------------------------------------------------------------
// One sweep: QT steps, each updating one line of a quadrant (a row, lanes =
// columns; or a column, lanes = rows) from the three pixels of the line
// before it, which the previous step stored.  A lane's pixel at step i sits
// at index o + i*ds of P; its two diagonal neighbours on the previous line
// are at +/- dl from the previous pixel, where the edge lanes find the halo
// or the neighbouring quadrant, so no lane needs a special case.  With
// R <= M everywhere, max(R, min(m, M)) = min(max(R, m), M).  __syncwarp
// orders each step's stores before the next step's loads; a neighbouring
// quadrant's edge may be read while its warp updates it, which only ever
// yields a value that is still a lower bound of R.
__device__ __forceinline__ void sweep(uint16_t* P, int o, int ds, int dl) {
    uint8_t* R = reinterpret_cast<uint8_t*>(P);  // R of pixel i is byte 2 i
    int prev = R[2 * (o - ds)];
#pragma unroll 8
    for (int i = 0; i < QT; i++, o += ds) {
        const int a = R[2 * (o - ds - dl)], b = R[2 * (o - ds + dl)];
        const uint32_t rm = P[o];
        const int nv = min(max((int)(rm & 0xffu), __vimax3_s32(prev, a, b)), (int)(rm >> 8));
        R[2 * o] = (uint8_t)nv;
        prev = nv;
        __syncwarp();
    }
}

// One round of the four sweeps over quadrant (qy, qx): down, up, right, left.
__device__ __forceinline__ void sweep_round(CtaTile& S, int qy, int qx, int lane) {
    sweep(S.P, pidx(qy, qx + lane), HS, 1);
    sweep(S.P, pidx(qy + QT - 1, qx + lane), -HS, 1);
    sweep(S.P, pidx(qy + lane, qx), 1, HS);
    sweep(S.P, pidx(qy + lane, qx + QT - 1), -1, HS);
}

// Whether some pixel of the quadrant can still be raised by one of its 8
// neighbours: the exact convergence test, for all pixels in parallel (lane
// = column), so it has no dependent chain.
__device__ __forceinline__ bool can_raise(CtaTile& S, int qy, int qx, int lane) {
    const int x = qx + lane;
    int a = __vimax3_s32(SR(qy - 1, x - 1), SR(qy - 1, x), SR(qy - 1, x + 1));
    int b = __vimax3_s32(SR(qy, x - 1), SR(qy, x), SR(qy, x + 1));
    bool v = false;
#pragma unroll 4
    for (int y = 0; y < QT; y++) {
        const int c = __vimax3_s32(SR(qy + y + 1, x - 1), SR(qy + y + 1, x), SR(qy + y + 1, x + 1));
        const uint32_t rm = S.P[pidx(qy + y, x)];
        v |= min(__vimax3_s32(a, b, c), (int)(rm >> 8)) > (int)(rm & 0xffu);
        a = b;
        b = c;
    }
    return __any_sync(FULL, v);
}

// Whether a pixel of a neighbouring quadrant can raise one of this
// quadrant's pixels on the two lines it shares with them.  When this
// quadrant was at a fixed point and has not changed since, only those lines
// can have become raisable, so this is the exact test in that case.
__device__ __forceinline__ bool seam_can_raise(CtaTile& S, int qy, int qx, int lane) {
    const int ex = qx == 0 ? QT - 1 : QT, nx = qx == 0 ? QT : QT - 1;  // own / neighbouring column
    const int ey = qy == 0 ? QT - 1 : QT, ny = qy == 0 ? QT : QT - 1;  // own / neighbouring row
    const int x = qx + lane, y = qy + lane;
    const int mv = __vimax3_s32(SR(y - 1, nx), SR(y, nx), SR(y + 1, nx));
    const int mh = __vimax3_s32(SR(ny, x - 1), SR(ny, x), SR(ny, x + 1));
    const bool v = min(mv, (int)SM(y, ex)) > (int)SR(y, ex) || min(mh, (int)SM(ey, x)) > (int)SR(ey, x);
    return __any_sync(FULL, v);
}

// Whether a halo pixel can raise a pixel of this quadrant's part of the tile
// border.  When the tile's interior was at a fixed point before the halo
// grew, only border pixels can have become raisable, so this is the exact
// test in that case.
__device__ __forceinline__ bool border_can_raise(CtaTile& S, int qy, int qx, int lane) {
    const int by = qy == 0 ? 0 : RT - 1, hy = qy == 0 ? -1 : RT;
    const int bx = qx == 0 ? 0 : RT - 1, hx = qx == 0 ? -1 : RT;
    const int x = qx + lane, y = qy + lane;
    const int mh = __vimax3_s32(SR(hy, x - 1), SR(hy, x), SR(hy, x + 1));
    const int mv = __vimax3_s32(SR(y - 1, hx), SR(y, hx), SR(y + 1, hx));
    const bool v = min(mh, (int)SM(by, x)) > (int)SR(by, x) || min(mv, (int)SM(y, bx)) > (int)SR(y, bx);
    return __any_sync(FULL, v);
}

// ---- neighbour requests ---------------------------------------------------------------
// Side s (0 top, 1 bottom, 2 left, 3 right) of the tile, evaluated by warp s
// after the tile is at a fixed point: halo pixel h of the side (h = -1..RT
// along it) needs its tile queued when a border pixel changed since the last
// requests and next to h can raise it.  h = -1 and h = RT are the halo
// corners, which belong to the diagonal neighbours.  The side's border then
// becomes the reference for the next requests.
__device__ __forceinline__ int side_border(int s, int p) {
    return s == 0 ? pidx(0, p) : s == 1 ? pidx(RT - 1, p) : s == 2 ? pidx(p, 0) : pidx(p, RT - 1);
}
__device__ __forceinline__ int side_halo(int s, int h) {
    return s == 0 ? pidx(-1, h) : s == 1 ? pidx(RT, h) : s == 2 ? pidx(h, -1) : pidx(h, RT);
}
__device__ __forceinline__ void side_requests(CtaTile& S, int s, int lane) {
    const uint8_t* R8 = reinterpret_cast<const uint8_t*>(S.P);
    auto cv = [&](int p) -> int {  // border value at p if it changed since the last requests, else 0
        if (p < 0 || p >= RT) return 0;
        const int v = R8[2 * side_border(s, p)];
        return v != S.B0[s][p] ? v : 0;
    };
    auto raises = [&](int m, int h) -> bool {
        const uint32_t hv = S.P[side_halo(s, h)];
        return min(m, (int)(hv >> 8)) > (int)(hv & 0xffu);
    };
    bool line = false;
#pragma unroll
    for (int u = 0; u < RT / 32; u++) {
        const int h = lane * (RT / 32) + u;
        line |= raises(max(max(cv(h - 1), cv(h)), cv(h + 1)), h);
    }
    const bool lo = lane == 0 && raises(cv(0), -1);
    const bool hi = lane == 31 && raises(cv(RT - 1), RT);
    const bool anyl = __any_sync(FULL, line), anylo = __any_sync(FULL, lo), anyhi = __any_sync(FULL, hi);
    if (lane == 0) {
        // corners: top -> UL, UR; bottom -> DL, DR; left -> UL, DL; right -> UR, DR
        const int cl = s == 0 ? 4 : s == 1 ? 6 : s == 2 ? 4 : 5;
        const int ch = s == 0 ? 5 : s == 1 ? 7 : s == 2 ? 6 : 7;
        if (anyl) S.flags[s] = 1;
        if (anylo) S.flags[cl] = 1;
        if (anyhi) S.flags[ch] = 1;
    }
    __syncwarp();
    for (int p = lane; p < RT; p += 32) S.B0[s][p] = R8[2 * side_border(s, p)];
}

__global__ void __launch_bounds__(RT_WARPS * 32, RECON_MIN_BLOCKS) k_recon(Launch L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    CtaTile& S = *reinterpret_cast<CtaTile*>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qy = (warp >> 1) * QT, qx = (warp & 1) * QT;  // this warp's quadrant
    int visits = 0;  // tile processings of this CTA (diagnostic), added once at exit
    if (threadIdx.x < 9) S.flags[threadIdx.x] = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned it = 0;
            S.ok = wl_pop(L, &it) ? 1 : 0;
            S.item = it;
        }
        __syncthreads();
        if (!S.ok) break;
        const unsigned item = S.item;
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
        if (threadIdx.x == 0) atomicExch(&L.wl_state[t], WL_RUNNING);
        visits++;
        __threadfence();
        __syncthreads();
        load_quadrant(S, Rg, Mg, W, H, x0, y0, qy, qx, lane);
        __syncthreads();
        // the border as loaded is the reference for the first requests; it is
        // taken before any warp sweeps
        for (int p = lane; p < RT; p += 32) S.B0[warp][p] = reinterpret_cast<const uint8_t*>(S.P)[2 * side_border(warp, p)];
        __syncthreads();
        for (;;) {
            int nr = 0;
            bool more = false;
            // this quadrant may still change: all of them on a first visit; on a
            // later one, those whose part of the tile border (or, after a round
            // limit, any pixel) a halo pixel can raise -- the others start at
            // a fixed point, and the seam tests wake them if needed
            bool qgo = true;
            if (!sweep_now) qgo = full_check ? can_raise(S, qy, qx, lane) : border_can_raise(S, qy, qx, lane);
            bool go = sweep_now || __syncthreads_or(qgo);
            sweep_now = false;
            while (go) {
                if (nr >= MAX_ROUNDS) { more = true; break; }
                if (qgo) sweep_round(S, qy, qx, lane);
                __syncthreads();
                nr++;
                // a quadrant that did not sweep was at a fixed point and is
                // unchanged: only its seams with the others can have moved
                qgo = qgo ? can_raise(S, qy, qx, lane) : seam_can_raise(S, qy, qx, lane);
                go = __syncthreads_or(qgo);
            }
            full_check = more;  // otherwise the interior is at a fixed point now
            bool grew = false;
            if (nr > 0) {
                // the halo read only decides which neighbours to queue; it is
                // issued before the write-back so that the two overlap (a stale
                // value can only cause a needless request)
                uint8_t hr[3];
                load_halo(hr, nullptr, Rg, Mg, W, H, x0, y0, qy, qx, lane);
                store_quadrant(S, Rg, W, H, x0, y0, qy, qx, lane);
                __threadfence();  // this tile's pixels before any request
                grew = __syncthreads_or(merge_halo(S, hr, qy, qx, lane));
                side_requests(S, warp, lane);
                if (more && threadIdx.x == 0) S.flags[8] = 1;  // not converged within MAX_ROUNDS: run again
                __syncthreads();
                if (threadIdx.x < 9 && S.flags[threadIdx.x]) {
                    int target = -1;
                    switch (threadIdx.x) {
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
                    S.flags[threadIdx.x] = 0;
                    if (target >= 0) wl_request(L, ti, base, target);
                }
            }
            // every request (and the pending count it adds) comes before this
            // tile stops counting as running
            __syncthreads();
            if (grew) continue;  // the fresher halo may raise pixels: check again
            if (threadIdx.x == 0) {
                // no fence needed here: every write-back above was followed by
                // one, and the requests' pending counts precede this update in
                // the counter's order through the CTA barrier
                const int st = atomicCAS(&L.wl_state[t], WL_RUNNING, WL_IDLE);
                if (st == WL_RUNNING) {
                    atomicAdd(&L.sh->tp, ~0ull);  // pending - 1
                    S.again = 0;
                } else {
                    // a neighbour raised the halo meanwhile: take the tile again
                    atomicExch(&L.wl_state[t], WL_RUNNING);
                    S.again = 1;
                }
            }
            __syncthreads();
            if (!S.again) break;
            visits++;
            __threadfence();
            // every thread of the CTA must take the same branch around the barriers
            if (__syncthreads_or(ld_vol(&L.sh->err) != 0)) break;
            // only the halo can have changed: the interior belongs to this worker
            uint8_t hr[3];
            load_halo(hr, nullptr, Rg, Mg, W, H, x0, y0, qy, qx, lane);
            merge_halo(S, hr, qy, qx, lane);
            __syncthreads();
        }
        __syncthreads();  // the next pop rewrites S.ok and S.item
    }
    if (threadIdx.x == 0 && visits) atomicAdd(&L.sh->processed, visits);
}

// resident CTAs of the reconstruction kernel
int recon_grid(int device) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const size_t smem = sizeof(CtaTile);
    cudaFuncSetAttribute(k_recon, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_recon, RT_WARPS * 32, smem);
    return sms * (per < 1 ? 1 : per);
}

void launch_recon(const Launch& L, int grid_cap, cudaStream_t s, Profiler* pf) {
    if (L.n_rt == 0) return;
    pf->begin("recon_init", s);
    k_wl_init<<<(L.n_rt + 255) / 256, 256, 0, s>>>(L);
    pf->end("recon_init", s);
    const int grid = L.n_rt < grid_cap ? L.n_rt : grid_cap;  // one work tile per CTA at a time
    pf->begin("recon", s);
    k_recon<<<grid, RT_WARPS * 32, sizeof(CtaTile), s>>>(L);
    pf->end("recon", s);
}

}  // namespace nucseg
