// Watershed split of labelled objects on the distance transform (Table I:
// "Pre-Watershed" -- the distance transform and the markers -- and
// "Watershed").  The paper names the operations only; the definition built
// here, for each object k of the label plane:
//   d  = min(255, floor(sqrt(edt))) on the object's pixels;
//   R  = reconstruction by dilation, 8-connected, of max(d - h, 0) under d
//        (the h-maxima of d);
//   markers = maximal 8-connected plateaus of equal R with no 8-neighbour in
//        the object of larger R, each named by its first pixel in raster order;
//   flooding in synchronous waves: with F the unnamed object pixels that have
//        a named 8-neighbour and L = max d over F, every pixel of F with
//        d >= L takes, in one wave, the name of its named neighbour of largest
//        edt (then smallest name); waves repeat at L while any pixel is named,
//        then L is taken again from the new F;
//   out = basins numbered object by object in label order, within an object
//        by the raster order of each basin's first pixel; 0 off the objects.
//
// Objects are independent: two labels are never 8-adjacent (they would be
// one component), and d = 0 off the object keeps R, the plateaus and the
// flooding inside it.  So one warp owns one object: its bounding box plus a
// 1-px margin is staged in shared memory (d, R and later flags in one 16-bit
// word per pixel, edt, and one 32-bit work word), and every step runs there
// with __syncwarp between passes:
//   1. relaxation passes, alternately in raster and anti-raster order, update
//      R in place until a pass changes nothing (monotone updates from below,
//      so the fixed point reached is the reconstruction);
//   2. plateaus by union-find over the work words (roots are the smallest
//      index, i.e. the first pixel), a flag on the root of every plateau with
//      a higher neighbour;
//   3. flooding: the work word holds (wave stamp, name); a pass names the
//      pixels of F at level L with stamp = wave, and only neighbours with an
//      older stamp count, so a pass is exactly one synchronous wave; a pass
//      that names nothing yields the next L from the same reads.  F itself
//      is kept as a list (double-buffered, pixels entered once through an
//      atomic flag), so a wave costs the frontier, not the box;
//   4. each basin's first pixel by atomicMin on its root's word, a ballot
//      prefix over the box in raster order for the ranks.
// Boxes up to WS_STAGE pixels (with margin) go to four-warp CTAs; larger
// ones to one-warp CTAs with a large dynamic stage, launched on a side
// stream so that the few large objects overlap the many small ones; boxes
// beyond that stage run the same steps (with a full-box scan per wave) on
// image-sized scratch planes in global memory.  A scan of the per-object
// basin counts and a pass adding each object's offset finish the numbering.
#include "internal.cuh"

namespace nucseg {

constexpr int WS_WARPS = 4;      // objects in flight per CTA of the small-box kernel (one per warp)
constexpr int WS_STAGE = 1024;   // staged box (with margin) capacity per warp of that kernel, pixels
constexpr int WS_PX_BYTES = 14;  // stage bytes per pixel: e 4, w 4, dr 2, two frontier lists 2 + 2
constexpr int WS_LARGE_SMEM = 96 * 1024;  // dynamic stage of a large-box CTA (one warp)
constexpr unsigned WFULL = 0xffffffffu;

__device__ __forceinline__ int ws_isqrt(int v) {  // floor(sqrt(v)), exact
    if (v <= 0) return 0;
    int r = (int)sqrtf((float)v);
    while ((long long)r * r > v) r--;
    while ((long long)(r + 1) * (r + 1) <= v) r++;
    return r;
}

// Flat positions f = lane, lane+32, ... of a row-major box of width ww, with
// (y, x) of f kept without a division per step.
struct Walk {
    int f, y, x, qy, qx, ww;
    __device__ __forceinline__ Walk(int f0, int ww_) : f(f0), ww(ww_) {
        y = f0 / ww;
        x = f0 - y * ww;
        qy = 32 / ww;
        qx = 32 - qy * ww;
    }
    __device__ __forceinline__ void next() {
        f += 32;
        x += qx;
        y += qy;
        if (x >= ww) { x -= ww; y++; }
    }
    __device__ __forceinline__ void prev() {
        f -= 32;
        x -= qx;
        y -= qy;
        if (x < 0) { x += ww; y--; }
    }
};

// Shared-memory box: the object's box plus a 1-px margin, row stride ww.
// Pixels off the object (margin, background, other objects) are staged with
// dr = 0 and w = all ones, so neighbour reads need no bounds or label tests.
struct SBox {
    using Wt = uint32_t;
    static constexpr bool GLOBAL = false;
    static constexpr int SH = 16;               // name bits (indices < 2^16)
    volatile uint16_t* dr;                      // d | R << 8; later bit 8 marker, 9 first pixel, 10 in F once
    volatile int32_t* e;                        // edt
    volatile Wt* w;                             // work word
    volatile uint16_t *la, *lb;                 // frontier lists, n entries each
    int ww, n;                                  // walk width, flat size
    int gx0, gy0, W;                            // image position of flat (0, 0)
    __device__ __forceinline__ int stor(const Walk& it) const { return it.f; }
    __device__ __forceinline__ bool in(int s) const { return (dr[s] & 0xFF) != 0; }
    __device__ __forceinline__ int nb(const Walk&, int s, int dy, int dx) const { return s + dy * ww + dx; }
    __device__ __forceinline__ size_t gidx(const Walk& it) const {
        return (size_t)(gy0 + it.y) * W + (gx0 + it.x);
    }
};

// Global box: the object's box (no margin) inside image-sized scratch planes
// (row stride W); membership from the label plane, bounds tested.
struct GBox {
    using Wt = unsigned long long;
    static constexpr bool GLOBAL = true;
    static constexpr int SH = 32;
    volatile uint16_t* dr;
    const int32_t* e;
    volatile Wt* w;
    const int32_t* lab;
    int k;
    int ww, bh, n;
    int gx0, gy0, W;
    __device__ __forceinline__ int stor(const Walk& it) const { return it.y * W + it.x; }
    __device__ __forceinline__ bool in(int s) const { return lab[s] == k; }
    __device__ __forceinline__ int nb(const Walk& it, int s, int dy, int dx) const {
        return ((unsigned)(it.y + dy) < (unsigned)bh && (unsigned)(it.x + dx) < (unsigned)ww) ? s + dy * W + dx
                                                                                              : -1;
    }
    __device__ __forceinline__ size_t gidx(const Walk& it) const {
        return (size_t)(gy0 + it.y) * W + (gx0 + it.x);
    }
};

template <class B>
__device__ __forceinline__ bool ws_nb_in(const B& b, int q) {
    if constexpr (B::GLOBAL) return q >= 0 && b.in(q);
    else return b.in(q);
}

template <class B>
__device__ __forceinline__ int ws_find(const B& b, int x) {
    // path halving: a non-root is pointed at its grandparent (an ancestor,
    // whatever concurrent unions do, so the forest stays valid); without it
    // the walks over a plateau of a thousand pixels grow with its size
    constexpr typename B::Wt IDX = ((typename B::Wt)1 << B::SH) - 1;
    for (;;) {
        const int p = (int)(b.w[x] & IDX);
        if (p == x) return x;
        const int gp = (int)(b.w[p] & IDX);
        if (gp != p) b.w[x] = (typename B::Wt)gp;
        x = gp;
    }
}

// Union of the plateaus of a and b; the larger root is linked under the
// smaller, so every root is its set's first pixel.
template <class B>
__device__ __forceinline__ void ws_unite(const B& b, int a, int c) {
    using Wt = typename B::Wt;
    for (;;) {
        a = ws_find(b, a);
        c = ws_find(b, c);
        if (a == c) return;
        if (a < c) { const int t = a; a = c; c = t; }
        const Wt old = atomicCAS((Wt*)(b.w + a), (Wt)a, (Wt)c);
        if (old == (Wt)a) return;
    }
}

// The four steps on one object.  Returns the number of basins (0 on a wave
// count beyond the cap, after setting the status word).
template <class B>
__device__ int ws_object(const B& b, int lane, int32_t* out, int* status) {
    using Wt = typename B::Wt;
    constexpr Wt IDX = ((Wt)1 << B::SH) - 1;
    constexpr Wt FLAG = (Wt)1 << (sizeof(Wt) * 8 - 1);
    constexpr Wt UNNAMED = ~(Wt)0;

    // 1. R: relaxation passes until one changes nothing
    for (int pass = 0;; pass++) {
        bool ch = false;
        auto relax = [&](const Walk& it) {
            const int s = b.stor(it);
            if (!b.in(s)) return;
            const unsigned v = b.dr[s];
            const int d = v & 0xFF, r = v >> 8;
            int m = r;
#pragma unroll
            for (int j = 0; j < 9; j++) {
                if (j == 4) continue;
                const int q = b.nb(it, s, j / 3 - 1, j % 3 - 1);
                if constexpr (B::GLOBAL) {
                    if (!ws_nb_in(b, q)) continue;
                }
                m = max(m, (int)(b.dr[q] >> 8));
            }
            m = min(m, d);
            if (m != r) {
                b.dr[s] = (uint16_t)(d | (m << 8));
                ch = true;
            }
        };
        if ((pass & 1) == 0) {
            for (Walk it(lane, b.ww); it.f < b.n; it.next()) relax(it);
        } else {
            const int last = b.n - 1 - lane;
            if (last >= 0)
                for (Walk it(last, b.ww); it.f >= 0; it.prev()) relax(it);
        }
        __syncwarp();
        if (!__any_sync(WFULL, ch)) break;
    }

    // 2. plateaus of equal R: union-find, then the non-maximal flag on roots
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {
        const int s = b.stor(it);
        if (b.in(s)) b.w[s] = (Wt)s;
    }
    __syncwarp();
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {
        const int s = b.stor(it);
        if (!b.in(s)) continue;
        const int r = b.dr[s] >> 8;
#pragma unroll
        for (int j = 0; j < 4; j++) {  // the neighbours before s in raster order
            const int q = b.nb(it, s, j < 3 ? -1 : 0, j < 3 ? j - 1 : -1);
            if (!ws_nb_in(b, q)) continue;
            if ((int)(b.dr[q] >> 8) == r) ws_unite(b, s, q);
        }
    }
    __syncwarp();
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {
        const int s = b.stor(it);
        if (b.in(s)) b.w[s] = (Wt)ws_find(b, s);
    }
    __syncwarp();
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {
        const int s = b.stor(it);
        if (!b.in(s)) continue;
        const int r = b.dr[s] >> 8;
        bool higher = false;
#pragma unroll
        for (int j = 0; j < 9; j++) {
            if (j == 4) continue;
            const int q = b.nb(it, s, j / 3 - 1, j % 3 - 1);
            if (!ws_nb_in(b, q)) continue;
            higher |= (int)(b.dr[q] >> 8) > r;
        }
        if (higher) atomicOr((Wt*)(b.w + (int)(b.w[s] & IDX)), FLAG);
    }
    __syncwarp();
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {  // bit 8 of dr: a marker pixel (R no longer needed)
        const int s = b.stor(it);
        if (!b.in(s)) continue;
        const bool mk = !(b.w[(int)(b.w[s] & IDX)] & FLAG);
        b.dr[s] = (uint16_t)((b.dr[s] & 0xFF) | (mk ? 0x100 : 0));
    }
    __syncwarp();
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {  // markers: stamp 0, name = root
        const int s = b.stor(it);
        if (!b.in(s)) continue;
        b.w[s] = (b.dr[s] & 0x100) ? (b.w[s] & IDX) : UNNAMED;
    }
    __syncwarp();

    // 3. flooding in synchronous waves
    {
        const unsigned cap = (unsigned)min((long long)b.n + 300, (long long)IDX - 1);
        if constexpr (B::GLOBAL) {
            // full-box scan per wave (boxes beyond every stage: rare)
            int L = 256;  // above every d: the first pass only measures F
            for (unsigned wave = 1;; wave++) {
                if (wave >= cap) {
                    if (lane == 0) set_status(status, ST_OVERFLOW);
                    return 0;
                }
                int named = 0, fmax = -1;
                for (Walk it(lane, b.ww); it.f < b.n; it.next()) {
                    const int s = b.stor(it);
                    if (!b.in(s) || b.w[s] != UNNAMED) continue;
                    int be = 0;
                    Wt bn = IDX;
#pragma unroll
                    for (int j = 0; j < 9; j++) {
                        if (j == 4) continue;
                        const int q = b.nb(it, s, j / 3 - 1, j % 3 - 1);
                        if (!ws_nb_in(b, q)) continue;
                        const Wt wq = b.w[q];
                        if ((wq >> B::SH) >= (Wt)wave) continue;  // unnamed, or named in this wave
                        const int eq = b.e[q];
                        const Wt nq = wq & IDX;
                        if (eq > be || (eq == be && nq < bn)) {
                            be = eq;
                            bn = nq;
                        }
                    }
                    if (be > 0) {
                        const int d = b.dr[s] & 0xFF;
                        fmax = max(fmax, d);
                        if (d >= L) {
                            b.w[s] = ((Wt)wave << B::SH) | bn;
                            named++;
                        }
                    }
                }
                __syncwarp();
                named = __reduce_add_sync(WFULL, (unsigned)named);
                fmax = (int)__reduce_max_sync(WFULL, (unsigned)(fmax + 1)) - 1;
                if (!named) {
                    if (fmax < 0) break;
                    L = fmax;
                }
            }
        } else {
            // F as a list: entries enter once (bit 10 of dr, set atomically on
            // the 32-bit word holding it; nothing else writes dr meanwhile)
            const unsigned lt = (1u << lane) - 1;
            auto enter = [&](int q) -> bool {
                const uintptr_t a = (uintptr_t)(b.dr + q);
                const unsigned sh = (unsigned)(a & 2) * 8;
                const unsigned old = atomicOr((unsigned*)(a & ~(uintptr_t)3), 0x400u << sh);
                return !((old >> sh) & 0x400u);
            };
            volatile uint16_t* cur = b.la;
            volatile uint16_t* nxt = b.lb;
            int m = 0;
            for (int f0 = 0; f0 < b.n; f0 += 32) {  // neighbours of the markers
                const int s = f0 + lane;
                const bool mk = s < b.n && b.w[s] != UNNAMED;
#pragma unroll
                for (int j = 0; j < 9; j++) {
                    if (j == 4) continue;
                    const int q = s + (j / 3 - 1) * b.ww + (j % 3 - 1);
                    const bool add = mk && b.in(q) && b.w[q] == UNNAMED && enter(q);
                    const unsigned bal = __ballot_sync(WFULL, add);
                    if (add) cur[m + __popc(bal & lt)] = (uint16_t)q;
                    m += __popc(bal);
                }
            }
            __syncwarp();
            int L = 256;
            for (unsigned wave = 1; m > 0; wave++) {
                if (wave >= cap) {
                    if (lane == 0) set_status(status, ST_OVERFLOW);
                    return 0;
                }
                int named = 0, fmax = -1, nm = 0;
                for (int i0 = 0; i0 < m; i0 += 32) {
                    const int i = i0 + lane;
                    const int s = i < m ? (int)cur[i] : -1;
                    bool took = false;
                    if (s >= 0) {
                        int be = 0;
                        Wt bn = IDX;
#pragma unroll
                        for (int j = 0; j < 9; j++) {
                            if (j == 4) continue;
                            const int q = s + (j / 3 - 1) * b.ww + (j % 3 - 1);
                            const Wt wq = b.w[q];
                            if ((wq >> B::SH) >= (Wt)wave) continue;  // unnamed, or named in this wave
                            const int eq = b.e[q];
                            const Wt nq = wq & IDX;
                            if (eq > be || (eq == be && nq < bn)) {
                                be = eq;
                                bn = nq;
                            }
                        }
                        if (be > 0) {
                            const int d = b.dr[s] & 0xFF;
                            fmax = max(fmax, d);
                            if (d >= L) {
                                b.w[s] = ((Wt)wave << B::SH) | bn;
                                named++;
                                took = true;
                            }
                        }
                    }
                    const bool keep = s >= 0 && !took;
                    unsigned bal = __ballot_sync(WFULL, keep);
                    if (keep) nxt[nm + __popc(bal & lt)] = (uint16_t)s;
                    nm += __popc(bal);
#pragma unroll
                    for (int j = 0; j < 9; j++) {  // unnamed neighbours of a pixel just named enter F
                        if (j == 4) continue;
                        const int q = s + (j / 3 - 1) * b.ww + (j % 3 - 1);
                        const bool add = took && b.in(q) && b.w[q] == UNNAMED && enter(q);
                        bal = __ballot_sync(WFULL, add);
                        if (add) nxt[nm + __popc(bal & lt)] = (uint16_t)q;
                        nm += __popc(bal);
                    }
                }
                __syncwarp();
                named = __reduce_add_sync(WFULL, (unsigned)named);
                fmax = (int)__reduce_max_sync(WFULL, (unsigned)(fmax + 1)) - 1;
                if (!named) {
                    if (fmax < 0) break;
                    L = fmax;
                }
                volatile uint16_t* t = cur;
                cur = nxt;
                nxt = t;
                m = nm;
            }
        }
    }

    // 4. ranks of the basins by first pixel
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {  // roots: first-pixel field to "none"
        const int s = b.stor(it);
        if (b.in(s) && (int)(b.w[s] & IDX) == s) b.w[s] = (IDX << B::SH) | (Wt)s;
    }
    __syncwarp();
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {
        const int s = b.stor(it);
        if (!b.in(s)) continue;
        const Wt nm = b.w[s] & IDX;
        atomicMin((Wt*)(b.w + (int)nm), ((Wt)s << B::SH) | nm);
    }
    __syncwarp();
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {  // bit 9 of dr: the first pixel of its basin
        const int s = b.stor(it);
        if (!b.in(s)) continue;
        const int nm = (int)(b.w[s] & IDX);
        if ((int)(b.w[nm] >> B::SH) == s) b.dr[s] = (uint16_t)(b.dr[s] | 0x200);
    }
    __syncwarp();
    int run = 0;
    for (int f0 = 0; f0 < b.n; f0 += 32) {  // raster order: rank = first pixels up to this one
        const int f = f0 + lane;
        bool first = false;
        int s = 0;
        if (f < b.n) {
            const Walk it(f, b.ww);
            s = b.stor(it);
            first = b.in(s) && (b.dr[s] & 0x200);
        }
        const unsigned bal = __ballot_sync(WFULL, first);
        if (first) {
            const Wt nm = b.w[s] & IDX;
            const int rank = run + __popc(bal & ((1u << lane) - 1)) + 1;
            b.w[(int)nm] = ((Wt)rank << B::SH) | nm;
        }
        run += __popc(bal);
    }
    __syncwarp();
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {
        const int s = b.stor(it);
        if (!b.in(s)) continue;
        out[b.gidx(it)] = (int32_t)(b.w[(int)(b.w[s] & IDX)] >> B::SH);
    }
    return run;
}

// Large boxes: the same steps on global scratch planes, kept out of line.
__device__ __noinline__ int ws_object_global(const int32_t* labels, const int32_t* edt, int W, int k, int4 bx,
                                             int h, uint16_t* gdr, unsigned long long* gw, int32_t* out,
                                             int* status, int lane) {
    GBox b;
    const size_t o = (size_t)bx.y * W + bx.x;
    b.dr = gdr + o;
    b.e = edt + o;
    b.w = gw + o;
    b.lab = labels + o;
    b.k = k;
    b.ww = bx.z - bx.x + 1;
    b.bh = bx.w - bx.y + 1;
    b.n = b.ww * b.bh;
    b.gx0 = bx.x;
    b.gy0 = bx.y;
    b.W = W;
    for (Walk it(lane, b.ww); it.f < b.n; it.next()) {
        const int s = b.stor(it);
        if (!b.in(s)) continue;
        const int d = min(255, ws_isqrt(b.e[s]));
        b.dr[s] = (uint16_t)(d | ((d > h ? d - h : 0) << 8));
    }
    __syncwarp();
    return ws_object(b, lane, out, status);
}

// Stages one object's box plus margin into a shared-memory stage of `cap`
// pixels (e, w, dr and the two frontier lists, laid out back to back) and
// splits it there.
__device__ __forceinline__ int ws_staged(const int32_t* __restrict__ labels, const int32_t* __restrict__ edt,
                                         int W, int H, int k, int4 bx, int h, char* stage, int cap,
                                         int32_t* out, int* status, int lane) {
    const int BW = bx.z - bx.x + 3, BH = bx.w - bx.y + 3;
    SBox b;
    b.e = (int32_t*)stage;
    b.w = (uint32_t*)(stage + 4 * cap);
    b.dr = (uint16_t*)(stage + 8 * cap);
    b.la = (uint16_t*)(stage + 10 * cap);
    b.lb = (uint16_t*)(stage + 12 * cap);
    b.ww = BW;
    b.n = BW * BH;
    b.gx0 = bx.x - 1;
    b.gy0 = bx.y - 1;
    b.W = W;
    for (Walk it(lane, BW); it.f < b.n; it.next()) {
        const int gy = b.gy0 + it.y, gx = b.gx0 + it.x;
        int ev = 0;
        if ((unsigned)gy < (unsigned)H && (unsigned)gx < (unsigned)W) {
            const size_t g = (size_t)gy * W + gx;
            if (labels[g] == k) ev = edt[g];
        }
        const int d = ev > 0 ? min(255, ws_isqrt(ev)) : 0;
        b.dr[it.f] = (uint16_t)(d | ((d > h ? d - h : 0) << 8));
        b.e[it.f] = ev;
        b.w[it.f] = 0xffffffffu;
    }
    __syncwarp();
    return ws_object(b, lane, out, status);
}

__device__ __forceinline__ int ws_box_px(int4 bx) { return (bx.z - bx.x + 3) * (bx.w - bx.y + 3); }

// The next entry for this warp from a launch-wide counter (entries go to
// whichever warp is free, so a warp that drew a slow object takes no more).
__device__ __forceinline__ int ws_next(int* next, int lane) {
    int v = 0;
    if (lane == 0) v = atomicAdd(next, 1);
    return __shfl_sync(WFULL, v, 0);
}

// Sorts the objects before the two object kernels: an absent object
// (empty box) gets count 0; an object whose box exceeds the small stage is
// appended to the large list (next[1] entries).
__global__ void k_ws_classify(const int4* __restrict__ bbox, int total, int* cnt, int* next, int* list) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int4 bx = bbox[i];
    if (bx.z < bx.x) cnt[i] = 0;
    else if (ws_box_px(bx) > WS_STAGE) list[atomicAdd(next + 1, 1)] = i;
}

// Small boxes: persistent warps drawing objects from a launch-wide counter
// (next[2]), WS_STAGE pixels of stage each.  Writes the basin's rank inside
// the object to out and the basin count to cnt[object]; absent objects and
// larger boxes were sorted out by k_ws_classify.
__global__ void __launch_bounds__(WS_WARPS * 32) k_ws_objects(const int32_t* __restrict__ labels,
                                                               const int32_t* __restrict__ edt, int W, int H,
                                                               int K, int h, const int4* __restrict__ bbox,
                                                               int32_t* out, int* cnt, int* next, int* status) {
    extern __shared__ __align__(16) char ws_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    char* stage = ws_smem + (size_t)warp * WS_STAGE * WS_PX_BYTES;
    for (int obj = ws_next(next + 2, lane); obj < K; obj = ws_next(next + 2, lane)) {
        const int4 bx = bbox[obj];
        if (bx.z < bx.x || ws_box_px(bx) > WS_STAGE) continue;
        const int c = ws_staged(labels, edt, W, H, obj + 1, bx, h, stage, WS_STAGE, out, status, lane);
        if (lane == 0) cnt[obj] = c;
        __syncwarp();
    }
}

// Large boxes: one warp per CTA with a stage of `cap` pixels, drawing from
// the large list (next[0] the draw counter, next[1] its length); boxes
// beyond the stage run on the global scratch planes.
__global__ void __launch_bounds__(32) k_ws_large(const int32_t* __restrict__ labels, const int32_t* __restrict__ edt,
                                                 int W, int H, int h, const int4* __restrict__ bbox, int32_t* out,
                                                 int* cnt, int cap, uint16_t* gdr, unsigned long long* gw, int* next,
                                                 const int* __restrict__ list, int* status) {
    extern __shared__ __align__(16) char ws_smem[];
    const int lane = threadIdx.x;
    const int nl = next[1];
    for (int i = ws_next(next, lane); i < nl; i = ws_next(next, lane)) {
        const int obj = list[i];
        const int4 bx = bbox[obj];
        const int c = ws_box_px(bx) <= cap
                          ? ws_staged(labels, edt, W, H, obj + 1, bx, h, ws_smem, cap, out, status, lane)
                          : ws_object_global(labels, edt, W, obj + 1, bx, h, gdr, gw, out, status, lane);
        if (lane == 0) cnt[obj] = c;
        __syncwarp();
    }
}

// In place: cnt[i] -> exclusive prefix; total -> *n_basins (one CTA of 1024).
__device__ __forceinline__ void ws_scan_block(int* cnt, int K, int32_t* n_basins) {
    __shared__ int wsum[32];
    __shared__ int carry;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < K; base += 1024) {
        const int i = base + t;
        const int v = i < K ? cnt[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(WFULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(WFULL, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const int excl = carry + (wid ? wsum[wid - 1] : 0) + x - v;
        if (i < K) cnt[i] = excl;
        __syncthreads();
        if (t == 1023) carry = excl + v;
        __syncthreads();
    }
    if (t == 0) *n_basins = carry;
}

__global__ void __launch_bounds__(1024) k_ws_scan(int* cnt, int K, int32_t* n_basins) {
    ws_scan_block(cnt, K, n_basins);
}

// out += o on the pixels of object k inside box bx (one warp).
__device__ __forceinline__ void ws_offset_obj(const int32_t* __restrict__ labels, int W, int k, int4 bx, int o,
                                              int32_t* out, int lane) {
    const int bw = bx.z - bx.x + 1, n = bw * (bx.w - bx.y + 1);
    for (Walk it(lane, bw); it.f < n; it.next()) {
        const size_t g = (size_t)(bx.y + it.y) * W + (bx.x + it.x);
        if (labels[g] == k) out[g] += o;
    }
}

// out += the object's first basin number - 1 on the object's pixels.
__global__ void __launch_bounds__(256) k_ws_offset(const int32_t* __restrict__ labels, int W, int K,
                                                   const int4* __restrict__ bbox, const int* __restrict__ off,
                                                   int32_t* out) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int obj = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); obj < K; obj += nw) {
        const int o = off[obj];
        const int4 bx = bbox[obj];
        if (o == 0 || bx.z < bx.x) continue;
        ws_offset_obj(labels, W, obj + 1, bx, o, out, lane);
    }
}

// ---- batched form: the objects of many tiles in one launch per pass ----------------
// Items are objects numbered across the tiles; the tile of an item is the last
// descriptor whose obj_base is <= the item (seg_base likewise for box segments).
__device__ __forceinline__ int ws_desc_of(const WsDesc* __restrict__ D, int n, int item, bool by_seg) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((by_seg ? D[mid].seg_base : D[mid].obj_base) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int WS_DESC_PACK = 16;
struct WsDescPack {
    int first, n;
    WsDesc d[WS_DESC_PACK];
};

__global__ void k_ws_set_desc(WsDesc* dst, WsDescPack pk) {
    if ((int)threadIdx.x < pk.n) dst[pk.first + threadIdx.x] = pk.d[threadIdx.x];
}

__global__ void k_ws_bbox_init_b(int4* bbox, int total) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) bbox[i] = make_int4(0x7fffffff, 0x7fffffff, -1, -1);
}

__global__ void __launch_bounds__(256) k_ws_bbox_b(const WsDesc* __restrict__ D, int n, int total_segs,
                                                   int4* bbox) {
    const int lane = threadIdx.x & 31;
    const int gw = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (gw >= total_segs) return;
    const WsDesc& T = D[ws_desc_of(D, n, gw, true)];
    const int k = gw - T.seg_base, spr = (T.W + FB_SEG - 1) / FB_SEG;
    const int y = k / spr, xs = (k - y * spr) * FB_SEG;
    bbox_segment(T.labels + (size_t)y * T.W, T.W, T.K, y, xs, bbox + T.obj_base, lane);
}

__global__ void __launch_bounds__(WS_WARPS * 32) k_ws_objects_b(const WsDesc* __restrict__ D, int n, int total,
                                                                 int h, const int4* __restrict__ bbox, int* cnt,
                                                                 int* next, int* status) {
    extern __shared__ __align__(16) char ws_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    char* stage = ws_smem + (size_t)warp * WS_STAGE * WS_PX_BYTES;
    for (int item = ws_next(next + 2, lane); item < total; item = ws_next(next + 2, lane)) {
        const int4 bx = bbox[item];
        if (bx.z < bx.x || ws_box_px(bx) > WS_STAGE) continue;
        const WsDesc& T = D[ws_desc_of(D, n, item, false)];
        const int c = ws_staged(T.labels, T.edt, T.W, T.H, item - T.obj_base + 1, bx, h, stage, WS_STAGE, T.out,
                                status, lane);
        if (lane == 0) cnt[item] = c;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(32) k_ws_large_b(const WsDesc* __restrict__ D, int n, int h,
                                                   const int4* __restrict__ bbox, int* cnt, int cap, uint16_t* gdr,
                                                   unsigned long long* gw, int* next, const int* __restrict__ list,
                                                   int* status) {
    extern __shared__ __align__(16) char ws_smem[];
    const int lane = threadIdx.x;
    const int nl = next[1];
    for (int i = ws_next(next, lane); i < nl; i = ws_next(next, lane)) {
        const int item = list[i];
        const int4 bx = bbox[item];
        const WsDesc& T = D[ws_desc_of(D, n, item, false)];
        const int k = item - T.obj_base + 1;
        const int c = ws_box_px(bx) <= cap
                          ? ws_staged(T.labels, T.edt, T.W, T.H, k, bx, h, ws_smem, cap, T.out, status, lane)
                          : ws_object_global(T.labels, T.edt, T.W, k, bx, h, gdr + T.px_base, gw + T.px_base,
                                             T.out, status, lane);
        if (lane == 0) cnt[item] = c;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(1024) k_ws_scan_b(const WsDesc* __restrict__ D, int* cnt) {
    const WsDesc& T = D[blockIdx.x];
    ws_scan_block(cnt + T.obj_base, T.K, T.n_basins);
}

__global__ void __launch_bounds__(256) k_ws_offset_b(const WsDesc* __restrict__ D, int n, int total,
                                                     const int4* __restrict__ bbox, const int* __restrict__ off) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < total; item += nw) {
        const int o = off[item];
        const int4 bx = bbox[item];
        if (o == 0 || bx.z < bx.x) continue;
        const WsDesc& T = D[ws_desc_of(D, n, item, false)];
        ws_offset_obj(T.labels, T.W, item - T.obj_base + 1, bx, o, T.out, lane);
    }
}

size_t watershed_scratch_bytes(int W, int H) {
    return (size_t)W * H * (sizeof(unsigned long long) + sizeof(uint16_t));
}

void launch_watershed(const int32_t* labels, const int32_t* edt, int W, int H, int K, int h, int32_t* out,
                      int32_t* n_basins, int4* bbox, int* cnt, int* next, void* scratch, int* status, int sms,
                      cudaStream_t s, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join, Profiler* pf) {
    static bool attrs[64] = {};  // opt-in shared memory above 48 KB, once per device
    const int small_smem = WS_WARPS * WS_STAGE * WS_PX_BYTES;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attrs[dev]) {
        cudaFuncSetAttribute(k_ws_objects, cudaFuncAttributeMaxDynamicSharedMemorySize, small_smem);
        cudaFuncSetAttribute(k_ws_large, cudaFuncAttributeMaxDynamicSharedMemorySize, WS_LARGE_SMEM);
        if (dev >= 0 && dev < 64) attrs[dev] = true;
    }
    const size_t N = (size_t)W * H;
    cudaMemsetAsync(out, 0, N * sizeof(int32_t), s);
    if (K <= 0) {
        cudaMemsetAsync(n_basins, 0, sizeof(int32_t), s);
        return;
    }
    launch_object_boxes(labels, W, H, K, bbox, s, pf);
    unsigned long long* gw = (unsigned long long*)scratch;
    uint16_t* gdr = (uint16_t*)(gw + N);
    int* list = next + 3;
    cudaMemsetAsync(next, 0, 3 * sizeof(int), s);
    pf->begin("ws_classify", s);
    k_ws_classify<<<(K + 255) / 256, 256, 0, s>>>(bbox, K, cnt, next, list);
    pf->end("ws_classify", s);
    // the large boxes on the (higher-priority) side stream, overlapping the small ones
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(side, fork, 0);
    pf->begin("ws_large", side);
    k_ws_large<<<K < sms ? K : sms, 32, WS_LARGE_SMEM, side>>>(labels, edt, W, H, h, bbox, out, cnt,
                                                           WS_LARGE_SMEM / WS_PX_BYTES, gdr, gw, next, list,
                                                           status);
    pf->end("ws_large", side);
    cudaEventRecord(join, side);
    const int ctas = (K + WS_WARPS - 1) / WS_WARPS;
    pf->begin("ws_objects", s);
    k_ws_objects<<<ctas < sms * 4 ? ctas : sms * 4, WS_WARPS * 32, small_smem, s>>>(labels, edt, W, H, K, h, bbox,
                                                                                 out, cnt, next, status);
    pf->end("ws_objects", s);
    cudaStreamWaitEvent(s, join, 0);
    pf->begin("ws_scan", s);
    k_ws_scan<<<1, 1024, 0, s>>>(cnt, K, n_basins);
    pf->end("ws_scan", s);
    const int octas = (K + 7) / 8;
    pf->begin("ws_offset", s);
    k_ws_offset<<<octas < sms * 8 ? octas : sms * 8, 256, 0, s>>>(labels, W, K, bbox, cnt, out);
    pf->end("ws_offset", s);
}

void launch_watershed_batch(const std::vector<WsDesc>& descs, WsDesc* d_descs, int h, int4* bbox, int* cnt,
                            int* next, void* scratch, size_t scratch_px, int* status, int sms, cudaStream_t s,
                            cudaStream_t side, cudaEvent_t fork, cudaEvent_t join, Profiler* pf) {
    static bool attrs[64] = {};  // opt-in shared memory above 48 KB, once per device
    const int small_smem = WS_WARPS * WS_STAGE * WS_PX_BYTES;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attrs[dev]) {
        cudaFuncSetAttribute(k_ws_objects_b, cudaFuncAttributeMaxDynamicSharedMemorySize, small_smem);
        cudaFuncSetAttribute(k_ws_large_b, cudaFuncAttributeMaxDynamicSharedMemorySize, WS_LARGE_SMEM);
        if (dev >= 0 && dev < 64) attrs[dev] = true;
    }
    const int n = (int)descs.size();
    int total = 0, segs = 0;
    for (const WsDesc& d : descs) {
        cudaMemsetAsync(d.out, 0, (size_t)d.W * d.H * sizeof(int32_t), s);
        total += d.K;
        segs += (d.W + FB_SEG - 1) / FB_SEG * d.H;
    }
    for (int i = 0; i < n; i += WS_DESC_PACK) {
        WsDescPack pk;
        pk.first = i;
        pk.n = n - i < WS_DESC_PACK ? n - i : WS_DESC_PACK;
        for (int k = 0; k < pk.n; k++) pk.d[k] = descs[i + k];
        k_ws_set_desc<<<1, WS_DESC_PACK, 0, s>>>(d_descs, pk);
    }
    if (total > 0) {
        unsigned long long* gw = (unsigned long long*)scratch;
        uint16_t* gdr = (uint16_t*)(gw + scratch_px);
        pf->begin("ws_bbox_init", s);
        k_ws_bbox_init_b<<<(total + 255) / 256, 256, 0, s>>>(bbox, total);
        pf->end("ws_bbox_init", s);
        pf->begin("ws_bbox", s);
        k_ws_bbox_b<<<(unsigned)(((long long)segs * 32 + 255) / 256), 256, 0, s>>>(d_descs, n, segs, bbox);
        pf->end("ws_bbox", s);
        int* list = next + 3;
        cudaMemsetAsync(next, 0, 3 * sizeof(int), s);
        pf->begin("ws_classify", s);
        k_ws_classify<<<(total + 255) / 256, 256, 0, s>>>(bbox, total, cnt, next, list);
        pf->end("ws_classify", s);
        cudaEventRecord(fork, s);
        cudaStreamWaitEvent(side, fork, 0);
        pf->begin("ws_large", side);
        k_ws_large_b<<<total < sms ? total : sms, 32, WS_LARGE_SMEM, side>>>(
            d_descs, n, h, bbox, cnt, WS_LARGE_SMEM / WS_PX_BYTES, gdr, gw, next, list, status);
        pf->end("ws_large", side);
        cudaEventRecord(join, side);
        const int ctas = (total + WS_WARPS - 1) / WS_WARPS;
        pf->begin("ws_objects", s);
        k_ws_objects_b<<<ctas < sms * 4 ? ctas : sms * 4, WS_WARPS * 32, small_smem, s>>>(d_descs, n, total, h, bbox,
                                                                                        cnt, next, status);
        pf->end("ws_objects", s);
        cudaStreamWaitEvent(s, join, 0);
    }
    pf->begin("ws_scan", s);
    k_ws_scan_b<<<n, 1024, 0, s>>>(d_descs, cnt);
    pf->end("ws_scan", s);
    if (total > 0) {
        const int octas = (total + 7) / 8;
        pf->begin("ws_offset", s);
        k_ws_offset_b<<<octas < sms * 8 ? octas : sms * 8, 256, 0, s>>>(d_descs, n, total, bbox, cnt);
        pf->end("ws_offset", s);
    }
}

}  // namespace nucseg
