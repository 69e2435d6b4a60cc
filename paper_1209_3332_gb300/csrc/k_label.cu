// K3 + K4: fill holes (Table I, "FillHoles"), 8-connected labelling
// (Table I, "BWLabel") with the area filter (Table I, "AreaThreshold") and
// a deterministic raster-order relabel.
//
// Both steps are connected-component problems solved with the same block
// union-find scheme:
//  * one warp labels a 32x32 block: lane y holds the 32-bit class word of
//    row y, runs of set bits are the union-find nodes, and only runs of
//    adjacent rows that touch are unioned (links point to the smaller
//    index, so every local root is the first pixel, row-major, of its local
//    component);
//  * local roots get a slot in the sparse global arrays P (parent) and A
//    (payload) at their own pixel index and are appended to a root list;
//  * block edges publish the local roots of their edge pixels; a merge
//    kernel unions facing edge pixels in P with atomicMin links, so global
//    roots are again component-first pixels;
//  * later kernels recompute the local labelling from the 2 MB bitmaps
//    instead of storing a full plane of provisional labels;
//  * a warp's only large shared array is its 1024-entry union-find table
//    (4 KB), whose root entries also carry a component's payload in bits
//    16 and up, so that 14 CTAs of 4 warps fit on an SM.
// Fill holes labels the background with 4-connectivity (dual of the 8-conn
// foreground) and marks components that touch the image border; every
// background pixel of an unmarked component is a hole.  Labelling then
// counts areas per root, marks roots whose area is in [amin, amax] in a
// root bitmap, and numbers them by an exclusive popcount prefix over that
// bitmap -- which is the row-major order of first pixels.
#include "internal.cuh"

namespace nucseg {

constexpr unsigned FULLM = 0xffffffffu;

// ---- shared-memory union-find ---------------------------------------------------
// A warp's table holds one entry per pixel of its 32x32 block, local index
// i = 32 y + x.  Entry i lives in slot 32 y + ((x + y) mod 32): the lanes of a
// warp (rows) then reach the entries of one column in 32 different banks.
struct UF {
    int* p;
    __device__ __forceinline__ int& operator[](int i) const { return p[(i & ~31) | ((i + (i >> 5)) & 31)]; }
};

__device__ __forceinline__ int s_find(UF par, int a) {
    int p = par[a];
    while (p != a) { a = p; p = par[a]; }
    return a;
}
__device__ __forceinline__ void s_union(UF par, int a, int b) {
    bool done;
    do {
        a = s_find(par, a);
        b = s_find(par, b);
        if (a < b) {
            int old = atomicMin(&par[b], a);
            done = (old == b);
            b = old;
        } else if (b < a) {
            int old = atomicMin(&par[a], b);
            done = (old == a);
            a = old;
        } else {
            done = true;
        }
    } while (!done);
}

// ---- global union-find -----------------------------------------------------------
// find with path halving; the shortcut is written with atomicMin, so it can
// only lower a link to an ancestor and never undoes a concurrent union
__device__ __forceinline__ int g_find(int* P, int a) {
    int p = __ldcg(P + a);
    while (p != a) {
        int gp = __ldcg(P + p);
        if (gp != p) atomicMin(P + a, gp);
        a = p;
        p = gp;
    }
    return a;
}
__device__ __forceinline__ void g_union(int* P, int a, int b) {
    bool done;
    do {
        a = g_find(P, a);
        b = g_find(P, b);
        if (a < b) {
            int old = atomicMin(P + b, a);
            done = (old == b);
            b = old;
        } else if (b < a) {
            int old = atomicMin(P + a, b);
            done = (old == a);
            a = old;
        } else {
            done = true;
        }
    } while (!done);
}

// ---- run-based local labelling, one warp per 32x32 block --------------------------
// Lane y holds the class word of row y (bit x = pixel (y, x)).  Runs of
// consecutive set bits are the nodes: a run is named by the pixel index of
// its first bit, par[] (per-warp shared memory, 1024 ints) holds union-find
// links at run starts only, and links always point to the smaller index, so
// a root is the first pixel (row-major) of its local component.  Only runs of
// adjacent rows that touch are unioned: a run of the row above covering
// columns [a, e] touches the runs of this row that meet [a, e] (4-conn) or
// [a-1, e+1] (8-conn).

__device__ __forceinline__ uint32_t below_or_at(int x) { return (2u << x) - 1u; }  // bits 0..x

// first bit of the run (of starts `st`) containing column x
__device__ __forceinline__ int run_start(uint32_t st, int x) { return 31 - __clz(st & below_or_at(x)); }

template <int CONN>
__device__ __forceinline__ void warp_ccl(uint32_t w, uint32_t st, int lane, UF par) {
    // Uniform fast path: every class row is one run, the class rows are
    // contiguous and each overlaps (CONN-adjacency) the row above -- the whole
    // block is one component whose root is its first pixel.  Typical for the
    // background of a block, and for blocks without any class pixel.
    {
        uint32_t wu = __shfl_up_sync(FULLM, w, 1);
        if (lane == 0) wu = 0u;
        const uint32_t adj = CONN == 8 ? (wu | (wu << 1) | (wu >> 1)) : wu;
        const unsigned has = __ballot_sync(FULLM, w != 0u);
        if (has == 0u) return;
        const int lo = __ffs(has) - 1;
        const uint32_t span = has >> lo;
        const bool contiguous = (span & (span + 1u)) == 0u;
        const bool bad = (w != 0u) && (__popc(st) != 1 || (lane != lo && (w & adj) == 0u));
        if (contiguous && __ballot_sync(FULLM, bad) == 0u) {
            const uint32_t w0 = __shfl_sync(FULLM, w, lo);
            const int root = lo * CB + __ffs(w0) - 1;
            if (st) par[lane * CB + __ffs(st) - 1] = root;
            __syncwarp();
            return;
        }
    }
    for (uint32_t m = st; m; m &= m - 1) {
        int i = lane * CB + __ffs(m) - 1;
        par[i] = i;
    }
    __syncwarp();
    uint32_t wu = __shfl_up_sync(FULLM, w, 1);
    if (lane == 0) wu = 0u;
    const uint32_t stu = wu & ~(wu << 1);
    for (uint32_t m = stu; m; m &= m - 1) {
        const int a = __ffs(m) - 1;
        const uint32_t rest = ~wu & (0xffffffffu << a);
        const int e = rest ? __ffs(rest) - 2 : 31;
        const int lo = CONN == 8 ? max(a - 1, 0) : a, hi = CONN == 8 ? min(e + 1, 31) : e;
        const uint32_t t = w & below_or_at(hi) & (0xffffffffu << lo);
        if (!t) continue;
        const int up = (lane - 1) * CB + a;
        const int s0 = run_start(st, __ffs(t) - 1);
        s_union(par, up, lane * CB + s0);
        for (uint32_t m2 = st & t & ~(1u << s0); m2; m2 &= m2 - 1) s_union(par, up, lane * CB + __ffs(m2) - 1);
    }
    __syncwarp();
    for (uint32_t m = st; m; m &= m - 1) {
        int i = lane * CB + __ffs(m) - 1;
        par[i] = s_find(par, i);
    }
    __syncwarp();
}

// mask of the run starting at bit s in word w
__device__ __forceinline__ uint32_t run_mask(uint32_t w, int s) {
    uint32_t rest = ~w & (0xffffffffu << s);
    int e = rest ? __ffs(rest) - 2 : 31;
    return below_or_at(e) & (0xffffffffu << s);
}

struct WarpGeo {
    int ti, bx, by, x0, y0, bw, bh, lb;
};

// The tile of a labelling block: a search over the first-block indices that
// travel in the launch parameters (up to LAUNCH_TAB tiles), else over the
// descriptors in global memory.
__device__ __forceinline__ int tile_of_block(const Launch& L, int gb) {
    if (L.ntiles > LAUNCH_TAB) return find_tile(L.tiles, L.ntiles, gb, &TileDev::cb_base);
    int lo = 0, hi = L.ntiles - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (L.cb_first[mid] <= gb) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ WarpGeo warp_geo(const Launch& L, int gb) {
    WarpGeo g;
    g.ti = tile_of_block(L, gb);
    const TileDev T = L.tiles[g.ti];  // by value: stores below cannot force reloads
    g.lb = gb - T.cb_base;
    g.by = g.lb / T.cbx;
    g.bx = g.lb - g.by * T.cbx;
    g.x0 = g.bx * CB;
    g.y0 = g.by * CB;
    g.bw = min(CB, T.W - g.x0);
    g.bh = min(CB, T.H - g.y0);
    return g;
}
__device__ __forceinline__ uint32_t valid_mask(int bw) { return bw >= 32 ? FULLM : ((1u << bw) - 1u); }
// word of row r of the block in a block-major bitmap
__device__ __forceinline__ size_t block_word(const TileDev& T, const WarpGeo& g, int r) {
    return ((size_t)g.by * T.cbx + g.bx) * CB + r;
}
__device__ __forceinline__ int gidx(const TileDev& T, const WarpGeo& g, int li) {
    return (g.y0 + (li >> 5)) * T.W + g.x0 + (li & 31);
}

// A union-find entry: the local root index in bits 0..9; a root's own entry
// may carry its component's payload in bits 16 and up.
constexpr int PAR_IDX = 0x3ff;
__device__ __forceinline__ int par_root(UF par, int i) { return par[i] & PAR_IDX; }

// Edge roots: [0,CB) left column, [CB,2CB) right column (x=31), [2CB,3CB)
// top row, [3CB,4CB) bottom row (y=31); -1 where the pixel is not in the class.
__device__ __forceinline__ void publish_edges(const TileDev& T, const WarpGeo& g, uint32_t w, uint32_t st,
                                              UF par, int lane) {
    int* e = T.border + (size_t)g.lb * 4 * CB;
    e[lane] = (w & 1u) ? gidx(T, g, par_root(par, lane * CB)) : -1;
    e[CB + lane] = (w >> 31) ? gidx(T, g, par_root(par, lane * CB + run_start(st, 31))) : -1;
    uint32_t w0 = __shfl_sync(FULLM, w, 0), s0 = __shfl_sync(FULLM, st, 0);
    uint32_t w31 = __shfl_sync(FULLM, w, 31), s31 = __shfl_sync(FULLM, st, 31);
    e[2 * CB + lane] = ((w0 >> lane) & 1u) ? gidx(T, g, par_root(par, run_start(s0, lane))) : -1;
    e[3 * CB + lane] = ((w31 >> lane) & 1u) ? gidx(T, g, par_root(par, 31 * CB + run_start(s31, lane))) : -1;
}

// Record this block's local roots (run starts that are roots) in the block's
// own slice of the root list (RL_CAP entries: a 32x32 block has at most 512
// 4-connected and 256 8-connected components) and initialise P/A at their
// global index with payload pay(root).  No global counter is involved.
template <typename Pay>
__device__ __forceinline__ void register_roots(const TileDev& T, const WarpGeo& g, uint32_t st, UF par,
                                               Pay pay, int lane) {
    uint32_t rs = 0;
    for (uint32_t m = st; m; m &= m - 1) {
        int s = __ffs(m) - 1;
        if (par_root(par, lane * CB + s) == lane * CB + s) rs |= 1u << s;
    }
    int n = __popc(rs), incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULLM, incl, o);
        if (lane >= o) incl += y;
    }
    int* list = T.rootlist + (size_t)g.lb * RL_CAP;
    int k = incl - n;
    for (uint32_t m = rs; m; m &= m - 1) {
        int li = lane * CB + __ffs(m) - 1;
        int gi = gidx(T, g, li);
        T.P[gi] = gi;
        T.A[gi] = pay(li);
        list[k++] = gi;
    }
    if (lane == 31) T.blkroots[g.lb] = incl;
}


// ---- K3a: foreground from the h-dome, background local components ---------------
__global__ void __launch_bounds__(CCL_WARPS * 32, 12) k_fill_local(Launch L) {
    __shared__ int par_sm[CCL_WARPS][CB * CB];
    __shared__ uint32_t touch_sm[CCL_WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = blockIdx.x * CCL_WARPS + warp;
    if (gb >= L.n_cb) return;
    const UF par{par_sm[warp]};
    uint32_t* touch = touch_sm[warp];
    const WarpGeo g = warp_geo(L, gb);
    const TileDev T = L.tiles[g.ti];  // by value: stores below cannot force reloads
    const uint32_t vm = valid_mask(g.bw);
    uint32_t fg = 0;
    // hem8 - R >= thr per byte: R <= hem8 bytewise, so the 32-bit difference
    // has no borrow between bytes; each byte plus 256 - thr (in its own
    // 16-bit lane) carries into bit 8 of the lane exactly when it is >= thr
    const uint32_t bias2 = (uint32_t)max(0, 256 - L.thr) * 0x00010001u;
    if (g.bw == 32 && (T.W & 15) == 0 &&
        ((reinterpret_cast<uintptr_t>(T.hem8) | reinterpret_cast<uintptr_t>(T.R)) & 15) == 0) {
        // lanes 2r and 2r+1 read the two 16-byte halves of row r (then of row
        // r+16), so every load covers 16 whole sectors; each half yields 16
        // foreground bits, and two shuffles assemble row y's word in lane y
        uint32_t half[2];
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int row = (lane >> 1) + 16 * i;
            half[i] = 0;
            if (row < g.bh) {
                const size_t o = (size_t)(g.y0 + row) * T.W + g.x0 + (lane & 1) * 16;
                const uint4 hv = __ldg(reinterpret_cast<const uint4*>(T.hem8 + o));
                const uint4 rv = __ldcg(reinterpret_cast<const uint4*>(T.R + o));
                const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, rw[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t d = hw[k] - rw[k];
                    const uint32_t e = (d & 0x00ff00ffu) + bias2, o = ((d >> 8) & 0x00ff00ffu) + bias2;
                    half[i] |= (((e >> 8) & 1u) | ((o >> 7) & 2u) | ((e >> 22) & 4u) | ((o >> 21) & 8u)) << (k * 4);
                }
            }
        }
        const int src = 2 * (lane & 15);
        const uint32_t lo0 = __shfl_sync(FULLM, half[0], src), hi0 = __shfl_sync(FULLM, half[0], src + 1);
        const uint32_t lo1 = __shfl_sync(FULLM, half[1], src), hi1 = __shfl_sync(FULLM, half[1], src + 1);
        fg = lane < 16 ? (lo0 | (hi0 << 16)) : (lo1 | (hi1 << 16));
        if (lane >= g.bh) fg = 0;
    } else if (lane < g.bh) {
        const size_t o = (size_t)(g.y0 + lane) * T.W + g.x0;
        for (int x = 0; x < g.bw; x++)
            if ((int)T.hem8[o + x] - (int)__ldcg(T.R + o + x) >= L.thr) fg |= 1u << x;
    }
    if (lane < g.bh) T.fgbits[block_word(T, g, lane)] = fg;
    const uint32_t bg = lane < g.bh ? (~fg & vm) : 0u;
    const uint32_t st = bg & ~(bg << 1);
    warp_ccl<4>(bg, st, lane, par);
    touch[lane] = 0u;
    __syncwarp();
    // a component touching the image border marks its root (one bit per pixel)
    const int gy = g.y0 + lane;
    for (uint32_t m = st; m; m &= m - 1) {
        int s = __ffs(m) - 1;
        uint32_t rm = run_mask(bg, s);
        bool tb = gy == 0 || gy == T.H - 1 || (g.x0 == 0 && (rm & 1u)) ||
                  (T.W - 1 - g.x0 < 32 && ((rm >> (T.W - 1 - g.x0)) & 1u));
        if (tb) {
            const int r = par_root(par, lane * CB + s);
            atomicOr(&touch[r >> 5], 1u << (r & 31));
        }
    }
    __syncwarp();
    register_roots(T, g, st, par, [&](int li) { return (int)((touch[li >> 5] >> (li & 31)) & 1u); }, lane);
    publish_edges(T, g, bg, st, par, lane);
}

// ---- merge facing edge pixels of neighbouring blocks ------------------------------
template <int CONN>
__device__ __forceinline__ int edge_root(const TileDev& T, int bx, int by, int side, int j) {
    if (bx < 0 || by < 0 || bx >= T.cbx || by >= T.cby || j < 0 || j >= CB) return -1;
    return T.border[(size_t)(by * T.cbx + bx) * 4 * CB + side * CB + j];
}

// One warp per block: lanes walk the right column and then the bottom row.
// Consecutive edge pixels mostly repeat the same pair of local roots, so a
// lane unions only when its pair differs from the previous lane's.
__device__ __forceinline__ void union_dedup(int* P, int a, int b, int lane) {
    int pa = __shfl_up_sync(FULLM, a, 1), pb = __shfl_up_sync(FULLM, b, 1);
    bool same = lane > 0 && pa == a && pb == b;
    if (a >= 0 && b >= 0 && !same) g_union(P, a, b);
}

template <int CONN>
__global__ void __launch_bounds__(CCL_WARPS * 32) k_merge(Launch L) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = blockIdx.x * CCL_WARPS + warp;
    if (gb >= L.n_cb) return;
    const WarpGeo g = warp_geo(L, gb);
    const TileDev T = L.tiles[g.ti];  // by value: stores below cannot force reloads
    const int* e = T.border + (size_t)g.lb * 4 * CB;
    // right column pixel (lane, 31) against the next block(s) to the right
    {
        int a = e[CB + lane];
        int b = edge_root<CONN>(T, g.bx + 1, g.by, 0, lane);
        union_dedup(T.P, a, b, lane);
        if (CONN == 8) {
            int up = lane == 0 ? edge_root<CONN>(T, g.bx + 1, g.by - 1, 0, CB - 1)
                               : edge_root<CONN>(T, g.bx + 1, g.by, 0, lane - 1);
            union_dedup(T.P, a, up, lane);
            int dn = lane == CB - 1 ? edge_root<CONN>(T, g.bx + 1, g.by + 1, 0, 0)
                                    : edge_root<CONN>(T, g.bx + 1, g.by, 0, lane + 1);
            union_dedup(T.P, a, dn, lane);
        }
    }
    // bottom row pixel (31, lane) against the block(s) below
    {
        int a = e[3 * CB + lane];
        int b = edge_root<CONN>(T, g.bx, g.by + 1, 2, lane);
        union_dedup(T.P, a, b, lane);
        if (CONN == 8) {
            int l = lane == 0 ? edge_root<CONN>(T, g.bx - 1, g.by + 1, 2, CB - 1)
                              : edge_root<CONN>(T, g.bx, g.by + 1, 2, lane - 1);
            union_dedup(T.P, a, l, lane);
            int r = lane == CB - 1 ? edge_root<CONN>(T, g.bx + 1, g.by + 1, 2, 0)
                                   : edge_root<CONN>(T, g.bx, g.by + 1, 2, lane + 1);
            union_dedup(T.P, a, r, lane);
        }
    }
}

// ---- root-list passes (grid-stride over every tile's list) -----------------------
constexpr int HOLE_BIT = 1 << 30;  // in a block's root count between the fill and the labelling
// mode 0: border flag of a local root -> its global root
// mode 1: copy the global root's flag back to every local root; compress P;
//         mark the blocks that hold a hole (HOLE_BIT in their root count)
//         (the labelling pass must read the flag at its own local roots: a
//         hole's global root can become a foreground root there, whose entry
//         that pass overwrites while other blocks would still follow links to it)
// mode 2: add local areas into the global root; compress P
// mode 3: mark kept global roots in the root bitmap
// Each warp strides over the labelling blocks (a grid of a warp per block,
// or of a few CTAs per SM: most blocks have one or two roots).
__global__ void __launch_bounds__(CCL_WARPS * 32) k_roots(Launch L, int mode) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int gb = blockIdx.x * CCL_WARPS + warp; gb < L.n_cb; gb += gridDim.x * CCL_WARPS) {
        const int ti = tile_of_block(L, gb);
        const TileDev T = L.tiles[ti];  // by value: stores below cannot force reloads
        const int lb = gb - T.cb_base;
        const int n = T.blkroots[lb];
        const int* list = T.rootlist + (size_t)lb * RL_CAP;
        bool hole = false;  // mode 1: a background component of this block is a hole
        for (int j = lane; j < n; j += 32) {
            int r = list[j];
            if (mode == 0) {
                if (T.A[r]) {
                    int g = g_find(T.P, r);
                    if (g != r) T.A[g] = 1;
                }
            } else if (mode == 1) {
                int g = g_find(T.P, r);
                int f = T.A[r];
                if (g != r) {
                    f = __ldcg(T.A + g);
                    T.A[r] = f;
                    T.P[r] = g;
                }
                hole |= f == 0;
            } else if (mode == 2) {
                int g = g_find(T.P, r);
                if (g != r) {
                    atomicAdd(T.A + g, T.A[r]);
                    T.P[r] = g;
                }
            } else {
                if (T.P[r] == r) {
                    int a = T.A[r];
                    if (a >= L.amin && a <= L.amax) {
                        int y = r / T.W, x = r - y * T.W;
                        atomicOr(T.rootbits + (size_t)y * T.wpr + (x >> 5), 1u << (x & 31));
                    }
                }
            }
        }
        if (mode == 1 && __any_sync(FULLM, hole) && lane == 0) T.blkroots[lb] = n | HOLE_BIT;
    }
}

// ---- K4a: holes -> filled; foreground local components ----------------------------
__global__ void __launch_bounds__(CCL_WARPS * 32, 12) k_label_local(Launch L) {
    __shared__ int par_sm[CCL_WARPS][CB * CB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = blockIdx.x * CCL_WARPS + warp;
    if (gb >= L.n_cb) return;
    const UF par{par_sm[warp]};
    const WarpGeo g = warp_geo(L, gb);
    const TileDev T = L.tiles[g.ti];  // by value: stores below cannot force reloads
    const uint32_t vm = valid_mask(g.bw);
    const size_t wrow = (size_t)(g.y0 + lane) * T.wpr + g.bx;  // row-major (root bitmap)
    const size_t wblk = block_word(T, g, lane);                // block-major (fg, filled)
    const uint32_t fg = lane < g.bh ? T.fgbits[wblk] : 0u;
    // background runs whose component does not reach the border are holes;
    // only blocks that hold one (most hold none) label their background again
    uint32_t filled = fg;
    if (__ldcg(T.blkroots + g.lb) & HOLE_BIT) {
        const uint32_t bg = lane < g.bh ? (~fg & vm) : 0u;
        const uint32_t sb = bg & ~(bg << 1);
        warp_ccl<4>(bg, sb, lane, par);
        for (uint32_t m = sb; m; m &= m - 1) {
            int s = __ffs(m) - 1;
            int gr = gidx(T, g, par[lane * CB + s]);
            if (!__ldcg(T.A + gr)) filled |= run_mask(bg, s);
        }
    }
    if (lane < g.bh) {
        T.filledbits[wblk] = filled;
        T.rootbits[wrow] = 0u;
    }
    __syncwarp();
    const uint32_t st = filled & ~(filled << 1);
    warp_ccl<8>(filled, st, lane, par);
    // local areas: each run adds its length to its root's entry, bits 16 and up
    for (uint32_t m = st; m; m &= m - 1) {
        int s = __ffs(m) - 1;
        atomicAdd(&par[par_root(par, lane * CB + s)], __popc(run_mask(filled, s)) << 16);
    }
    __syncwarp();
    register_roots(T, g, st, par, [&](int li) { return par[li] >> 16; }, lane);
    publish_edges(T, g, filled, st, par, lane);
}

// ---- K4e: exclusive popcount prefix of the root bitmap ----------------------------
__device__ __forceinline__ int block_exclusive_scan(int v, int* tmp /*[32]*/, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULLM, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < nw ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULLM, s, o);
            if (lane >= o) s += y;
        }
        tmp[lane] = s;
    }
    __syncthreads();
    int excl = x - v + (warp > 0 ? tmp[warp - 1] : 0);
    if (total) *total = tmp[nw - 1];
    __syncthreads();
    return excl;
}

// per chunk of SCAN_CHUNK words: chunk popcount (pass 0) or word prefixes
// (pass 1); each thread takes four consecutive words (one 16-byte load where
// the chunk lies inside the bitmap: chunks start at multiples of 16 KB)
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_chunks(Launch L, int pass) {
    __shared__ int tmp[32];
    int gc = blockIdx.x;
    int ti = find_tile(L.tiles, L.ntiles, gc, &TileDev::chunk_base);
    const TileDev& T = L.tiles[ti];
    int c = gc - T.chunk_base;
    const size_t nwords = (size_t)T.H * T.wpr;
    const size_t w = (size_t)c * SCAN_CHUNK + 4 * (size_t)threadIdx.x;
    uint32_t b[4] = {0u, 0u, 0u, 0u};
    if (w + 4 <= nwords) {
        const uint4 v = __ldcg(reinterpret_cast<const uint4*>(T.rootbits + w));
        b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
    } else {
        for (int i = 0; i < 4; i++)
            if (w + i < nwords) b[i] = T.rootbits[w + i];
    }
    const int p0 = __popc(b[0]), p1 = __popc(b[1]), p2 = __popc(b[2]), p3 = __popc(b[3]);
    int total = 0;
    const int excl = block_exclusive_scan(p0 + p1 + p2 + p3, tmp, &total);
    if (pass == 0) {
        if (threadIdx.x == 0) T.chunksum[c] = total;
    } else {
        const int base = excl + T.chunksum[c];
        const int v[4] = {base, base + p0, base + p0 + p1, base + p0 + p1 + p2};
        if (w + 4 <= nwords) {
            *reinterpret_cast<int4*>(T.wordprefix + w) = make_int4(v[0], v[1], v[2], v[3]);
        } else {
            for (int i = 0; i < 4; i++)
                if (w + i < nwords) T.wordprefix[w + i] = v[i];
        }
    }
}

// one block per tile: exclusive scan of the chunk sums; K = total
__global__ void __launch_bounds__(1024) k_scan_tiles(Launch L) {
    __shared__ int tmp[32];
    const TileDev& T = L.tiles[blockIdx.x];
    int carry = 0;
    for (int base = 0; base < T.nchunks; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < T.nchunks ? T.chunksum[i] : 0;
        int total = 0;
        int excl = block_exclusive_scan(v, tmp, &total);
        if (i < T.nchunks) T.chunksum[i] = excl + carry;
        carry += total;
    }
    if (threadIdx.x == 0) *T.n_objects = carry;
}

// ---- K4f: final labels, kept bitmap, EDT column summaries, object boxes ----------
// The final label is looked up once per local root (global root, root
// bitmap word, word prefix), and stored in the root's own entry with bit 31
// set; every run then takes its root's label from shared memory.  Each lane
// writes its row of labels from registers, four labels per 16-byte store.
constexpr int LAB_FLAG = (int)0x80000000u;
__global__ void __launch_bounds__(CCL_WARPS * 32, 12) k_relabel(Launch L, int want_bbox) {
    __shared__ int par_sm[CCL_WARPS][CB * CB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = blockIdx.x * CCL_WARPS + warp;
    if (gb >= L.n_cb) return;
    const UF par{par_sm[warp]};
    const WarpGeo g = warp_geo(L, gb);
    const TileDev T = L.tiles[g.ti];  // by value: stores below cannot force reloads
    const uint32_t filled = lane < g.bh ? T.filledbits[block_word(T, g, lane)] : 0u;
    const uint32_t st = filled & ~(filled << 1);
    warp_ccl<8>(filled, st, lane, par);
    // roots of this lane's row: label (0 if filtered out) into the root's entry
    uint32_t rs = 0;
    for (uint32_t m = st; m; m &= m - 1) {
        const int i = lane * CB + __ffs(m) - 1;
        if (par[i] == i) rs |= 1u << (i & 31);
    }
    uint32_t todo = rs;
    while (todo) {
        // up to four roots at a time, so that their lookups overlap
        int idx[4], gr[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            idx[k] = todo ? lane * CB + __ffs(todo) - 1 : -1;
            todo &= todo - 1;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) gr[k] = idx[k] >= 0 ? __ldcg(T.P + gidx(T, g, idx[k])) : 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (idx[k] < 0) continue;
            const int yy = gr[k] / T.W, xx = gr[k] - yy * T.W;
            const size_t w = (size_t)yy * T.wpr + (xx >> 5);
            const uint32_t bits = T.rootbits[w];
            const int wp = T.wordprefix[w];  // read unconditionally: both loads overlap
            const int lab = ((bits >> (xx & 31)) & 1u) ? wp + __popc(bits & ((1u << (xx & 31)) - 1u)) + 1 : 0;
            par[idx[k]] = lab | LAB_FLAG;
        }
    }
    __syncwarp();
    // runs: label from the root's entry; kept bits and object boxes.  The
    // lanes take their k-th runs together, so the runs of one object in this
    // block meet their box with one set of atomics from the group's first lane.
    uint32_t kept = 0;
    const int gy = g.y0 + lane;
    for (uint32_t m = st; __any_sync(FULLM, m != 0u);) {
        int lab = 0, xs = 0, xe = 0;
        if (m) {
            const int s = __ffs(m) - 1;
            m &= m - 1;
            const int v = par[lane * CB + s];
            lab = (v & LAB_FLAG) ? (v & ~LAB_FLAG) : (par[v] & ~LAB_FLAG);
            if (lab) {
                const uint32_t rm = run_mask(filled, s);
                kept |= rm;
                xs = g.x0 + s;
                xe = g.x0 + 31 - __clz(rm);
            }
        }
        if (want_bbox) {
            const bool box = lab != 0 && lab <= T.feats_cap;
            const unsigned grp = __match_any_sync(FULLM, box ? lab : 0);
            if (box) {
                const int x_lo = __reduce_min_sync(grp, xs), x_hi = __reduce_max_sync(grp, xe);
                const int y_lo = __reduce_min_sync(grp, gy), y_hi = __reduce_max_sync(grp, gy);
                if (lane == __ffs(grp) - 1) {
                    int4* b = T.bbox + (lab - 1);
                    atomicMin(&b->x, x_lo);
                    atomicMax(&b->z, x_hi);
                    atomicMin(&b->y, y_lo);
                    atomicMax(&b->w, y_hi);
                }
            }
        }
    }
    // label of the run starting at column s of this row
    auto run_label = [&](int s) -> int {
        const int v = par[lane * CB + s];
        return (v & LAB_FLAG) ? (v & ~LAB_FLAG) : (par[v] & ~LAB_FLAG);
    };
    if (g.bw == CB && (T.W & 3) == 0) {
        // lanes 8r..8r+7 write row 4q+r, four labels each: every store covers
        // four whole 128-byte rows of the block
        const int c4 = (lane & 7) * 4;
#pragma unroll 2
        for (int q = 0; q < CB / 4; q++) {
            const int y = 4 * q + (lane >> 3);
            const uint32_t sty = __shfl_sync(FULLM, st, y), kpy = __shfl_sync(FULLM, kept, y);
            if (y < g.bh) {
                int v[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int x = c4 + u;
                    int lab = 0;
                    if ((kpy >> x) & 1u) {
                        const int e = par[y * CB + run_start(sty, x)];
                        lab = (e & LAB_FLAG) ? (e & ~LAB_FLAG) : (par[e] & ~LAB_FLAG);
                    }
                    v[u] = lab;
                }
                reinterpret_cast<int4*>(T.labels + (size_t)(g.y0 + y) * T.W + g.x0)[lane & 7] =
                    make_int4(v[0], v[1], v[2], v[3]);
            }
        }
    } else if (lane < g.bh) {
        int32_t* dst = T.labels + (size_t)gy * T.W + g.x0;
        for (int x = 0; x < g.bw; x++) dst[x] = ((kept >> x) & 1u) ? run_label(run_start(st, x)) : 0;
    }
    // EDT input: this chunk's 32 kept bits of each column, as one word per
    // column: a 32x32 bit transpose across the lanes in five exchange stages
    if (T.edt) {
        uint32_t col = kept;
        const uint32_t msk[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const int j = 16 >> k;
            const uint32_t y = __shfl_xor_sync(FULLM, col, j);
            col = (lane & j) ? ((col & ~msk[k]) | ((y & ~msk[k]) >> j)) : ((col & msk[k]) | ((y & msk[k]) << j));
        }
        if (lane < g.bw) T.colbits[(size_t)g.by * T.W + g.x0 + lane] = col;
    }
}

// every box slot a tile can use (feats_cap of them) starts empty
__global__ void k_bbox_init(Launch L) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (int ti = 0; ti < L.ntiles; ti++) {
        const TileDev& T = L.tiles[ti];
        int n = T.feats_cap;
        for (int j = i; j < n; j += gridDim.x * blockDim.x)
            T.bbox[j] = make_int4(0x7fffffff, 0x7fffffff, -1, -1);
    }
}

__global__ void k_counters_reset(Launch L) {
    for (int i = threadIdx.x; i < L.ntiles; i += blockDim.x) L.tile_status[i] = 0;
}

// a block-major bitmap (CB words per labelling block) as one byte per pixel
__global__ void k_unpack_bits(const uint32_t* bits, int W, int H, int cbx, uint8_t* out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)W * H) return;
    int y = (int)(i / W), x = (int)(i - (long long)y * W);
    const size_t w = ((size_t)(y / CB) * cbx + x / CB) * CB + (y % CB);
    out[i] = (uint8_t)((bits[w] >> (x & 31)) & 1u);
}

void launch_unpack_bits(const uint32_t* bits, int W, int H, int cbx, uint8_t* out, cudaStream_t s,
                        Profiler* pf) {
    long long n = (long long)W * H;
    if (n == 0) return;
    pf->begin("unpack_bits", s);
    k_unpack_bits<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(bits, W, H, cbx, out);
    pf->end("unpack_bits", s);
}

void launch_label(const Launch& L, int want_bbox, int max_objects, int sms, cudaStream_t s, Profiler* pf) {
    if (L.n_cb == 0) return;
    const int rgrid = sms * 8;
    pf->begin("label_reset", s);
    k_counters_reset<<<1, 1024, 0, s>>>(L);
    pf->end("label_reset", s);
    if (want_bbox) {
        pf->begin("bbox_init", s);
        k_bbox_init<<<rgrid, 256, 0, s>>>(L);
        pf->end("bbox_init", s);
    }
    pf->begin("fill_local", s);
    k_fill_local<<<(L.n_cb + CCL_WARPS - 1) / CCL_WARPS, CCL_WARPS * 32, 0, s>>>(L);
    pf->end("fill_local", s);
    const int wg = (L.n_cb + CCL_WARPS - 1) / CCL_WARPS;
    // the area and keep passes stride over the blocks with a few CTAs per SM;
    // the flag passes, whose finds wait on global links, keep a warp per block
    const int rg = std::min(wg, sms * 16);
    pf->begin("fill_merge", s);
    k_merge<4><<<wg, CCL_WARPS * 32, 0, s>>>(L);
    pf->end("fill_merge", s);
    pf->begin("fill_roots_flag", s);
    k_roots<<<wg, CCL_WARPS * 32, 0, s>>>(L, 0);
    pf->end("fill_roots_flag", s);
    pf->begin("fill_roots_copy", s);
    k_roots<<<wg, CCL_WARPS * 32, 0, s>>>(L, 1);
    pf->end("fill_roots_copy", s);
    pf->begin("label_local", s);
    k_label_local<<<(L.n_cb + CCL_WARPS - 1) / CCL_WARPS, CCL_WARPS * 32, 0, s>>>(L);
    pf->end("label_local", s);
    pf->begin("label_merge", s);
    k_merge<8><<<wg, CCL_WARPS * 32, 0, s>>>(L);
    pf->end("label_merge", s);
    pf->begin("label_roots_area", s);
    k_roots<<<rg, CCL_WARPS * 32, 0, s>>>(L, 2);
    pf->end("label_roots_area", s);
    pf->begin("label_roots_keep", s);
    k_roots<<<rg, CCL_WARPS * 32, 0, s>>>(L, 3);
    pf->end("label_roots_keep", s);
    pf->begin("scan_chunks", s);
    k_scan_chunks<<<L.n_chunks, SCAN_THREADS, 0, s>>>(L, 0);
    pf->end("scan_chunks", s);
    pf->begin("scan_tiles", s);
    k_scan_tiles<<<L.ntiles, 1024, 0, s>>>(L);
    pf->end("scan_tiles", s);
    pf->begin("scan_words", s);
    k_scan_chunks<<<L.n_chunks, SCAN_THREADS, 0, s>>>(L, 1);
    pf->end("scan_words", s);
    pf->begin("relabel", s);
    k_relabel<<<(L.n_cb + CCL_WARPS - 1) / CCL_WARPS, CCL_WARPS * 32, 0, s>>>(L, want_bbox);
    pf->end("relabel", s);
}

}  // namespace nucseg
