// K3 + K4: fill holes (Table I, "FillHoles"), 8-connected labelling
// (Table I, "BWLabel") with the area filter (Table I, "AreaThreshold") and
// a deterministic raster-order relabel.
//
// Both steps are connected-component problems solved with the same block
// union-find scheme:
//  * a 32x32 labelling block stages its class bits (one 32-bit word per
//    row) and labels its local components in shared memory with union-find
//    whose links always point to the smaller index, so every local root is
//    the first pixel (row-major) of its local component;
//  * local roots get a slot in the sparse global arrays P (parent) and A
//    (payload) at their own pixel index and are appended to a root list;
//  * block edges publish the local roots of their edge pixels; a merge
//    kernel unions facing edge pixels in P with atomicMin links, so global
//    roots are again component-first pixels;
//  * later kernels recompute the local labelling from the 2 MB bitmaps
//    instead of storing a full plane of provisional labels.
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
__device__ __forceinline__ int s_find(const int* par, int a) {
    int p = par[a];
    while (p != a) { a = p; p = par[a]; }
    return a;
}
__device__ __forceinline__ void s_union(int* par, int a, int b) {
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
__device__ __forceinline__ int g_find(int* P, int a) {
    int p = __ldcg(P + a);
    while (p != a) { a = p; p = __ldcg(P + a); }
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

// Local components of the class bits cls[CB] (bit x of word y = pixel (y,x))
// of one block.  On return par[i] is the local root (first pixel) of pixel i,
// or -1 when i is not in the class.
template <int CONN>
__device__ void local_ccl(const uint32_t* cls, int* par) {
    for (int i = threadIdx.x; i < CB * CB; i += blockDim.x) {
        int y = i >> 5, x = i & 31;
        par[i] = ((cls[y] >> x) & 1u) ? i : -1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < CB * CB; i += blockDim.x) {
        int y = i >> 5, x = i & 31;
        uint32_t row = cls[y];
        if (!((row >> x) & 1u)) continue;
        if (x > 0 && ((row >> (x - 1)) & 1u)) s_union(par, i, i - 1);
        if (y > 0) {
            uint32_t up = cls[y - 1];
            if ((up >> x) & 1u) s_union(par, i, i - CB);
            if (CONN == 8) {
                if (x > 0 && ((up >> (x - 1)) & 1u)) s_union(par, i, i - CB - 1);
                if (x < CB - 1 && ((up >> (x + 1)) & 1u)) s_union(par, i, i - CB + 1);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < CB * CB; i += blockDim.x)
        if (par[i] >= 0) par[i] = s_find(par, i);
    __syncthreads();
}

struct BlockGeo {
    int ti, bx, by, x0, y0, bw, bh, lb;  // lb: block index within its tile
};
__device__ __forceinline__ BlockGeo block_geo(const Launch& L, int gb) {
    BlockGeo g;
    g.ti = find_tile(L.tiles, L.ntiles, gb, &TileDev::cb_base);
    const TileDev& T = L.tiles[g.ti];
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

// Publish edge local roots: [0,CB) left column, [CB,2CB) right column (x=31),
// [2CB,3CB) top row, [3CB,4CB) bottom row (y=31); -1 = not in class.
__device__ void publish_edges(const TileDev& T, const BlockGeo& g, const int* par) {
    int* e = T.border + (size_t)g.lb * 4 * CB;
    for (int k = threadIdx.x; k < 4 * CB; k += blockDim.x) {
        int side = k / CB, j = k % CB;
        int ly = side == 0 || side == 1 ? j : (side == 2 ? 0 : CB - 1);
        int lx = side == 2 || side == 3 ? j : (side == 0 ? 0 : CB - 1);
        int r = par[ly * CB + lx];
        int v = -1;
        if (r >= 0) v = (g.y0 + (r >> 5)) * T.W + g.x0 + (r & 31);
        e[k] = v;
    }
}

// Append local roots (pixels with par[i]==i) to the tile's root list and
// initialise P/A at their global index with payload pay[i].
__device__ void register_roots(const TileDev& T, const BlockGeo& g, const int* par, const int* pay,
                               int counter) {
    for (int i = threadIdx.x; i < CB * CB; i += blockDim.x) {
        bool root = par[i] == i;
        unsigned m = __ballot_sync(FULLM, root);
        if (!m) continue;
        int lane = threadIdx.x & 31;
        int base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(T.counters + counter, __popc(m));
        base = __shfl_sync(FULLM, base, __ffs(m) - 1);
        if (root) {
            int gi = (g.y0 + (i >> 5)) * T.W + g.x0 + (i & 31);
            T.P[gi] = gi;
            T.A[gi] = pay[i];
            T.rootlist[base + __popc(m & ((1u << lane) - 1u))] = gi;
        }
    }
}

// ---- K3a: foreground from the h-dome, background local components ---------------
__global__ void __launch_bounds__(CB_THREADS) k_fill_local(Launch L) {
    __shared__ uint32_t fgw[CB], bgw[CB];
    __shared__ int par[CB * CB];
    __shared__ int flag[CB * CB];
    const BlockGeo g = block_geo(L, blockIdx.x);
    const TileDev& T = L.tiles[g.ti];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t vm = valid_mask(g.bw);
    for (int ly = warp; ly < CB; ly += CB_THREADS / 32) {
        bool in = ly < g.bh && lane < g.bw;
        bool fg = false;
        if (in) {
            size_t o = (size_t)(g.y0 + ly) * T.W + g.x0 + lane;
            fg = (int)__ldg(T.hem8 + o) - (int)__ldcg(T.R + o) >= L.thr;
        }
        uint32_t b = __ballot_sync(FULLM, fg);
        if (lane == 0) {
            fgw[ly] = b;
            bgw[ly] = ly < g.bh ? (~b & vm) : 0u;
            if (ly < g.bh) T.fgbits[(size_t)(g.y0 + ly) * T.wpr + g.bx] = b;
        }
    }
    for (int i = threadIdx.x; i < CB * CB; i += blockDim.x) flag[i] = 0;
    __syncthreads();
    local_ccl<4>(bgw, par);
    // a local component touching the image border marks its root
    for (int i = threadIdx.x; i < CB * CB; i += blockDim.x) {
        int r = par[i];
        if (r < 0) continue;
        int gy = g.y0 + (i >> 5), gx = g.x0 + (i & 31);
        if (gy == 0 || gx == 0 || gy == T.H - 1 || gx == T.W - 1) flag[r] = 1;
    }
    __syncthreads();
    register_roots(T, g, par, flag, 0);
    publish_edges(T, g, par);
}

// ---- merge facing edge pixels of neighbouring blocks ------------------------------
template <int CONN>
__device__ __forceinline__ int edge_root(const TileDev& T, int bx, int by, int side, int j) {
    if (bx < 0 || by < 0 || bx >= T.cbx || by >= T.cby || j < 0 || j >= CB) return -1;
    return T.border[(size_t)(by * T.cbx + bx) * 4 * CB + side * CB + j];
}

template <int CONN>
__global__ void __launch_bounds__(256) k_merge(Launch L) {
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    int gb = gid / (2 * CB), k = gid % (2 * CB);
    if (gb >= L.n_cb) return;
    const BlockGeo g = block_geo(L, gb);
    const TileDev& T = L.tiles[g.ti];
    const int* e = T.border + (size_t)g.lb * 4 * CB;
    if (k < CB) {  // right column pixel (k, 31) against the next block(s) to the right
        int a = e[CB + k];
        if (a < 0) return;
        int b = edge_root<CONN>(T, g.bx + 1, g.by, 0, k);
        if (b >= 0) g_union(T.P, a, b);
        if (CONN == 8) {
            int up = k == 0 ? edge_root<CONN>(T, g.bx + 1, g.by - 1, 0, CB - 1)
                            : edge_root<CONN>(T, g.bx + 1, g.by, 0, k - 1);
            if (up >= 0) g_union(T.P, a, up);
            int dn = k == CB - 1 ? edge_root<CONN>(T, g.bx + 1, g.by + 1, 0, 0)
                                 : edge_root<CONN>(T, g.bx + 1, g.by, 0, k + 1);
            if (dn >= 0) g_union(T.P, a, dn);
        }
    } else {  // bottom row pixel (31, j) against the block(s) below
        int j = k - CB;
        int a = e[3 * CB + j];
        if (a < 0) return;
        int b = edge_root<CONN>(T, g.bx, g.by + 1, 2, j);
        if (b >= 0) g_union(T.P, a, b);
        if (CONN == 8) {
            int l = j == 0 ? edge_root<CONN>(T, g.bx - 1, g.by + 1, 2, CB - 1)
                           : edge_root<CONN>(T, g.bx, g.by + 1, 2, j - 1);
            if (l >= 0) g_union(T.P, a, l);
            int r = j == CB - 1 ? edge_root<CONN>(T, g.bx + 1, g.by + 1, 2, 0)
                                : edge_root<CONN>(T, g.bx, g.by + 1, 2, j + 1);
            if (r >= 0) g_union(T.P, a, r);
        }
    }
}

// ---- root-list passes (grid-stride over every tile's list) -----------------------
// mode 0: border flag of a local root -> its global root
// mode 1: copy the global root's flag back to every local root; compress P
// mode 2: add local areas into the global root; compress P
// mode 3: mark kept global roots in the root bitmap
__global__ void __launch_bounds__(256) k_roots(Launch L, int counter, int mode) {
    const int stride = gridDim.x * blockDim.x;
    for (int ti = 0; ti < L.ntiles; ti++) {
        const TileDev& T = L.tiles[ti];
        const int n = __ldcg(T.counters + counter);
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
            int r = T.rootlist[j];
            if (mode == 0) {
                if (T.A[r]) {
                    int g = g_find(T.P, r);
                    if (g != r) T.A[g] = 1;
                }
            } else if (mode == 1) {
                int g = g_find(T.P, r);
                if (g != r) {
                    T.A[r] = __ldcg(T.A + g);
                    T.P[r] = g;
                }
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
    }
}

// ---- K4a: holes -> filled; foreground local components ----------------------------
__global__ void __launch_bounds__(CB_THREADS) k_label_local(Launch L) {
    __shared__ uint32_t fgw[CB], bgw[CB], flw[CB];
    __shared__ int par[CB * CB];
    __shared__ int cnt[CB * CB];
    const BlockGeo g = block_geo(L, blockIdx.x);
    const TileDev& T = L.tiles[g.ti];
    const uint32_t vm = valid_mask(g.bw);
    for (int ly = threadIdx.x; ly < CB; ly += blockDim.x) {
        uint32_t b = ly < g.bh ? T.fgbits[(size_t)(g.y0 + ly) * T.wpr + g.bx] : 0u;
        fgw[ly] = b;
        bgw[ly] = ly < g.bh ? (~b & vm) : 0u;
        flw[ly] = b;
    }
    for (int i = threadIdx.x; i < CB * CB; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    local_ccl<4>(bgw, par);
    // background pixels whose component does not reach the border are holes
    for (int i = threadIdx.x; i < CB * CB; i += blockDim.x) {
        int r = par[i];
        if (r < 0) continue;
        int gr = (g.y0 + (r >> 5)) * T.W + g.x0 + (r & 31);
        if (!__ldcg(T.A + gr)) atomicOr(&flw[i >> 5], 1u << (i & 31));
    }
    __syncthreads();
    for (int ly = threadIdx.x; ly < g.bh; ly += blockDim.x) {
        size_t w = (size_t)(g.y0 + ly) * T.wpr + g.bx;
        T.filledbits[w] = flw[ly];
        T.rootbits[w] = 0u;
    }
    local_ccl<8>(flw, par);
    for (int i = threadIdx.x; i < CB * CB; i += blockDim.x)
        if (par[i] >= 0) atomicAdd(&cnt[par[i]], 1);
    __syncthreads();
    register_roots(T, g, par, cnt, 1);
    publish_edges(T, g, par);
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

// per chunk of SCAN_CHUNK words: chunk popcount (pass 0) or word prefixes (pass 1)
__global__ void __launch_bounds__(SCAN_CHUNK) k_scan_chunks(Launch L, int pass) {
    __shared__ int tmp[32];
    int gc = blockIdx.x;
    int ti = find_tile(L.tiles, L.ntiles, gc, &TileDev::chunk_base);
    const TileDev& T = L.tiles[ti];
    int c = gc - T.chunk_base;
    size_t nwords = (size_t)T.H * T.wpr;
    size_t w = (size_t)c * SCAN_CHUNK + threadIdx.x;
    int v = w < nwords ? __popc(T.rootbits[w]) : 0;
    int total = 0;
    int excl = block_exclusive_scan(v, tmp, &total);
    if (pass == 0) {
        if (threadIdx.x == 0) T.chunksum[c] = total;
    } else if (w < nwords) {
        T.wordprefix[w] = excl + T.chunksum[c];
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
__global__ void __launch_bounds__(CB_THREADS) k_relabel(Launch L, int want_bbox) {
    __shared__ uint32_t flw[CB], keep[CB];
    __shared__ int par[CB * CB];
    const BlockGeo g = block_geo(L, blockIdx.x);
    const TileDev& T = L.tiles[g.ti];
    for (int ly = threadIdx.x; ly < CB; ly += blockDim.x) {
        flw[ly] = ly < g.bh ? T.filledbits[(size_t)(g.y0 + ly) * T.wpr + g.bx] : 0u;
        keep[ly] = 0u;
    }
    __syncthreads();
    local_ccl<8>(flw, par);
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < CB * CB; i += blockDim.x) {
        int ly = i >> 5, lx = i & 31;
        int lab = 0;
        int r = par[i];
        if (r >= 0) {
            int gl = (g.y0 + (r >> 5)) * T.W + g.x0 + (r & 31);
            int gr = __ldcg(T.P + gl);
            int yy = gr / T.W, xx = gr - yy * T.W;
            size_t w = (size_t)yy * T.wpr + (xx >> 5);
            uint32_t bits = T.rootbits[w];
            if ((bits >> (xx & 31)) & 1u) lab = T.wordprefix[w] + __popc(bits & ((1u << (xx & 31)) - 1u)) + 1;
        }
        if (ly < g.bh && lx < g.bw) {
            T.labels[(size_t)(g.y0 + ly) * T.W + g.x0 + lx] = lab;
            if (want_bbox && lab > 0) {
                // warp-aggregated box update per label
                unsigned grp = __match_any_sync(__activemask(), lab);
                int gx = g.x0 + lx, gy = g.y0 + ly;
                int mnx = __reduce_min_sync(grp, (unsigned)gx), mxx = __reduce_max_sync(grp, (unsigned)gx);
                int mny = __reduce_min_sync(grp, (unsigned)gy), mxy = __reduce_max_sync(grp, (unsigned)gy);
                if (lane == __ffs(grp) - 1 && lab <= T.feats_cap) {
                    int4* b = T.bbox + (lab - 1);
                    atomicMin(&b->x, mnx); atomicMin(&b->y, mny);
                    atomicMax(&b->z, mxx); atomicMax(&b->w, mxy);
                }
            }
        }
        unsigned kb = __ballot_sync(FULLM, lab > 0);
        if (lane == 0) keep[ly] = kb;
    }
    __syncthreads();
    for (int ly = threadIdx.x; ly < g.bh; ly += blockDim.x)
        T.keptbits[(size_t)(g.y0 + ly) * T.wpr + g.bx] = keep[ly];
    // EDT column summaries of this 32-row chunk: first and last background row
    if (T.edt && threadIdx.x < 32) {
        int lx = threadIdx.x;
        int fb = -1, lb = -1;
        if (lx < g.bw) {
            for (int ly = 0; ly < g.bh; ly++) {
                if (!((keep[ly] >> lx) & 1u)) {
                    if (fb < 0) fb = g.y0 + ly;
                    lb = g.y0 + ly;
                }
            }
            size_t o = (size_t)g.by * T.W + g.x0 + lx;
            T.edtF[o] = fb;
            T.edtL[o] = lb;
        }
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
    for (int i = threadIdx.x; i < L.ntiles; i += blockDim.x) {
        L.tiles[i].counters[0] = 0;
        L.tiles[i].counters[1] = 0;
        L.tile_status[i] = 0;
    }
}

__global__ void k_unpack_bits(const uint32_t* bits, int W, int H, int wpr, uint8_t* out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)W * H) return;
    int y = (int)(i / W), x = (int)(i - (long long)y * W);
    out[i] = (uint8_t)((bits[(size_t)y * wpr + (x >> 5)] >> (x & 31)) & 1u);
}

void launch_unpack_bits(const uint32_t* bits, int W, int H, int wpr, uint8_t* out, cudaStream_t s,
                        Profiler* pf) {
    long long n = (long long)W * H;
    if (n == 0) return;
    pf->begin("unpack_bits", s);
    k_unpack_bits<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(bits, W, H, wpr, out);
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
    k_fill_local<<<L.n_cb, CB_THREADS, 0, s>>>(L);
    pf->end("fill_local", s);
    int mg = (L.n_cb * 2 * CB + 255) / 256;
    pf->begin("fill_merge", s);
    k_merge<4><<<mg, 256, 0, s>>>(L);
    pf->end("fill_merge", s);
    pf->begin("fill_roots_flag", s);
    k_roots<<<rgrid, 256, 0, s>>>(L, 0, 0);
    pf->end("fill_roots_flag", s);
    pf->begin("fill_roots_copy", s);
    k_roots<<<rgrid, 256, 0, s>>>(L, 0, 1);
    pf->end("fill_roots_copy", s);
    pf->begin("label_local", s);
    k_label_local<<<L.n_cb, CB_THREADS, 0, s>>>(L);
    pf->end("label_local", s);
    pf->begin("label_merge", s);
    k_merge<8><<<mg, 256, 0, s>>>(L);
    pf->end("label_merge", s);
    pf->begin("label_roots_area", s);
    k_roots<<<rgrid, 256, 0, s>>>(L, 1, 2);
    pf->end("label_roots_area", s);
    pf->begin("label_roots_keep", s);
    k_roots<<<rgrid, 256, 0, s>>>(L, 1, 3);
    pf->end("label_roots_keep", s);
    pf->begin("scan_chunks", s);
    k_scan_chunks<<<L.n_chunks, SCAN_CHUNK, 0, s>>>(L, 0);
    pf->end("scan_chunks", s);
    pf->begin("scan_tiles", s);
    k_scan_tiles<<<L.ntiles, 1024, 0, s>>>(L);
    pf->end("scan_tiles", s);
    pf->begin("scan_words", s);
    k_scan_chunks<<<L.n_chunks, SCAN_CHUNK, 0, s>>>(L, 1);
    pf->end("scan_words", s);
    pf->begin("relabel", s);
    k_relabel<<<L.n_cb, CB_THREADS, 0, s>>>(L, want_bbox);
    pf->end("relabel", s);
}

}  // namespace nucseg
