/*
 * CPU oracle (test infrastructure only; see oracle.h).  Plain C,
 * single-threaded, integer arithmetic for every plane, FP64 for features.
 * Each function states the passage of the paper it follows and the reading
 * taken where the paper is silent.
 */
#include "oracle.h"

#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Colour deconvolution (Sec. V-A, feature-stage transforms)          */
/* ------------------------------------------------------------------ */

static void normalize3(double v[3]) {
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n; v[1] /= n; v[2] /= n;
}

void oracle_deconv_tables(int32_t od_lut[256], int32_t wq[3], double w_out[3]) {
    /* Stain optical-density vectors (Ruifrok & Johnston 2001): hematoxylin,
       eosin, and the residual as their normalised cross product. */
    double Hs[3] = {0.650, 0.704, 0.286}, Es[3] = {0.072, 0.990, 0.105}, Rs[3];
    normalize3(Hs);
    normalize3(Es);
    Rs[0] = Hs[1] * Es[2] - Hs[2] * Es[1];
    Rs[1] = Hs[2] * Es[0] - Hs[0] * Es[2];
    Rs[2] = Hs[0] * Es[1] - Hs[1] * Es[0];
    normalize3(Rs);
    /* M has rows H, E, R; concentrations c = od * M^-1 (od as a row vector),
       so the hematoxylin weight of channel k is (M^-1)[k][0]. */
    double M[3][3] = {{Hs[0], Hs[1], Hs[2]}, {Es[0], Es[1], Es[2]}, {Rs[0], Rs[1], Rs[2]}};
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                 M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                 M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    /* first column of the inverse = first column of the adjugate / det */
    double w[3];
    w[0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / det;
    w[1] = -(M[1][0] * M[2][2] - M[1][2] * M[2][0]) / det;
    w[2] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / det;
    for (int v = 0; v < 256; v++) od_lut[v] = (int32_t)floor(-log((v + 1) / 256.0) * 256.0 + 0.5);
    for (int k = 0; k < 3; k++) {
        wq[k] = (int32_t)llround(100.0 * w[k] * 2048.0);
        if (w_out) w_out[k] = w[k];
    }
}

void oracle_deconv(const uint8_t* rgb, int W, int H, size_t pitch, uint8_t* hem8) {
    int32_t lut[256], wq[3];
    oracle_deconv_tables(lut, wq, NULL);
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            const uint8_t* p = rgb + (size_t)y * pitch + (size_t)x * 3;
            int32_t acc = wq[0] * lut[p[0]] + wq[1] * lut[p[1]] + wq[2] * lut[p[2]];
            int32_t v = acc < 0 ? 0 : (acc + (1 << 18)) >> 19;
            hem8[(size_t)y * W + x] = (uint8_t)(v > 255 ? 255 : v);
        }
}

/* ------------------------------------------------------------------ */
/* Morphological reconstruction (Table I, ReconToNuclei)              */
/* ------------------------------------------------------------------ */

typedef struct { int32_t* a; size_t head, tail, cap; } fifo;
static int fifo_push(fifo* f, int32_t v) {
    if (f->tail == f->cap) {
        if (f->head > 0) { /* compact */
            memmove(f->a, f->a + f->head, (f->tail - f->head) * sizeof(int32_t));
            f->tail -= f->head;
            f->head = 0;
        }
        if (f->tail == f->cap) {
            size_t nc = f->cap ? 2 * f->cap : 1024;
            int32_t* na = (int32_t*)realloc(f->a, nc * sizeof(int32_t));
            if (!na) return -1;
            f->a = na;
            f->cap = nc;
        }
    }
    f->a[f->tail++] = v;
    return 0;
}

static const int DY8[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
static const int DX8[8] = {-1, 0, 1, -1, 1, -1, 0, 1};

int oracle_recon(const uint8_t* marker, const uint8_t* mask, int W, int H, uint8_t* J,
                 oracle_recon_stats* st) {
    size_t N = (size_t)W * H;
    for (size_t i = 0; i < N; i++) {
        if (marker[i] > mask[i]) return -1;
        J[i] = marker[i];
    }
    const uint8_t* I = mask;
    /* raster sweep: causal half-neighbourhood (up-left, up, up-right, left) */
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            size_t p = (size_t)y * W + x;
            int m = J[p];
            for (int k = 0; k < 4; k++) {
                int yy = y + DY8[k], xx = x + DX8[k];
                if (yy < 0 || xx < 0 || xx >= W) continue;
                int v = J[(size_t)yy * W + xx];
                if (v > m) m = v;
            }
            J[p] = (uint8_t)(m < I[p] ? m : I[p]);
        }
    /* anti-raster sweep: anti-causal half (right, down-left, down, down-right);
       pixels that can still raise an anti-causal neighbour seed the queue */
    fifo f = {NULL, 0, 0, 0};
    uint32_t* depth = NULL;
    if (st) {
        depth = (uint32_t*)calloc(N, sizeof(uint32_t));
        st->fifo_pushes = 0;
        st->max_depth = 0;
    }
    for (int y = H - 1; y >= 0; y--)
        for (int x = W - 1; x >= 0; x--) {
            size_t p = (size_t)y * W + x;
            int m = J[p];
            for (int k = 4; k < 8; k++) {
                int yy = y + DY8[k], xx = x + DX8[k];
                if (yy >= H || xx < 0 || xx >= W) continue;
                int v = J[(size_t)yy * W + xx];
                if (v > m) m = v;
            }
            J[p] = (uint8_t)(m < I[p] ? m : I[p]);
            for (int k = 4; k < 8; k++) {
                int yy = y + DY8[k], xx = x + DX8[k];
                if (yy >= H || xx < 0 || xx >= W) continue;
                size_t q = (size_t)yy * W + xx;
                if (J[q] < J[p] && J[q] < I[q]) {
                    fifo_push(&f, (int32_t)p);
                    break;
                }
            }
        }
    /* breadth-first propagation until no pixel can be raised */
    while (f.head < f.tail) {
        int32_t p = f.a[f.head++];
        int y = p / W, x = p % W;
        for (int k = 0; k < 8; k++) {
            int yy = y + DY8[k], xx = x + DX8[k];
            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            size_t q = (size_t)yy * W + xx;
            if (J[q] < J[p] && I[q] != J[q]) {
                J[q] = (uint8_t)(J[p] < I[q] ? J[p] : I[q]);
                fifo_push(&f, (int32_t)q);
                if (st) {
                    st->fifo_pushes++;
                    depth[q] = depth[p] + 1;
                    if ((int)depth[q] > st->max_depth) st->max_depth = (int)depth[q];
                }
            }
        }
    }
    free(f.a);
    free(depth);
    return 0;
}

int oracle_recon_plain(const uint8_t* marker, const uint8_t* mask, int W, int H, uint8_t* R) {
    size_t N = (size_t)W * H;
    uint8_t* nx = (uint8_t*)malloc(N ? N : 1);
    for (size_t i = 0; i < N; i++) R[i] = marker[i];
    int iters = 0;
    for (;;) {
        int changed = 0;
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                int m = 0;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        int yy = y + dy, xx = x + dx;
                        if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                        int v = R[(size_t)yy * W + xx];
                        if (v > m) m = v;
                    }
                size_t p = (size_t)y * W + x;
                int v = m < mask[p] ? m : mask[p];
                nx[p] = (uint8_t)v;
                if (v != R[p]) changed = 1;
            }
        memcpy(R, nx, N);
        if (!changed) break;
        iters++;
    }
    free(nx);
    return iters;
}

/* The same synchronous iteration as oracle_recon_plain, R_{k+1} =
 * min(dilate8(R_k), mask), evaluated only where it can change: a pixel's
 * value in R_{k+1} differs from R_k only if some pixel of its 3x3
 * neighbourhood changed in step k, so after the first full step only the
 * neighbourhoods of the previous step's changes are re-evaluated (against
 * an unmodified R_k; changes are applied after the step).  Every R_k, and
 * hence the number of steps that change something, equals the plain
 * iteration's.  That number is the distance, in 8-connected steps, that the
 * slowest reconstruction front travels. */
int oracle_recon_rounds(const uint8_t* marker, const uint8_t* mask, int W, int H, uint8_t* R,
                        long long* evaluated) {
    size_t N = (size_t)W * H;
    int32_t* cand = (int32_t*)malloc((N ? N : 1) * sizeof(int32_t));
    int32_t* next = (int32_t*)malloc((N ? N : 1) * sizeof(int32_t));
    int32_t* chg = (int32_t*)malloc((N ? N : 1) * sizeof(int32_t));
    uint8_t* val = (uint8_t*)malloc(N ? N : 1);
    int32_t* stamp = (int32_t*)malloc((N ? N : 1) * sizeof(int32_t));
    for (size_t i = 0; i < N; i++) { R[i] = marker[i]; cand[i] = (int32_t)i; stamp[i] = 0; }
    size_t nc = N;
    long long evals = 0;
    int steps = 0;
    for (;;) {
        size_t nch = 0;
        for (size_t c = 0; c < nc; c++) {
            int p = cand[c], y = p / W, x = p % W, m = 0;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    int v = R[(size_t)yy * W + xx];
                    if (v > m) m = v;
                }
            int v = m < mask[p] ? m : mask[p];
            if (v != R[p]) { chg[nch] = p; val[nch] = (uint8_t)v; nch++; }
        }
        evals += (long long)nc;
        if (nch == 0) break;
        steps++;
        for (size_t k = 0; k < nch; k++) R[chg[k]] = val[k];
        size_t nn = 0;
        for (size_t k = 0; k < nch; k++) {
            int p = chg[k], y = p / W, x = p % W;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    int q = yy * W + xx;
                    if (stamp[q] != steps) { stamp[q] = steps; next[nn++] = q; }
                }
        }
        int32_t* t = cand; cand = next; next = t;
        nc = nn;
    }
    if (evaluated) *evaluated = evals;
    free(cand); free(next); free(chg); free(val); free(stamp);
    return steps;
}

void oracle_hdome(const uint8_t* hem8, int W, int H, int h, int thr, uint8_t* R, uint8_t* fg,
                  oracle_recon_stats* st) {
    size_t N = (size_t)W * H;
    uint8_t* mk = (uint8_t*)malloc(N ? N : 1);
    uint8_t* r = R ? R : (uint8_t*)malloc(N ? N : 1);
    for (size_t i = 0; i < N; i++) mk[i] = (uint8_t)(hem8[i] > h ? hem8[i] - h : 0);
    oracle_recon(mk, hem8, W, H, r, st);
    if (fg)
        for (size_t i = 0; i < N; i++) fg[i] = (uint8_t)((int)hem8[i] - (int)r[i] >= thr);
    free(mk);
    if (!R) free(r);
}

/* ------------------------------------------------------------------ */
/* Fill holes (Table I, FillHoles)                                     */
/* ------------------------------------------------------------------ */

void oracle_fill_holes(const uint8_t* fg, int W, int H, uint8_t* filled) {
    size_t N = (size_t)W * H;
    uint8_t* reach = (uint8_t*)calloc(N ? N : 1, 1);
    int32_t* q = (int32_t*)malloc((N ? N : 1) * sizeof(int32_t));
    size_t qh = 0, qt = 0;
    /* seeds: background pixels on the image border */
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            if (y != 0 && y != H - 1 && x != 0 && x != W - 1) continue;
            size_t p = (size_t)y * W + x;
            if (!fg[p] && !reach[p]) { reach[p] = 1; q[qt++] = (int32_t)p; }
        }
    static const int dy4[4] = {-1, 1, 0, 0}, dx4[4] = {0, 0, -1, 1};
    while (qh < qt) {
        int32_t p = q[qh++];
        int y = p / W, x = p % W;
        for (int k = 0; k < 4; k++) {
            int yy = y + dy4[k], xx = x + dx4[k];
            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            size_t n = (size_t)yy * W + xx;
            if (!fg[n] && !reach[n]) { reach[n] = 1; q[qt++] = (int32_t)n; }
        }
    }
    for (size_t i = 0; i < N; i++) filled[i] = (uint8_t)(!reach[i]);
    free(reach);
    free(q);
}

/* ------------------------------------------------------------------ */
/* Labelling + area filter (Table I, BWLabel and AreaThreshold)        */
/* ------------------------------------------------------------------ */

int oracle_label(const uint8_t* filled, int W, int H, int amin, int amax, int32_t* labels) {
    size_t N = (size_t)W * H;
    int32_t* q = (int32_t*)malloc((N ? N : 1) * sizeof(int32_t));
    for (size_t i = 0; i < N; i++) labels[i] = 0;
    int K = 0;
    /* raster order: the first unvisited foreground pixel starts a component,
       so components are discovered in order of their first pixel */
    uint8_t* seen = (uint8_t*)calloc(N ? N : 1, 1);
    for (size_t s = 0; s < N; s++) {
        if (!filled[s] || seen[s]) continue;
        size_t qh = 0, qt = 0;
        seen[s] = 1;
        q[qt++] = (int32_t)s;
        while (qh < qt) {
            int32_t p = q[qh++];
            int y = p / W, x = p % W;
            for (int k = 0; k < 8; k++) {
                int yy = y + DY8[k], xx = x + DX8[k];
                if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                size_t n = (size_t)yy * W + xx;
                if (filled[n] && !seen[n]) { seen[n] = 1; q[qt++] = (int32_t)n; }
            }
        }
        int area = (int)qt;
        if (area >= amin && area <= amax) {
            K++;
            for (size_t i = 0; i < qt; i++) labels[q[i]] = K;
        }
    }
    free(q);
    free(seen);
    return K;
}

/* ------------------------------------------------------------------ */
/* Exact squared EDT (Table I, Pre-Watershed distance transform)       */
/* ------------------------------------------------------------------ */

static inline int64_t floordiv64(int64_t a, int64_t b) { /* b > 0 */
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q--;
    return q;
}

void oracle_edt(const int32_t* labels, int W, int H, int32_t* edt) {
    size_t N = (size_t)W * H;
    const int64_t INF = (int64_t)W + H; /* larger than any in-image distance */
    int64_t* g = (int64_t*)malloc((N ? N : 1) * sizeof(int64_t));
    int any_bg = 0;
    /* phase 1: per column, distance to the nearest background pixel */
    for (int x = 0; x < W; x++) {
        g[x] = labels[x] == 0 ? 0 : INF;
        for (int y = 1; y < H; y++) {
            size_t p = (size_t)y * W + x;
            g[p] = labels[p] == 0 ? 0 : (g[p - W] >= INF ? INF : g[p - W] + 1);
        }
        for (int y = H - 2; y >= 0; y--) {
            size_t p = (size_t)y * W + x;
            if (g[p + W] < g[p]) g[p] = g[p + W] + 1;
        }
    }
    for (size_t i = 0; i < N; i++)
        if (labels[i] == 0) { any_bg = 1; break; }
    /* phase 2: per row, lower envelope of parabolas f_i(u) = (u-i)^2 + g_i^2 */
    int* s = (int*)malloc((W ? W : 1) * sizeof(int));
    int* t = (int*)malloc((W ? W : 1) * sizeof(int));
    for (int y = 0; y < H; y++) {
        const int64_t* gr = g + (size_t)y * W;
#define F(u, i) ((int64_t)((u) - (i)) * ((u) - (i)) + gr[i] * gr[i])
        int qn = 0;
        s[0] = 0;
        t[0] = 0;
        for (int u = 1; u < W; u++) {
            while (qn >= 0 && F(t[qn], s[qn]) > F(t[qn], u)) qn--;
            if (qn < 0) {
                qn = 0;
                s[0] = u;
            } else {
                int i = s[qn];
                int64_t num = (int64_t)u * u - (int64_t)i * i + gr[u] * gr[u] - gr[i] * gr[i];
                int64_t w = 1 + floordiv64(num, 2 * (int64_t)(u - i));
                if (w < W) {
                    qn++;
                    s[qn] = u;
                    t[qn] = (int)w;
                }
            }
        }
        for (int u = W - 1; u >= 0; u--) {
            int64_t d = F(u, s[qn]);
            edt[(size_t)y * W + u] = any_bg ? (int32_t)d : INT32_MAX;
            if (u == t[qn]) qn--;
        }
#undef F
    }
    free(s);
    free(t);
    free(g);
}

/* ------------------------------------------------------------------ */
/* Per-object features (Sec. II feature families; Sec. V-A transforms) */
/* ------------------------------------------------------------------ */

static const int GLCM_DX[4] = {1, 0, 1, 1};
static const int GLCM_DY[4] = {0, 1, 1, -1};

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Sobel on hem8 with replicate (clamp-to-edge) border; returns gx^2+gy^2 */
static int sobel_m2(const uint8_t* I, int W, int H, int y, int x) {
#define P(yy, xx) ((int)I[(size_t)clampi(yy, 0, H - 1) * W + clampi(xx, 0, W - 1)])
    int gx = (P(y - 1, x + 1) + 2 * P(y, x + 1) + P(y + 1, x + 1)) -
             (P(y - 1, x - 1) + 2 * P(y, x - 1) + P(y + 1, x - 1));
    int gy = (P(y + 1, x - 1) + 2 * P(y + 1, x) + P(y + 1, x + 1)) -
             (P(y - 1, x - 1) + 2 * P(y - 1, x) + P(y - 1, x + 1));
#undef P
    return gx * gx + gy * gy;
}

void oracle_features(const uint8_t* hem8, const int32_t* labels, int W, int H, int K,
                     double* feats) {
    if (K <= 0) return;
    long long* n = (long long*)calloc(K + 1, sizeof(long long));
    long long* per = (long long*)calloc(K + 1, sizeof(long long));
    long long* S = (long long*)calloc(K + 1, sizeof(long long));
    long long* Qs = (long long*)calloc(K + 1, sizeof(long long));
    int* mn = (int*)malloc((K + 1) * sizeof(int));
    int* mx = (int*)malloc((K + 1) * sizeof(int));
    double* gs = (double*)calloc(K + 1, sizeof(double));
    double* gss = (double*)calloc(K + 1, sizeof(double));
    int* gmn = (int*)malloc((K + 1) * sizeof(int));
    int* gmx = (int*)malloc((K + 1) * sizeof(int));
    long long* C = (long long*)calloc((size_t)(K + 1) * 4 * 64, sizeof(long long));
    for (int k = 0; k <= K; k++) { mn[k] = INT_MAX; mx[k] = -1; gmn[k] = INT_MAX; gmx[k] = -1; }

    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            size_t p = (size_t)y * W + x;
            int l = labels[p];
            if (l <= 0 || l > K) continue;
            int v = hem8[p];
            n[l]++;
            S[l] += v;
            Qs[l] += (long long)v * v;
            if (v < mn[l]) mn[l] = v;
            if (v > mx[l]) mx[l] = v;
            /* crack length: 4-neighbours outside the object or the image */
            static const int dy4[4] = {-1, 1, 0, 0}, dx4[4] = {0, 0, -1, 1};
            for (int k = 0; k < 4; k++) {
                int yy = y + dy4[k], xx = x + dx4[k];
                if (yy < 0 || yy >= H || xx < 0 || xx >= W || labels[(size_t)yy * W + xx] != l)
                    per[l]++;
            }
            int m2 = sobel_m2(hem8, W, H, y, x);
            gs[l] += sqrt((double)m2);
            if (m2 < gmn[l]) gmn[l] = m2;
            if (m2 > gmx[l]) gmx[l] = m2;
            /* co-occurrence: both ends inside the same object; 8 levels */
            for (int o = 0; o < 4; o++) {
                int yy = y + GLCM_DY[o], xx = x + GLCM_DX[o];
                if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                size_t q = (size_t)yy * W + xx;
                if (labels[q] != l) continue;
                C[((size_t)l * 4 + o) * 64 + (v >> 5) * 8 + (hem8[q] >> 5)]++;
            }
        }
    /* second pass: squared deviations of the gradient magnitude from its mean */
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            size_t p = (size_t)y * W + x;
            int l = labels[p];
            if (l <= 0 || l > K) continue;
            double d = sqrt((double)sobel_m2(hem8, W, H, y, x)) - gs[l] / (double)n[l];
            gss[l] += d * d;
        }

    for (int l = 1; l <= K; l++) {
        double* f = feats + (size_t)(l - 1) * ORACLE_NFEAT;
        if (n[l] == 0) {
            for (int k = 0; k < ORACLE_NFEAT; k++) f[k] = 0.0;
            continue;
        }
        double N = (double)n[l];
        f[0] = N;
        f[1] = (double)per[l];
        f[2] = (double)S[l] / N;
        __int128 var_num = (__int128)n[l] * Qs[l] - (__int128)S[l] * S[l]; /* N*Q - S^2 >= 0 */
        f[3] = sqrt((double)var_num) / N;
        f[4] = mn[l];
        f[5] = mx[l];
        f[6] = gs[l] / N;
        f[7] = sqrt(gss[l] / N);
        f[8] = sqrt((double)gmn[l]);
        f[9] = sqrt((double)gmx[l]);
        double acc[5] = {0, 0, 0, 0, 0};
        int used = 0;
        for (int o = 0; o < 4; o++) {
            const long long* c = C + ((size_t)l * 4 + o) * 64;
            long long T = 0, si = 0, sj = 0, sii = 0, sjj = 0, sij = 0;
            for (int i = 0; i < 8; i++)
                for (int j = 0; j < 8; j++) {
                    long long v = c[i * 8 + j];
                    T += v; si += i * v; sj += j * v;
                    sii += (long long)i * i * v; sjj += (long long)j * j * v; sij += (long long)i * j * v;
                }
            if (T == 0) continue;
            used++;
            double con = 0, ene = 0, hom = 0, ent = 0;
            for (int i = 0; i < 8; i++)
                for (int j = 0; j < 8; j++) {
                    long long v = c[i * 8 + j];
                    if (!v) continue;
                    double P = (double)v / (double)T;
                    con += (double)((i - j) * (i - j)) * P;
                    ene += P * P;
                    hom += P / (1.0 + (double)((i - j) * (i - j)));
                    ent -= P * log(P);
                }
            /* correlation from exact integer moments: T^2 * cov and T^2 * var
               are integers, so a constant marginal gives exactly 0 */
            long long vi = T * sii - si * si, vj = T * sjj - sj * sj, cv = T * sij - si * sj;
            double cor = (vi == 0 || vj == 0) ? 0.0 : (double)cv / sqrt((double)vi * (double)vj);
            acc[0] += con; acc[1] += ene; acc[2] += hom; acc[3] += ent; acc[4] += cor;
        }
        for (int k = 0; k < 5; k++) f[10 + k] = used ? acc[k] / used : 0.0;
    }
    free(n); free(per); free(S); free(Qs); free(mn); free(mx);
    free(gs); free(gss); free(gmn); free(gmx); free(C);
}

/* ---- morphological opening by a disk (Table I "Morph. Open") ---------------
 * Reading: the paper names the operation and its 19 x 19 disk only.  The disk
 * of radius r is {(dx, dy) : dx^2 + dy^2 <= r^2}; pixels outside the image
 * take no part (erosion and dilation range over in-image pixels only). */
void oracle_morph_disk(const uint8_t* src, int W, int H, int r, int is_max, uint8_t* out) {
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int v = is_max ? 0 : 255;
            for (int dy = -r; dy <= r; dy++) {
                const int yy = y + dy;
                if (yy < 0 || yy >= H) continue;
                for (int dx = -r; dx <= r; dx++) {
                    const int xx = x + dx;
                    if (xx < 0 || xx >= W || dx * dx + dy * dy > r * r) continue;
                    const int s = src[(size_t)yy * W + xx];
                    v = is_max ? (s > v ? s : v) : (s < v ? s : v);
                }
            }
            out[(size_t)y * W + x] = (uint8_t)v;
        }
}

int oracle_morph_open(const uint8_t* src, int W, int H, int r, uint8_t* out) {
    if (W <= 0 || H <= 0 || r < 0 || !src || !out) return -1;
    uint8_t* e = (uint8_t*)malloc((size_t)W * H);
    if (!e) return -1;
    oracle_morph_disk(src, W, H, r, 0, e);
    oracle_morph_disk(e, W, H, r, 1, out);
    free(e);
    return 0;
}

/* ---- watershed split of objects (Table I "Pre-Watershed", "Watershed") -------
 * Readings: the paper names the operations only.  Markers are the regional
 * maxima of the h-maxima of the integer distance; flooding goes down the
 * levels of the integer distance in synchronous waves, with ties decided by
 * the squared distance and then the marker's name, so that the result is one
 * exact function of the input (see oracle.h). */
static int isqrt_floor(long long v) {
    if (v <= 0) return 0;
    long long r = (long long)sqrt((double)v);
    while (r * r > v) r--;
    while ((r + 1) * (r + 1) <= v) r++;
    return (int)r;
}

int oracle_watershed(const int32_t* labels, const int32_t* edt, int W, int H, int h, int32_t* out) {
    if (W <= 0 || H <= 0 || h < 0 || !labels || !edt || !out) return -1;
    const size_t N = (size_t)W * H;
    uint8_t* d = (uint8_t*)malloc(N);
    uint8_t* m = (uint8_t*)malloc(N);
    uint8_t* R = (uint8_t*)malloc(N);
    int32_t* name = (int32_t*)malloc(N * sizeof(int32_t));   /* marker / basin name, -1 unset */
    int32_t* nxt = (int32_t*)malloc(N * sizeof(int32_t));
    int32_t* stk = (int32_t*)malloc(N * sizeof(int32_t));
    if (!d || !m || !R || !name || !nxt || !stk) {
        free(d); free(m); free(R); free(name); free(nxt); free(stk);
        return -1;
    }
    for (size_t i = 0; i < N; i++) {
        const int v = labels[i] > 0 ? isqrt_floor(edt[i]) : 0;
        d[i] = (uint8_t)(v > 255 ? 255 : v);
        m[i] = (uint8_t)(d[i] > h ? d[i] - h : 0);
        name[i] = -1;
    }
    oracle_recon(m, d, W, H, R, NULL);
    /* markers: flood each plateau of equal R (object pixels, 8-connected) from
       its first pixel in raster order; it is a marker if no pixel of it has a
       higher neighbour */
    int32_t* plateau = nxt;  /* reused as the plateau id of each pixel */
    for (size_t i = 0; i < N; i++) plateau[i] = -1;
    for (size_t i0 = 0; i0 < N; i0++) {
        if (labels[i0] <= 0 || plateau[i0] >= 0) continue;
        int top = 0, maximal = 1;
        size_t cnt = 0;
        stk[top++] = (int32_t)i0;
        plateau[i0] = (int32_t)i0;
        while (top) {
            const int32_t p = stk[--top];
            cnt++;
            const int y = p / W, x = p - y * W;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    if (!dy && !dx) continue;
                    const int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    const size_t q = (size_t)yy * W + xx;
                    if (labels[q] <= 0) continue;
                    if (R[q] > R[p]) maximal = 0;
                    if (R[q] == R[p] && plateau[q] < 0) {
                        plateau[q] = (int32_t)i0;
                        stk[top++] = (int32_t)q;
                    }
                }
        }
        (void)cnt;
        if (maximal) name[i0] = (int32_t)i0;  /* provisional: spread below */
    }
    for (size_t i = 0; i < N; i++)
        if (labels[i] > 0 && name[plateau[i]] == plateau[i]) name[i] = plateau[i];
    /* flooding in synchronous waves */
    for (;;) {
        long long L = -1;
        for (size_t i = 0; i < N; i++) {
            if (labels[i] <= 0 || name[i] >= 0) continue;
            const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
            int front = 0;
            for (int dy = -1; dy <= 1 && !front; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int yy = y + dy, xx = x + dx;
                    if ((!dy && !dx) || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    if (name[(size_t)yy * W + xx] >= 0) { front = 1; break; }
                }
            if (front && d[i] > L) L = d[i];
        }
        if (L < 0) break;
        for (;;) {
            int n = 0;
            for (size_t i = 0; i < N; i++) {
                nxt[i] = -1;
                if (labels[i] <= 0 || name[i] >= 0 || d[i] < L) continue;
                const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
                int best = -1;
                long long bd = -1;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        const int yy = y + dy, xx = x + dx;
                        if ((!dy && !dx) || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                        const size_t q = (size_t)yy * W + xx;
                        if (name[q] < 0) continue;
                        if (edt[q] > bd || (edt[q] == bd && name[q] < best)) {
                            bd = edt[q];
                            best = name[q];
                        }
                    }
                if (best >= 0) { nxt[i] = best; n++; }
            }
            if (!n) break;
            for (size_t i = 0; i < N; i++)
                if (nxt[i] >= 0) name[i] = nxt[i];
        }
    }
    /* numbering: per object (input label order), basins by first pixel */
    int K = 0;
    for (size_t i = 0; i < N; i++)
        if (labels[i] > K) K = labels[i];
    int* cnt = (int*)calloc((size_t)K + 2, sizeof(int));
    int32_t* first = stk;  /* first[name] = 1 when pixel name's basin starts at pixel i: via a rank map */
    for (size_t i = 0; i < N; i++) first[i] = 0;
    /* rank of a basin inside its object = number of basins of that object
       whose first pixel precedes it; basins are met in raster order of their
       first pixels, so a running count per object gives the rank */
    int32_t* rank = nxt;
    for (size_t i = 0; i < N; i++) rank[i] = 0;
    for (size_t i = 0; i < N; i++) {
        if (labels[i] <= 0) continue;
        const int32_t b = name[i];
        if (!first[b]) {
            first[b] = 1;
            rank[b] = ++cnt[labels[i]];
        }
    }
    int* off = (int*)calloc((size_t)K + 2, sizeof(int));
    int total = 0;
    for (int k = 1; k <= K; k++) {
        off[k] = total;
        total += cnt[k];
    }
    for (size_t i = 0; i < N; i++) out[i] = labels[i] > 0 ? off[labels[i]] + rank[name[i]] : 0;
    free(cnt); free(off);
    free(d); free(m); free(R); free(name); free(nxt); free(stk);
    return total;
}

/* RBC detection: red dominance, then the mask components that hold a marker
 * pixel, found by a breadth-first flood from the markers (raster order of
 * the seeds; the result does not depend on it). */
long long oracle_rbc(const uint8_t* rgb, int W, int H, size_t pitch, int t_lo, int t_hi, uint8_t* out,
                     int16_t* red) {
    if (W < 1 || H < 1 || pitch < (size_t)W * 3 || t_lo < 0 || t_hi < t_lo || t_hi > 255) return -1;
    const size_t N = (size_t)W * H;
    int16_t* d = (int16_t*)malloc(N * sizeof(int16_t));
    int32_t* q = (int32_t*)malloc(N * sizeof(int32_t));
    if (!d || !q) { free(d); free(q); return -1; }
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            const uint8_t* p = rgb + (size_t)y * pitch + (size_t)x * 3;
            const int gb = p[1] > p[2] ? p[1] : p[2];
            d[(size_t)y * W + x] = (int16_t)(p[0] - gb);
        }
    if (red) memcpy(red, d, N * sizeof(int16_t));
    memset(out, 0, N);
    size_t head = 0, tail = 0;
    for (size_t i = 0; i < N; i++)
        if (d[i] >= t_hi) { out[i] = 1; q[tail++] = (int32_t)i; }
    while (head < tail) {
        const int i = q[head++], y = i / W, x = i % W;
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                const int yy = y + dy, xx = x + dx;
                if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                const size_t j = (size_t)yy * W + xx;
                if (!out[j] && d[j] >= t_lo) { out[j] = 1; q[tail++] = (int32_t)j; }
            }
    }
    free(d);
    free(q);
    return (long long)tail;
}

/* ---- Canny edges (Sec. V-A feature-stage transform; Table I "Features
 * comp.") -- readings in oracle.h ------------------------------------------ */

static void sobel_gxgy(const uint8_t* I, int W, int H, int y, int x, int* gx, int* gy) {
    int v[3][3];
    for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++)
            v[dy + 1][dx + 1] = I[(size_t)clampi(y + dy, 0, H - 1) * W + clampi(x + dx, 0, W - 1)];
    *gx = (v[0][2] + 2 * v[1][2] + v[2][2]) - (v[0][0] + 2 * v[1][0] + v[2][0]);
    *gy = (v[2][0] + 2 * v[2][1] + v[2][2]) - (v[0][0] + 2 * v[0][1] + v[0][2]);
}

long long oracle_canny(const uint8_t* I, int W, int H, int low, int high, uint8_t* out, int32_t* mag,
                       uint8_t* cls) {
    if (W < 1 || H < 1 || low < 0 || high < low || !I || !out) return -1;
    const size_t N = (size_t)W * H;
    int32_t* m = (int32_t*)malloc(N * sizeof(int32_t));
    int32_t* gxs = (int32_t*)malloc(N * sizeof(int32_t));
    int32_t* gys = (int32_t*)malloc(N * sizeof(int32_t));
    uint8_t* c = (uint8_t*)malloc(N);
    int32_t* stk = (int32_t*)malloc(N * sizeof(int32_t));
    if (!m || !gxs || !gys || !c || !stk) {
        free(m); free(gxs); free(gys); free(c); free(stk);
        return -1;
    }
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int gx, gy;
            sobel_gxgy(I, W, H, y, x, &gx, &gy);
            const size_t i = (size_t)y * W + x;
            gxs[i] = gx;
            gys[i] = gy;
            m[i] = abs(gx) + abs(gy);
        }
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            const size_t i = (size_t)y * W + x;
            const long long ax = abs(gxs[i]), ay = abs(gys[i]);
            int ay_, ax_, by_, bx_;  /* offsets of a and b */
            if ((ax + ay) * (ax + ay) < 2 * ax * ax) {
                ay_ = 0; ax_ = -1; by_ = 0; bx_ = 1;
            } else if (ay > ax && (ay - ax) * (ay - ax) > 2 * ax * ax) {
                ay_ = -1; ax_ = 0; by_ = 1; bx_ = 0;
            } else if ((long long)gxs[i] * gys[i] > 0) {
                ay_ = -1; ax_ = -1; by_ = 1; bx_ = 1;
            } else {
                ay_ = -1; ax_ = 1; by_ = 1; bx_ = -1;
            }
            const int ya = y + ay_, xa = x + ax_, yb = y + by_, xb = x + bx_;
            const int ma = (ya >= 0 && ya < H && xa >= 0 && xa < W) ? m[(size_t)ya * W + xa] : 0;
            const int mb = (yb >= 0 && yb < H && xb >= 0 && xb < W) ? m[(size_t)yb * W + xb] : 0;
            const int keep = m[i] > ma && m[i] >= mb;
            c[i] = (uint8_t)(keep && m[i] > high ? 2 : (keep && m[i] > low ? 1 : 0));
        }
    /* hysteresis: flood from every strong pixel through candidates, 8-connected */
    memset(out, 0, N);
    long long n = 0;
    for (size_t i0 = 0; i0 < N; i0++) {
        if (c[i0] != 2 || out[i0]) continue;
        int top = 0;
        stk[top++] = (int32_t)i0;
        out[i0] = 1;
        while (top) {
            const int32_t p = stk[--top];
            n++;
            const int y = p / W, x = p - y * W;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int yy = y + dy, xx = x + dx;
                    if ((!dy && !dx) || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    const size_t q = (size_t)yy * W + xx;
                    if (c[q] && !out[q]) {
                        out[q] = 1;
                        stk[top++] = (int32_t)q;
                    }
                }
        }
    }
    if (mag) memcpy(mag, m, N * sizeof(int32_t));
    if (cls) memcpy(cls, c, N);
    free(m); free(gxs); free(gys); free(c); free(stk);
    return n;
}

void oracle_edge_counts(const uint8_t* edges, const int32_t* labels, int W, int H, int K, int r, int32_t* cnt) {
    for (int k = 0; k < K; k++) cnt[k] = 0;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            if (!edges[(size_t)y * W + x]) continue;
            /* the distinct labels within the disk around the pixel, each counted once */
            int seen[64], ns = 0;
            for (int dy = -r; dy <= r; dy++)
                for (int dx = -r; dx <= r; dx++) {
                    const int yy = y + dy, xx = x + dx;
                    if (dx * dx + dy * dy > r * r || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    const int l = labels[(size_t)yy * W + xx];
                    if (l < 1 || l > K) continue;
                    int dup = 0;
                    for (int j = 0; j < ns; j++) dup |= seen[j] == l;
                    if (!dup && ns < 64) seen[ns++] = l;
                }
            for (int j = 0; j < ns; j++) cnt[seen[j] - 1]++;
        }
}

int oracle_seg(const uint8_t* rgb, int W, int H, size_t pitch, int h, int thr, int amin, int amax,
               uint8_t* hem8, uint8_t* R, uint8_t* fg, uint8_t* filled, int32_t* labels,
               int32_t* edt) {
    if (W <= 0 || H <= 0 || pitch < (size_t)W * 3 || !hem8 || !labels) return -1;
    size_t N = (size_t)W * H;
    uint8_t* f = fg ? fg : (uint8_t*)malloc(N);
    uint8_t* fl = filled ? filled : (uint8_t*)malloc(N);
    oracle_deconv(rgb, W, H, pitch, hem8);
    oracle_hdome(hem8, W, H, h, thr, R, f, NULL);
    oracle_fill_holes(f, W, H, fl);
    int K = oracle_label(fl, W, H, amin, amax, labels);
    if (edt) oracle_edt(labels, W, H, edt);
    if (!fg) free(f);
    if (!filled) free(fl);
    return K;
}
