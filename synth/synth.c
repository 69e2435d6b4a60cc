/*
 * Seeded synthetic H&E-like RGB tiles: the shared INPUT of the CUDA path and
 * of the CPU oracle.  It holds none of the segmentation/feature arithmetic;
 * it only paints colours.  The paper's own tiles (glioblastoma 4Kx4K tiles,
 * Sec. V-A) are not available, so these stand in for them with the paper's
 * tile size and its nuclei-per-tile scale (10^5..10^7 nuclei per 50K..100K
 * square slide, Sec. II).
 *
 * Every random draw is a counter-based SplitMix64 value (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014), so pixel
 * noise does not depend on evaluation order and the generator is reentrant
 * across threads.  Noise, blur and rounding are integer arithmetic, so the
 * bytes are the same on every host architecture; only the ellipse geometry
 * uses libm cos/sin.
 *
 * Paint order: background -> stroma blobs -> nuclei -> red blood cells ->
 * serpentine corridor -> per-channel noise (Irwin-Hall sum of 12 uniforms, sd 6) -> separable
 * Gaussian blur sigma 1 (radius 3, mirror border) -> round half to even and
 * clamp to uint8.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include "synth.h"

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* value number `ctr` of stream `stream` under `seed` */
static inline uint64_t rnd(uint64_t seed, uint64_t stream, uint64_t ctr) {
    uint64_t key = sm64_mix(seed * 0x9E3779B97F4A7C15ULL + stream + 1);
    return sm64_mix(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}

typedef struct { uint64_t seed, stream, ctr; } rstream;
static inline uint64_t rs_next(rstream* s) { return rnd(s->seed, s->stream, s->ctr++); }
static inline double rs_unif(rstream* s) { return (double)(rs_next(s) >> 11) * (1.0 / 9007199254740992.0); }
static inline int rs_int(rstream* s, int lo, int hi) { /* inclusive */
    return lo + (int)(rs_next(s) % (uint64_t)(hi - lo + 1));
}

#define Q 256 /* canvas fixed point: value * 256 */

typedef struct { int W, H; int32_t* c; } canvas; /* c: H*W*3 */

static void fill_ellipse(canvas* cv, double cx, double cy, double a, double b, double th,
                         const int col[3]) {
    double ct = cos(th), st = sin(th);
    double r = a > b ? a : b;
    int x0 = (int)floor(cx - r - 1), x1 = (int)ceil(cx + r + 1);
    int y0 = (int)floor(cy - r - 1), y1 = (int)ceil(cy + r + 1);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > cv->W - 1) x1 = cv->W - 1;
    if (y1 > cv->H - 1) y1 = cv->H - 1;
    for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++) {
            double dx = x - cx, dy = y - cy;
            double u = dx * ct + dy * st, v = -dx * st + dy * ct;
            if ((u * u) / (a * a) + (v * v) / (b * b) <= 1.0) {
                int32_t* p = cv->c + ((size_t)y * cv->W + x) * 3;
                p[0] = col[0] * Q; p[1] = col[1] * Q; p[2] = col[2] * Q;
            }
        }
}

static void fill_disc_q(canvas* cv, double cx, double cy, double rad, const int32_t colq[3]) {
    int x0 = (int)floor(cx - rad), x1 = (int)ceil(cx + rad);
    int y0 = (int)floor(cy - rad), y1 = (int)ceil(cy + rad);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > cv->W - 1) x1 = cv->W - 1;
    if (y1 > cv->H - 1) y1 = cv->H - 1;
    for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++) {
            double dx = x - cx, dy = y - cy;
            if (dx * dx + dy * dy <= rad * rad) {
                int32_t* p = cv->c + ((size_t)y * cv->W + x) * 3;
                p[0] = colq[0]; p[1] = colq[1]; p[2] = colq[2];
            }
        }
}

static const int BG[3] = {225, 215, 228};
static const int NUC[3] = {90, 60, 140};
static const int STROMA[3] = {200, 150, 190};
static const int CORR_END[3] = {160, 110, 170};
static const int RBC[3] = {200, 60, 70};

/* one nucleus: semi-axes uniform in [4,12], angle uniform in [0,pi), colour +-8 jitter */
typedef struct { double cx, cy, a, b, th; } nuc;

static nuc draw_nuc(rstream* rs, double cx, double cy) {
    nuc n;
    n.cx = cx; n.cy = cy;
    n.a = 4.0 + 8.0 * rs_unif(rs);
    n.b = 4.0 + 8.0 * rs_unif(rs);
    n.th = M_PI * rs_unif(rs);
    return n;
}
static void paint_nuc(canvas* cv, rstream* rs, const nuc* n) {
    int col[3];
    for (int c = 0; c < 3; c++) col[c] = NUC[c] + rs_int(rs, -8, 8);
    fill_ellipse(cv, n->cx, n->cy, n->a, n->b, n->th, col);
}
static double nuc_rad(const nuc* n) { return 0.5 * (n->a + n->b); }

/* Serpentine band: `runs` horizontal runs 128 px in from the left and right
   edges, joined by vertical runs of 256 px, its colour ramped linearly (in
   RGB) along the arc length from STROMA to CORR_END.  It is painted after
   the nuclei, over a clearance strip of background 14 px wide on each side
   of its centre line, so no nucleus touches it and the reconstruction front
   entering at its high end has to travel along it. */
static void corridor_pass(canvas* cv, int W, int H, double rad, int ramp) {
    const int runs = 3, margin = 128, step = 256;
    const int run_len = W - 2 * margin;
    if (run_len < 16 || H < (runs - 1) * step + 2 * margin) return;
    const double total = (double)runs * run_len + (runs - 1) * step;
    double s = 0.0;
    int x = margin, y = margin, dir = 1;
    for (int r = 0; r < runs; r++) {
        for (int i = 0; i < run_len + (r == runs - 1 ? 0 : step); i++) {
            int32_t colq[3];
            for (int c = 0; c < 3; c++)
                colq[c] = ramp ? (int32_t)llround((STROMA[c] + (CORR_END[c] - STROMA[c]) * (s / total)) * Q)
                               : BG[c] * Q;
            fill_disc_q(cv, x, y, rad, colq);
            if (i < run_len) x += dir; else y += 1;
            s += 1.0;
        }
        dir = -dir;
    }
}

static void paint_corridor(canvas* cv, int W, int H) {
    corridor_pass(cv, W, H, 14.0, 0);
    corridor_pass(cv, W, H, 4.0, 1);
}

/* Q16 taps of exp(-k^2/2), k=-3..3, normalised to sum 65536 */
static const int32_t BLUR[7] = {291, 3539, 15862, 26152, 15862, 3539, 291};

static inline int mirror(int i, int n) {
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * n - 2 - i;
    }
    return i;
}

int synth_tile(const synth_cfg* cfg, uint8_t* out, size_t pitch) {
    int W = cfg->W, H = cfg->H;
    if (W <= 0 || H <= 0 || pitch < (size_t)W * 3) return 1;
    canvas cv = {W, H, NULL};
    size_t n = (size_t)W * H * 3;
    cv.c = (int32_t*)malloc(n * sizeof(int32_t));
    int32_t* tmp = (int32_t*)malloc(n * sizeof(int32_t));
    if (!cv.c || !tmp) { free(cv.c); free(tmp); return 2; }
    for (size_t i = 0; i < (size_t)W * H; i++) {
        cv.c[3 * i + 0] = BG[0] * Q; cv.c[3 * i + 1] = BG[1] * Q; cv.c[3 * i + 2] = BG[2] * Q;
    }
    uint64_t seed = cfg->seed;
    rstream geo = {seed, 1, 0};

    /* stroma: large faint discs, radius in [rmin, rmax], colour +-5 jitter */
    for (int i = 0; i < cfg->n_stroma; i++) {
        double cx = W * rs_unif(&geo), cy = H * rs_unif(&geo);
        double rad = cfg->stroma_rmin + (cfg->stroma_rmax - cfg->stroma_rmin) * rs_unif(&geo);
        int32_t colq[3];
        for (int c = 0; c < 3; c++) colq[c] = (STROMA[c] + rs_int(&geo, -5, 5)) * Q;
        fill_disc_q(&cv, cx, cy, rad, colq);
    }

    /* nuclei: singles, overlapping pairs, touching clusters (2..6), chains */
    int placed = 0;
    nuc prev = {0, 0, 8, 8, 0};
    int have_prev = 0;
    while (placed < cfg->n_nuclei) {
        double u = rs_unif(&geo);
        if (u < cfg->frac_chain) {
            int len = rs_int(&geo, 10, 30);
            nuc n = draw_nuc(&geo, W * rs_unif(&geo), H * rs_unif(&geo));
            double phi = 2 * M_PI * rs_unif(&geo);
            for (int k = 0; k < len && placed < cfg->n_nuclei; k++) {
                paint_nuc(&cv, &geo, &n);
                placed++;
                phi += (rs_unif(&geo) - 0.5);
                nuc m = draw_nuc(&geo, 0, 0);
                double d = 0.85 * (nuc_rad(&n) + nuc_rad(&m));
                m.cx = n.cx + d * cos(phi); m.cy = n.cy + d * sin(phi);
                n = m;
            }
            have_prev = 0;
        } else if (u < cfg->frac_chain + cfg->frac_cluster) {
            int len = rs_int(&geo, 2, 6);
            nuc first = draw_nuc(&geo, W * rs_unif(&geo), H * rs_unif(&geo));
            nuc cur = first;
            for (int k = 0; k < len && placed < cfg->n_nuclei; k++) {
                paint_nuc(&cv, &geo, &cur);
                placed++;
                double phi = 2 * M_PI * rs_unif(&geo);
                nuc m = draw_nuc(&geo, 0, 0);
                double d = 0.9 * (nuc_rad(&cur) + nuc_rad(&m));
                m.cx = cur.cx + d * cos(phi); m.cy = cur.cy + d * sin(phi);
                cur = m;
            }
            have_prev = 0;
        } else if (have_prev && u < cfg->frac_chain + cfg->frac_cluster + cfg->frac_overlap) {
            /* centre distance below a1+a2: overlapping a previous nucleus */
            double phi = 2 * M_PI * rs_unif(&geo);
            nuc m = draw_nuc(&geo, 0, 0);
            double d = (0.3 + 0.4 * rs_unif(&geo)) * (nuc_rad(&prev) + nuc_rad(&m));
            m.cx = prev.cx + d * cos(phi); m.cy = prev.cy + d * sin(phi);
            paint_nuc(&cv, &geo, &m);
            placed++;
            prev = m;
        } else {
            nuc m = draw_nuc(&geo, W * rs_unif(&geo), H * rs_unif(&geo));
            paint_nuc(&cv, &geo, &m);
            placed++;
            prev = m;
            have_prev = 1;
        }
    }

    /* red blood cells: discs of radius uniform in [3.5, 5.5] px, colour +-8
       jitter; 30% of the draws start a touching clump of 2..5 (rouleaux).
       Their draws come from a stream of their own, so the rest of a tile
       does not depend on n_rbc. */
    rstream rbc = {seed, 3, 0};
    for (int placed_rbc = 0; placed_rbc < cfg->n_rbc;) {
        int len = rs_unif(&rbc) < 0.3 ? rs_int(&rbc, 2, 5) : 1;
        double cx = W * rs_unif(&rbc), cy = H * rs_unif(&rbc);
        double rad = 3.5 + 2.0 * rs_unif(&rbc);
        double phi = 2 * M_PI * rs_unif(&rbc);
        for (int k = 0; k < len && placed_rbc < cfg->n_rbc; k++) {
            int32_t colq[3];
            for (int c = 0; c < 3; c++) colq[c] = (RBC[c] + rs_int(&rbc, -8, 8)) * Q;
            fill_disc_q(&cv, cx, cy, rad, colq);
            placed_rbc++;
            double r2 = 3.5 + 2.0 * rs_unif(&rbc);
            phi += 0.6 * (rs_unif(&rbc) - 0.5);
            cx += 0.9 * (rad + r2) * cos(phi);
            cy += 0.9 * (rad + r2) * sin(phi);
            rad = r2;
        }
    }

    if (cfg->corridor) paint_corridor(&cv, W, H);

    /* noise: per pixel and channel, 12 16-bit uniforms from 3 counter draws;
       (sum - 12*32767.5) / 65536 has sd 1; scaled by 6 into Q8 units */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int c = 0; c < 3; c++) {
                uint64_t ctr = (((uint64_t)y * W + x) * 3 + c) * 3;
                int64_t s = 0;
                for (int k = 0; k < 3; k++) {
                    uint64_t r = rnd(seed, 2, ctr + k);
                    s += (int64_t)(r & 0xFFFF) + (int64_t)((r >> 16) & 0xFFFF) +
                         (int64_t)((r >> 32) & 0xFFFF) + (int64_t)(r >> 48);
                }
                int64_t z = (2 * s - 786420) * 6; /* 2*(s - 12*32767.5): sd 1 is 131072 units */
                int32_t nq = (int32_t)(z >= 0 ? (z + 256) / 512 : -((-z + 256) / 512)); /* -> Q8 */
                cv.c[((size_t)y * W + x) * 3 + c] += nq;
            }

    /* separable blur, Q8 in and out, rounding to nearest (ties up) */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int c = 0; c < 3; c++) {
                int64_t acc = 0;
                for (int k = -3; k <= 3; k++)
                    acc += (int64_t)BLUR[k + 3] * cv.c[((size_t)y * W + mirror(x + k, W)) * 3 + c];
                tmp[((size_t)y * W + x) * 3 + c] = (int32_t)((acc + 32768) >> 16);
            }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int c = 0; c < 3; c++) {
                int64_t acc = 0;
                for (int k = -3; k <= 3; k++)
                    acc += (int64_t)BLUR[k + 3] * tmp[((size_t)mirror(y + k, H) * W + x) * 3 + c];
                int32_t v = (int32_t)((acc + 32768) >> 16); /* Q8 */
                int32_t qv = v >> 8, fr = v & 255;
                if (fr > 128 || (fr == 128 && (qv & 1))) qv++;
                if (qv < 0) qv = 0;
                if (qv > 255) qv = 255;
                out[(size_t)y * pitch + (size_t)x * 3 + c] = (uint8_t)qv;
            }
    free(cv.c);
    free(tmp);
    return 0;
}
