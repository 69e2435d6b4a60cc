/*
 * CPU oracle for the per-tile nucleus pipeline: plain, slow, single-threaded,
 * FP64 for every floating-point feature.  TEST INFRASTRUCTURE ONLY: it is
 * called by the tests, by the smoke check and by the benchmark's CPU-baseline
 * leg, never by the library.  It shares no code, header or table with the
 * CUDA path; both sides rebuild the colour-deconvolution constants from the
 * same formulas.
 *
 * Paper: Teodoro et al., "High-throughput Execution of Hierarchical Analysis
 * Pipelines on Hybrid Cluster Platforms".  The pipeline is the segmentation
 * and feature stages of Sec. II / Fig. 1; the operations are those of
 * Table I (ReconToNuclei, FillHoles, BWLabel + AreaThreshold, the distance
 * transform of Pre-Watershed) and the feature-stage transforms of Sec. V-A
 * (colour deconvolution, gradient) with the feature families of Sec. II.
 * The paper gives no formulas; the readings taken for every silent point are
 * stated at each function.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_NFEAT 15

/* Fixed-point colour deconvolution constants (Sec. V-A "Color
 * deconvolution"; stain vectors of Ruifrok & Johnston 2001):
 * od_lut[v] = floor(-ln((v+1)/256)*256 + 0.5), wq[c] = round(100*w_c*2^11)
 * with w the hematoxylin column of the inverse stain matrix. */
void oracle_deconv_tables(int32_t od_lut[256], int32_t wq[3], double w[3]);

/* hem8 = clamp((sum_c wq[c]*od_lut[rgb_c] + 2^18) >> 19, 0, 255), 0 when the
 * sum is negative.  rgb: H rows of 3*W bytes at `pitch`; hem8: H*W. */
void oracle_deconv(const uint8_t* rgb, int W, int H, size_t pitch, uint8_t* hem8);

typedef struct {
    long long fifo_pushes;   /* pixels queued by the propagation phase */
    int max_depth;           /* longest chain of queue hops from a seed */
} oracle_recon_stats;

/* Grayscale reconstruction by dilation, 8-connected (Table I
 * "ReconToNuclei": Vincent's MR).  R = lim R_k, R_0 = marker,
 * R_{k+1} = min(dilate8(R_k), mask); neighbours outside the image are
 * ignored.  Algorithm: Vincent 1993 hybrid (raster sweep, anti-raster sweep,
 * FIFO propagation).  Requires marker <= mask; returns -1 otherwise. */
int oracle_recon(const uint8_t* marker, const uint8_t* mask, int W, int H, uint8_t* R,
                 oracle_recon_stats* stats);

/* The plain definition iterated to stability (slow; small inputs).
 * Returns the number of iterations that changed something. */
int oracle_recon_plain(const uint8_t* marker, const uint8_t* mask, int W, int H, uint8_t* R);

/* The plain iteration of oracle_recon_plain, restricted after its first
 * step to the 3x3 neighbourhoods of the previous step's changes (exactly
 * the same sequence R_k).  Returns the number of steps that changed
 * something: the distance, in 8-connected steps, that the slowest front
 * travels.  *evaluated (may be NULL) receives the pixel evaluations. */
int oracle_recon_rounds(const uint8_t* marker, const uint8_t* mask, int W, int H, uint8_t* R,
                        long long* evaluated);

/* h-dome: marker = max(hem8 - h, 0), R = recon(marker | hem8),
 * fg = (hem8 - R >= thr).  R and fg may be NULL. */
void oracle_hdome(const uint8_t* hem8, int W, int H, int h, int thr, uint8_t* R, uint8_t* fg,
                  oracle_recon_stats* stats);

/* Fill holes (Table I "FillHoles"): background pixels not 4-connected,
 * through background, to the image border become foreground. */
void oracle_fill_holes(const uint8_t* fg, int W, int H, uint8_t* filled);

/* 8-connected components of `filled` (Table I "BWLabel"); components whose
 * area lies in [amin, amax] (Table I "AreaThreshold") are numbered 1..K in
 * row-major order of their first pixel, the rest become 0.  Returns K. */
int oracle_label(const uint8_t* filled, int W, int H, int amin, int amax, int32_t* labels);

/* Exact squared Euclidean distance to the nearest pixel with label 0, over
 * in-image pixels (Table I "Pre-Watershed" distance transform); 0 on
 * background; INT32_MAX everywhere when no pixel has label 0.  Algorithm:
 * Meijster, Roerdink, Hesselink 2000 (separable, exact). */
void oracle_edt(const int32_t* labels, int W, int H, int32_t* edt);

/* Per-object features for labels 1..K (Sec. II feature families: pixel
 * statistics, gradient statistics, Haralick texture, morphometry), FP64,
 * feats[K][15]:
 *  0 area, 1 perimeter (crack length), 2 mean, 3 std (population) of hem8,
 *  4 min, 5 max of hem8, 6..9 mean/std/min/max of the Sobel magnitude,
 *  10..14 GLCM contrast, energy, homogeneity, entropy, correlation, averaged
 *  over the offsets (dx,dy) in {(1,0),(0,1),(1,1),(1,-1)} with any pair. */
void oracle_features(const uint8_t* hem8, const int32_t* labels, int W, int H, int K,
                     double* feats);

/* Grayscale erosion (is_max = 0) or dilation (is_max = 1) by a disk of
 * radius r: out(p) = min (max) of src over the in-image pixels q with
 * |q - p|^2 <= r^2 (the disk is the set of integer offsets (dx, dy) with
 * dx^2 + dy^2 <= r^2; r = 9 spans 19 x 19).  Plain definition, O(W H r^2). */
void oracle_morph_disk(const uint8_t* src, int W, int H, int r, int is_max, uint8_t* out);

/* Morphological opening by that disk (Table I "Morph. Open", 19 x 19 disk):
 * the dilation of the erosion.  Returns -1 on bad arguments. */
int oracle_morph_open(const uint8_t* src, int W, int H, int r, uint8_t* out);

/* Watershed split of labelled objects on the distance transform (Table I
 * "Pre-Watershed" and "Watershed"; the paper names the operations only, and
 * states that its CPU and GPU versions differ).  Definition:
 *  d = min(255, floor(sqrt(edt))) on object pixels (labels > 0), 0 elsewhere;
 *  R = reconstruction by dilation, 8-connected, of max(d - h, 0) under d;
 *  markers = maximal 8-connected plateaus of equal R among object pixels
 *    with no 8-neighbour of larger R; a marker is named by the raster index
 *    of its first pixel;
 *  flooding in synchronous waves: with F the unlabelled object pixels that
 *    have a labelled 8-neighbour and L = max of d over F, every pixel of F
 *    with d >= L takes, in one wave, the name of its labelled 8-neighbour
 *    with the largest edt (then the smallest name); waves repeat at L until
 *    none qualifies, then L is taken again from the new F;
 *  out = basins numbered object by object in the order of the input labels,
 *    within an object in raster order of each basin's first pixel; 0 on
 *    background.  Returns the number of basins, or -1 on bad arguments. */
int oracle_watershed(const int32_t* labels, const int32_t* edt, int W, int H, int h, int32_t* out);

/* Canny edge map of a uint8 plane (Sec. V-A lists Canny among the
 * feature-stage transforms applied to the deconvolved image; Table I
 * "Features comp." uses OpenCV's Canny; the paper gives no parameter).
 * Definition:
 *  gx, gy = 3x3 Sobel with replicated border (the gradient of the features);
 *  m = |gx| + |gy|;
 *  sector of the gradient, with ax = |gx|, ay = |gy| (exact integer tests):
 *    horizontal if ay < ax tan(22.5 deg)  <=>  (ax + ay)^2 < 2 ax^2;
 *    vertical   if ay > ax tan(67.5 deg)  <=>  ay > ax and (ay - ax)^2 > 2 ax^2;
 *    otherwise diagonal, along (+x,+y) if gx gy > 0, along (+x,-y) if < 0;
 *  the two neighbours along the sector: a = (y, x-1), b = (y, x+1) for the
 *    horizontal sector; a = (y-1, x), b = (y+1, x) for the vertical one;
 *    a = (y-1, x-1), b = (y+1, x+1) along (+x,+y); a = (y-1, x+1),
 *    b = (y+1, x-1) along (+x,-y); m outside the image counts as 0;
 *  non-maximum suppression: p survives iff m(p) > m(a) and m(p) >= m(b);
 *  candidates: survivors with m > low; strong: survivors with m > high;
 *  edges: candidates 8-connected through candidates to a strong pixel.
 * out = 1 on edges, 0 elsewhere.  mag (may be NULL) receives m; cls (may be
 * NULL) receives 0 / 1 (candidate) / 2 (strong).  Returns -1 on bad
 * arguments (W, H < 1, low < 0 or high < low), else the number of edge
 * pixels. */
long long oracle_canny(const uint8_t* I, int W, int H, int low, int high, uint8_t* out, int32_t* mag,
                       uint8_t* cls);

/* Edge features of the objects (Sec. II "edge" feature family): cnt[k-1] =
 * the number of edge pixels (edges == 1) within the disk dilation of object
 * k, i.e. at an offset (dx, dy) with dx^2 + dy^2 <= r^2 from one of its
 * pixels, k = 1..K (0 <= r <= 4).  The steepest gradient of a nucleus lies
 * on its visible border, a few pixels outside the dome-top mask the
 * segmentation keeps; a pixel near two objects counts for both. */
void oracle_edge_counts(const uint8_t* edges, const int32_t* labels, int W, int H, int K, int r, int32_t* cnt);

/* Red blood cell detection (Table I "RBC detection": OpenCV colour
 * operations and Vincent's MR; the paper gives no definition).  Our reading:
 *  red dominance d = R - max(G, B) per pixel (an integer in [-255, 255]);
 *  marker = {d >= t_hi}, mask = {d >= t_lo}, 0 <= t_lo <= t_hi <= 255;
 *  out = the binary reconstruction by dilation, 8-connected, of the marker
 *    under the mask: 1 on the 8-connected components of the mask that hold
 *    a marker pixel, 0 elsewhere.
 * Plain definition: a breadth-first flood from every marker pixel through
 * the mask.  rgb: H rows of 3*W bytes at `pitch`; out: H*W; red (may be
 * NULL) receives d.  Returns the number of RBC pixels, or -1 on bad
 * arguments. */
long long oracle_rbc(const uint8_t* rgb, int W, int H, size_t pitch, int t_lo, int t_hi, uint8_t* out,
                     int16_t* red);

/* Whole segmentation: deconv -> h-dome -> fill holes -> label -> EDT.
 * Any of R, fg, filled may be NULL.  Returns K, or -1 on bad arguments. */
int oracle_seg(const uint8_t* rgb, int W, int H, size_t pitch, int h, int thr, int amin, int amax,
               uint8_t* hem8, uint8_t* R, uint8_t* fg, uint8_t* filled, int32_t* labels,
               int32_t* edt);

#ifdef __cplusplus
}
#endif
#endif
