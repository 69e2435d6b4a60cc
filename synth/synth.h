/* Seeded synthetic H&E-like RGB tiles (input generator shared by the CUDA
 * path's tests/benchmarks and the CPU oracle; holds no method arithmetic). */
#ifndef SYNTH_H
#define SYNTH_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif
typedef struct {
    int W, H;             /* tile size in pixels */
    uint64_t seed;        /* all draws derive from this */
    int n_nuclei;         /* ellipses with colour (90,60,140) +-8 */
    double frac_overlap;  /* share placed overlapping the previous single nucleus */
    double frac_cluster;  /* share of draws starting a touching cluster of 2..6 */
    double frac_chain;    /* share of draws starting a chain of 10..30 touching nuclei */
    int n_stroma;         /* discs with colour (200,150,190) +-5 */
    double stroma_rmin, stroma_rmax;
    int corridor;         /* 1: paint a serpentine low-contrast ramp band */
    int n_rbc;            /* red blood cells: discs with colour (200,60,70) +-8 */
} synth_cfg;

/* Writes H rows of W*3 bytes (R,G,B interleaved) at `out` with row pitch
 * `pitch` bytes.  Returns 0, 1 on bad sizes, 2 on allocation failure. */
int synth_tile(const synth_cfg* cfg, uint8_t* out, size_t pitch);
#ifdef __cplusplus
}
#endif
#endif
