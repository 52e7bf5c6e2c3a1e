/* Host-side inspection of the B300 MHD library's work plan: the split of
 * the fused substep over persistent CTAs.  Not part of the method (the paper
 * has no counterpart; its library autotunes a thread-block decomposition,
 * Sec. 3.2); it exists so the plan can be checked without a GPU.
 *
 * The fused substep kernel is persistent and walks a table of tiles, each a
 * (column, z-range): a column is a tw x th block of (x, y) points of one run
 * over all z.  Every CTA takes whole columns first, then a contiguous share
 * of the remaining columns that brings it to the common load; the table is
 * round-robin (entry c + G*j is tile j of CTA c) and padded with empty tiles
 * (z0 == z1). */
#ifndef MHD_PLAN_H
#define MHD_PLAN_H

#include "mhd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The substep plan of a context with parameters p if it ran grid_ctas
 * persistent CTAs (the library uses CTAs-per-SM x SM count, at most 592).
 * Writes up to max_tiles tiles as 5 ints each (x0, y0, z0, z1, run) into
 * tiles (may be NULL), the table length into *ntiles and the number of CTAs
 * the plan uses into *grid.  Host only; no CUDA call.  Errors: MHD_EINVAL
 * (invalid parameters, grid_ctas < 1, NULL ntiles or grid). */
int mhd_substep_plan(const mhd_params *p, int grid_ctas, int *tiles, int max_tiles, int *ntiles, int *grid);

#ifdef __cplusplus
}
#endif
#endif
