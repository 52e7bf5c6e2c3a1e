/* Debug check of the B300 MHD library: NaN canaries in the alignment padding
 * of the state buffers.  Not part of the method (the paper has no
 * counterpart); it stands in for a memory checker where none can run.
 *
 * Every field of both state buffers is a padded array whose x-rows are px
 * values wide: column 0 and columns nx+7 .. px-1 lie outside the interior
 * (columns 4 .. nx+3) and its periodic ghost zones (1..3 and nx+4..nx+6), and
 * no kernel may read or write them.  mhd_create fills them with NaN; a kernel
 * writing there would replace the canaries, and one reading them would turn
 * its results into NaN. */
#ifndef MHD_CHECK_H
#define MHD_CHECK_H

#include "mhd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Counts the words of the padding columns of both state buffers (all fields,
 * all rows) that are not NaN into *bad (0 when every canary is intact).
 * Synchronising.  Errors: MHD_EINVAL (NULL argument), MHD_ECUDA. */
int mhd_padding_check(mhd_ctx *ctx, long long *bad);

/* Self-test of the bounded waits: one CTA waits, with the bounded mbarrier
 * wait every TMA kernel uses (its poll count cut by a known factor), on an
 * mbarrier that nothing arrives on (no copy is issued: a flag that nothing
 * sets).  The wait must give up and the kernel must report it as the kernels
 * do (status bit 1) and return, leaving the context usable.
 * stream: cudaStream_t (NULL: legacy stream).  *seconds (may be NULL)
 * receives the time the wait took, *kernel_bound_seconds (may be NULL) that
 * time scaled to the kernels' own poll count: how long a TMA kernel waits for
 * a copy before it gives up.  Returns MHD_ETIMEOUT when the wait gave up (the
 * expected outcome), MHD_OK if it completed, MHD_ECUDA on a CUDA error.
 * Synchronising. */
int mhd_wait_selftest(void *stream, double *seconds, double *kernel_bound_seconds);

#ifdef __cplusplus
}
#endif
#endif
