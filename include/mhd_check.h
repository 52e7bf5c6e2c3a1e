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

#ifdef __cplusplus
}
#endif
#endif
