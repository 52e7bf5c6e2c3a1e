// Tile variants of the paired-point substep kernel (kernels_x2.cu), FP32:
// id -> (TY rows of 64 points, TMA stages, planes between CTA barriers,
// warp-specialised, interleaved w layout).  Each thread computes two
// neighbouring x-points; a CTA of 32 x TY compute threads covers a 64 x TY
// column.  Prefetch distance NS - 3 - BAR >= 1 planes (tiles 23, 24: two and
// three planes ahead).
// Tiles 25-28: a producer warpgroup issues the copies against per-stage
// "empty" mbarriers, no CTA barrier; up to NS - 4 planes ahead.  Tiles 26 and
// 28 (6 stages) and 25 (7) also have room for a ring of 3 / 2 stages of w,
// which the producer fills one output plane at a time.  Tile 28 is tile 26
// with w's fields 0-5 in the interleaved layout (WP): 16-byte w stores and
// ring reads; the FP32 default.
#pragma once
#define MHD_X2_VARIANTS(X) \
  X(17, 8, 6, 2, 0, 0)     \
  X(18, 8, 7, 3, 0, 0)     \
  X(19, 4, 5, 1, 0, 0)     \
  X(20, 6, 6, 2, 0, 0)     \
  X(21, 8, 5, 1, 0, 0)     \
  X(22, 8, 8, 4, 0, 0)     \
  X(23, 8, 8, 3, 0, 0)     \
  X(24, 8, 8, 2, 0, 0)     \
  X(25, 8, 7, 0, 1, 0)     \
  X(26, 8, 6, 0, 1, 0)     \
  X(27, 8, 8, 0, 1, 0)     \
  X(28, 8, 6, 0, 1, 1)
#define MHD_X2_FIRST 17
#define MHD_X2_LAST 28
