/* Measurement helper of the B300 MHD library: the arithmetic-unit peak that
 * the FP64 step is compared against.  Not part of the method; the method's
 * interface is mhd.h.
 *
 * The FP64 step is bound by the GPU's FP64 fused multiply-add throughput,
 * not by HBM bandwidth, so its roofline needs a measured FMA peak of the same
 * device; the FP32 figure is given beside it for the FP32 step's arithmetic. */
#ifndef MHD_MEASURE_H
#define MHD_MEASURE_H

#include "mhd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* FMA throughput of the current device, measured with independent
 * multiply-add chains on every SM (grid: a multiple of the SM count, enough
 * warps per scheduler to hide the pipeline latency).
 *   dtype:   MHD_F32 (scalar fused multiply-add), MHD_F64, or 2 for FP32
 *            packed pairs (two FP32 lanes per instruction).
 *   stream:  cudaStream_t to launch on (NULL: legacy default stream).
 *   flops:   out, floating-point operations per second (an FMA counts 2),
 *            median of five timed launches after one warm-up launch.
 *   ms:      out (may be NULL), median duration of one launch in ms.
 * Synchronises the stream.  Allocates 4 KiB of device memory per call (the
 * sink that keeps the chains alive) and frees it before returning.
 * Returns MHD_OK, MHD_EINVAL for a NULL flops pointer or an unknown dtype,
 * MHD_ECUDA on a CUDA error (message in mhd_last_error(NULL)). */
int mhd_alu_peak(int dtype, void* stream, double* flops, double* ms);

#ifdef __cplusplus
}
#endif
#endif
