// mhd_alu_peak: measured fused multiply-add throughput of the device, the
// denominator of the FP64 step's arithmetic roofline (the FP64 step on B300
// is bound by FP64 FMA throughput, not by HBM).  Contract in
// include/mhd_measure.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "../../include/mhd_measure.h"
#include "mhd_internal.h"

namespace mhd {
namespace {

constexpr int FP_THREADS = 256;
constexpr int FP_BLOCKS_PER_SM = 8;   // 2048 threads per SM: 16 warps per scheduler
constexpr int FP_CHAINS = 8;          // independent chains per thread
constexpr int FP_UNROLL = 16;
constexpr int FP_SINK = 512;          // sink elements (4 KiB of doubles)

__device__ __forceinline__ float fma_op(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_op(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 fma_op(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ double as_double(float v) { return v; }
__device__ __forceinline__ double as_double(double v) { return v; }
__device__ __forceinline__ double as_double(float2 v) { return (double)v.x + (double)v.y; }

template <typename V> __device__ __forceinline__ V seed_value(int t);
template <> __device__ __forceinline__ float seed_value<float>(int t) { return 1e-3f * (float)(t & 63); }
template <> __device__ __forceinline__ double seed_value<double>(int t) { return 1e-3 * (double)(t & 63); }
template <> __device__ __forceinline__ float2 seed_value<float2>(int t) {
  return make_float2(1e-3f * (float)(t & 63), 2e-3f * (float)(t & 31));
}

// a <- a*b + c on FP_CHAINS independent chains; with 0 < b < 1 the chains
// converge to c/(1-b) and stay normal.  The sum of the chains is stored so
// that no chain is dead code.
template <typename V>
__global__ void __launch_bounds__(FP_THREADS) k_fma_peak(double *sink, V b, V c, int iters) {
  const int t = blockIdx.x * FP_THREADS + threadIdx.x;
  V a[FP_CHAINS];
#pragma unroll
  for (int i = 0; i < FP_CHAINS; ++i) a[i] = seed_value<V>(t + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < FP_UNROLL; ++u) {
#pragma unroll
      for (int i = 0; i < FP_CHAINS; ++i) a[i] = fma_op(a[i], b, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < FP_CHAINS; ++i) s += as_double(a[i]);
  sink[t & (FP_SINK - 1)] = s;
}

template <typename V>
int time_peak(V b, V c, int iters, int lanes, cudaStream_t s, double *flops, double *ms_out) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return MHD_ECUDA;
  }
  const int grid = sms * FP_BLOCKS_PER_SM;
  double *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms[5] = {};
  e = cudaMalloc(&sink, FP_SINK * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_fma_peak<V><<<grid, FP_THREADS, 0, s>>>(sink, b, c, iters);  // warm-up
    e = cudaGetLastError();
  }
  for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, s);
    k_fma_peak<V><<<grid, FP_THREADS, 0, s>>>(sink, b, c, iters);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[r], e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return MHD_ECUDA;
  }
  std::sort(ms, ms + 5);
  const double med = ms[2];
  const double ops = 2.0 * lanes * (double)grid * FP_THREADS * (double)iters * FP_UNROLL * FP_CHAINS;
  *flops = ops / (med * 1e-3);
  if (ms_out) *ms_out = med;
  return MHD_OK;
}

}  // namespace
}  // namespace mhd

extern "C" int mhd_alu_peak(int dtype, void *stream, double *flops, double *ms) {
  using namespace mhd;
  if (!flops) {
    set_last_error("mhd_alu_peak: flops is NULL");
    return MHD_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  switch (dtype) {
    case MHD_F32:
      return time_peak<float>(0.999999f, 1e-7f, 8192, 1, s, flops, ms);
    case MHD_F64:
      return time_peak<double>(0.999999, 1e-7, 128, 1, s, flops, ms);
    case 2:
      return time_peak<float2>(make_float2(0.999999f, 0.999998f), make_float2(1e-7f, 2e-7f), 4096, 2, s,
                               flops, ms);
    default:
      set_last_error("mhd_alu_peak: dtype must be MHD_F32, MHD_F64 or 2 (packed FP32 pairs)");
      return MHD_EINVAL;
  }
}
