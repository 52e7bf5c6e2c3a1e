// Magnetic energy spectrum E_B(k) (Sec. 5, power spectra): B = curl A with
// the first-derivative stencil (the B of every other diagnostic), its
// discrete Fourier transform (cuFFT, real-to-complex, in the working
// precision) and a shell sum in FP64 whose order is fixed, so the result is
// bitwise reproducible.
//
// Shell sum in two passes over the half spectrum (kx >= 0, nh = nx/2 + 1
// modes per row; modes 0 < kx < nx/2 stand for their conjugate partners
// too and count twice):
//   1. one warp per row (ky, kz): along a row |k| grows with kx and the
//      shell index m = floor(|k| + 1/2) rises by at most one per step, so a
//      row's modes form consecutive runs of equal m.  A segmented scan
//      across the warp's lanes (fixed shuffle network) sums each run; the
//      row's sums go to rowsum[row][m - m_min(row)].
//   2. one block per shell m: the sum over rows in row order, then a fixed
//      block tree.
#include <cuda_runtime.h>
#include <cufft.h>

#include <climits>
#include <cmath>

#include "mhd_internal.h"
#include "physics.cuh"
#include "step_device.cuh"

namespace mhd {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SPEC_THREADS = 256;

__device__ __forceinline__ int shell_of(long long k2) { return (int)floor(sqrt((double)k2) + 0.5); }

template <typename T>
__global__ void __launch_bounds__(SPEC_THREADS)
    k_spec_rows(const Cplx<T> *__restrict__ bh, long long odist, int nx, int ny, int nz, double norm,
                double *__restrict__ rowsum, int2 *__restrict__ rowinfo) {
  const int lane = threadIdx.x & 31;
  const long long row = ((long long)blockIdx.x * SPEC_THREADS + threadIdx.x) >> 5;
  const long long nrows = (long long)ny * nz;
  if (row >= nrows) return;  // warp-uniform
  const int nh = nx / 2 + 1;
  const int iz = (int)(row / ny), iy = (int)(row % ny);
  const long long ky = iy <= ny / 2 ? iy : iy - ny;
  const long long kz = iz <= nz / 2 ? iz : iz - nz;
  const long long kyz2 = ky * ky + kz * kz;
  const int smin = shell_of(kyz2);
  const int smax = shell_of((long long)(nh - 1) * (nh - 1) + kyz2);
  const Cplx<T> *r0 = bh + row * nh;
  double *out = rowsum + row * nh;
  double carry = 0.0;
  int cshell = smin;
  for (int base = 0; base < nh; base += 32) {
    const int kx = base + lane;
    const bool v = kx < nh;
    double e = 0.0;
    int s = INT_MAX;
    if (v) {
      double a2 = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const Cplx<T> z = r0[c * odist + kx];
        a2 += (double)z.re * (double)z.re + (double)z.im * (double)z.im;
      }
      const double wgt = (kx == 0 || 2 * kx == nx) ? 1.0 : 2.0;
      e = wgt * norm * a2;
      s = shell_of((long long)kx * kx + kyz2);
    }
    // inclusive scan within runs of equal s (keys do not decrease across lanes)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const double eo = __shfl_up_sync(FULL, e, d);
      const int so = __shfl_up_sync(FULL, s, d);
      if (lane >= d && so == s) e += eo;
    }
    const int s0 = __shfl_sync(FULL, s, 0);
    const int last = min(31, nh - 1 - base);
    const int slast = __shfl_sync(FULL, s, last);
    if (base > 0) {
      if (s0 != cshell) {
        if (lane == 0) out[cshell - smin] = carry;  // the carried run ended at the boundary
      } else if (s == cshell) {
        e += carry;  // the first run continues the carried one
      }
    }
    const int snext = __shfl_down_sync(FULL, s, 1);
    const bool end = v && (lane == last || snext != s);
    if (end && s != slast) out[s - smin] = e;
    carry = __shfl_sync(FULL, e, last);
    cshell = slast;
  }
  if (lane == 0) {
    out[cshell - smin] = carry;
    rowinfo[row] = make_int2(smin, smax);
  }
}

__global__ void __launch_bounds__(SPEC_THREADS)
    k_spec_shells(const double *__restrict__ rowsum, const int2 *__restrict__ rowinfo, long long nrows,
                  int nh, double *__restrict__ out) {
  __shared__ double sh[SPEC_THREADS];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (long long r = threadIdx.x; r < nrows; r += SPEC_THREADS) {
    const int2 mm = rowinfo[r];
    if (s >= mm.x && s <= mm.y) acc += rowsum[r * nh + (s - mm.x)];
  }
  const double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) out[s] = tot;
}

}  // namespace

int spectrum_nshells(int nx, int ny, int nz) {
  const long long hx = nx / 2, hy = ny / 2, hz = nz / 2;
  return (int)std::floor(std::sqrt((double)(hx * hx + hy * hy + hz * hz)) + 0.5) + 1;
}

size_t spectrum_scratch_bytes(int nx, int ny, int nz) {
  const long long nrows = (long long)ny * nz, nh = nx / 2 + 1;
  return (size_t)(nrows * nh * 8 + 16 + nrows * 8 + 16 + (long long)spectrum_nshells(nx, ny, nz) * 8);
}

int launch_spectrum_bins(int dtype, const void *bh, long long odist, int nx, int ny, int nz, void *scratch,
                         double *shells_out, cudaStream_t s) {
  const long long nrows = (long long)ny * nz, nh = nx / 2 + 1;
  const double n = (double)nx * ny * nz;
  const double norm = 0.5 / (n * n);
  char *p = static_cast<char *>(scratch);
  double *rowsum = reinterpret_cast<double *>(p);
  size_t off = (size_t)(nrows * nh * 8 + 15) / 16 * 16;
  int2 *rowinfo = reinterpret_cast<int2 *>(p + off);
  const long long blocks = (nrows * 32 + SPEC_THREADS - 1) / SPEC_THREADS;
  if (dtype == 0)
    k_spec_rows<float><<<(unsigned)blocks, SPEC_THREADS, 0, s>>>(static_cast<const Cplx<float> *>(bh), odist,
                                                                 nx, ny, nz, norm, rowsum, rowinfo);
  else
    k_spec_rows<double><<<(unsigned)blocks, SPEC_THREADS, 0, s>>>(static_cast<const Cplx<double> *>(bh), odist,
                                                                  nx, ny, nz, norm, rowsum, rowinfo);
  int e = (int)cudaGetLastError();
  if (e) return e;
  k_spec_shells<<<spectrum_nshells(nx, ny, nz), SPEC_THREADS, 0, s>>>(rowsum, rowinfo, nrows, (int)nh,
                                                                     shells_out);
  return (int)cudaGetLastError();
}

}  // namespace mhd
