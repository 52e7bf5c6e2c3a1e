// Magnetic energy spectrum E_B(k) (Sec. 5, power spectra): B = curl A with
// the first-derivative stencil (the B of every other diagnostic), its
// discrete Fourier transform (cuFFT, real-to-complex, in the working
// precision) and a shell sum in FP64 whose order is fixed, so the result is
// bitwise reproducible.
//
// Shell sum in two passes over the half spectrum (kx >= 0, nh = nx/2 + 1
// modes per row; modes 0 < kx < nx/2 stand for their conjugate partners
// too and count twice):
//   1. one thread per row (ky, kz), k_x in increasing order: along a row
//      |k|^2 = kx^2 + ky^2 + kz^2 grows by 2 kx + 1 per step and the shell
//      m = floor(|k| + 1/2) -- the least m >= 0 with |k|^2 <= m^2 + m, exact
//      in integers -- rises by at most one per step, so each shell's modes
//      of a row are consecutive; their sum goes to rowsum[row][m - m_min(row)].
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

constexpr int SPEC_THREADS = 256;

// Least m >= 0 with k2 <= m^2 + m (= floor(sqrt(k2) + 1/2) for integer k2):
// a single-precision square-root estimate corrected in integers.
__device__ __forceinline__ int shell_of(long long k2) {
  long long m = (long long)sqrtf((float)k2);
  while (m * m + m < k2) ++m;
  while (m > 0 && (m - 1) * (m - 1) + (m - 1) >= k2) --m;
  return (int)m;
}

template <typename T>
__global__ void __launch_bounds__(SPEC_THREADS)
    k_spec_rows(const Cplx<T> *__restrict__ bh, long long odist, int nx, int ny, int nz, double norm,
                double *__restrict__ rowsum, int2 *__restrict__ rowinfo) {
  const long long row = (long long)blockIdx.x * SPEC_THREADS + threadIdx.x;
  const long long nrows = (long long)ny * nz;
  if (row >= nrows) return;
  const int nh = nx / 2 + 1;
  const int iz = (int)(row / ny), iy = (int)(row % ny);
  const long long ky = iy <= ny / 2 ? iy : iy - ny;
  const long long kz = iz <= nz / 2 ? iz : iz - nz;
  const long long kyz2 = ky * ky + kz * kz;
  const int smin = shell_of(kyz2);
  long long m = smin, top = (long long)smin * smin + smin;  // |k|^2 <= top inside shell m
  const Cplx<T> *r0 = bh + row * nh;
  const Cplx<T> *r1 = r0 + odist, *r2 = r1 + odist;
  double *out = rowsum + row * nh;
  double acc = 0.0;
  long long k2 = kyz2;
  for (int kx = 0; kx < nh; ++kx) {
    if (k2 > top) {  // the row leaves shell m (at most one shell per step)
      out[m - smin] = acc;
      acc = 0.0;
      ++m;
      top += 2 * m;
    }
    const Cplx<T> a = r0[kx], b = r1[kx], c = r2[kx];
    const T a2 = a.re * a.re + a.im * a.im + b.re * b.re + b.im * b.im + c.re * c.re + c.im * c.im;
    acc += ((kx == 0 || 2 * kx == nx) ? norm : 2.0 * norm) * (double)a2;
    k2 += 2 * kx + 1;
  }
  out[m - smin] = acc;
  rowinfo[row] = make_int2(smin, (int)m);
}

constexpr int SHELL_THREADS = 1024;

__global__ void __launch_bounds__(SHELL_THREADS)
    k_spec_shells(const double *__restrict__ rowsum, const int2 *__restrict__ rowinfo, long long nrows,
                  int nh, double *__restrict__ out) {
  __shared__ double sh[SHELL_THREADS];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (long long r = threadIdx.x; r < nrows; r += SHELL_THREADS) {
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
  const long long blocks = (nrows + SPEC_THREADS - 1) / SPEC_THREADS;
  if (dtype == 0)
    k_spec_rows<float><<<(unsigned)blocks, SPEC_THREADS, 0, s>>>(static_cast<const Cplx<float> *>(bh), odist,
                                                                 nx, ny, nz, norm, rowsum, rowinfo);
  else
    k_spec_rows<double><<<(unsigned)blocks, SPEC_THREADS, 0, s>>>(static_cast<const Cplx<double> *>(bh), odist,
                                                                  nx, ny, nz, norm, rowsum, rowinfo);
  int e = (int)cudaGetLastError();
  if (e) return e;
  k_spec_shells<<<spectrum_nshells(nx, ny, nz), SHELL_THREADS, 0, s>>>(rowsum, rowinfo, nrows, (int)nh,
                                                                     shells_out);
  return (int)cudaGetLastError();
}

}  // namespace mhd
