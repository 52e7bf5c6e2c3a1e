// mhd_diagnostics_noalloc: the diagnostics reduction for callers that must
// not allocate device memory.  Its scratch (per-block partial sums and the
// last-block counter) is a file-scope static device array of fixed size
// instead of a context workspace.  See include/mhd.h for the contract.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/mhd.h"
#include "mhd_internal.h"
#include "physics.cuh"
#include "step_device.cuh"

namespace mhd {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_THREAD = 16;
constexpr long long NA_CELLS_PER_BLOCK = (long long)NA_THREADS * NA_CELLS_PER_THREAD;
constexpr int NA_MAX_BLOCKS = (int)(MHD_NOALLOC_MAX_POINTS / NA_CELLS_PER_BLOCK);  // 4096
constexpr int NA_HEADER = 32;  // 64-bit words before the partials (counter in word 0)
constexpr int NA_WORDS = NA_HEADER + NA_MAX_BLOCKS * NPART;

// The scratch.  Every GPU that loads this library holds it until the
// process exits (NA_WORDS * 8 bytes = 256 KiB + 256 B).
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NA_WORDS];

int na_fail(int code, const char *msg) {
  set_last_error(msg);  // reported by mhd_last_error(NULL)
  return code;
}

// Device address of g_noalloc_scratch, looked up once per device with that
// device current.  In host code the symbol name is only a host-side stand-in;
// the kernel must be given this address.
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
void *g_na_addr[NA_MAX_DEVICES] = {};

int scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(MHD_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(MHD_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return na_fail(MHD_ECUDA, cudaGetErrorString(e));
    g_na_addr[dev] = p;
  }
  *out = g_na_addr[dev];
  return MHD_OK;
}

struct DenseGrid {
  int nx, ny, nz;
  long long n;  // nx * ny * nz
  double inv_h[3];
  double cs2;
};

template <typename T>
__device__ __forceinline__ long long at(const DenseGrid &g, int i, int j, int k) {
  i = (i % g.nx + g.nx) % g.nx;
  j = (j % g.ny + g.ny) % g.ny;
  k = (k % g.nz + g.nz) % g.nz;
  return ((long long)k * g.ny + j) * g.nx + i;
}

// First derivative along `ax` of field f at (i, j, k), periodic wrap; same
// weights and operation order as the context path.
template <typename T>
__device__ __forceinline__ T d1w(const DenseGrid &g, const T *f, int i, int j, int k, int ax,
                                 const T *w) {
  const int di = ax == 0, dj = ax == 1, dk = ax == 2;
  auto v = [&](int s) { return f[at<T>(g, i + s * di, j + s * dj, k + s * dk)]; };
  return w[1] * (v(1) - v(-1)) + w[2] * (v(2) - v(-2)) + w[3] * (v(3) - v(-3));
}

// Component c of B = curl A at (i, j, k).
template <typename T>
__device__ __forceinline__ T curl_c(const DenseGrid &g, const T *q, int i, int j, int k, int c,
                                    const T (*w)[4]) {
  const T *Ax = q + 4 * g.n, *Ay = q + 5 * g.n, *Az = q + 6 * g.n;
  if (c == 0) return d1w(g, Az, i, j, k, 1, w[1]) - d1w(g, Ay, i, j, k, 2, w[2]);
  if (c == 1) return d1w(g, Ax, i, j, k, 2, w[2]) - d1w(g, Az, i, j, k, 0, w[0]);
  return d1w(g, Ay, i, j, k, 0, w[0]) - d1w(g, Ax, i, j, k, 1, w[1]);
}

template <typename T>
__global__ void __launch_bounds__(NA_THREADS)
    k_diag_noalloc(const T *__restrict__ q, DenseGrid g, unsigned long long *scratch,
                   double *__restrict__ out) {
  __shared__ double sh[NA_THREADS];
  __shared__ int last;
  T w[3][4];
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 4; ++s) w[a][s] = T(W1(s) * g.inv_h[a]);
  double su2 = 0, sb2 = 0, sk = 0, sm = 0, mu = 0, mb = 0, mv = 0, md = 0;
  const long long base = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
  for (int r = 0; r < NA_CELLS_PER_THREAD; ++r) {
    const long long c = base + (long long)r * NA_THREADS + threadIdx.x;
    if (c >= g.n) break;
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((long long)g.nx * g.ny));
    const double ux = q[g.n + c], uy = q[2 * g.n + c], uz = q[3 * g.n + c];
    const double bx = curl_c(g, q, i, j, k, 0, w), by = curl_c(g, q, i, j, k, 1, w),
                 bz = curl_c(g, q, i, j, k, 2, w);
    T div = T(0);
    {
      // div B with the first-derivative stencil applied to B itself
      T dx = T(0), dy = T(0), dz = T(0);
      dx = w[0][1] * (curl_c(g, q, i + 1, j, k, 0, w) - curl_c(g, q, i - 1, j, k, 0, w)) +
           w[0][2] * (curl_c(g, q, i + 2, j, k, 0, w) - curl_c(g, q, i - 2, j, k, 0, w)) +
           w[0][3] * (curl_c(g, q, i + 3, j, k, 0, w) - curl_c(g, q, i - 3, j, k, 0, w));
      dy = w[1][1] * (curl_c(g, q, i, j + 1, k, 1, w) - curl_c(g, q, i, j - 1, k, 1, w)) +
           w[1][2] * (curl_c(g, q, i, j + 2, k, 1, w) - curl_c(g, q, i, j - 2, k, 1, w)) +
           w[1][3] * (curl_c(g, q, i, j + 3, k, 1, w) - curl_c(g, q, i, j - 3, k, 1, w));
      dz = w[2][1] * (curl_c(g, q, i, j, k + 1, 2, w) - curl_c(g, q, i, j, k - 1, 2, w)) +
           w[2][2] * (curl_c(g, q, i, j, k + 2, 2, w) - curl_c(g, q, i, j, k - 2, 2, w)) +
           w[2][3] * (curl_c(g, q, i, j, k + 3, 2, w) - curl_c(g, q, i, j, k - 3, 2, w));
      div = dx + dy + dz;
    }
    const double u2 = ux * ux + uy * uy + uz * uz, b2 = bx * bx + by * by + bz * bz;
    const double rho = exp((double)q[c]);
    su2 += u2;
    sb2 += b2;
    sk += rho * u2;
    sm += rho;
    mu = fmax(mu, sqrt(u2));
    mb = fmax(mb, sqrt(b2));
    mv = fmax(mv, sqrt(u2) + sqrt(g.cs2 + b2 / rho));
    md = fmax(md, fabs((double)div));
  }
  const double vals[NPART] = {su2, sb2, sk, sm, mu, mb, mv, md};
  const int t = threadIdx.x;
  for (int v = 0; v < NPART; ++v) {
    const double r = v < 4 ? block_sum(vals[v], sh) : block_max(vals[v], sh);
    if (t == 0) scratch[NA_HEADER + (long long)blockIdx.x * NPART + v] = __double_as_longlong(r);
  }
  __threadfence();
  __syncthreads();
  if (t == 0) last = (atomicAdd(&scratch[0], 1ull) == (unsigned long long)(gridDim.x - 1));
  __syncthreads();
  if (!last || t != 0) return;
  __threadfence();
  double tot[NPART] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (unsigned b = 0; b < gridDim.x; ++b)
    for (int v = 0; v < NPART; ++v) {
      const double p = __longlong_as_double(
          (long long)*((volatile unsigned long long *)&scratch[NA_HEADER + (long long)b * NPART + v]));
      tot[v] = v < 4 ? tot[v] + p : fmax(tot[v], p);
    }
  const double n = (double)g.n;
  out[0] = sqrt(tot[0] / n);
  out[1] = sqrt(tot[1] / n);
  out[2] = tot[4];
  out[3] = tot[5];
  out[4] = 0.5 * tot[2] / n;
  out[5] = 0.5 * tot[1] / n;
  out[6] = tot[7];
  out[7] = tot[3] / n;
  out[8] = tot[6];
  scratch[0] = 0ull;
}

}  // namespace
}  // namespace mhd

using namespace mhd;

extern "C" int mhd_diagnostics_noalloc(const void *state_dev, int dtype, int nx, int ny, int nz,
                                       double lx, double ly, double lz, double cs, double *out_dev,
                                       void *stream) {
  if (!state_dev || !out_dev) return na_fail(MHD_EINVAL, "state_dev and out_dev must be non-NULL");
  if (dtype != MHD_F32 && dtype != MHD_F64) return na_fail(MHD_EINVAL, "dtype must be MHD_F32 or MHD_F64");
  if (nx < 1 || ny < 1 || nz < 1) return na_fail(MHD_EINVAL, "nx, ny, nz must be >= 1");
  if (!(lx > 0 && ly > 0 && lz > 0) || !(cs > 0)) return na_fail(MHD_EINVAL, "box sizes and cs must be > 0");
  const long long n = (long long)nx * ny * nz;
  const long long blocks = (n + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK;
  if (blocks > NA_MAX_BLOCKS) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "grid of %lld points exceeds the no-allocation limit of %lld points "
             "(%d blocks of %lld points in the static scratch)",
             n, (long long)NA_MAX_BLOCKS * NA_CELLS_PER_BLOCK, NA_MAX_BLOCKS, NA_CELLS_PER_BLOCK);
    return na_fail(MHD_EINVAL, buf);
  }
  void *scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DenseGrid g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.n = n;
  g.inv_h[0] = nx / lx;
  g.inv_h[1] = ny / ly;
  g.inv_h[2] = nz / lz;
  g.cs2 = cs * cs;
  // the counter must start at zero (a previous call that was interrupted
  // could have left it elsewhere); clearing is a memset, not an allocation
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return na_fail(MHD_ECUDA, cudaGetErrorString(e));
  unsigned long long *sc = static_cast<unsigned long long *>(scratch);
  if (dtype == MHD_F32)
    k_diag_noalloc<float><<<(unsigned)blocks, NA_THREADS, 0, s>>>(static_cast<const float *>(state_dev), g, sc, out_dev);
  else
    k_diag_noalloc<double><<<(unsigned)blocks, NA_THREADS, 0, s>>>(static_cast<const double *>(state_dev), g, sc, out_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(MHD_ECUDA, cudaGetErrorString(e));
  return MHD_OK;
}
