// mhd_diagnostics_noalloc: the diagnostics reduction for callers that must
// not allocate device memory.  Its scratch (per-block partial sums and the
// last-block counter) is a file-scope static device array of fixed size
// instead of a context workspace.  See include/mhd.h for the contract.
#include <cuda.h>
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

// Device address of g_noalloc_scratch in the calling thread's current CUDA
// context.  In host code the symbol name is only a host-side stand-in; the
// kernel must be given this address.  The array is instantiated once per
// context, so the address is looked up with cudaGetSymbolAddress once per
// context and cached under the context's unique id (cuCtxGetId): a device
// reset or a new context has a new id and gets a fresh lookup at its first
// call, and a cached address is never used in a context it does not belong to.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

template <typename F>
F driver_fn(const char *name) {
  void *f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(f);
}

constexpr int NA_CACHE = 64;
std::mutex g_na_mu;
unsigned long long g_na_ctx[NA_CACHE] = {};  // context ids (0: empty slot)
void *g_na_addr[NA_CACHE] = {};
int g_na_next = 0;

int scratch_address(void **out) {
  static CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
  static CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
  if (!get_current || !get_id) return na_fail(MHD_ECUDA, "cuCtxGetCurrent / cuCtxGetId not available from the driver");
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return na_fail(MHD_ECUDA, "cuCtxGetCurrent failed");
  cudaError_t e;
  if (!ctx) {
    // no context yet on this thread: make the current device's primary
    // context current (cudaSetDevice initialises it; nothing is allocated)
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e != cudaSuccess) return na_fail(MHD_ECUDA, cudaGetErrorString(e));
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return na_fail(MHD_ECUDA, "no current CUDA context");
  }
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return na_fail(MHD_ECUDA, "cuCtxGetId failed");
  std::lock_guard<std::mutex> lock(g_na_mu);
  for (int i = 0; i < NA_CACHE; ++i)
    if (g_na_ctx[i] == id) {
      *out = g_na_addr[i];
      return MHD_OK;
    }
  void *p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return na_fail(MHD_ECUDA, cudaGetErrorString(e));
  g_na_ctx[g_na_next] = id;
  g_na_addr[g_na_next] = p;
  g_na_next = (g_na_next + 1) % NA_CACHE;
  *out = p;
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

// First derivative along `ax` of field f at (i, j, k), periodic wrap, with
// the fixed rounding sequence every reduction of the library uses (d1_vals).
template <typename T>
__device__ __forceinline__ T d1w(const DenseGrid &g, const T *f, int i, int j, int k, int ax,
                                 const T *w) {
  const int di = ax == 0, dj = ax == 1, dk = ax == 2;
  auto v = [&](int s) { return f[at<T>(g, i + s * di, j + s * dj, k + s * dk)]; };
  return d1_vals(v(1), v(-1), v(2), v(-2), v(3), v(-3), w);
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
  // per-point values in the working precision, sums accumulated in FP64,
  // maxima kept in the working precision (exact): as mhd_diagnostics forms them
  double su2 = 0, sb2 = 0, sk = 0, sm = 0;
  T mu = 0, mb = 0, mv = 0, md = 0;
  const T cs2 = T(g.cs2);
  const long long base = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
  for (int r = 0; r < NA_CELLS_PER_THREAD; ++r) {
    const long long c = base + (long long)r * NA_THREADS + threadIdx.x;
    if (c >= g.n) break;
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((long long)g.nx * g.ny));
    const T ux = q[g.n + c], uy = q[2 * g.n + c], uz = q[3 * g.n + c];
    const T bx = curl_c(g, q, i, j, k, 0, w), by = curl_c(g, q, i, j, k, 1, w), bz = curl_c(g, q, i, j, k, 2, w);
    // div B with the first-derivative stencil applied to B itself
    auto bxa = [&](int s) { return curl_c(g, q, i + s, j, k, 0, w); };
    auto bya = [&](int s) { return curl_c(g, q, i, j + s, k, 1, w); };
    auto bza = [&](int s) { return curl_c(g, q, i, j, k + s, 2, w); };
    const T div = d1_vals(bxa(1), bxa(-1), bxa(2), bxa(-2), bxa(3), bxa(-3), w[0]) +
                  d1_vals(bya(1), bya(-1), bya(2), bya(-2), bya(3), bya(-3), w[1]) +
                  d1_vals(bza(1), bza(-1), bza(2), bza(-2), bza(3), bza(-3), w[2]);
    const T u2 = ux * ux + uy * uy + uz * uz, b2 = norm2_rn(bx, by, bz);
    const T rho = exp(q[c]);
    const T umag = sqrt(u2);
    su2 += (double)u2;
    sb2 += (double)b2;
    sk += (double)(rho * u2);
    sm += (double)rho;
    mu = fmax(mu, umag);
    mb = fmax(mb, sqrt(b2));
    mv = fmax(mv, umag + sqrt(cs2 + b2 / rho));
    md = fmax(md, fabs(div));
  }
  const double vals[NPART] = {su2, sb2, sk, sm, (double)mu, (double)mb, (double)mv, (double)md};
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
