// Reductions and per-step set-up kernels:
//  * step prologue: max over the grid of |u| + sqrt(cs^2 + |B|^2 / rho) for
//    the CFL time step, finalised by the last tile of each run, which also
//    draws the forcing of the step (Sec. 4, Eqs. 4-6) and advances the
//    device clock;
//  * diagnostics: FP64-accumulated volume means and maxima (u_rms, B_rms,
//    energies, max |div B|, mass) in a fixed reduction order;
//  * forcing-draw and coefficient set-up helpers.
#include <cuda_runtime.h>

#include "mhd_internal.h"
#include "physics.cuh"
#include "step_device.cuh"

namespace mhd {

template <typename T, int AX>
__device__ __forceinline__ T d1_at(const T *f, long long c, long long stride, const T *w) {
  return d1_vals(f[c + stride], f[c - stride], f[c + 2 * stride], f[c - 2 * stride], f[c + 3 * stride],
                 f[c - 3 * stride], w);
}

// ---------------------------------------------------------------------------
// Step prologue
// ---------------------------------------------------------------------------
// Plain-load version (used with the plane-ring substep kernel); the TMA
// version lives in kernels_tma.cu.  A CTA sweeps its tile along z, so the
// z-neighbours of A stay in L1.
constexpr int PRO_SPLIT = 1;
static_assert(PRO_SPLIT <= NPART, "sub-maxima must fit the tile's partial slot");

template <typename T>
__global__ void __launch_bounds__(MAX_TILE_THREADS) k_prologue(const RunDesc *__restrict__ runs,
                                                  const Tile *__restrict__ tiles) {
  __shared__ double sh[MAX_TILE_THREADS];
  __shared__ int flag;
  const Tile tile = tiles[blockIdx.x];
  const RunDesc &R = runs[tile.run];
  const long long step = R.clock->step;
  double vmax = 0.0;
  if (R.dt_fixed <= 0.0) {
    const T *q = static_cast<const T *>(R.q[step & 1]);
    const long long fs = R.fstride, sy = R.px, sz = (long long)R.px * R.py;
    T w[3][4];
    for (int a = 0; a < 3; ++a)
      for (int s = 0; s < 4; ++s) w[a][s] = T(W1(s) * R.inv_h[a]);
    const T cs2 = T(R.cs2);
    const int x = tile.x0 + threadIdx.x, y = tile.y0 + threadIdx.y;
    // running maximum in the working precision (a maximum is exact in any
    // precision; FP64 per point would run on B300's 1/64-rate FP64 pipe),
    // NaN tracked apart so that a blown-up run still reports NaN
    T vm = T(0);
    bool bad = false;
    if (x < R.nx && y < R.ny) {
      const T *Ax = q + 4 * fs, *Ay = q + 5 * fs, *Az = q + 6 * fs;
      for (int z = tile.z0 + (int)blockIdx.y; z < tile.z1; z += PRO_SPLIT) {
        const long long c = ((long long)(z + OZ) * R.py + (y + OY)) * R.px + (x + OX);
        const T Bx = d1_at<T, 1>(Az, c, sy, w[1]) - d1_at<T, 2>(Ay, c, sz, w[2]);
        const T By = d1_at<T, 2>(Ax, c, sz, w[2]) - d1_at<T, 0>(Az, c, 1, w[0]);
        const T Bz = d1_at<T, 0>(Ay, c, 1, w[0]) - d1_at<T, 1>(Ax, c, sy, w[1]);
        const T ux = q[fs + c], uy = q[2 * fs + c], uz = q[3 * fs + c];
        const T v = sqrt(ux * ux + uy * uy + uz * uz) +
                    sqrt(cs2 + norm2_rn(Bx, By, Bz) * exp(-q[c]));
        bad |= isnan(v);
        vm = fmax(vm, v);
      }
    }
    vmax = bad ? __longlong_as_double(0x7ff8000000000000ll) : (double)vm;
    vmax = block_max(vmax, sh);
  }
  if (threadIdx.x == 0 && threadIdx.y == 0)
    R.partials[(long long)tile.slot * NPART + blockIdx.y] = vmax;
  if (!last_tile_done(&R.counter[0], R.ntiles * PRO_SPLIT, &flag)) return;
  finalize_step(R, step, PRO_SPLIT, sh);
}

int launch_prologue_plain(int dtype, const RunDesc *runs, const Tile *tiles, int ntiles, int tw, int th,
                          cudaStream_t s) {
  if (ntiles <= 0) return 0;
  const dim3 grid(ntiles, PRO_SPLIT);
  if (dtype == 0)
    k_prologue<float><<<grid, dim3(tw, th), 0, s>>>(runs, tiles);
  else
    k_prologue<double><<<grid, dim3(tw, th), 0, s>>>(runs, tiles);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagnostics: B = curl A into scratch (the RK register, dead between
// steps), periodic halo of B, then one reduction pass.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(MAX_TILE_THREADS) k_curl(const RunDesc *__restrict__ runs,
                                              const Tile *__restrict__ tiles) {
  const Tile tile = tiles[blockIdx.x];
  const RunDesc &R = runs[tile.run];
  const T *q = static_cast<const T *>(R.q[R.clock->step & 1]);
  T *B = static_cast<T *>(R.w);
  const long long fs = R.fstride, sy = R.px, sz = (long long)R.px * R.py;
  T w[3][4];
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 4; ++s) w[a][s] = T(W1(s) * R.inv_h[a]);
  const int x = tile.x0 + threadIdx.x, y = tile.y0 + threadIdx.y;
  if (x >= R.nx || y >= R.ny) return;
  const T *Ax = q + 4 * fs, *Ay = q + 5 * fs, *Az = q + 6 * fs;
  // z-neighbours come from L1 (the block sweeps its tile along z); register
  // pencils of A_x, A_y measured 2.4x slower here: at 92 registers only one
  // 12-warp block fits an SM instead of four
  for (int z = tile.z0; z < tile.z1; ++z) {
    const long long c = ((long long)(z + OZ) * R.py + (y + OY)) * R.px + (x + OX);
    B[c] = d1_at<T, 1>(Az, c, sy, w[1]) - d1_at<T, 2>(Ay, c, sz, w[2]);
    B[fs + c] = d1_at<T, 2>(Ax, c, sz, w[2]) - d1_at<T, 0>(Az, c, 1, w[0]);
    B[2 * fs + c] = d1_at<T, 0>(Ay, c, 1, w[0]) - d1_at<T, 1>(Ax, c, sy, w[1]);
  }
}

template <typename T>
__global__ void __launch_bounds__(MAX_TILE_THREADS) k_diag(const RunDesc *__restrict__ runs,
                                              const Tile *__restrict__ tiles) {
  __shared__ double sh[MAX_TILE_THREADS];
  __shared__ int flag;
  const Tile tile = tiles[blockIdx.x];
  const RunDesc &R = runs[tile.run];
  const T *q = static_cast<const T *>(R.q[R.clock->step & 1]);
  const T *B = static_cast<const T *>(R.w);
  const long long fs = R.fstride, sy = R.px, sz = (long long)R.px * R.py;
  T w[3][4];
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 4; ++s) w[a][s] = T(W1(s) * R.inv_h[a]);
  const double cs2 = R.cs2;
  double su2 = 0, sb2 = 0, sk = 0, sm = 0;  // sums: FP64 accumulation
  T mu = 0, mb = 0, mv = 0, md = 0;         // maxima: exact in any precision
  const int x = tile.x0 + threadIdx.x, y = tile.y0 + threadIdx.y;
  if (x < R.nx && y < R.ny) {
    for (int z = tile.z0; z < tile.z1; ++z) {
      const long long c = ((long long)(z + OZ) * R.py + (y + OY)) * R.px + (x + OX);
      // per-point values in the working precision (FP64 arithmetic runs at
      // 1/64 rate on B300), sums accumulated in FP64
      const T ux = q[fs + c], uy = q[2 * fs + c], uz = q[3 * fs + c];
      const T bx = B[c], by = B[fs + c], bz = B[2 * fs + c];
      const T u2 = ux * ux + uy * uy + uz * uz, b2 = norm2_rn(bx, by, bz);
      const T rho = exp(q[c]);
      const T div = d1_at<T, 0>(B, c, 1, w[0]) + d1_at<T, 1>(B + fs, c, sy, w[1]) +
                    d1_at<T, 2>(B + 2 * fs, c, sz, w[2]);
      const T umag = sqrt(u2);
      su2 += (double)u2;
      sb2 += (double)b2;
      sk += (double)(rho * u2);
      sm += (double)rho;
      mu = fmax(mu, umag);
      mb = fmax(mb, sqrt(b2));
      mv = fmax(mv, umag + sqrt(T(cs2) + b2 / rho));
      md = fmax(md, fabs(div));
    }
  }
  const double vals[NPART] = {su2, sb2, sk, sm, (double)mu, (double)mb, (double)mv, (double)md};
  double red[NPART];
  for (int i = 0; i < 4; ++i) red[i] = block_sum(vals[i], sh);
  for (int i = 4; i < NPART; ++i) red[i] = block_max(vals[i], sh);
  if (threadIdx.x == 0 && threadIdx.y == 0)
    for (int i = 0; i < NPART; ++i) R.partials[(long long)tile.slot * NPART + i] = red[i];
  if (!last_tile_done(&R.counter[1], R.ntiles, &flag)) return;
  // the last tile reduces all partials: thread t takes tiles t, t+nthr, ...
  // in order, then the fixed block tree; the order depends only on the tile
  // table, so the result is the same on every run
  const int nthr = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
  double loc[NPART] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int t = tid; t < R.ntiles; t += nthr)
    for (int i = 0; i < NPART; ++i) {
      const double p = __ldcg(&R.partials[(long long)t * NPART + i]);
      loc[i] = i < 4 ? loc[i] + p : fmax(loc[i], p);
    }
  double tot[NPART];
  for (int i = 0; i < 4; ++i) tot[i] = block_sum(loc[i], sh);
  for (int i = 4; i < NPART; ++i) tot[i] = block_max(loc[i], sh);
  if (tid != 0) return;
  const double n = (double)R.nx * R.ny * R.nzg;  // all points of the (possibly decomposed) grid
  R.diag[0] = sqrt(tot[0] / n);  // u_rms
  R.diag[1] = sqrt(tot[1] / n);  // B_rms
  R.diag[2] = tot[4];            // max |u|
  R.diag[3] = tot[5];            // max |B|
  R.diag[4] = 0.5 * tot[2] / n;  // E_kin
  R.diag[5] = 0.5 * tot[1] / n;  // E_mag
  R.diag[6] = tot[7];            // max |div B|
  R.diag[7] = tot[3] / n;        // <rho>
  R.diag[8] = tot[6];            // CFL speed
  R.counter[1] = 0u;
}

// B_rms alone (the quantity sampled every step of a growth-rate run): B = curl A
// straight from the state and sum |B|^2 in FP64, with the tiles, per-thread
// z order, block tree and final tile order of k_diag, so the value equals the
// B_rms of the full diagnostics without storing B or filling its halo.
template <typename T>
__global__ void __launch_bounds__(MAX_TILE_THREADS) k_brms(const RunDesc *__restrict__ runs,
                                              const Tile *__restrict__ tiles) {
  __shared__ double sh[MAX_TILE_THREADS];
  __shared__ int flag;
  const Tile tile = tiles[blockIdx.x];
  const RunDesc &R = runs[tile.run];
  const T *q = static_cast<const T *>(R.q[R.clock->step & 1]);
  const long long fs = R.fstride, sy = R.px, sz = (long long)R.px * R.py;
  T w[3][4];
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 4; ++s) w[a][s] = T(W1(s) * R.inv_h[a]);
  double sb2 = 0;
  const int x = tile.x0 + threadIdx.x, y = tile.y0 + threadIdx.y;
  if (x < R.nx && y < R.ny) {
    const T *Ax = q + 4 * fs, *Ay = q + 5 * fs, *Az = q + 6 * fs;
    for (int z = tile.z0; z < tile.z1; ++z) {
      const long long c = ((long long)(z + OZ) * R.py + (y + OY)) * R.px + (x + OX);
      const T bx = d1_at<T, 1>(Az, c, sy, w[1]) - d1_at<T, 2>(Ay, c, sz, w[2]);
      const T by = d1_at<T, 2>(Ax, c, sz, w[2]) - d1_at<T, 0>(Az, c, 1, w[0]);
      const T bz = d1_at<T, 0>(Ay, c, 1, w[0]) - d1_at<T, 1>(Ax, c, sy, w[1]);
      sb2 += (double)norm2_rn(bx, by, bz);
    }
  }
  const double red = block_sum(sb2, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) R.partials[(long long)tile.slot * NPART + 1] = red;
  if (!last_tile_done(&R.counter[2], R.ntiles, &flag)) return;
  const int nthr = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
  double loc = 0;
  for (int t = tid; t < R.ntiles; t += nthr) loc += __ldcg(&R.partials[(long long)t * NPART + 1]);
  const double tot = block_sum(loc, sh);
  if (tid != 0) return;
  R.diag[1] = sqrt(tot / ((double)R.nx * R.ny * R.nzg));
  R.counter[2] = 0u;
}

int launch_brms(int dtype, const RunDesc *run_dev, const Tile *tiles, int ntiles, int tw, int th,
                cudaStream_t s) {
  if (dtype == 0)
    k_brms<float><<<ntiles, dim3(tw, th), 0, s>>>(run_dev, tiles);
  else
    k_brms<double><<<ntiles, dim3(tw, th), 0, s>>>(run_dev, tiles);
  return (int)cudaGetLastError();
}

int launch_curl(int dtype, const RunDesc *run_dev, const Tile *tiles, int ntiles, int tw, int th,
                cudaStream_t s) {
  if (dtype == 0)
    k_curl<float><<<ntiles, dim3(tw, th), 0, s>>>(run_dev, tiles);
  else
    k_curl<double><<<ntiles, dim3(tw, th), 0, s>>>(run_dev, tiles);
  return (int)cudaGetLastError();
}

int launch_diagnostics(int dtype, const RunDesc *run_dev, const RunDesc &run_host,
                       const Tile *tiles, int ntiles, int tw, int th, cudaStream_t s) {
  int e;
  if (dtype == 0) {
    k_curl<float><<<ntiles, dim3(tw, th), 0, s>>>(run_dev, tiles);
  } else {
    k_curl<double><<<ntiles, dim3(tw, th), 0, s>>>(run_dev, tiles);
  }
  if ((e = (int)cudaGetLastError())) return e;
  if ((e = launch_halo(dtype, run_host.w, 3, run_host.fstride, run_host.nx, run_host.ny,
                       run_host.nz, run_host.px, run_host.py, s)))
    return e;
  if (dtype == 0)
    k_diag<float><<<ntiles, dim3(tw, th), 0, s>>>(run_dev, tiles);
  else
    k_diag<double><<<ntiles, dim3(tw, th), 0, s>>>(run_dev, tiles);
  return (int)cudaGetLastError();
}

// The reduction pass of the diagnostics alone (B and its halo already in
// the RK register): used by decomposed domains, whose B halo along z comes
// from the neighbouring slabs.
int launch_diag_pass(int dtype, const RunDesc *runs, const Tile *tiles, int ntiles, int tw, int th,
                     cudaStream_t s) {
  if (ntiles <= 0) return 0;
  if (dtype == 0)
    k_diag<float><<<ntiles, dim3(tw, th), 0, s>>>(runs, tiles);
  else
    k_diag<double><<<ntiles, dim3(tw, th), 0, s>>>(runs, tiles);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Single-thread helpers
// ---------------------------------------------------------------------------
__global__ void k_coeffs(const RunDesc *R, long long draw_step, double dt_update,
                         double dt_forcing, int parity) {
  make_coeffs(*R, draw_step, dt_update, dt_forcing, parity, R->coeffs);
}

int launch_coeffs(int dtype, const RunDesc *run, int64_t draw_step, double dt_update,
                  double dt_forcing, int parity, cudaStream_t s) {
  (void)dtype;
  k_coeffs<<<1, 1, 0, s>>>(run, (long long)draw_step, dt_update, dt_forcing, parity);
  return (int)cudaGetLastError();
}

__global__ void k_forcing_draw(const RunDesc *R, long long step, double *out) {
  Draw D;
  forcing_draw(*R, step, D);
  for (int d = 0; d < 3; ++d) {
    out[d] = D.k[d];
    out[4 + d] = D.e[d];
    out[7 + d] = D.a[d];
    out[10 + d] = D.b[d];
  }
  out[3] = D.phi;
}

int launch_forcing_draw(const RunDesc *run, int64_t step, double *out13, cudaStream_t s) {
  k_forcing_draw<<<1, 1, 0, s>>>(run, (long long)step, out13);
  return (int)cudaGetLastError();
}

}  // namespace mhd
