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

namespace mhd {

// ---------------------------------------------------------------------------
// Forcing draw on the device.  Random numbers: SplitMix64 (Steele, Lea &
// Flood 2014) used as a counter-based generator: output c of the stream with
// key `seed` mixes seed + (c + 1) * 0x9E3779B97F4A7C15.  Draw j of step n
// uses counter 64 n + j, so any step's forcing can be regenerated from
// (seed, n) alone -- checkpoints need no generator state.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long key,
                                                         unsigned long long ctr) {
  unsigned long long z = key + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double unit_uniform(unsigned long long key, unsigned long long ctr) {
  return (double)(splitmix64(key, ctr) >> 11) * 0x1.0p-53;  // [0, 1), 53 random bits
}

struct Draw {
  int k[3];
  double phi, e[3], a[3], b[3], kk;
};

// k uniform over the shell list; phi uniform in [-pi, pi); e isotropic,
// redrawn while nearly parallel to k; f_k = a + i b from Eq. 6.
__device__ void forcing_draw(const RunDesc &R, long long step, Draw &D) {
  const double PI = 3.14159265358979323846;
  const unsigned long long ctr0 = (unsigned long long)step * 64ull;
  int idx = (int)(unit_uniform(R.seed, ctr0) * R.nk);
  idx = idx < R.nk - 1 ? idx : R.nk - 1;
  double kp[3];
  for (int d = 0; d < 3; ++d) {
    D.k[d] = R.kshell[3 * idx + d];
    kp[d] = R.kscale[d] * D.k[d];
  }
  D.phi = PI * (2.0 * unit_uniform(R.seed, ctr0 + 1) - 1.0);
  D.kk = sqrt(kp[0] * kp[0] + kp[1] * kp[1] + kp[2] * kp[2]);
  for (int t = 0; t < 31; ++t) {
    const double ez = 2.0 * unit_uniform(R.seed, ctr0 + 2 + 2 * t) - 1.0;
    const double psi = 2.0 * PI * unit_uniform(R.seed, ctr0 + 3 + 2 * t);
    const double r = sqrt(fmax(0.0, 1.0 - ez * ez));
    double sp, cp;
    sincos(psi, &sp, &cp);
    D.e[0] = r * cp;
    D.e[1] = r * sp;
    D.e[2] = ez;
    if (fabs(kp[0] * D.e[0] + kp[1] * D.e[1] + kp[2] * D.e[2]) <= 0.99 * D.kk) break;
  }
  // k x e and k x (k x e)
  const double c1[3] = {kp[1] * D.e[2] - kp[2] * D.e[1], kp[2] * D.e[0] - kp[0] * D.e[2],
                        kp[0] * D.e[1] - kp[1] * D.e[0]};
  const double c2[3] = {kp[1] * c1[2] - kp[2] * c1[1], kp[2] * c1[0] - kp[0] * c1[2],
                        kp[0] * c1[1] - kp[1] * c1[0]};
  const double ke = kp[0] * D.e[0] + kp[1] * D.e[1] + kp[2] * D.e[2];
  const double k2 = D.kk * D.kk;
  const double norm = sqrt(1.0 + R.sigma * R.sigma) * k2 * sqrt(1.0 - ke * ke / k2);
  for (int d = 0; d < 3; ++d) {
    D.a[d] = c2[d] / norm;
    D.b[d] = -R.sigma * D.kk * c1[d] / norm;
  }
}

// Step constants: dt for the update; forcing normalised with dt_forcing
// (Eq. 5: N = f0 cs sqrt(|k| cs / dt)).
__device__ void make_coeffs(const RunDesc &R, long long draw_step, double dt_update,
                            double dt_forcing, int parity, StepCoeffs *C) {
  C->dt = dt_update;
  C->parity = parity;
  C->forcing = 0;
  C->cphi = 1.0;
  C->sphi = 0.0;
  for (int d = 0; d < 3; ++d) {
    C->fa[d] = C->fb[d] = 0.0;
    C->kmod[d] = 0;
  }
  if (R.f0 > 0.0 && R.nk > 0 && dt_forcing > 0.0) {
    Draw D;
    forcing_draw(R, draw_step, D);
    const double amp = R.f0 * R.cs * sqrt(D.kk * R.cs / dt_forcing);
    const int n[3] = {R.nx, R.ny, R.nz};
    for (int d = 0; d < 3; ++d) {
      C->fa[d] = amp * D.a[d];
      C->fb[d] = amp * D.b[d];
      C->kmod[d] = ((D.k[d] % n[d]) + n[d]) % n[d];
    }
    sincos(D.phi, &C->sphi, &C->cphi);
    C->forcing = 1;
  }
}

// ---------------------------------------------------------------------------
// Block reduction helpers (fixed tree order: deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double *sh) {
  const int n = blockDim.x * blockDim.y, t = threadIdx.y * blockDim.x + threadIdx.x;
  __syncthreads();
  sh[t] = v;
  __syncthreads();
  for (int s = n / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  return sh[0];
}

__device__ __forceinline__ double block_max(double v, double *sh) {
  const int n = blockDim.x * blockDim.y, t = threadIdx.y * blockDim.x + threadIdx.x;
  __syncthreads();
  sh[t] = v;
  __syncthreads();
  for (int s = n / 2; s > 0; s >>= 1) {
    if (t < s) {
      const double a = sh[t], b = sh[t + s];
      sh[t] = (isnan(a) || isnan(b)) ? (a + b) : fmax(a, b);
    }
    __syncthreads();
  }
  return sh[0];
}

// Returns true in the one block that finished last among the run's tiles.
__device__ __forceinline__ bool last_tile_done(unsigned int *counter, int ntiles, int *flag_sh) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const unsigned int prev = atomicAdd(counter, 1u);
    *flag_sh = (prev == (unsigned int)(ntiles - 1));
  }
  __syncthreads();
  if (*flag_sh) __threadfence();
  return *flag_sh != 0;
}

template <typename T, int AX>
__device__ __forceinline__ T d1_at(const T *f, long long c, long long stride, const T *w) {
  return w[1] * (f[c + stride] - f[c - stride]) + w[2] * (f[c + 2 * stride] - f[c - 2 * stride]) +
         w[3] * (f[c + 3 * stride] - f[c - 3 * stride]);
}

// ---------------------------------------------------------------------------
// Step prologue
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_prologue(const RunDesc *__restrict__ runs,
                                                  const Tile *__restrict__ tiles) {
  __shared__ double sh[256];
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
    if (x < R.nx && y < R.ny) {
      for (int z = tile.z0; z < tile.z1; ++z) {
        const long long c = ((long long)(z + OZ) * R.py + (y + OY)) * R.px + (x + OX);
        const T *Ax = q + 4 * fs, *Ay = q + 5 * fs, *Az = q + 6 * fs;
        const T Bx = d1_at<T, 1>(Az, c, sy, w[1]) - d1_at<T, 2>(Ay, c, sz, w[2]);
        const T By = d1_at<T, 2>(Ax, c, sz, w[2]) - d1_at<T, 0>(Az, c, 1, w[0]);
        const T Bz = d1_at<T, 0>(Ay, c, 1, w[0]) - d1_at<T, 1>(Ax, c, sy, w[1]);
        const T ux = q[fs + c], uy = q[2 * fs + c], uz = q[3 * fs + c];
        const T v = sqrt(ux * ux + uy * uy + uz * uz) +
                    sqrt(cs2 + (Bx * Bx + By * By + Bz * Bz) * exp(-q[c]));
        const double vd = (double)v;
        vmax = (isnan(vd) || isnan(vmax)) ? vd + vmax : fmax(vmax, vd);
      }
    }
    vmax = block_max(vmax, sh);
  }
  if (threadIdx.x == 0 && threadIdx.y == 0) R.partials[(long long)tile.slot * NPART] = vmax;
  if (!last_tile_done(&R.counter[0], R.ntiles, &flag)) return;
  if (threadIdx.x != 0 || threadIdx.y != 0) return;
  // finalise: this block is the last of the run's tiles
  Clock *clk = R.clock;
  double dt;
  bool bad = false;
  if (R.dt_fixed > 0.0) {
    dt = R.dt_fixed;
  } else {
    double v = 0.0;
    for (int t = 0; t < R.ntiles; ++t) {
      const double p = *((volatile double *)&R.partials[(long long)t * NPART]);
      bad |= !isfinite(p);
      v = fmax(v, p);
    }
    dt = R.cfl * R.dmin / v;
    const double diff = fmax(R.nu, R.eta);
    if (diff > 0.0) dt = fmin(dt, R.cfl_visc * R.dmin * R.dmin / diff);
  }
  bad |= !(dt > 0.0) || !isfinite(dt);
  if (bad) clk->status |= 1;
  make_coeffs(R, step, dt, dt, (int)(step & 1), R.coeffs);
  clk->dt_last = dt;
  clk->t += dt;
  clk->step = step + 1;
  R.counter[0] = 0u;
}

int launch_prologue(int dtype, const RunDesc *runs, const Tile *tiles, int ntiles, int tw, int th,
                    cudaStream_t s) {
  if (ntiles <= 0) return 0;
  if (dtype == 0)
    k_prologue<float><<<ntiles, dim3(tw, th), 0, s>>>(runs, tiles);
  else
    k_prologue<double><<<ntiles, dim3(tw, th), 0, s>>>(runs, tiles);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagnostics: B = curl A into scratch (the RK register, dead between
// steps), periodic halo of B, then one reduction pass.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_curl(const RunDesc *__restrict__ runs,
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
  for (int z = tile.z0; z < tile.z1; ++z) {
    const long long c = ((long long)(z + OZ) * R.py + (y + OY)) * R.px + (x + OX);
    B[c] = d1_at<T, 1>(Az, c, sy, w[1]) - d1_at<T, 2>(Ay, c, sz, w[2]);
    B[fs + c] = d1_at<T, 2>(Ax, c, sz, w[2]) - d1_at<T, 0>(Az, c, 1, w[0]);
    B[2 * fs + c] = d1_at<T, 0>(Ay, c, 1, w[0]) - d1_at<T, 1>(Ax, c, sy, w[1]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_diag(const RunDesc *__restrict__ runs,
                                              const Tile *__restrict__ tiles) {
  __shared__ double sh[256];
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
  double su2 = 0, sb2 = 0, sk = 0, sm = 0, mu = 0, mb = 0, mv = 0, md = 0;
  const int x = tile.x0 + threadIdx.x, y = tile.y0 + threadIdx.y;
  if (x < R.nx && y < R.ny) {
    for (int z = tile.z0; z < tile.z1; ++z) {
      const long long c = ((long long)(z + OZ) * R.py + (y + OY)) * R.px + (x + OX);
      const double ux = q[fs + c], uy = q[2 * fs + c], uz = q[3 * fs + c];
      const double bx = B[c], by = B[fs + c], bz = B[2 * fs + c];
      const double u2 = ux * ux + uy * uy + uz * uz, b2 = bx * bx + by * by + bz * bz;
      const double rho = exp((double)q[c]);
      const double div = (double)(d1_at<T, 0>(B, c, 1, w[0]) + d1_at<T, 1>(B + fs, c, sy, w[1]) +
                                  d1_at<T, 2>(B + 2 * fs, c, sz, w[2]));
      su2 += u2;
      sb2 += b2;
      sk += rho * u2;
      sm += rho;
      mu = fmax(mu, sqrt(u2));
      mb = fmax(mb, sqrt(b2));
      mv = fmax(mv, sqrt(u2) + sqrt(cs2 + b2 / rho));
      md = fmax(md, fabs(div));
    }
  }
  const double vals[NPART] = {su2, sb2, sk, sm, mu, mb, mv, md};
  double red[NPART];
  for (int i = 0; i < 4; ++i) red[i] = block_sum(vals[i], sh);
  for (int i = 4; i < NPART; ++i) red[i] = block_max(vals[i], sh);
  if (threadIdx.x == 0 && threadIdx.y == 0)
    for (int i = 0; i < NPART; ++i) R.partials[(long long)tile.slot * NPART + i] = red[i];
  if (!last_tile_done(&R.counter[1], R.ntiles, &flag)) return;
  if (threadIdx.x != 0 || threadIdx.y != 0) return;
  double tot[NPART] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int t = 0; t < R.ntiles; ++t)
    for (int i = 0; i < NPART; ++i) {
      const double p = *((volatile double *)&R.partials[(long long)t * NPART + i]);
      tot[i] = i < 4 ? tot[i] + p : fmax(tot[i], p);
    }
  const double n = (double)R.nx * R.ny * R.nz;
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
