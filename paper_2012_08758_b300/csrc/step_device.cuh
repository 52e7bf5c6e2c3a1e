// Device-side pieces of a time step shared by the kernels: the forcing draw
// (Sec. 4, Eqs. 4-6), the step constants, deterministic block reductions and
// the end-of-prologue finaliser (dt, forcing of the step, device clock).
#pragma once
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
__device__ __forceinline__ void forcing_draw(const RunDesc &R, long long step, Draw &D) {
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
__device__ __forceinline__ void make_coeffs(const RunDesc &R, long long draw_step, double dt_update,
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
    const int n[3] = {R.nx, R.ny, R.nzg};  // k mod N of the whole (possibly decomposed) grid
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
// Block reduction helpers (fixed order: deterministic).
// ---------------------------------------------------------------------------
// A butterfly of warp shuffles inside each warp, the warp results through
// shared memory, then the same butterfly in the first warp.  Every lane of a
// butterfly ends with the same value (both combining operations are
// commutative), and the order is fixed, so the result is bitwise
// reproducible.  Blocks are whole warps (every launch uses 32 x TY, 256 or
// 1024 threads); sh holds at least one double per warp.
__device__ __forceinline__ double nan_max(double a, double b) {
  return (isnan(a) || isnan(b)) ? (a + b) : fmax(a, b);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
  const int nw = (blockDim.x * blockDim.y) >> 5, t = threadIdx.y * blockDim.x + threadIdx.x;
  v = warp_sum(v);
  __syncthreads();  // sh[0] may still be read after the previous call
  if ((t & 31) == 0) sh[t >> 5] = v;
  __syncthreads();
  if (t < 32) {
    const double w = warp_sum(t < nw ? sh[t] : 0.0);
    __syncwarp();
    if (t == 0) sh[0] = w;
  }
  __syncthreads();
  return sh[0];
}

// Maximum with NaN kept (a non-finite partial poisons the result).
__device__ __forceinline__ double block_max(double v, double *sh) {
  const int nw = (blockDim.x * blockDim.y) >> 5, t = threadIdx.y * blockDim.x + threadIdx.x;
  v = warp_max(v);
  __syncthreads();
  if ((t & 31) == 0) sh[t >> 5] = v;
  __syncthreads();
  if (t < 32) {
    const double w = warp_max(t < nw ? sh[t] : -INFINITY);
    __syncwarp();
    if (t == 0) sh[0] = w;
  }
  __syncthreads();
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

// Called by every thread of the last block of a run in a step prologue
// (sh: blockDim-sized shared scratch): reduces the per-tile maxima (nsub per
// tile slot) in parallel, then thread 0 sets dt (CFL rule or dt_fixed),
// draws the forcing of this step, writes the step constants and advances
// the clock.
__device__ __forceinline__ void finalize_step(const RunDesc &R, long long step, int nsub, double *sh) {
  const int nthr = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (R.dt_fixed <= 0.0 && R.clock->cache_tag == step + 1) {
    v = R.clock->cache_vmax;  // taken by a B_rms reduction of this very state
  } else if (R.dt_fixed <= 0.0) {
    const int n = R.ntiles * nsub;
    for (int i = tid; i < n; i += nthr) {
      const double p = __ldcg(&R.partials[(long long)(i / nsub) * NPART + (i % nsub)]);
      // a non-finite tile maximum poisons the result (block_max keeps NaN)
      v = isfinite(p) ? fmax(v, p) : __longlong_as_double(0x7ff8000000000000ll);
      if (!isfinite(p)) break;
    }
  }
  v = block_max(v, sh);
  if (tid != 0) return;
  Clock *clk = R.clock;
  double dt;
  bool bad = false;
  if (R.dt_fixed > 0.0) {
    dt = R.dt_fixed;
  } else {
    bad = !isfinite(v);
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

}  // namespace mhd
