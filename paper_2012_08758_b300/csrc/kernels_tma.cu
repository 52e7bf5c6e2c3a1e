// Substep kernel, TMA variant (the fast path).
//
// Same arithmetic as the plane-ring kernel (one stage of the 3rd-order
// 2N-storage Runge-Kutta scheme of Sec. 2 on the right-hand side of
// Eqs. 1-3 with the forcing of Eqs. 4-6), organised for sm_103a:
//
//  * a CTA owns a 32 x TY column and sweeps it along z;
//  * every z-plane of all seven fields (with 3-point x/y halos) is brought
//    into shared memory by one cp.async.bulk.tensor (TMA) copy, issued
//    P = NS-3-BAR planes ahead and completed on an mbarrier, so the memory
//    system always has planes in flight while the SM computes; the CTA
//    synchronises only after every BAR-th plane, so its warps may drift
//    apart by up to BAR planes;
//  * each thread keeps its seven z-values of every field in registers (a
//    pencil), so z-derivatives need no shared-memory traffic;
//  * the mixed derivatives in the x-z and y-z planes are accumulated in
//    registers: the diagonal sum S_s(z0) = dx_s(z0+s) - dx_s(z0-s) is built
//    from the x-differences dx_s = f(x+s) - f(x-s) of each plane as it
//    arrives, so only four planes (output plane to lead plane) must stay in
//    shared memory;
//  * x/y derivatives and the x-y mixed derivatives come from the output
//    plane in shared memory.
// Every wait on an mbarrier is bounded; on time-out the CTA records an
// error in the run's clock (status bit 1), waits (bounded) for the copies it
// issued and returns without writing further results.
#include <cuda.h>
#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mhd_internal.h"
#include "physics.cuh"
#include "step_device.cuh"
#include "tma_util.cuh"
#include "x2_variants.h"

namespace mhd {

using namespace tma;

namespace {


}  // namespace

// One thread waits with the bounded wait, cut to SELFTEST_TRIES polls, on an
// mbarrier that nothing arrives on; out[0] = 2 (status bit 1) when it gave
// up, 0 if it completed.  The kernels' own bound is MAX_TRIES polls, so the
// time of this wait times MAX_TRIES / SELFTEST_TRIES is theirs.
constexpr uint32_t SELFTEST_TRIES = 1u << 10;

__global__ void k_wait_selftest(int *out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) out[0] = mbar_wait<SELFTEST_TRIES>(&bar, 0) ? 0 : 2;
}

int launch_wait_selftest(int *out, cudaStream_t s, double *scale) {
  k_wait_selftest<<<1, 32, 0, s>>>(out);
  if (scale) *scale = (double)MAX_TRIES / SELFTEST_TRIES;
  return (int)cudaGetLastError();
}

template <int V>
struct Phase {
  static constexpr int value = V;
};

template <typename T, int TY, int NS, bool UNROLL7, bool ISO, int BAR>
__global__ void __launch_bounds__(32 * TY, TY <= 6 ? 2 : 1)
    k_substep_tma(const RunDesc *__restrict__ runs, const Tile *__restrict__ tiles, int ntiles,
                  int substep) {
  using SH = TmaShape<T, TY>;
  constexpr int TX = SH::TX, SX = SH::SX, FIELD = SH::FIELD;
  // Prefetch distance in planes.  The CTA synchronises after every BAR-th
  // plane (and after a tile's last one); a stage is refilled NS - P planes
  // after it was the lead plane, i.e. NS - P - 3 planes after it was last read
  // as the output plane, which must be at least BAR planes.
  constexpr int P = NS - 3 - BAR;
  static_assert(P >= 1, "need at least one plane of prefetch");
  static_assert(BAR >= 1 && BAR <= 8, "one to eight planes between barriers");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * SH::STAGE_BYTES);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();

  unsigned long long G = 0;  // planes issued by this CTA before the current tile
  bool failed = false, waits_ok = true;
  int fail_run = -1, fail_p = 0, issued_hi = 0;

  for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
    const Tile tile = tiles[t];
    if (tile.z1 <= tile.z0) continue;  // padding entry of the work split
    const RunDesc &R = runs[tile.run];
    const StepCoeffs &K = *R.coeffs;
    StencilCoefs<T, ISO> c;
    c.load(R);
    const int nx = R.nx, ny = R.ny, nz = R.nz, px = R.px, py = R.py, nzg = R.nzg;
    const bool zper = R.z_open == 0;
    const long long fs = R.fstride;
    const int par = (K.parity + substep) & 1;
    const CUtensorMap *map = &R.tmap[par];
    T *__restrict__ qout = static_cast<T *>(R.q[par ^ 1]);
    T *__restrict__ w = static_cast<T *>(R.w);
    const T dt = T(K.dt);
    const T alpha = T(RK_ALPHA(substep)), beta = T(RK_BETA(substep));
    const int x = tile.x0 + tx, y = tile.y0 + ty;
    const bool active = x < nx && y < ny;
    const bool edge_xy = x < RAD || x >= nx - RAD || y < RAD || y >= ny - RAD;
    const int npl = (tile.z1 - tile.z0) + 2 * RAD;  // lead planes z0-3 .. z1+2

    const bool forcing = K.forcing != 0;
    const bool force_in_rhs = forcing && R.forcing_mode == 0;
    const bool force_at_end = forcing && R.forcing_mode == 1 && substep == 2;
    Cplx<T> exy = {T(1), T(0)};
    T fa[3] = {T(0), T(0), T(0)}, fb[3] = {T(0), T(0), T(0)};
    int mz = 0;  // (k_z * z_out) mod nz, advanced plane by plane
    if (forcing) {
      const Cplx<T> *rx = static_cast<const Cplx<T> *>(R.roots[0]);
      const Cplx<T> *ry = static_cast<const Cplx<T> *>(R.roots[1]);
      if (active)
        exy = cmul(rx[(int)(((long long)K.kmod[0] * x) % nx)], ry[(int)(((long long)K.kmod[1] * y) % ny)]);
      for (int a = 0; a < 3; ++a) {
        fa[a] = T(K.fa[a]);
        fb[a] = T(K.fb[a]);
      }
      mz = (int)(((long long)K.kmod[2] * (tile.z0 + R.z_off)) % R.nzg);  // global plane index
    }
    const int kz = K.kmod[2];
    const Cplx<T> ephi = {T(K.cphi), T(K.sphi)};
    const Cplx<T> *rz = static_cast<const Cplx<T> *>(R.roots[2]);

    // ring position of the first plane of this tile, advanced incrementally
    int slot = (int)(G % NS);
    uint32_t phase = (uint32_t)((G / NS) & 1ull);
    auto issue = [&](int p, int sl) {
      uint64_t *bar = &bars[sl];
      mbar_arrive_expect_tx(bar, (uint32_t)(NF * FIELD * sizeof(T)));
      tma_load_4d(smem + sl * SH::STAGE_BYTES, map, bar, tile.x0, tile.y0, tile.z0 + p, 0);
    };
    if (tid == 0) {
      fence_proxy_async_smem();
      const int first = npl < P ? npl : P;
      for (int p = 0; p < first; ++p) issue(p, (slot + p) % NS);
      issued_hi = first;
    }

    // Register rings (physical index = (logical + phase) mod 7): pencils
    // pen[f][.] hold lead planes p-6 .. p; the accumulators hold the x-z /
    // y-z mixed sums of output planes p-3 .. p+3.
    T pen[NF][7];
    T aX1[7], aY1[7], aZ1[7], aX2[7], aY2[7], aZ2[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
#pragma unroll
      for (int f = 0; f < NF; ++f) pen[f][k] = T(0);
      aX1[k] = aY1[k] = aZ1[k] = aX2[k] = aY2[k] = aZ2[k] = T(0);
    }
    const int cxy = (ty + RAD) * SX + tx + 4;  // thread's point inside a field plane
    const bool need_w = substep > 0 && active;
    const long long wplane = (long long)py * px;
    // index of the output point of lead plane 6 (interior z = z0)
    long long cidx = ((long long)(tile.z0 + OZ) * py + (y + OY)) * px + (x + OX);
    T wn[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) wn[f] = T(0);

    auto plane = [&](auto PHc, int p) {
      constexpr int PH = decltype(PHc)::value;
      auto L = [](int k) { return (k + PH) % 7; };  // logical -> physical ring index
      if (tid == 0 && p + P < npl) {
        fence_proxy_async_smem();
        int sl = slot + P;
        if (sl >= NS) sl -= NS;
        issue(p + P, sl);
        issued_hi = p + P + 1;
      }
      T wc[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) wc[f] = wn[f];
      if (need_w && p >= 2 * RAD - 1 && p + 1 < npl) {
        const T *wp = w + cidx + (p >= 2 * RAD ? wplane : 0);
#pragma unroll
        for (int f = 0; f < NF; ++f, wp += fs) wn[f] = __ldcs(wp);
      }
      const bool ok = mbar_wait(&bars[slot], phase);
      const T *lead = reinterpret_cast<const T *>(smem + slot * SH::STAGE_BYTES) + cxy;
#pragma unroll
      for (int f = 0; f < NF; ++f) pen[f][L(6)] = lead[f * FIELD];
      auto dxs = [&](int f, int s) { return lead[f * FIELD + s] - lead[f * FIELD - s]; };
      auto dys = [&](int f, int s) { return lead[f * FIELD + s * SX] - lead[f * FIELD - s * SX]; };
#pragma unroll
      for (int s = 1; s <= 3; ++s) {
        // plane p adds +w_s dx_s to output plane p-s and -w_s dx_s to p+s
        const T mxz = c.wm(1, s), myz = c.wm(2, s);
        const T ux_ = dxs(1, s), uy_ = dys(2, s), uzx = dxs(3, s), uzy = dys(3, s);
        const T Ax_ = dxs(4, s), Ay_ = dys(5, s), Azx = dxs(6, s), Azy = dys(6, s);
        aX1[L(3 - s)] = fma(mxz, uzx, aX1[L(3 - s)]);   // d_x d_z u_z
        aX1[L(3 + s)] = fma(-mxz, uzx, aX1[L(3 + s)]);
        aY1[L(3 - s)] = fma(myz, uzy, aY1[L(3 - s)]);   // d_y d_z u_z
        aY1[L(3 + s)] = fma(-myz, uzy, aY1[L(3 + s)]);
        aZ1[L(3 - s)] = fma(myz, uy_, fma(mxz, ux_, aZ1[L(3 - s)]));  // d_x d_z u_x + d_y d_z u_y
        aZ1[L(3 + s)] = fma(-myz, uy_, fma(-mxz, ux_, aZ1[L(3 + s)]));
        aX2[L(3 - s)] = fma(mxz, Azx, aX2[L(3 - s)]);   // d_x d_z A_z
        aX2[L(3 + s)] = fma(-mxz, Azx, aX2[L(3 + s)]);
        aY2[L(3 - s)] = fma(myz, Azy, aY2[L(3 - s)]);   // d_y d_z A_z
        aY2[L(3 + s)] = fma(-myz, Azy, aY2[L(3 + s)]);
        aZ2[L(3 - s)] = fma(myz, Ay_, fma(mxz, Ax_, aZ2[L(3 - s)]));  // d_x d_z A_x + d_y d_z A_y
        aZ2[L(3 + s)] = fma(-myz, Ay_, fma(-mxz, Ax_, aZ2[L(3 + s)]));
      }

      if (p >= 2 * RAD && ok && active) {
        const int z = tile.z0 + p - 2 * RAD;  // output plane (interior index)
        int oslot = slot - RAD;
        if (oslot < 0) oslot += NS;
        const T *o = reinterpret_cast<const T *>(smem + oslot * SH::STAGE_BYTES) + cxy;
        auto X = [&](int f, int s) { return o[f * FIELD + s]; };
        auto Y = [&](int f, int s) { return o[f * FIELD + s * SX]; };
        auto D = [&](int f, int sa, int sb) { return o[f * FIELD + sa + sb * SX]; };
        auto Z = [&](int f, int k) { return pen[f][L(k + 3)]; };  // z offset k in -3..3
        auto d1x = [&](int f) {
          return c.w1(0, 1) * (X(f, 1) - X(f, -1)) + c.w1(0, 2) * (X(f, 2) - X(f, -2)) +
                 c.w1(0, 3) * (X(f, 3) - X(f, -3));
        };
        auto d1y = [&](int f) {
          return c.w1(1, 1) * (Y(f, 1) - Y(f, -1)) + c.w1(1, 2) * (Y(f, 2) - Y(f, -2)) +
                 c.w1(1, 3) * (Y(f, 3) - Y(f, -3));
        };
        auto d1z = [&](int f) {
          return c.w1(2, 1) * (Z(f, 1) - Z(f, -1)) + c.w1(2, 2) * (Z(f, 2) - Z(f, -2)) +
                 c.w1(2, 3) * (Z(f, 3) - Z(f, -3));
        };
        auto d2x = [&](int f) {
          return c.w2(0, 0) * Z(f, 0) + c.w2(0, 1) * (X(f, 1) + X(f, -1)) +
                 c.w2(0, 2) * (X(f, 2) + X(f, -2)) + c.w2(0, 3) * (X(f, 3) + X(f, -3));
        };
        auto d2y = [&](int f) {
          return c.w2(1, 0) * Z(f, 0) + c.w2(1, 1) * (Y(f, 1) + Y(f, -1)) +
                 c.w2(1, 2) * (Y(f, 2) + Y(f, -2)) + c.w2(1, 3) * (Y(f, 3) + Y(f, -3));
        };
        auto d2z = [&](int f) {
          return c.w2(2, 0) * Z(f, 0) + c.w2(2, 1) * (Z(f, 1) + Z(f, -1)) +
                 c.w2(2, 2) * (Z(f, 2) + Z(f, -2)) + c.w2(2, 3) * (Z(f, 3) + Z(f, -3));
        };
        auto dxy = [&](int f) {
          T r = T(0);
#pragma unroll
          for (int s = 1; s <= 3; ++s)
            r += c.wm(0, s) * ((D(f, s, s) - D(f, -s, s)) - (D(f, s, -s) - D(f, -s, -s)));
          return r;
        };

        Derivs<T> d;
        d.lnr = Z(0, 0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          d.u[a] = Z(1 + a, 0);
          d.A[a] = Z(4 + a, 0);
        }
        d.g[0] = d1x(0);
        d.g[1] = d1y(0);
        d.g[2] = d1z(0);
        d.up = T(0);
        if (c.upwind)
          d.up = c.w6(0) * fabs(d.u[0]) * delta6(X(0, -3), X(0, -2), X(0, -1), Z(0, 0), X(0, 1), X(0, 2), X(0, 3)) +
                 c.w6(1) * fabs(d.u[1]) * delta6(Y(0, -3), Y(0, -2), Y(0, -1), Z(0, 0), Y(0, 1), Y(0, 2), Y(0, 3)) +
                 c.w6(2) * fabs(d.u[2]) * delta6(Z(0, -3), Z(0, -2), Z(0, -1), Z(0, 0), Z(0, 1), Z(0, 2), Z(0, 3));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          d.G[a][0] = d1x(1 + a);
          d.G[a][1] = d1y(1 + a);
          d.G[a][2] = d1z(1 + a);
        }
        d.gA[0][0] = d.gA[1][1] = d.gA[2][2] = T(0);  // not used by B = curl A
        d.gA[0][1] = d1y(4);
        d.gA[0][2] = d1z(4);
        d.gA[1][0] = d1x(5);
        d.gA[1][2] = d1z(5);
        d.gA[2][0] = d1x(6);
        d.gA[2][1] = d1y(6);
        const T uxx = d2x(1), uxy_ = d2y(1), uxz_ = d2z(1);
        const T uyx = d2x(2), uyy = d2y(2), uyz_ = d2z(2);
        const T uzx = d2x(3), uzy = d2y(3), uzz = d2z(3);
        d.lapu[0] = uxx + uxy_ + uxz_;
        d.lapu[1] = uyx + uyy + uyz_;
        d.lapu[2] = uzx + uzy + uzz;
        d.gdu[0] = uxx + dxy(2) + aX1[L(0)];
        d.gdu[1] = dxy(1) + uyy + aY1[L(0)];
        d.gdu[2] = aZ1[L(0)] + uzz;
        const T Axx = d2x(4), Axy_ = d2y(4), Axz_ = d2z(4);
        const T Ayx = d2x(5), Ayy = d2y(5), Ayz_ = d2z(5);
        const T Azx = d2x(6), Azy = d2y(6), Azz = d2z(6);
        d.lapA[0] = Axx + Axy_ + Axz_;
        d.lapA[1] = Ayx + Ayy + Ayz_;
        d.lapA[2] = Azx + Azy + Azz;
        d.jc[0] = dxy(5) + aX2[L(0)] - Axy_ - Axz_;
        d.jc[1] = dxy(4) + aY2[L(0)] - Ayx - Ayz_;
        d.jc[2] = aZ2[L(0)] - Azx - Azy;

        T f[3] = {T(0), T(0), T(0)};
        if (forcing) {
          const Cplx<T> e = cmul(exy, cmul(rz[mz], ephi));
#pragma unroll
          for (int a = 0; a < 3; ++a) f[a] = fa[a] * e.re - fb[a] * e.im;
        }
        const T fr[3] = {force_in_rhs ? f[0] : T(0), force_in_rhs ? f[1] : T(0), force_in_rhs ? f[2] : T(0)};
        T r[NF];
        rhs_point(d, c, fr, r);
        T qn[NF];
        T *wp = w + cidx;
#pragma unroll
        for (int fld = 0; fld < NF; ++fld, wp += fs) {
          T wv = dt * r[fld];
          if (substep > 0) wv += alpha * wc[fld];
          if (substep < 2) __stcs(wp, wv);
          qn[fld] = Z(fld, 0) + beta * wv;
        }
        if (force_at_end)
          for (int a = 0; a < 3; ++a) qn[1 + a] += dt * f[a];
        store_with_images<T, true>(qout, fs, cidx, qn, edge_xy || z < RAD || z >= nz - RAD, x, y, z, nx, ny, nz,
                                   px, py, zper);
      }
      if (p >= 2 * RAD) {
        cidx += wplane;
        if (forcing) {
          mz += kz;
          if (mz >= nzg) mz -= nzg;
        }
      }
      // retire the accumulators of the output plane: its ring slot becomes
      // the one of output plane p+4 at the next phase
      aX1[L(0)] = aY1[L(0)] = aZ1[L(0)] = aX2[L(0)] = aY2[L(0)] = aZ2[L(0)] = T(0);
      if (++slot == NS) {
        slot = 0;
        phase ^= 1u;
      }
      if constexpr (BAR == 1) {
        if (__syncthreads_or(!ok)) {
          failed = true;
          fail_run = tile.run;
          fail_p = p;
        }
      } else {
        // a wait that gave up between barriers is remembered and caught at
        // the next one; the clean-up then waits again from the earliest
        // plane it could concern
        waits_ok &= ok;
        if (p % BAR == BAR - 1 || p == npl - 1) {
          if (__syncthreads_or(!waits_ok)) {
            failed = true;
            fail_run = tile.run;
            fail_p = p >= BAR - 1 ? p - (BAR - 1) : 0;
          }
        }
      }
    };

    if constexpr (UNROLL7) {
      // seven planes per iteration: the ring indices rotate at compile time
      for (int p = 0; p < npl && !failed; p += 7) {
        plane(Phase<0>{}, p);
        if (p + 1 < npl && !failed) plane(Phase<1>{}, p + 1);
        if (p + 2 < npl && !failed) plane(Phase<2>{}, p + 2);
        if (p + 3 < npl && !failed) plane(Phase<3>{}, p + 3);
        if (p + 4 < npl && !failed) plane(Phase<4>{}, p + 4);
        if (p + 5 < npl && !failed) plane(Phase<5>{}, p + 5);
        if (p + 6 < npl && !failed) plane(Phase<6>{}, p + 6);
      }
    } else {
      // one plane per iteration; the rings are shifted by register moves
      for (int p = 0; p < npl && !failed; ++p) {
        plane(Phase<0>{}, p);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
#pragma unroll
          for (int f = 0; f < NF; ++f) pen[f][k] = pen[f][k + 1];
          aX1[k] = aX1[k + 1]; aY1[k] = aY1[k + 1]; aZ1[k] = aZ1[k + 1];
          aX2[k] = aX2[k + 1]; aY2[k] = aY2[k + 1]; aZ2[k] = aZ2[k + 1];
        }
        aX1[6] = aY1[6] = aZ1[6] = aX2[6] = aY2[6] = aZ2[6] = T(0);
      }
    }
    if (!failed) G += npl;
  }

  if (failed && tid == 0) {
    // record the time-out, then wait (bounded) for the copies still in flight
    atomicOr(&runs[fail_run].clock->status, 2);
    for (int p = fail_p; p < issued_hi; ++p) {
      const unsigned long long g = G + p;
      mbar_wait(&bars[(int)(g % NS)], (uint32_t)((g / NS) & 1ull));
    }
  }
}

// ---------------------------------------------------------------------------
// Packed-FP32 variant (FP32, isotropic grid).  Same pipeline and arithmetic as
// k_substep_tma, but derivatives of two fields that share their stencil
// weights are computed together with the sm_100-family paired FP32
// instructions (__ffma2_rn, __fadd2_rn, __fmul2_rn): (u_x, u_y), (A_x, A_y),
// (u_z, A_z), and cross-axis pairs such as (d_y A_x, d_x A_y) or
// (d_x ln rho, d_y ln rho), whose weights coincide when h_x = h_y = h_z.
// Pencils and the x-z / y-z accumulators are kept as pairs too.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

template <int TY, int NS>
__global__ void __launch_bounds__(32 * TY, 1)
    k_substep_tma_f2(const RunDesc *__restrict__ runs, const Tile *__restrict__ tiles, int ntiles,
                     int substep) {
  using T = float;
  using SH = TmaShape<T, TY>;
  constexpr int TX = SH::TX, SX = SH::SX, F = SH::FIELD;
  constexpr int P = NS - 4;
  static_assert(P >= 1, "need at least one plane of prefetch");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * SH::STAGE_BYTES);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) mbar_init(&bars[q], 1);
    mbar_fence_init();
  }
  __syncthreads();

  unsigned long long G = 0;
  bool failed = false;
  int fail_run = -1, fail_p = 0, issued_hi = 0;

  for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
    const Tile tile = tiles[t];
    if (tile.z1 <= tile.z0) continue;  // padding entry of the work split
    const RunDesc &R = runs[tile.run];
    const StepCoeffs &K = *R.coeffs;
    StencilCoefs<T, true> c;
    c.load(R);
    const float2 M1 = pk(-1.f, -1.f);
    float2 W1[4], W2[4], WMp[4], WMn[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      W1[q] = pk(c.w1(0, q), c.w1(0, q));
      W2[q] = pk(c.w2(0, q), c.w2(0, q));
      WMp[q] = pk(c.wm(0, q), c.wm(0, q));
      WMn[q] = pk(-c.wm(0, q), -c.wm(0, q));
    }
    const int nx = R.nx, ny = R.ny, nz = R.nz, px = R.px, py = R.py, nzg = R.nzg;
    const bool zper = R.z_open == 0;
    const long long fs = R.fstride;
    const int par = (K.parity + substep) & 1;
    const CUtensorMap *map = &R.tmap[par];
    T *__restrict__ qout = static_cast<T *>(R.q[par ^ 1]);
    T *__restrict__ w = static_cast<T *>(R.w);
    const T dt = T(K.dt);
    const T alpha = T(RK_ALPHA(substep)), beta = T(RK_BETA(substep));
    const int x = tile.x0 + tx, y = tile.y0 + ty;
    const bool active = x < nx && y < ny;
    const bool edge_xy = x < RAD || x >= nx - RAD || y < RAD || y >= ny - RAD;
    const int npl = (tile.z1 - tile.z0) + 2 * RAD;

    const bool forcing = K.forcing != 0;
    const bool force_in_rhs = forcing && R.forcing_mode == 0;
    const bool force_at_end = forcing && R.forcing_mode == 1 && substep == 2;
    Cplx<T> exy = {T(1), T(0)};
    T fa[3] = {T(0), T(0), T(0)}, fb[3] = {T(0), T(0), T(0)};
    int mz = 0;
    if (forcing) {
      const Cplx<T> *rx = static_cast<const Cplx<T> *>(R.roots[0]);
      const Cplx<T> *ry = static_cast<const Cplx<T> *>(R.roots[1]);
      if (active)
        exy = cmul(rx[(int)(((long long)K.kmod[0] * x) % nx)], ry[(int)(((long long)K.kmod[1] * y) % ny)]);
      for (int a = 0; a < 3; ++a) {
        fa[a] = T(K.fa[a]);
        fb[a] = T(K.fb[a]);
      }
      mz = (int)(((long long)K.kmod[2] * (tile.z0 + R.z_off)) % R.nzg);  // global plane index
    }
    const int kz = K.kmod[2];
    const Cplx<T> ephi = {T(K.cphi), T(K.sphi)};
    const Cplx<T> *rz = static_cast<const Cplx<T> *>(R.roots[2]);

    int slot = (int)(G % NS);
    uint32_t phase = (uint32_t)((G / NS) & 1ull);
    auto issue = [&](int p, int sl) {
      uint64_t *bar = &bars[sl];
      mbar_arrive_expect_tx(bar, (uint32_t)(NF * F * sizeof(T)));
      tma_load_4d(smem + sl * SH::STAGE_BYTES, map, bar, tile.x0, tile.y0, tile.z0 + p, 0);
    };
    if (tid == 0) {
      fence_proxy_async_smem();
      const int first = npl < P ? npl : P;
      for (int p = 0; p < first; ++p) issue(p, (slot + p) % NS);
      issued_hi = first;
    }

    // pencils: pU = (u_x, u_y), pA = (A_x, A_y), pZ = (u_z, A_z), pL = ln rho;
    // index k holds lead plane p-6+k
    float2 pU[7], pA[7], pZ[7];
    float pL[7];
    // accumulators of output planes p-3 .. p+3:
    // aU = (d_x d_z u_z, d_y d_z u_z), aA = (d_x d_z A_z, d_y d_z A_z),
    // zU = d_x d_z u_x + d_y d_z u_y, zA = d_x d_z A_x + d_y d_z A_y
    float2 aU[7], aA[7];
    float zU[7], zA[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      pU[k] = pA[k] = pZ[k] = aU[k] = aA[k] = pk(0.f, 0.f);
      pL[k] = zU[k] = zA[k] = 0.f;
    }
    const int cxy = (ty + RAD) * SX + tx + 4;
    const bool need_w = substep > 0 && active;
    const long long wplane = (long long)py * px;
    long long cidx = ((long long)(tile.z0 + OZ) * py + (y + OY)) * px + (x + OX);
    T wn[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) wn[f] = T(0);

    for (int p = 0; p < npl && !failed; ++p) {
      if (tid == 0 && p + P < npl) {
        fence_proxy_async_smem();
        int sl = slot + P;
        if (sl >= NS) sl -= NS;
        issue(p + P, sl);
        issued_hi = p + P + 1;
      }
      T wc[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) wc[f] = wn[f];
      if (need_w && p >= 2 * RAD - 1 && p + 1 < npl) {
        const T *wp = w + cidx + (p >= 2 * RAD ? wplane : 0);
#pragma unroll
        for (int f = 0; f < NF; ++f, wp += fs) wn[f] = __ldcs(wp);
      }
      const bool ok = mbar_wait(&bars[slot], phase);
      const T *lead = reinterpret_cast<const T *>(smem + slot * SH::STAGE_BYTES) + cxy;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        pU[k] = pU[k + 1];
        pA[k] = pA[k + 1];
        pZ[k] = pZ[k + 1];
        pL[k] = pL[k + 1];
      }
      pL[6] = lead[0];
      pU[6] = pk(lead[1 * F], lead[2 * F]);
      pZ[6] = pk(lead[3 * F], lead[6 * F]);
      pA[6] = pk(lead[4 * F], lead[5 * F]);
#pragma unroll
      for (int s = 1; s <= 3; ++s) {
        // (f(+s) - f(-s)) along x for the first lane and along y for the second
        const float2 dUZ = fma2(pk(lead[3 * F - s], lead[3 * F - s * SX]), M1, pk(lead[3 * F + s], lead[3 * F + s * SX]));
        const float2 dAZ = fma2(pk(lead[6 * F - s], lead[6 * F - s * SX]), M1, pk(lead[6 * F + s], lead[6 * F + s * SX]));
        const float2 dUU = fma2(pk(lead[1 * F - s], lead[2 * F - s * SX]), M1, pk(lead[1 * F + s], lead[2 * F + s * SX]));
        const float2 dAA = fma2(pk(lead[4 * F - s], lead[5 * F - s * SX]), M1, pk(lead[4 * F + s], lead[5 * F + s * SX]));
        aU[3 - s] = fma2(WMp[s], dUZ, aU[3 - s]);
        aU[3 + s] = fma2(WMn[s], dUZ, aU[3 + s]);
        aA[3 - s] = fma2(WMp[s], dAZ, aA[3 - s]);
        aA[3 + s] = fma2(WMn[s], dAZ, aA[3 + s]);
        const float su = dUU.x + dUU.y, sa = dAA.x + dAA.y;
        zU[3 - s] = fmaf(WMp[s].x, su, zU[3 - s]);
        zU[3 + s] = fmaf(WMn[s].x, su, zU[3 + s]);
        zA[3 - s] = fmaf(WMp[s].x, sa, zA[3 - s]);
        zA[3 + s] = fmaf(WMn[s].x, sa, zA[3 + s]);
      }

      if (p >= 2 * RAD && ok && active) {
        const int z = tile.z0 + p - 2 * RAD;
        int oslot = slot - RAD;
        if (oslot < 0) oslot += NS;
        const T *o = reinterpret_cast<const T *>(smem + oslot * SH::STAGE_BYTES) + cxy;
        // paired first derivative from samples g(s), s = +-1..3
        auto d1p = [&](auto g) {
          const float2 t1 = fma2(g(-1), M1, g(1));
          const float2 t2 = fma2(g(-2), M1, g(2));
          const float2 t3 = fma2(g(-3), M1, g(3));
          return fma2(W1[3], t3, fma2(W1[2], t2, mul2(W1[1], t1)));
        };
        // paired second derivative, centre values c0
        auto d2p = [&](float2 c0, auto g) {
          const float2 s1 = add2(g(1), g(-1)), s2 = add2(g(2), g(-2)), s3 = add2(g(3), g(-3));
          return fma2(W2[3], s3, fma2(W2[2], s2, fma2(W2[1], s1, mul2(W2[0], c0))));
        };
        // paired x-y mixed derivative of fields fa (lane 0) and fb (lane 1)
        auto dxyp = [&](int f0, int f1) {
          float2 r = pk(0.f, 0.f);
#pragma unroll
          for (int q = 1; q <= 3; ++q) {
            auto D = [&](int sa, int sb) { return pk(o[f0 * F + sa + sb * SX], o[f1 * F + sa + sb * SX]); };
            const float2 S = add2(fma2(D(-q, q), M1, D(q, q)), fma2(D(q, -q), M1, D(-q, -q)));
            r = fma2(WMp[q], S, r);
          }
          return r;
        };
        auto xs = [&](int f0, int f1) { return [=](int q) { return pk(o[f0 * F + q], o[f1 * F + q]); }; };
        auto ys = [&](int f0, int f1) { return [=](int q) { return pk(o[f0 * F + q * SX], o[f1 * F + q * SX]); }; };

        Derivs<T> d;
        d.lnr = pL[3];
        d.u[0] = pU[3].x; d.u[1] = pU[3].y; d.u[2] = pZ[3].x;
        d.A[0] = pA[3].x; d.A[1] = pA[3].y; d.A[2] = pZ[3].y;
        const float2 Ux = d1p(xs(1, 2)), Uy = d1p(ys(1, 2)), Uz = d1p([&](int q) { return pU[3 + q]; });
        const float2 Zx = d1p(xs(3, 6)), Zy = d1p(ys(3, 6));
        const float2 Az = d1p([&](int q) { return pA[3 + q]; });
        const float2 Ac = d1p([&](int q) { return pk(o[4 * F + q * SX], o[5 * F + q]); });  // (d_y A_x, d_x A_y)
        const float2 Lg = d1p([&](int q) { return pk(o[q], o[q * SX]); });                   // (d_x ln rho, d_y ln rho)
        const float uzz1 = c.w1(0, 1) * (pZ[4].x - pZ[2].x) + c.w1(0, 2) * (pZ[5].x - pZ[1].x) +
                           c.w1(0, 3) * (pZ[6].x - pZ[0].x);
        const float lz1 = c.w1(0, 1) * (pL[4] - pL[2]) + c.w1(0, 2) * (pL[5] - pL[1]) + c.w1(0, 3) * (pL[6] - pL[0]);
        d.g[0] = Lg.x; d.g[1] = Lg.y; d.g[2] = lz1;
        d.up = 0.f;
        if (c.upwind)
          d.up = c.w6(0) * (fabsf(d.u[0]) * delta6(o[-3], o[-2], o[-1], pL[3], o[1], o[2], o[3]) +
                            fabsf(d.u[1]) * delta6(o[-3 * SX], o[-2 * SX], o[-SX], pL[3], o[SX], o[2 * SX], o[3 * SX]) +
                            fabsf(d.u[2]) * delta6(pL[0], pL[1], pL[2], pL[3], pL[4], pL[5], pL[6]));
        d.G[0][0] = Ux.x; d.G[0][1] = Uy.x; d.G[0][2] = Uz.x;
        d.G[1][0] = Ux.y; d.G[1][1] = Uy.y; d.G[1][2] = Uz.y;
        d.G[2][0] = Zx.x; d.G[2][1] = Zy.x; d.G[2][2] = uzz1;
        d.gA[0][0] = d.gA[1][1] = d.gA[2][2] = 0.f;  // not used by B = curl A
        d.gA[0][1] = Ac.x; d.gA[0][2] = Az.x;
        d.gA[1][0] = Ac.y; d.gA[1][2] = Az.y;
        d.gA[2][0] = Zx.y; d.gA[2][1] = Zy.y;
        // second derivatives: lane 0 / lane 1 of each pair
        const float2 UUx = d2p(pU[3], xs(1, 2)), UUy = d2p(pU[3], ys(1, 2)),
                     UUz = d2p(pU[3], [&](int q) { return pU[3 + q]; });
        const float2 AAx = d2p(pA[3], xs(4, 5)), AAy = d2p(pA[3], ys(4, 5)),
                     AAz = d2p(pA[3], [&](int q) { return pA[3 + q]; });
        const float2 ZZx = d2p(pZ[3], xs(3, 6)), ZZy = d2p(pZ[3], ys(3, 6)),
                     ZZz = d2p(pZ[3], [&](int q) { return pZ[3 + q]; });
        const float2 lapU = add2(add2(UUx, UUy), UUz);  // (lap u_x, lap u_y)
        const float2 lapA = add2(add2(AAx, AAy), AAz);  // (lap A_x, lap A_y)
        const float2 lapZ = add2(add2(ZZx, ZZy), ZZz);  // (lap u_z, lap A_z)
        d.lapu[0] = lapU.x; d.lapu[1] = lapU.y; d.lapu[2] = lapZ.x;
        d.lapA[0] = lapA.x; d.lapA[1] = lapA.y; d.lapA[2] = lapZ.y;
        const float2 DU = dxyp(1, 2);  // (d_x d_y u_x, d_x d_y u_y)
        const float2 DA = dxyp(4, 5);  // (d_x d_y A_x, d_x d_y A_y)
        d.gdu[0] = UUx.x + DU.y + aU[0].x;
        d.gdu[1] = DU.x + UUy.y + aU[0].y;
        d.gdu[2] = zU[0] + ZZz.x;
        d.jc[0] = DA.y + aA[0].x - AAy.x - AAz.x;
        d.jc[1] = DA.x + aA[0].y - AAx.y - AAz.y;
        d.jc[2] = zA[0] - ZZx.y - ZZy.y;

        T fz[3] = {T(0), T(0), T(0)};
        if (forcing) {
          const Cplx<T> e = cmul(exy, cmul(rz[mz], ephi));
#pragma unroll
          for (int a = 0; a < 3; ++a) fz[a] = fa[a] * e.re - fb[a] * e.im;
        }
        const T fr[3] = {force_in_rhs ? fz[0] : T(0), force_in_rhs ? fz[1] : T(0), force_in_rhs ? fz[2] : T(0)};
        T r[NF];
        rhs_point(d, c, fr, r);
        const T qc[NF] = {d.lnr, d.u[0], d.u[1], d.u[2], d.A[0], d.A[1], d.A[2]};
        T qn[NF];
        T *wp = w + cidx;
#pragma unroll
        for (int fld = 0; fld < NF; ++fld, wp += fs) {
          T wv = dt * r[fld];
          if (substep > 0) wv += alpha * wc[fld];
          if (substep < 2) __stcs(wp, wv);
          qn[fld] = qc[fld] + beta * wv;
        }
        if (force_at_end)
          for (int a = 0; a < 3; ++a) qn[1 + a] += dt * fz[a];
        store_with_images<T, true>(qout, fs, cidx, qn, edge_xy || z < RAD || z >= nz - RAD, x, y, z, nx, ny, nz,
                                   px, py, zper);
      }
      if (p >= 2 * RAD) {
        cidx += wplane;
        if (forcing) {
          mz += kz;
          if (mz >= nzg) mz -= nzg;
        }
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        aU[k] = aU[k + 1];
        aA[k] = aA[k + 1];
        zU[k] = zU[k + 1];
        zA[k] = zA[k + 1];
      }
      aU[6] = aA[6] = pk(0.f, 0.f);
      zU[6] = zA[6] = 0.f;
      if (++slot == NS) {
        slot = 0;
        phase ^= 1u;
      }
      if (__syncthreads_or(!ok)) {
        failed = true;
        fail_run = tile.run;
        fail_p = p;
      }
    }
    if (!failed) G += npl;
  }

  if (failed && tid == 0) {
    atomicOr(&runs[fail_run].clock->status, 2);
    for (int p = fail_p; p < issued_hi; ++p) {
      const unsigned long long g = G + p;
      mbar_wait(&bars[(int)(g % NS)], (uint32_t)((g / NS) & 1ull));
    }
  }
}

// Step prologue over TMA-staged planes: max over the run's points of
// |u| + sqrt(cs^2 + |B|^2 / rho), B = curl A with the first-derivative
// stencil.  Each plane is used only while it is the lead plane: its x/y
// derivatives of A, |u| and 1/rho go into a three-plane register delay
// line, and the z-derivatives of A_x, A_y come from register pencils, so
// every shared-memory stage but the current one holds a plane in flight.
// One CTA per tile; the last CTA of each run sets dt, draws the forcing and
// advances the clock (finalize_step).
// Stage count of the prologue: small enough for two CTAs per SM.
template <typename T, int TY, int TXW = 32>
__host__ __device__ constexpr int pro_stages() {
  return TmaShape<T, TY, TXW>::STAGE_BYTES * 6 <= 110 * 1024 ? 6 : 5;
}

// MODE 0: the step prologue.  MODE 1: the same sweep as a B_rms reduction of
// the current state (|B|^2 summed in FP64 per point, in the tile, thread-z,
// block and tile order of every other B_rms reduction); its CFL maximum is
// kept in the clock, tagged with the step, and the prologue of that step
// takes it instead of sweeping the state again.
template <typename T, int TY, int MODE, int TXW>
__global__ void __launch_bounds__(TXW * TY, TXW == 32 ? 2 : 1)
    k_prologue_tma(const RunDesc *__restrict__ runs, const Tile *__restrict__ tiles) {
  using SH = TmaShape<T, TY, TXW>;
  constexpr int TX = SH::TX, SX = SH::SX, FIELD = SH::FIELD, NS = pro_stages<T, TY, TXW>(), P = NS - 1;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double sh[TXW * TY];
  __shared__ int flag;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * SH::STAGE_BYTES);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const Tile tile = tiles[blockIdx.x];
  const RunDesc &R = runs[tile.run];
  const long long step = R.clock->step;
  const bool cached = MODE == 0 && R.clock->cache_tag == step + 1;
  double vmax = 0.0, sb2 = 0.0;
  if (MODE == 1 || (R.dt_fixed <= 0.0 && !cached)) {
    if (tid == 0) {
      for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
      mbar_fence_init();
    }
    __syncthreads();
    const CUtensorMap *map = &R.rmap[step & 1];
    const int npl = (tile.z1 - tile.z0) + 2 * RAD;
    auto issue = [&](int p) {
      const int sl = p % NS;
      mbar_arrive_expect_tx(&bars[sl], (uint32_t)(NF * FIELD * sizeof(T)));
      tma_load_4d(smem + sl * SH::STAGE_BYTES, map, &bars[sl], tile.x0, tile.y0, tile.z0 + p, 0);
    };
    int issued = 0;
    if (tid == 0) {
      issued = npl < P ? npl : P;
      for (int p = 0; p < issued; ++p) issue(p);
    }
    T w[3][4];
    for (int a = 0; a < 3; ++a)
      for (int s = 0; s < 4; ++s) w[a][s] = T(W1(s) * R.inv_h[a]);
    const T cs2 = T(R.cs2);
    const int x = tile.x0 + tx, y = tile.y0 + ty;
    const bool active = x < R.nx && y < R.ny;
    const int cxy = (ty + RAD) * SX + tx + 4;
    // pencils of A_x, A_y over planes p-6 .. p; delay line of the lead-plane
    // values (d_y A_z, d_x A_z, d_x A_y, d_y A_x, |u|, 1/rho) of planes p-3 .. p
    // rings indexed by the plane: A_x, A_y of planes p-7 .. p in slot p & 7,
    // the lead-plane values of planes p-3 .. p in slot p & 3; the plane loop
    // is unrolled by 8 so that every ring index is a constant and no value
    // moves between registers as the sweep advances
    T ax[8], ay[8], dl[4][6];
#pragma unroll
    for (int k = 0; k < 8; ++k) ax[k] = ay[k] = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int v = 0; v < 6; ++v) dl[k][v] = T(0);
    // running maximum in the working precision (exact; FP64 per point would
    // run on B300's 1/64-rate FP64 pipe), NaN tracked apart
    T vm = T(0);
    bool bad = false;
    bool failed = false;
    int p = 0;
    // one plane of the sweep at phase PH = p mod 8; false once a wait gave up
    auto plane = [&](auto PH) -> bool {
      constexpr int K = decltype(PH)::value;
      if (tid == 0 && p + P < npl) {
        fence_proxy_async_smem();
        issue(p + P);  // into the stage of plane p-1, released at the end of the last iteration
        issued = p + P + 1;
      }
      const int sl = p % NS;
      const bool ok = mbar_wait(&bars[sl], (uint32_t)((p / NS) & 1));
      const T *o = reinterpret_cast<const T *>(smem + sl * SH::STAGE_BYTES) + cxy;
      auto dx = [&](int f) {
        const T *r = o + f * FIELD;
        return d1_vals(r[1], r[-1], r[2], r[-2], r[3], r[-3], w[0]);
      };
      auto dy = [&](int f) {
        const T *r = o + f * FIELD;
        return d1_vals(r[SX], r[-SX], r[2 * SX], r[-2 * SX], r[3 * SX], r[-3 * SX], w[1]);
      };
      ax[K] = o[4 * FIELD];
      ay[K] = o[5 * FIELD];
      T *d = dl[K & 3];
      if (active) {
        const T ux = o[FIELD], uy = o[2 * FIELD], uz = o[3 * FIELD];
        d[0] = dy(6);
        d[1] = dx(6);
        d[2] = dx(5);
        d[3] = dy(4);
        d[4] = sqrt(ux * ux + uy * uy + uz * uz);
        d[5] = exp(-o[0]);
      }
      if (p >= 2 * RAD && ok && active) {  // output plane p-3
        constexpr int c = (K + 5) & 7;     // slot of plane p-3
        const T dzAx = d1_vals(ax[(c + 1) & 7], ax[(c + 7) & 7], ax[(c + 2) & 7], ax[(c + 6) & 7], ax[(c + 3) & 7],
                               ax[(c + 5) & 7], w[2]);
        const T dzAy = d1_vals(ay[(c + 1) & 7], ay[(c + 7) & 7], ay[(c + 2) & 7], ay[(c + 6) & 7], ay[(c + 3) & 7],
                               ay[(c + 5) & 7], w[2]);
        const T *e = dl[(K + 1) & 3];  // lead-plane values of plane p-3
        const T Bx = e[0] - dzAy;
        const T By = dzAx - e[1];
        const T Bz = e[2] - e[3];
        const T b2 = norm2_rn(Bx, By, Bz);
        const T v = e[4] + sqrt(cs2 + b2 * e[5]);
        bad |= isnan(v);
        vm = fmax(vm, v);
        if constexpr (MODE == 1) sb2 += (double)b2;
      }
      return !__syncthreads_or(!ok);
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using I4 = std::integral_constant<int, 4>;
    using I5 = std::integral_constant<int, 5>;
    using I6 = std::integral_constant<int, 6>;
    using I7 = std::integral_constant<int, 7>;
    // npl is the same for every thread of the CTA, so the guards are uniform
    while (p < npl) {
      if (!plane(I0{})) break;
      if (++p == npl || !plane(I1{})) break;
      if (++p == npl || !plane(I2{})) break;
      if (++p == npl || !plane(I3{})) break;
      if (++p == npl || !plane(I4{})) break;
      if (++p == npl || !plane(I5{})) break;
      if (++p == npl || !plane(I6{})) break;
      if (++p == npl || !plane(I7{})) break;
      ++p;
    }
    failed = p < npl;
    vmax = bad ? __longlong_as_double(0x7ff8000000000000ll) : (double)vm;
    if (failed) {
      if (tid == 0) {
        atomicOr(&R.clock->status, 2);
        for (int q = p; q < issued; ++q) mbar_wait(&bars[q % NS], (uint32_t)((q / NS) & 1));
      }
      vmax = __longlong_as_double(0x7ff8000000000000ll);  // NaN: the step is marked bad
      sb2 = vmax;
    }
    vmax = block_max(vmax, sh);
  }
  if constexpr (MODE == 1) {
    const double red = block_sum(sb2, sh);
    if (tid == 0) {
      R.partials[(long long)tile.slot * NPART] = vmax;
      R.partials[(long long)tile.slot * NPART + 1] = red;
    }
    if (!last_tile_done(&R.counter[2], R.ntiles, &flag)) return;
    // the CFL maximum as finalize_step would form it, and the |B|^2 sum
    const int nthr = TXW * TY;
    double v = 0.0, sum = 0.0;
    for (int t = tid; t < R.ntiles; t += nthr) {
      const double pm = __ldcg(&R.partials[(long long)t * NPART]);
      v = isfinite(pm) ? fmax(v, pm) : __longlong_as_double(0x7ff8000000000000ll);
      if (!isfinite(pm)) break;
    }
    for (int t = tid; t < R.ntiles; t += nthr) sum += __ldcg(&R.partials[(long long)t * NPART + 1]);
    v = block_max(v, sh);
    sum = block_sum(sum, sh);
    if (tid != 0) return;
    R.diag[1] = sqrt(sum / ((double)R.nx * R.ny * R.nzg));
    R.clock->cache_vmax = v;
    R.clock->cache_tag = step + 1;
    R.counter[2] = 0u;
    return;
  }
  if (tid == 0) R.partials[(long long)tile.slot * NPART] = vmax;
  if (!last_tile_done(&R.counter[0], R.ntiles, &flag)) return;
  finalize_step(R, step, 1, sh);
}

namespace {

template <typename T, int TY, int NS, bool U>
int tma_smem_bytes() {
  return NS * TmaShape<T, TY>::STAGE_BYTES + NS * 8;
}

template <typename T, int TY, int NS, bool U, int BR>
int prepare_tma() {
  int e = (int)cudaFuncSetAttribute(k_substep_tma<T, TY, NS, U, false, BR>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, tma_smem_bytes<T, TY, NS, U>());
  if (!e)
    e = (int)cudaFuncSetAttribute(k_substep_tma<T, TY, NS, U, true, BR>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, tma_smem_bytes<T, TY, NS, U>());
  return e;
}

template <typename T, int TY, int NS, bool U, int BR>
int launch_tma(const RunDesc *runs, const Tile *tiles, int ntiles, int substep, int grid, bool iso,
               cudaStream_t s) {
  if (grid <= 0 || grid > ntiles) grid = ntiles;
  if (grid == 0) return 0;
  const int smem = tma_smem_bytes<T, TY, NS, U>();
  if (iso)
    k_substep_tma<T, TY, NS, U, true, BR><<<grid, dim3(32, TY), smem, s>>>(runs, tiles, ntiles, substep);
  else
    k_substep_tma<T, TY, NS, U, false, BR><<<grid, dim3(32, TY), smem, s>>>(runs, tiles, ntiles, substep);
  return (int)cudaGetLastError();
}

template <typename T, int TY, int NS, bool U, int BR>
int occupancy_tma(int *bps) {
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_substep_tma<T, TY, NS, U, true, BR>, 32 * TY,
                                                            tma_smem_bytes<T, TY, NS, U>());
}

}  // namespace

// Tile variants of the TMA kernel: id -> (dtype, TY, stages, ring rotation
// by 7-fold unrolling instead of register moves, planes between barriers).
//   FP32: 1 = 32x8/6; 2 = 32x4/6; 3 = 32x8/8; 4 = 32x12/6; 5 = 32x12/5; 6 = 32x16/5;
//         9 = 32x6/5 (two CTAs per SM); 10 .. 14 = 32x12 with 6 .. 10 stages
//         and a barrier every 2nd .. 6th plane (one plane of prefetch);
//         15, 16 = 32x12 with 9, 10 stages, a barrier every 4th, 5th plane
//         and two planes of prefetch
//   FP32 packed (isotropic grids; anisotropic runs fall back to the tile
//   of the same shape above): 7 = 32x12/5; 8 = 32x8/6
//   FP64: 1 = 32x4/6; 2 = 32x4/6 unrolled; 3 = 32x8/6; 4 = 32x8/7 with a barrier every
//         second plane
// (the unrolled FP32 variants measured 1.7x slower on B300: the 7-fold body
// overflows the instruction cache)
#define MHD_TMA_VARIANTS(X)            \
  X(0, 1, float, 8, 6, false, 1)       \
  X(0, 2, float, 4, 6, false, 1)       \
  X(0, 3, float, 8, 8, false, 1)       \
  X(0, 4, float, 12, 6, false, 1)      \
  X(0, 5, float, 12, 5, false, 1)      \
  X(0, 6, float, 16, 5, false, 1)      \
  X(0, 9, float, 6, 5, false, 1)       \
  X(0, 10, float, 12, 6, false, 2)     \
  X(0, 11, float, 12, 7, false, 3)     \
  X(0, 12, float, 12, 8, false, 4)     \
  X(0, 13, float, 12, 9, false, 5)     \
  X(0, 14, float, 12, 10, false, 6)    \
  X(0, 15, float, 12, 9, false, 4)     \
  X(0, 16, float, 12, 10, false, 5)    \
  X(1, 1, double, 4, 6, false, 1)      \
  X(1, 2, double, 4, 6, true, 1)       \
  X(1, 3, double, 8, 6, false, 1)      \
  X(1, 4, double, 8, 7, false, 2)

int tma_num_tiles(int dtype) { return dtype == 0 ? MHD_X2_LAST : 4; }

template <typename T, int TY, int TXW = 32>
int pro_smem_bytes() {
  return pro_stages<T, TY, TXW>() * TmaShape<T, TY, TXW>::STAGE_BYTES + pro_stages<T, TY, TXW>() * 8;
}

static_assert(32 * 16 <= MAX_TILE_THREADS && 64 * 8 <= MAX_TILE_THREADS, "reduction kernels run with the tile's block shape");

// packed tiles: id -> (scalar tile of the same shape, TY, stages)
#define MHD_PACKED_VARIANTS(X) \
  X(7, 5, 12, 5)               \
  X(8, 1, 8, 6)

int tma_tile_shape(int dtype, int tile, int *tx, int *ty) {
  *tx = 32;
  if (dtype == 0 && x2_rows(tile) > 0) {  // paired-point variants: 64-point rows
    *tx = 64;
    *ty = x2_rows(tile);
    return 0;
  }
#define X(ID, SC, TY, NS) \
  if (dtype == 0 && tile == ID) { *ty = TY; return 0; }
  MHD_PACKED_VARIANTS(X)
#undef X
#define X(DT, ID, T, TY, NS, U, BR) \
  if (dtype == DT && tile == ID) { *ty = TY; return 0; }
  MHD_TMA_VARIANTS(X)
#undef X
  return -1;
}

int tma_prepare(int dtype, int tile) {
  if (dtype == 0 && x2_rows(tile) > 0) {  // the substep kernel, and the prologue of tile 13 (32 x 12)
    const int e = x2_prepare(tile);
    return e ? e : tma_prepare(0, 13);
  }
#define X(ID, SC, TY, NS)                                                                            \
  if (dtype == 0 && tile == ID) {                                                                    \
    int e = (int)cudaFuncSetAttribute(k_substep_tma_f2<TY, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      tma_smem_bytes<float, TY, NS, false>());                       \
    return e ? e : tma_prepare(0, SC);                                                               \
  }
  MHD_PACKED_VARIANTS(X)
#undef X
#define X(DT, ID, T, TY, NS, U, BR)                                                                          \
  if (dtype == DT && tile == ID) {                                                                       \
    int e = prepare_tma<T, TY, NS, U, BR>();                                                                 \
    if (!e)                                                                                              \
      e = (int)cudaFuncSetAttribute(k_prologue_tma<T, TY, 0, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    pro_smem_bytes<T, TY>());                                               \
    if (!e)                                                                                                 \
      e = (int)cudaFuncSetAttribute(k_prologue_tma<T, TY, 1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    pro_smem_bytes<T, TY>());                                               \
    return e;                                                                                            \
  }
  MHD_TMA_VARIANTS(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int tma_occupancy(int dtype, int tile, int *bps) {
  if (dtype == 0 && x2_rows(tile) > 0) return x2_occupancy(tile, bps);
#define X(ID, SC, TY, NS)                                                                                \
  if (dtype == 0 && tile == ID)                                                                          \
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_substep_tma_f2<TY, NS>, 32 * TY,    \
                                                              tma_smem_bytes<float, TY, NS, false>());
  MHD_PACKED_VARIANTS(X)
#undef X
#define X(DT, ID, T, TY, NS, U, BR) \
  if (dtype == DT && tile == ID) return occupancy_tma<T, TY, NS, U, BR>(bps);
  MHD_TMA_VARIANTS(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int tma_launch_prologue(int dtype, int tile, const RunDesc *runs, const Tile *tiles, int ntiles,
                        cudaStream_t s, int mode) {
  if (ntiles <= 0) return 0;
  if (dtype == 0 && x2_rows(tile) > 0) return tma_launch_prologue(0, 13, runs, tiles, ntiles, s, mode);
#define X(ID, SC, TY, NS) \
  if (dtype == 0 && tile == ID) return tma_launch_prologue(0, SC, runs, tiles, ntiles, s, mode);
  MHD_PACKED_VARIANTS(X)
#undef X
#define X(DT, ID, T, TY, NS, U, BR)                                                                       \
  if (dtype == DT && tile == ID) {                                                                    \
    if (mode == 1)                                                                                    \
      k_prologue_tma<T, TY, 1, 32><<<ntiles, dim3(32, TY), pro_smem_bytes<T, TY>(), s>>>(runs, tiles);    \
    else                                                                                              \
      k_prologue_tma<T, TY, 0, 32><<<ntiles, dim3(32, TY), pro_smem_bytes<T, TY>(), s>>>(runs, tiles);    \
    return (int)cudaGetLastError();                                                                   \
  }
  MHD_TMA_VARIANTS(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int tma_launch(int dtype, int tile, const RunDesc *runs, const Tile *tiles, int ntiles, int substep, int grid,
               int iso, cudaStream_t s) {
  if (dtype == 0 && x2_rows(tile) > 0) return x2_launch(tile, runs, tiles, ntiles, substep, grid, iso, s);
#define X(ID, SC, TY, NS)                                                                             \
  if (dtype == 0 && tile == ID) {                                                                     \
    if (!iso) return tma_launch(0, SC, runs, tiles, ntiles, substep, grid, iso, s);                   \
    if (grid <= 0 || grid > ntiles) grid = ntiles;                                                    \
    if (grid == 0) return 0;                                                                          \
    k_substep_tma_f2<TY, NS><<<grid, dim3(32, TY), tma_smem_bytes<float, TY, NS, false>(), s>>>(     \
        runs, tiles, ntiles, substep);                                                                \
    return (int)cudaGetLastError();                                                                   \
  }
  MHD_PACKED_VARIANTS(X)
#undef X
#define X(DT, ID, T, TY, NS, U, BR) \
  if (dtype == DT && tile == ID) return launch_tma<T, TY, NS, U, BR>(runs, tiles, ntiles, substep, grid, iso != 0, s);
  MHD_TMA_VARIANTS(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

}  // namespace mhd
