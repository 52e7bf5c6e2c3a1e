// Stencil weights and the right-hand side of the isothermal MHD equations
// (arXiv:2012.08758, Sec. 4 Eqs. 1-3), shared by every substep kernel.
#pragma once
#include "mhd_internal.h"

namespace mhd {

// 6th-order central weights (Sec. 2).  First derivative:
//   f' = [45 (f1 - f-1) - 9 (f2 - f-2) + (f3 - f-3)] / (60 h)
// second derivative:
//   f'' = [-490 f0 + 270 (f1 + f-1) - 27 (f2 + f-2) + 2 (f3 + f-3)] / (180 h^2)
// mixed derivative on the two diagonals of the a-b plane (the diagonal
// points of the stencil figure of Sec. 3.1):
//   f_ab = [270 S1 - 27 S2 + 2 S3] / (720 h_a h_b),
//   S_s = f(+s,+s) + f(-s,-s) - f(+s,-s) - f(-s,+s).
__host__ __device__ constexpr double W1(int s) {
  return s == 1 ? 45.0 / 60.0 : s == 2 ? -9.0 / 60.0 : s == 3 ? 1.0 / 60.0 : 0.0;
}
__host__ __device__ constexpr double W2(int s) {
  return s == 0 ? -490.0 / 180.0 : s == 1 ? 270.0 / 180.0 : s == 2 ? -27.0 / 180.0 : 2.0 / 180.0;
}
__host__ __device__ constexpr double WM(int s) {
  return s == 1 ? 270.0 / 720.0 : s == 2 ? -27.0 / 720.0 : s == 3 ? 2.0 / 720.0 : 0.0;
}

// Williamson (1980) low-storage RK3: w <- alpha_s w + dt RHS, q <- q + beta_s w.
__host__ __device__ constexpr double RK_ALPHA(int s) {
  return s == 0 ? 0.0 : s == 1 ? -5.0 / 9.0 : -153.0 / 128.0;
}
__host__ __device__ constexpr double RK_BETA(int s) {
  return s == 0 ? 1.0 / 3.0 : s == 1 ? 15.0 / 16.0 : 8.0 / 15.0;
}

// Per-run stencil and physics constants in the working precision.
template <typename T>
struct Coefs {
  T c1[3][4];   // first-derivative weights / h, per axis
  T c2[3][4];   // second-derivative weights / h^2, per axis
  T cm[3][4];   // mixed weights / (h_a h_b), index by the pair (xy=0, xz=1, yz=2)
  T c6[3];      // 1 / (60 h) per axis: weight of the upwinding sixth difference
  T cs2, nu, eta;
  int upwind;
  __device__ void load(const RunDesc &R) {
    for (int a = 0; a < 3; ++a)
      for (int s = 0; s < 4; ++s) {
        c1[a][s] = T(W1(s) * R.inv_h[a]);
        c2[a][s] = T(W2(s) * R.inv_h[a] * R.inv_h[a]);
      }
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    for (int p = 0; p < 3; ++p)
      for (int s = 0; s < 4; ++s) cm[p][s] = T(WM(s) * R.inv_h[pa[p]] * R.inv_h[pb[p]]);
    for (int a = 0; a < 3; ++a) c6[a] = T(R.inv_h[a] / 60.0);
    cs2 = T(R.cs2);
    nu = T(R.nu);
    eta = T(R.eta);
    upwind = R.upwind;
  }
};

// Derivatives at one point, as delivered by a kernel variant.
template <typename T>
struct Derivs {
  T lnr, u[3], A[3];   // centre values
  T g[3];              // grad ln rho
  T G[3][3];           // G[a][b] = d u_a / d x_b
  T gA[3][3];          // gA[a][b] = d A_a / d x_b
  T lapu[3];           // Laplacian of u_a
  T gdu[3];            // (grad div u)_a = sum_b d_a d_b u_b
  T lapA[3];           // Laplacian of A_a
  T jc[3];             // j = grad div A - lap A with the d_a d_a A_a terms
                       // cancelled analytically (mu0 = 1)
  T up;                // upwinding term of d ln rho / dt (0 when off)
};

// Sixth difference f(-3) - 6 f(-2) + 15 f(-1) - 20 f(0) + 15 f(1) - 6 f(2) + f(3)
// from the samples at offsets -3..3.  The fifth-order upwind-biased first
// derivative (the six points from three upstream to two downstream) equals
// the central sixth-order one minus sign(u) * delta6 / (60 h), so
// u d_up f = u D1 f - |u| delta6 / (60 h): upwinding adds |u_a| delta6_a / (60 h_a)
// to d ln rho / dt for every axis a.
template <typename T>
__device__ __forceinline__ T delta6(T m3, T m2, T m1, T c0, T p1, T p2, T p3) {
  return ((m3 + p3) - T(6) * (m2 + p2)) + (T(15) * (m1 + p1) - T(20) * c0);
}

// Stencil coefficients for the TMA kernel.  ISO: all three grid spacings
// equal (every configuration of the benchmarks), so the three axes -- and
// the three mixed pairs -- share one set of 10 weights, which frees
// registers for more warps per SM.
template <typename T, bool ISO>
struct StencilCoefs {
  static constexpr int NA = ISO ? 1 : 3;
  T c1[NA][4], c2[NA][4], cm[NA][4];
  T c6[NA];  // 1 / (60 h): weight of the upwinding sixth difference
  T cs2, nu, eta;
  int upwind;
  __device__ __forceinline__ void load(const RunDesc &R) {
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    for (int a = 0; a < NA; ++a) {
      for (int s = 0; s < 4; ++s) {
        c1[a][s] = T(W1(s) * R.inv_h[a]);
        c2[a][s] = T(W2(s) * R.inv_h[a] * R.inv_h[a]);
        cm[a][s] = T(WM(s) * R.inv_h[pa[a]] * R.inv_h[pb[a]]);
      }
      c6[a] = T(R.inv_h[a] / 60.0);
    }
    cs2 = T(R.cs2);
    nu = T(R.nu);
    eta = T(R.eta);
    upwind = R.upwind;
  }
  __device__ __forceinline__ T w6(int a) const { return c6[ISO ? 0 : a]; }
  __device__ __forceinline__ T w1(int a, int s) const { return c1[ISO ? 0 : a][s]; }
  __device__ __forceinline__ T w2(int a, int s) const { return c2[ISO ? 0 : a][s]; }
  __device__ __forceinline__ T wm(int pair, int s) const { return cm[ISO ? 0 : pair][s]; }
};

// 1/rho = exp(-ln rho): FP32 takes the hardware exponential (__expf, a few
// ulp: far inside the FP32 error budget of the step), FP64 the library exp.
__device__ __forceinline__ float inv_density(float lnr) { return __expf(-lnr); }
__device__ __forceinline__ double inv_density(double lnr) { return exp(-lnr); }

// dq/dt of Eqs. 1-3 at one point; f = forcing (already evaluated).
// C provides cs2, nu, eta in the working precision.
template <typename T, class C>
__device__ __forceinline__ void rhs_point(const Derivs<T> &d, const C &c, const T f[3], T out[NF]) {
  const T rho_inv = inv_density(d.lnr);
  const T divu = d.G[0][0] + d.G[1][1] + d.G[2][2];
  const T B[3] = {d.gA[2][1] - d.gA[1][2], d.gA[0][2] - d.gA[2][0], d.gA[1][0] - d.gA[0][1]};
  // Eq. 1: D ln rho / Dt = -div u
  out[0] = -(d.u[0] * d.g[0] + d.u[1] * d.g[1] + d.u[2] * d.g[2]) - divu + d.up;
  const T third = T(1.0 / 3.0);
  const T jxB[3] = {d.jc[1] * B[2] - d.jc[2] * B[1], d.jc[2] * B[0] - d.jc[0] * B[2],
                    d.jc[0] * B[1] - d.jc[1] * B[0]};
  const T uxB[3] = {d.u[1] * B[2] - d.u[2] * B[1], d.u[2] * B[0] - d.u[0] * B[2],
                    d.u[0] * B[1] - d.u[1] * B[0]};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // traceless rate of strain times grad ln rho
    T Sg = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      T S = T(0.5) * (d.G[a][b] + d.G[b][a]);
      if (a == b) S -= third * divu;
      Sg += S * d.g[b];
    }
    const T adv = d.u[0] * d.G[a][0] + d.u[1] * d.G[a][1] + d.u[2] * d.G[a][2];
    // Eq. 2
    out[1 + a] = -adv - c.cs2 * d.g[a] + jxB[a] * rho_inv +
                 c.nu * (d.lapu[a] + third * d.gdu[a] + T(2) * Sg) + f[a];
    // Eq. 3 (diffusive gauge)
    out[4 + a] = uxB[a] + c.eta * d.lapA[a];
  }
}

// Round-to-nearest operations the compiler may not fuse or reorder: every
// kernel that evaluates them gets the same bits.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// First derivative from the samples at offsets +-1, +-2, +-3 with the
// weights w[1..3] of one axis, and |B|^2, in one fixed sequence of roundings
// shared by every reduction (dt prologue, diagnostics, B_rms, curl), so they
// all see bit-identical B.
template <typename T>
__device__ __forceinline__ T d1_vals(T p1, T m1, T p2, T m2, T p3, T m3, const T *w) {
  return fma_rn(w[3], p3 - m3, fma_rn(w[2], p2 - m2, mul_rn(w[1], p1 - m1)));
}
template <typename T>
__device__ __forceinline__ T norm2_rn(T bx, T by, T bz) {
  return fma_rn(bz, bz, fma_rn(by, by, mul_rn(bx, bx)));
}

// Complex product helpers for the forcing phase.
template <typename T>
struct Cplx {
  T re, im;
};
template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// Periodic images of interior index i along an axis of n points: all
// j = i + m n with -RAD <= j < n + RAD.  Returns the count (<= 7).
__device__ __forceinline__ int periodic_images(int i, int n, int *out) {
  int j = -RAD + (i + RAD) % n;
  int c = 0;
  for (; j < n + RAD; j += n) out[c++] = j;
  return c;
}

// Stores the new values qn of interior point (x, y, z), padded index c, and
// -- for a point within RAD of a face (near) -- its periodic images in the
// ghost zones (Sec. 3.1: periodic boundaries as wrapped ghost zones), so the
// next substep finds its halo filled.  With at least 2 RAD + 1 points on
// every axis a point has at most one image per axis (i + n below RAD, i - n
// at or above n - RAD), so the images are the up to seven sums of those
// shifts; smaller grids take the general enumeration.  zper = false (a
// z-slab of a decomposed domain): no images along z, whose ghost planes the
// halo exchange fills from the neighbouring slabs.
template <typename T, bool STREAM>
__device__ __forceinline__ void store_with_images(T *qout, long long fs, long long c, const T qn[NF], bool near,
                                                  int x, int y, int z, int nx, int ny, int nz, int px, int py,
                                                  bool zper = true) {
  auto put = [&](long long o) {
    T *p = qout + o;
#pragma unroll
    for (int f = 0; f < NF; ++f, p += fs) {
      if (STREAM)
        __stcs(p, qn[f]);
      else
        *p = qn[f];
    }
  };
  put(c);
  if (!near) return;
  if (nx >= 2 * RAD + 1 && ny >= 2 * RAD + 1 && (nz >= 2 * RAD + 1 || !zper)) {
    const long long sy = px, sz = (long long)px * py;
    const long long dx = x < RAD ? nx : (x >= nx - RAD ? -nx : 0);
    const long long dy = y < RAD ? ny * sy : (y >= ny - RAD ? -ny * sy : 0);
    const long long dz = !zper ? 0 : z < RAD ? nz * sz : (z >= nz - RAD ? -nz * sz : 0);
    // the images are the non-empty subsets of the non-zero shifts; a
    // rolled loop over those subsets issues only the stores that exist
    const int mask = (dx != 0 ? 1 : 0) | (dy != 0 ? 2 : 0) | (dz != 0 ? 4 : 0);
#pragma unroll 1
    for (int m = mask; m != 0; m = (m - 1) & mask)
      put(c + ((m & 1) ? dx : 0) + ((m & 2) ? dy : 0) + ((m & 4) ? dz : 0));
  } else {
    int ix[7], iy[7], iz[7];
    const int cx = periodic_images(x, nx, ix);
    const int cy = periodic_images(y, ny, iy);
    int cz = 1;
    iz[0] = z;
    if (zper) cz = periodic_images(z, nz, iz);
    for (int a = 0; a < cz; ++a)
      for (int b = 0; b < cy; ++b)
        for (int e = 0; e < cx; ++e) put(((long long)(iz[a] + OZ) * py + (iy[b] + OY)) * px + (ix[e] + OX));
  }
}

}  // namespace mhd
