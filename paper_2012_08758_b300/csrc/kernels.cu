// Substep kernel (shared-memory plane ring variant), periodic halo fill and
// state conversion kernels.
//
// Substep = one stage of the 3rd-order 2N-storage Runge-Kutta scheme
// (Sec. 2): for every interior point, all derivatives of Eqs. 1-3 from the
// 6th-order stencils, the right-hand side with forcing (Eqs. 4-6), then
//   w <- alpha_s w + dt RHS,   q_out <- q_in + beta_s w,
// and q_out is also written to its periodic images in the ghost zones
// (Sec. 3.1: periodic boundaries = wrapped ghost zones), so the next stage
// finds its halo ready without a separate fill pass.
#include <cuda_runtime.h>

#include <type_traits>

#include "mhd_internal.h"
#include "physics.cuh"
#include "step_device.cuh"

namespace mhd {

// ---------------------------------------------------------------------------
// Shared-memory plane ring: a CTA owns a TX x TY column of the grid and
// sweeps it along z.  Seven consecutive z-planes of all seven fields, each
// with a 3-point halo in x and y, sit in a ring; the output plane is the
// middle one.  All derivatives are read from the ring.
// ---------------------------------------------------------------------------
template <typename T, int TX, int TY>
struct RingView {
  static constexpr int SX = TX + 2 * RAD, SY = TY + 2 * RAD;
  static constexpr int PLANE = NF * SY * SX;
  const T *ring;
  int off[7];
  int cxy;  // offset of (tx, ty) inside a field plane (halo included)
  // value of field f at offset (dx, dy, dz) from the thread's point
  __device__ __forceinline__ T at(int f, int dx, int dy, int dz) const {
    return ring[off[dz + RAD] + f * SY * SX + cxy + dy * SX + dx];
  }
  template <int AX>
  __device__ __forceinline__ T nb(int f, int s) const {
    return at(f, AX == 0 ? s : 0, AX == 1 ? s : 0, AX == 2 ? s : 0);
  }
  template <int AX>
  __device__ __forceinline__ T d1(int f, const Coefs<T> &c) const {
    return c.c1[AX][1] * (nb<AX>(f, 1) - nb<AX>(f, -1)) + c.c1[AX][2] * (nb<AX>(f, 2) - nb<AX>(f, -2)) +
           c.c1[AX][3] * (nb<AX>(f, 3) - nb<AX>(f, -3));
  }
  // second derivative without the centre term (added by the caller)
  template <int AX>
  __device__ __forceinline__ T d2_off(int f, const Coefs<T> &c) const {
    return c.c2[AX][1] * (nb<AX>(f, 1) + nb<AX>(f, -1)) + c.c2[AX][2] * (nb<AX>(f, 2) + nb<AX>(f, -2)) +
           c.c2[AX][3] * (nb<AX>(f, 3) + nb<AX>(f, -3));
  }
  // mixed derivative in the (A, B) plane, A < B; P = pair index
  template <int A, int B, int P>
  __device__ __forceinline__ T dmix(int f, const Coefs<T> &c) const {
    T r = T(0);
#pragma unroll
    for (int s = 1; s <= 3; ++s) {
      auto v = [&](int sa, int sb) {
        return at(f, (A == 0 ? sa : 0) + (B == 0 ? sb : 0), (A == 1 ? sa : 0) + (B == 1 ? sb : 0),
                  (A == 2 ? sa : 0) + (B == 2 ? sb : 0));
      };
      const T S = (v(s, s) - v(-s, s)) - (v(s, -s) - v(-s, -s));
      r += c.cm[P][s] * S;
    }
    return r;
  }
};

template <typename T, int TX, int TY>
__device__ __forceinline__ void derivs_from_ring(const RingView<T, TX, TY> &S, const Coefs<T> &c,
                                                 Derivs<T> &d) {
  d.lnr = S.at(0, 0, 0, 0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    d.u[a] = S.at(1 + a, 0, 0, 0);
    d.A[a] = S.at(4 + a, 0, 0, 0);
  }
  d.g[0] = S.template d1<0>(0, c);
  d.g[1] = S.template d1<1>(0, c);
  d.g[2] = S.template d1<2>(0, c);
  d.up = T(0);
  if (c.upwind) {
    auto d6 = [&](auto AXc) {
      constexpr int AX = decltype(AXc)::value;
      return delta6(S.template nb<AX>(0, -3), S.template nb<AX>(0, -2), S.template nb<AX>(0, -1), d.lnr,
                    S.template nb<AX>(0, 1), S.template nb<AX>(0, 2), S.template nb<AX>(0, 3));
    };
    d.up = c.c6[0] * fabs(d.u[0]) * d6(std::integral_constant<int, 0>{}) +
           c.c6[1] * fabs(d.u[1]) * d6(std::integral_constant<int, 1>{}) +
           c.c6[2] * fabs(d.u[2]) * d6(std::integral_constant<int, 2>{});
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    d.G[a][0] = S.template d1<0>(1 + a, c);
    d.G[a][1] = S.template d1<1>(1 + a, c);
    d.G[a][2] = S.template d1<2>(1 + a, c);
    d.gA[a][0] = S.template d1<0>(4 + a, c);
    d.gA[a][1] = S.template d1<1>(4 + a, c);
    d.gA[a][2] = S.template d1<2>(4 + a, c);
  }
  // second derivatives d_a d_a of each component, per axis
  T uxx[3][3], Axx[3][3];  // [component][axis]
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    uxx[a][0] = S.template d2_off<0>(1 + a, c) + c.c2[0][0] * d.u[a];
    uxx[a][1] = S.template d2_off<1>(1 + a, c) + c.c2[1][0] * d.u[a];
    uxx[a][2] = S.template d2_off<2>(1 + a, c) + c.c2[2][0] * d.u[a];
    Axx[a][0] = S.template d2_off<0>(4 + a, c) + c.c2[0][0] * d.A[a];
    Axx[a][1] = S.template d2_off<1>(4 + a, c) + c.c2[1][0] * d.A[a];
    Axx[a][2] = S.template d2_off<2>(4 + a, c) + c.c2[2][0] * d.A[a];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    d.lapu[a] = uxx[a][0] + uxx[a][1] + uxx[a][2];
    d.lapA[a] = Axx[a][0] + Axx[a][1] + Axx[a][2];
  }
  // mixed derivatives of u and A: pairs xy (P0), xz (P1), yz (P2)
  const T uxy_y = S.template dmix<0, 1, 0>(2, c), uxy_x = S.template dmix<0, 1, 0>(1, c);
  const T uxz_z = S.template dmix<0, 2, 1>(3, c), uxz_x = S.template dmix<0, 2, 1>(1, c);
  const T uyz_z = S.template dmix<1, 2, 2>(3, c), uyz_y = S.template dmix<1, 2, 2>(2, c);
  d.gdu[0] = uxx[0][0] + uxy_y + uxz_z;
  d.gdu[1] = uxy_x + uxx[1][1] + uyz_z;
  d.gdu[2] = uxz_x + uyz_y + uxx[2][2];
  const T Axy_y = S.template dmix<0, 1, 0>(5, c), Axy_x = S.template dmix<0, 1, 0>(4, c);
  const T Axz_z = S.template dmix<0, 2, 1>(6, c), Axz_x = S.template dmix<0, 2, 1>(4, c);
  const T Ayz_z = S.template dmix<1, 2, 2>(6, c), Ayz_y = S.template dmix<1, 2, 2>(5, c);
  d.jc[0] = Axy_y + Axz_z - Axx[0][1] - Axx[0][2];
  d.jc[1] = Axy_x + Ayz_z - Axx[1][0] - Axx[1][2];
  d.jc[2] = Axz_x + Ayz_y - Axx[2][0] - Axx[2][1];
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX *TY)
    k_substep_smem(const RunDesc *__restrict__ runs, const Tile *__restrict__ tiles, int ntiles,
                   int substep) {
  using RV = RingView<T, TX, TY>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *ring = reinterpret_cast<T *>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;

  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tile = tiles[t];
    if (tile.z1 <= tile.z0) continue;  // padding entry of the work split
    const RunDesc &R = runs[tile.run];
    const StepCoeffs &K = *R.coeffs;
    Coefs<T> c;
    c.load(R);
    const int nx = R.nx, ny = R.ny, nz = R.nz, px = R.px, py = R.py;
    const long long fs = R.fstride;
    const int par = (K.parity + substep) & 1;
    const T *__restrict__ qin = static_cast<const T *>(R.q[par]);
    T *__restrict__ qout = static_cast<T *>(R.q[par ^ 1]);
    T *__restrict__ w = static_cast<T *>(R.w);
    const T dt = T(K.dt);
    const T alpha = T(RK_ALPHA(substep)), beta = T(RK_BETA(substep));
    const int x = tile.x0 + tx, y = tile.y0 + ty;
    const bool active = x < nx && y < ny;

    // forcing: e^{i k.x} = e^{i kx x} e^{i ky y} e^{i kz z}, each factor a
    // root of unity looked up in the per-axis table (exact index arithmetic)
    const bool forcing = K.forcing != 0;
    const bool force_in_rhs = forcing && R.forcing_mode == 0;
    const bool force_at_end = forcing && R.forcing_mode == 1 && substep == 2;
    Cplx<T> exy = {T(1), T(0)};
    T fa[3], fb[3];
    if (forcing) {
      const Cplx<T> *rx = static_cast<const Cplx<T> *>(R.roots[0]);
      const Cplx<T> *ry = static_cast<const Cplx<T> *>(R.roots[1]);
      if (active) {
        Cplx<T> ex = rx[(int)(((long long)K.kmod[0] * x) % nx)];
        Cplx<T> ey = ry[(int)(((long long)K.kmod[1] * y) % ny)];
        exy = cmul(ex, ey);
      }
      for (int a = 0; a < 3; ++a) {
        fa[a] = T(K.fa[a]);
        fb[a] = T(K.fb[a]);
      }
    }
    const Cplx<T> ephi = {T(K.cphi), T(K.sphi)};
    const Cplx<T> *rz = static_cast<const Cplx<T> *>(R.roots[2]);

    RV S;
    S.ring = ring;
    S.cxy = (ty + RAD) * RV::SX + tx + RAD;
    const int nload = (tile.z1 - tile.z0) + 2 * RAD;
    for (int i = 0; i < nload; ++i) {
      // load interior plane z0 - 3 + i (padded Z = z0 + i) into slot i % 7
      const int Z = tile.z0 + i;
      T *dst = ring + (i % 7) * RV::PLANE;
      for (int e = tid; e < RV::PLANE; e += TX * TY) {
        const int f = e / (RV::SY * RV::SX);
        const int r = e - f * (RV::SY * RV::SX);
        const int yy = r / RV::SX, xx = r - yy * RV::SX;
        const int X = tile.x0 + xx + (OX - RAD), Y = tile.y0 + yy;
        T v = T(0);
        if (X < nx + OX + RAD && Y < ny + 2 * RAD)
          v = __ldg(qin + f * fs + ((long long)Z * py + Y) * px + X);
        dst[e] = v;
      }
      __syncthreads();
      if (i >= 2 * RAD) {
        const int z = tile.z0 + i - 2 * RAD;  // interior index of the output plane
#pragma unroll
        for (int dz = -RAD; dz <= RAD; ++dz) S.off[dz + RAD] = ((i - RAD + dz) % 7) * RV::PLANE;
        if (active) {
          Derivs<T> d;
          derivs_from_ring(S, c, d);
          T f[3] = {T(0), T(0), T(0)};
          if (forcing) {
            const Cplx<T> e = cmul(exy, cmul(rz[(int)(((long long)K.kmod[2] * (z + R.z_off)) % R.nzg)], ephi));
            for (int a = 0; a < 3; ++a) f[a] = fa[a] * e.re - fb[a] * e.im;
          }
          const T fr[3] = {force_in_rhs ? f[0] : T(0), force_in_rhs ? f[1] : T(0),
                           force_in_rhs ? f[2] : T(0)};
          T r[NF];
          rhs_point(d, c, fr, r);
          const long long cidx = ((long long)(z + OZ) * py + (y + OY)) * px + (x + OX);
          const T qc[NF] = {d.lnr, d.u[0], d.u[1], d.u[2], d.A[0], d.A[1], d.A[2]};
          T qn[NF];
#pragma unroll
          for (int fld = 0; fld < NF; ++fld) {
            T wv = dt * r[fld];
            if (substep > 0) wv += alpha * w[fld * fs + cidx];
            if (substep < 2) w[fld * fs + cidx] = wv;
            qn[fld] = qc[fld] + beta * wv;
          }
          if (force_at_end)
            for (int a = 0; a < 3; ++a) qn[1 + a] += dt * f[a];
          const bool near = x < RAD || x >= nx - RAD || y < RAD || y >= ny - RAD || z < RAD || z >= nz - RAD;
          store_with_images<T, false>(qout, fs, cidx, qn, near, x, y, z, nx, ny, nz, px, py, R.z_open == 0);
        }
      }
      __syncthreads();
    }
  }
}

template <typename T, int TX, int TY>
static int prepare_smem() {
  using RV = RingView<T, TX, TY>;
  const size_t smem = sizeof(T) * 7 * RV::PLANE;
  return (int)cudaFuncSetAttribute(k_substep_smem<T, TX, TY>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, int TX, int TY>
static int launch_smem(const RunDesc *runs, const Tile *tiles, int ntiles, int substep, int grid,
                       cudaStream_t s) {
  using RV = RingView<T, TX, TY>;
  const size_t smem = sizeof(T) * 7 * RV::PLANE;
  if (grid <= 0 || grid > ntiles) grid = ntiles;
  if (grid == 0) return 0;
  k_substep_smem<T, TX, TY><<<grid, dim3(TX, TY), smem, s>>>(runs, tiles, ntiles, substep);
  return (int)cudaGetLastError();
}

int substep_tile_shape(int dtype, int kernel, int tile, int *tx, int *ty) {
  if (kernel == 2) return tma_tile_shape(dtype, tile, tx, ty);
  *tx = 32;
  *ty = dtype == 0 ? 8 : 4;
  return 0;
}

// The paired-point variants (64-point substep tiles) reduce over 32 x 12
// tiles, with the prologue of the 32 x 12 scalar variant.
int reduction_tile_shape(int dtype, int kernel, int tile, int *tx, int *ty) {
  if (kernel == 2 && dtype == 0 && x2_rows(tile) > 0) {
    *tx = 32;
    *ty = 12;
    return 0;
  }
  return substep_tile_shape(dtype, kernel, tile, tx, ty);
}

int substep_max_grid(int dtype, int kernel, int tile, int *blocks_per_sm) {
  if (kernel == 2) return tma_occupancy(dtype, tile, blocks_per_sm);
  int n = 0;
  cudaError_t e;
  if (dtype == 0)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, k_substep_smem<float, 32, 8>, 256, sizeof(float) * 7 * RingView<float, 32, 8>::PLANE);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, k_substep_smem<double, 32, 4>, 128, sizeof(double) * 7 * RingView<double, 32, 4>::PLANE);
  *blocks_per_sm = n;
  return (int)e;
}

// Sets the kernel attributes (dynamic shared memory above 48 KB) on the
// current device; called when a context is created, outside any capture.
// kernel: 1 = shared-memory plane ring, 2 = TMA.
int prepare_substep(int dtype, int kernel, int tile) {
  if (kernel == 2) return tma_prepare(dtype, tile);
  return dtype == 0 ? prepare_smem<float, 32, 8>() : prepare_smem<double, 32, 4>();
}

int launch_prologue(int dtype, int kernel, int tile, const RunDesc *runs, const Tile *tiles, int ntiles,
                    int tw, int th, cudaStream_t s) {
  if (kernel == 2) return tma_launch_prologue(dtype, tile, runs, tiles, ntiles, s);
  return launch_prologue_plain(dtype, runs, tiles, ntiles, tw, th, s);
}

int launch_substep(int dtype, int kernel, int tile, const RunDesc *runs, const Tile *tiles,
                   int ntiles, int substep, int grid, int iso, cudaStream_t s) {
  if (kernel == 2) return tma_launch(dtype, tile, runs, tiles, ntiles, substep, grid, iso, s);
  if (dtype == 0) return launch_smem<float, 32, 8>(runs, tiles, ntiles, substep, grid, s);
  return launch_smem<double, 32, 4>(runs, tiles, ntiles, substep, grid, s);
}

// ---------------------------------------------------------------------------
// Periodic halo fill (Sec. 3.1): every ghost point takes the value of the
// interior point it wraps onto.  Reads interior points only, writes ghost
// points only, so there is no ordering hazard.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_halo(T *fields, int nfields, long long fstride, int nx, int ny, int nz, int px,
                       int py) {
  const int wx = nx + 2 * RAD, wy = ny + 2 * RAD, wz = nz + 2 * RAD;
  const long long total = (long long)wx * wy * wz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % wx) - RAD;
    const int j = (int)((e / wx) % wy) - RAD;
    const int k = (int)(e / ((long long)wx * wy)) - RAD;
    if (i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz) continue;
    const int si = (i % nx + nx) % nx, sj = (j % ny + ny) % ny, sk = (k % nz + nz) % nz;
    const long long dst = ((long long)(k + OZ) * py + (j + OY)) * px + (i + OX);
    const long long src = ((long long)(sk + OZ) * py + (sj + OY)) * px + (si + OX);
    for (int f = 0; f < nfields; ++f) fields[f * fstride + dst] = fields[f * fstride + src];
  }
}

int launch_halo(int dtype, void *fields, int nfields, long long fstride, int nx, int ny, int nz,
                int px, int py, cudaStream_t s) {
  const long long total = (long long)(nx + 6) * (ny + 6) * (nz + 6);
  int grid = (int)((total + 255) / 256);
  if (grid > 148 * 16) grid = 148 * 16;
  if (dtype == 0)
    k_halo<float><<<grid, 256, 0, s>>>(static_cast<float *>(fields), nfields, fstride, nx, ny, nz, px, py);
  else
    k_halo<double><<<grid, 256, 0, s>>>(static_cast<double *>(fields), nfields, fstride, nx, ny, nz, px, py);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dense <-> padded conversion of one field (host layout: x fastest, no halo).
// ---------------------------------------------------------------------------
template <typename T, typename H>
__global__ void k_set_field(const H *src, T *dst, int nx, int ny, int nz, int px, int py) {
  const long long total = (long long)nx * ny * nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long long)nx * ny));
    dst[((long long)(k + OZ) * py + (j + OY)) * px + (i + OX)] = T(src[e]);
  }
}

template <typename T>
__global__ void k_gather_points(const T *q, long long fstride, int px, int py, const int *ijk, int npts,
                                double *out, int wpairs) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= npts) return;
  const long long c = ((long long)(ijk[3 * n + 2] + OZ) * py + (ijk[3 * n + 1] + OY)) * px + (ijk[3 * n] + OX);
  for (int f = 0; f < NF; ++f) {
    const long long at =
        wpairs && f < 6 ? (long long)(f >> 1) * 2 * fstride + 4 * (c >> 1) + 2 * (f & 1) + (c & 1) : f * fstride + c;
    out[(long long)NF * n + f] = (double)q[at];
  }
}

int launch_gather_points(int dtype, const void *q, long long fstride, int px, int py, const int *ijk, int npts,
                         double *out, int wpairs, cudaStream_t s) {
  const int grid = (npts + 255) / 256;
  if (dtype == 0)
    k_gather_points<float><<<grid, 256, 0, s>>>(static_cast<const float *>(q), fstride, px, py, ijk, npts, out,
                                                 wpairs);
  else
    k_gather_points<double><<<grid, 256, 0, s>>>(static_cast<const double *>(q), fstride, px, py, ijk, npts,
                                                  out, wpairs);
  return (int)cudaGetLastError();
}

template <typename T, typename H>
__global__ void k_get_field(const T *src, H *dst, int nx, int ny, int nz, int px, int py, int pairs) {
  const long long total = (long long)nx * ny * nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long long)nx * ny));
    const long long c = ((long long)(k + OZ) * py + (j + OY)) * px + (i + OX);
    dst[e] = H(src[pairs ? 4 * (c >> 1) + (c & 1) : c]);
  }
}

// The paper's initial state (Sec. 4) at the interior points: ln rho = 0,
// u = 0 and A = amp * N(0,1) independently per component and point.  A points
// to field 4 of a state buffer; fields 0..3 are the NF - 3 fields before it.
// Normal number n = c * npts + e (component c, point e = (k ny + j) nx + i)
// by Box-Muller from SplitMix64 outputs 2n and 2n + 1 of the stream keyed by
// `seed` (u1 in (0, 1], u2 in [0, 1)), in FP64.  Only interior points are
// written, so the alignment padding keeps whatever it holds.
template <typename T>
__global__ void k_seed_field(T *A, long long fstride, int nx, int ny, int nz, int px, int py,
                             unsigned long long seed, double amp) {
  const long long npts = (long long)nx * ny * nz, total = 3 * npts;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < npts;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long long)nx * ny));
    const long long o = ((long long)(k + OZ) * py + (j + OY)) * px + (i + OX);
    for (int f = 0; f < 4; ++f) A[(f - 4) * fstride + o] = T(0);
  }
  const double TWO_PI = 6.283185307179586476925286766559;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < total;
       n += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(n / npts);
    const long long e = n - c * npts;
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long long)nx * ny));
    double g = 0.0;
    if (amp != 0.0) {  // the zero state (context creation) needs no random numbers
      const double u1 = (double)((splitmix64(seed, 2ull * (unsigned long long)n) >> 11) + 1ull) * 0x1.0p-53;
      const double u2 = (double)(splitmix64(seed, 2ull * (unsigned long long)n + 1ull) >> 11) * 0x1.0p-53;
      g = sqrt(-2.0 * log(u1)) * cos(TWO_PI * u2);
    }
    A[c * fstride + ((long long)(k + OZ) * py + (j + OY)) * px + (i + OX)] = T(amp * g);
  }
}

// Canary check of the alignment padding: counts the words of x-columns 0 and
// nx + OX + RAD .. px - 1 of nf fields that are not NaN.  No kernel reads or
// writes these columns; they are filled with NaN when a context is created.
template <typename T>
__global__ void k_padding_check(const T *q, int nf, long long fstride, int nx, int px, int py, int pz,
                                unsigned long long *bad) {
  const int first = nx + OX + RAD, ncols = 1 + (px - first);
  const long long rows = (long long)nf * py * pz, total = rows * ncols;
  unsigned long long cnt = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % ncols);
    const long long r = e / ncols;
    const int f = (int)(r / ((long long)py * pz));
    const long long row = r - (long long)f * py * pz;
    const int x = c == 0 ? 0 : first + c - 1;
    const T v = q[f * fstride + row * px + x];
    cnt += isnan(v) ? 0ull : 1ull;
  }
  if (cnt) atomicAdd(bad, cnt);
}

static int conv_grid(long long total) {
  long long g = (total + 255) / 256;
  return (int)(g > 148 * 32 ? 148 * 32 : (g < 1 ? 1 : g));
}

int launch_set_field(int dtype, int host_dtype, const void *src, void *dst_field, int nx, int ny,
                     int nz, int px, int py, cudaStream_t s) {
  const int g = conv_grid((long long)nx * ny * nz);
  if (dtype == 0 && host_dtype == 0)
    k_set_field<float, float><<<g, 256, 0, s>>>((const float *)src, (float *)dst_field, nx, ny, nz, px, py);
  else if (dtype == 0)
    k_set_field<float, double><<<g, 256, 0, s>>>((const double *)src, (float *)dst_field, nx, ny, nz, px, py);
  else if (host_dtype == 0)
    k_set_field<double, float><<<g, 256, 0, s>>>((const float *)src, (double *)dst_field, nx, ny, nz, px, py);
  else
    k_set_field<double, double><<<g, 256, 0, s>>>((const double *)src, (double *)dst_field, nx, ny, nz, px, py);
  return (int)cudaGetLastError();
}

int launch_seed_field(int dtype, void *A, long long fstride, int nx, int ny, int nz, int px, int py,
                      unsigned long long seed, double amp, cudaStream_t s) {
  const int g = conv_grid(3LL * nx * ny * nz);
  if (dtype == 0)
    k_seed_field<float><<<g, 256, 0, s>>>((float *)A, fstride, nx, ny, nz, px, py, seed, amp);
  else
    k_seed_field<double><<<g, 256, 0, s>>>((double *)A, fstride, nx, ny, nz, px, py, seed, amp);
  return (int)cudaGetLastError();
}

int launch_padding_check(int dtype, const void *q, int nf, long long fstride, int nx, int px, int py, int pz,
                         unsigned long long *bad, cudaStream_t s) {
  const int g = conv_grid((long long)nf * py * pz * (1 + px - (nx + OX + RAD)));
  if (dtype == 0)
    k_padding_check<float><<<g, 256, 0, s>>>((const float *)q, nf, fstride, nx, px, py, pz, bad);
  else
    k_padding_check<double><<<g, 256, 0, s>>>((const double *)q, nf, fstride, nx, px, py, pz, bad);
  return (int)cudaGetLastError();
}

int launch_get_field(int dtype, int host_dtype, const void *src_field, void *dst, int nx, int ny,
                     int nz, int px, int py, int pairs, cudaStream_t s) {
  const int g = conv_grid((long long)nx * ny * nz);
  if (dtype == 0 && host_dtype == 0)
    k_get_field<float, float><<<g, 256, 0, s>>>((const float *)src_field, (float *)dst, nx, ny, nz, px, py,
                                                pairs);
  else if (dtype == 0)
    k_get_field<float, double><<<g, 256, 0, s>>>((const float *)src_field, (double *)dst, nx, ny, nz, px, py,
                                                 pairs);
  else if (host_dtype == 0)
    k_get_field<double, float><<<g, 256, 0, s>>>((const double *)src_field, (float *)dst, nx, ny, nz, px, py,
                                                 pairs);
  else
    k_get_field<double, double><<<g, 256, 0, s>>>((const double *)src_field, (double *)dst, nx, ny, nz, px, py,
                                                  pairs);
  return (int)cudaGetLastError();
}

}  // namespace mhd
