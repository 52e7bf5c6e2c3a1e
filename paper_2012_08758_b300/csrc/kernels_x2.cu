// Substep kernel, paired-point TMA variant (FP32).
//
// The arithmetic of one stage of the 3rd-order 2N-storage Runge-Kutta scheme
// (Sec. 2) on the right-hand side of Eqs. 1-3 with the forcing of Eqs. 4-6,
// as in kernels_tma.cu, organised so that one thread computes TWO
// neighbouring x-points (x, x+1):
//
//  * a CTA owns a 64 x TY column and sweeps it along z; every z-plane of all
//    seven fields (3-point x/y halo) arrives by one TMA copy completed on an
//    mbarrier, P planes ahead;
//  * shared-memory reads are 64-bit pairs (f(x), f(x+1)), so one load serves
//    both points, and the arithmetic whose operands come as such pairs -- y
//    and z stencils, the right-hand side, the RK update -- runs on packed
//    FP32 pairs (__ffma2_rn / __fadd2_rn / __fmul2_rn); x-direction
//    differences, whose samples straddle pairs, are formed per point;
//  * the output plane o is computed once lead plane o+3 has arrived: its
//    z-neighbours o+1..o+3 are read from the stages still in shared memory,
//    only the three planes below (o-3..o-1) are kept in registers;
//  * the mixed x-z / y-z derivatives are split into the half from planes
//    above o, read from shared memory at o, and the half from planes below,
//    accumulated into a three-deep register ring as each plane passes
//    (S_s(o) = d_s(o+s) - d_s(o-s), d_s the x- or y-difference at distance s).
// Every wait on an mbarrier is bounded; on time-out the CTA records status
// bit 1 in the run's clock, waits (bounded) for its copies and returns.
#include <cuda.h>
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

__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
// Streaming 64-bit global load as a volatile asm statement: the w samples of
// the output plane keep their place before the wait for the lead plane, so
// that the latency of the read overlaps the plane's stencil work.
__device__ __forceinline__ float2 ldcs2_pinned(const float *p) {
  float2 v;
  asm volatile("ld.global.cs.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p) : "memory");
  return v;
}

// Stencil weights of the run as packed pairs (both lanes equal).
template <bool ISO>
struct PairCoefs {
  static constexpr int NA = ISO ? 1 : 3;
  float2 c1[NA][4], c2[NA][4], cm[NA][4];
  float2 cmn[NA][4];  // -cm (the half of a mixed derivative from planes below)
  float2 c6[NA];
  float2 cs2, nu, eta;
  int upwind;
  __device__ __forceinline__ void load(const RunDesc &R) {
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    for (int a = 0; a < NA; ++a) {
      for (int s = 0; s < 4; ++s) {
        c1[a][s] = bc(float(W1(s) * R.inv_h[a]));
        c2[a][s] = bc(float(W2(s) * R.inv_h[a] * R.inv_h[a]));
        cm[a][s] = bc(float(WM(s) * R.inv_h[pa[a]] * R.inv_h[pb[a]]));
        cmn[a][s] = bc(-float(WM(s) * R.inv_h[pa[a]] * R.inv_h[pb[a]]));
      }
      c6[a] = bc(float(R.inv_h[a] / 60.0));
    }
    cs2 = bc(float(R.cs2));
    nu = bc(float(R.nu));
    eta = bc(float(R.eta));
    upwind = R.upwind;
  }
  __device__ __forceinline__ float2 w1(int a, int s) const { return c1[ISO ? 0 : a][s]; }
  __device__ __forceinline__ float2 w2(int a, int s) const { return c2[ISO ? 0 : a][s]; }
  __device__ __forceinline__ float2 wm(int p, int s) const { return cm[ISO ? 0 : p][s]; }
  __device__ __forceinline__ float2 wmn(int p, int s) const { return cmn[ISO ? 0 : p][s]; }
  __device__ __forceinline__ float2 w6(int a) const { return c6[ISO ? 0 : a]; }
};

// First and second derivative from the paired differences d_s = f(+s) - f(-s)
// and sums e_s = f(+s) + f(-s), s = 1..3, and the centre c.
template <bool ISO>
__device__ __forceinline__ float2 d1p(const PairCoefs<ISO> &c, int a, float2 d1, float2 d2, float2 d3) {
  return fma2(c.w1(a, 3), d3, fma2(c.w1(a, 2), d2, mul2(c.w1(a, 1), d1)));
}
template <bool ISO>
__device__ __forceinline__ float2 d2p(const PairCoefs<ISO> &c, int a, float2 c0, float2 e1, float2 e2, float2 e3) {
  return fma2(c.w2(a, 3), e3, fma2(c.w2(a, 2), e2, fma2(c.w2(a, 1), e1, mul2(c.w2(a, 0), c0))));
}

}  // namespace

namespace {

// Derivatives at a pair of points (lane 0: x, lane 1: x+1).
struct PairDerivs {
  float2 lnr, u[3];
  float2 g[3];      // grad ln rho
  float2 G[3][3];   // G[a][b] = d u_a / d x_b
  float2 B[3];      // curl A (first-derivative stencil)
  float2 lapu[3], gdu[3], lapA[3];
  float2 jc[3];     // j = grad div A - lap A, d_a d_a A_a cancelled analytically (mu0 = 1)
  float2 up;        // upwinding term of d ln rho / dt (0 when off)
};

// dq/dt of Eqs. 1-3 at a pair of points, packed; f = forcing (zero when off).
// The same terms as rhs_point, with the scalar operations paired.
template <bool ISO>
__device__ __forceinline__ void rhs_pair(const PairDerivs &d, const PairCoefs<ISO> &c, const float2 f[3],
                                         float2 out[NF]) {
  const float2 M1 = bc(-1.f), third = bc(1.f / 3.f), mthird = bc(-1.f / 3.f), half = bc(0.5f), two = bc(2.f);
  const float2 rinv = pk(__expf(-d.lnr.x), __expf(-d.lnr.y));
  const float2 divu = add2(add2(d.G[0][0], d.G[1][1]), d.G[2][2]);
  // Eq. 1: D ln rho / Dt = -div u
  const float2 ug = fma2(d.u[2], d.g[2], fma2(d.u[1], d.g[1], mul2(d.u[0], d.g[0])));
  out[0] = sub2(sub2(d.up, ug), divu);
  const float2 nB[3] = {mul2(d.B[0], M1), mul2(d.B[1], M1), mul2(d.B[2], M1)};
  const float2 jxB[3] = {fma2(d.jc[1], d.B[2], mul2(d.jc[2], nB[1])), fma2(d.jc[2], d.B[0], mul2(d.jc[0], nB[2])),
                         fma2(d.jc[0], d.B[1], mul2(d.jc[1], nB[0]))};
  const float2 uxB[3] = {fma2(d.u[1], d.B[2], mul2(d.u[2], nB[1])), fma2(d.u[2], d.B[0], mul2(d.u[0], nB[2])),
                         fma2(d.u[0], d.B[1], mul2(d.u[1], nB[0]))};
  // traceless rate of strain (symmetric)
  float2 S[3][3];
  S[0][1] = S[1][0] = mul2(half, add2(d.G[0][1], d.G[1][0]));
  S[0][2] = S[2][0] = mul2(half, add2(d.G[0][2], d.G[2][0]));
  S[1][2] = S[2][1] = mul2(half, add2(d.G[1][2], d.G[2][1]));
#pragma unroll
  for (int a = 0; a < 3; ++a) S[a][a] = fma2(mthird, divu, d.G[a][a]);
  const float2 mcs2 = mul2(c.cs2, M1);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 Sg = fma2(S[a][2], d.g[2], fma2(S[a][1], d.g[1], mul2(S[a][0], d.g[0])));
    const float2 adv = fma2(d.u[2], d.G[a][2], fma2(d.u[1], d.G[a][1], mul2(d.u[0], d.G[a][0])));
    const float2 visc = fma2(two, Sg, fma2(third, d.gdu[a], d.lapu[a]));
    // Eq. 2
    out[1 + a] = fma2(c.nu, visc, fma2(jxB[a], rinv, fma2(mcs2, d.g[a], sub2(f[a], adv))));
    // Eq. 3 (diffusive gauge)
    out[4 + a] = fma2(c.eta, d.lapA[a], uxB[a]);
  }
}

}  // namespace

namespace {

// The samples of one field along x around a pair: 64-bit loads at x-4, x-2,
// x, x+2, x+4 (x even), and per point the differences d_s = f(+s) - f(-s)
// and sums e_s = f(+s) + f(-s), s = 1..3, paired.
struct XRow {
  float2 c, d1, d2, d3, e1, e2, e3;
};
__device__ __forceinline__ XRow xrow(const float *b) {
  const float2 A = ld2(b - 4), Bq = ld2(b - 2), C = ld2(b), D = ld2(b + 2), E = ld2(b + 4);
  XRow r;
  r.c = C;
  r.d1 = pk(C.y - Bq.y, D.x - C.x);
  r.d2 = pk(D.x - Bq.x, D.y - Bq.y);
  r.d3 = pk(D.y - A.y, E.x - Bq.x);
  r.e1 = pk(C.y + Bq.y, D.x + C.x);
  r.e2 = pk(D.x + Bq.x, D.y + Bq.y);
  r.e3 = pk(D.y + A.y, E.x + Bq.x);
  return r;
}

// The x-differences d_s = f(+s) - f(-s) of a pair in the row at b, for one s.
template <int S>
__device__ __forceinline__ float2 xdiff(const float *b) {
  if (S == 1) {
    const float2 Bq = ld2(b - 2), C = ld2(b), D = ld2(b + 2);
    return pk(C.y - Bq.y, D.x - C.x);
  } else if (S == 2) {
    const float2 Bq = ld2(b - 2), D = ld2(b + 2);
    return pk(D.x - Bq.x, D.y - Bq.y);
  } else {
    const float2 A = ld2(b - 4), Bq = ld2(b - 2), D = ld2(b + 2), E = ld2(b + 4);
    return pk(D.y - A.y, E.x - Bq.x);
  }
}

// Samples along y: d_s = f(y+s) - f(y-s), e_s = f(y+s) + f(y-s), paired.
struct YRow {
  float2 d1, d2, d3, e1, e2, e3;
};
template <int SX>
__device__ __forceinline__ YRow yrow(const float *b) {
  YRow r;
  float2 p = ld2(b + SX), m = ld2(b - SX);
  r.d1 = sub2(p, m);
  r.e1 = add2(p, m);
  p = ld2(b + 2 * SX), m = ld2(b - 2 * SX);
  r.d2 = sub2(p, m);
  r.e2 = add2(p, m);
  p = ld2(b + 3 * SX), m = ld2(b - 3 * SX);
  r.d3 = sub2(p, m);
  r.e3 = add2(p, m);
  return r;
}

// x-y mixed derivative of a pair on the two diagonals (R1):
// sum_s wm_s [(f(x+s, y+s) - f(x-s, y+s)) - (f(x+s, y-s) - f(x-s, y-s))].
template <int SX, bool ISO>
__device__ __forceinline__ float2 dxy_pair(const float *b, const PairCoefs<ISO> &c) {
  const float2 S1 = sub2(xdiff<1>(b + SX), xdiff<1>(b - SX));
  const float2 S2 = sub2(xdiff<2>(b + 2 * SX), xdiff<2>(b - 2 * SX));
  const float2 S3 = sub2(xdiff<3>(b + 3 * SX), xdiff<3>(b - 3 * SX));
  return fma2(c.wm(0, 3), S3, fma2(c.wm(0, 2), S2, mul2(c.wm(0, 1), S1)));
}

}  // namespace

// Warp-specialised variants (WS): a fifth warpgroup of the CTA only issues
// the TMA copies; each stage has a "full" mbarrier (the copy's bytes) and an
// "empty" one (one arrival per compute warp once the stage's plane has left
// its last use, three planes after it led), so the compute warps never meet
// at a CTA barrier.  The producer warpgroup gives its registers to the
// compute warpgroups (setmaxnreg): at launch 32 x (TY + 4) threads hold
// X2_WS_LAUNCH_REGS each; 4 x 32 producer threads keep X2_WS_PRODUCER_REGS
// and the TY warps of compute threads may use X2_WS_COMPUTE_REGS, with
// (TY + 4) * 32 * LAUNCH = TY * 32 * COMPUTE + 128 * PRODUCER for TY = 8.
constexpr int X2_WS_LAUNCH_REGS = 168, X2_WS_PRODUCER_REGS = 40, X2_WS_COMPUTE_REGS = 232;
static_assert(12 * 32 * X2_WS_LAUNCH_REGS == 8 * 32 * X2_WS_COMPUTE_REGS + 4 * 32 * X2_WS_PRODUCER_REGS,
              "register split of the warp-specialised variants");

// Shared memory of a variant: NS TMA stages of q; for the warp-specialised
// variants, where it fits, a ring of NW <= NS - 3 stages of w (the interior
// points of one z-plane of the tile, all fields; substeps 2 and 3 read w
// through it instead of from global memory); then the mbarriers (full /
// empty per stage of each ring).
//
// A w stage holds the seven fields' TY x 64 values.  Variants with the WP
// layout instead keep w's fields 0-5 as three interleaved arrays, m = 0..2,
// each 2 fstride values from 2 m fstride on: the points (2j, 2j+1) of fields
// 2m and 2m+1 are the four values 4j .. 4j+3 (field 2m at both points, then
// field 2m+1), field 6 as usual; a thread writes and reads its two points of
// a field pair as one 16-byte access, and a w stage holds the three arrays'
// TY x 128 values, then field 6's TY x 64.  (The second substep updates w in
// place, so every substep of a run uses the one layout.)
template <int TY>
__host__ __device__ constexpr int x2_wstage_bytes() {
  return NF * TY * 64 * (int)sizeof(float);
}
template <int TY>
__host__ __device__ constexpr int x2_wpair_bytes() {
  return 3 * TY * 128 * (int)sizeof(float);
}
template <int TY, int NS, int NW>
__host__ __device__ constexpr int x2_ws_bytes() {
  return NS * TmaShape<float, TY, 64>::STAGE_BYTES + NW * x2_wstage_bytes<TY>() + (2 * NS + 2 * NW) * 8;
}
// the largest w ring that fits the opt-in limit of dynamic shared memory per
// block (232448 bytes), 0 if none
template <int TY, int NS>
__host__ __device__ constexpr int x2_wring() {
  return x2_ws_bytes<TY, NS, NS - 3>() <= 232448   ? NS - 3
         : x2_ws_bytes<TY, NS, 2>() <= 232448      ? 2
         : 0;
}
template <int TY, int NS, bool WS>
__host__ __device__ constexpr int x2_smem_bytes() {
  return !WS ? NS * TmaShape<float, TY, 64>::STAGE_BYTES + NS * 8 : x2_ws_bytes<TY, NS, x2_wring<TY, NS>()>();
}

namespace {
// The producer: every plane of every tile of this CTA, in the compute warps'
// order, into stage g mod NS once the plane g - NS has been released.  On a
// wait that gives up it records status bit 1 and raises the CTA's abort flag;
// before returning it waits (bounded) for every copy it issued.  WT: after
// lead plane p it also copies w of output plane p - WL into the w ring, slot
// gw mod NW, once w plane gw - NW has been released; WL = NS - NW - 1, so
// that w arrives a plane before the compute warps reach that output plane
// (with the copy issued with the plane's own lead copy the third substep
// waited for it) and at most NW w planes are in flight; the w of the tile's
// last output planes follows its last lead plane.
template <int TY, int NS, int SUB, bool WT, bool WP>
__device__ __forceinline__ void x2_produce(const RunDesc *__restrict__ runs, const Tile *__restrict__ tiles,
                                           int ntiles, unsigned char *smem, uint64_t *full, uint64_t *empty,
                                           unsigned char *wst, uint64_t *wfull, uint64_t *wempty,
                                           volatile int *abort) {
  using SH = TmaShape<float, TY, 64>;
  constexpr int NW = x2_wring<TY, NS>() > 0 ? x2_wring<TY, NS>() : 1, WL = NS - NW - 1;
  // the w slot the producer waits for at lead p frees once output p - WL - NW
  // is done, which needs q planes up to p - WL - NW + RAD only: no cycle
  static_assert(!WT || WL + NW > RAD, "the w ring must not wait on planes not yet issued");
  unsigned long long g = 0, gw = 0;
  int fail_run = -1;
  for (int t = blockIdx.x; t < ntiles && fail_run < 0; t += gridDim.x) {
    const Tile tile = tiles[t];
    if (tile.z1 <= tile.z0) continue;
    const RunDesc &R = runs[tile.run];
    const CUtensorMap *map = &R.tmap[(R.coeffs->parity + SUB) & 1];
    const int npl = (tile.z1 - tile.z0) + 2 * RAD;
    // w of output plane o (lead index, padded z = z0 + o) into the ring
    auto issue_w = [&](int o) {
      const int ws = (int)(gw % NW);
      if ((gw >= NW && !mbar_wait(&wempty[ws], (uint32_t)(((gw / NW) - 1) & 1ull))) || *abort) return false;
      unsigned char *dst = wst + ws * x2_wstage_bytes<TY>();
      mbar_arrive_expect_tx(&wfull[ws], (uint32_t)x2_wstage_bytes<TY>());
      if constexpr (WP) {
        tma_load_4d(dst, &R.wpmap[0], &wfull[ws], 2 * (tile.x0 + OX), tile.y0 + OY, tile.z0 + o, 0);
        tma_load_4d(dst + x2_wpair_bytes<TY>(), &R.wpmap[1], &wfull[ws], tile.x0 + OX, tile.y0 + OY, tile.z0 + o,
                    0);
      } else {
        tma_load_4d(dst, &R.wmap, &wfull[ws], tile.x0 + OX, tile.y0 + OY, tile.z0 + o, 0);
      }
      ++gw;
      return true;
    };
    for (int p = 0; p < npl; ++p, ++g) {
      const int sl = (int)(g % NS);
      if ((g >= NS && !mbar_wait(&empty[sl], (uint32_t)(((g / NS) - 1) & 1ull))) || *abort) {
        fail_run = tile.run;
        break;
      }
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&full[sl], (uint32_t)(NF * SH::FIELD * sizeof(float)));
      tma_load_4d(smem + sl * SH::STAGE_BYTES, map, &full[sl], tile.x0, tile.y0, tile.z0 + p, 0);
      if constexpr (WT) {
        const int ow = p - WL;
        if (ow >= RAD && ow < npl - RAD && !issue_w(ow)) {
          fail_run = tile.run;
          ++g;
          break;
        }
      }
    }
    if constexpr (WT) {
      // the w of the tile's last output planes
      for (int o = npl - WL; fail_run < 0 && o < npl - RAD; ++o)
        if (o >= RAD && !issue_w(o)) fail_run = tile.run;
    }
  }
  if (fail_run >= 0) {
    atomicOr(&runs[fail_run].clock->status, 2);
    *abort = 1;
  }
  for (unsigned long long q = g > (unsigned long long)NS ? g - NS : 0; q < g; ++q)
    mbar_wait(&full[q % NS], (uint32_t)((q / NS) & 1ull));
  if constexpr (WT)
    for (unsigned long long q = gw > (unsigned long long)NW ? gw - NW : 0; q < gw; ++q)
      mbar_wait(&wfull[q % NW], (uint32_t)((q / NW) & 1ull));
}
}  // namespace

// SUB: the RK substep (0, 1, 2), a compile-time constant so that each
// instantiation carries only its own w traffic (none read at 0, none written
// at 2) and its own RK coefficients.
template <int TY, int NS, int BAR, bool ISO, int SUB, bool WS, bool WP>
__global__ void __launch_bounds__(32 * TY + (WS ? 128 : 0), 1)
    k_substep_x2(const RunDesc *__restrict__ runs, const Tile *__restrict__ tiles, int ntiles) {
  constexpr int substep = SUB;
  using SH = TmaShape<float, TY, 64>;
  constexpr int SX = SH::SX, FIELD = SH::FIELD;
  // Prefetch distance: the stage of plane q is last read when q is the output
  // plane (lead plane q+3) and refilled by plane q+NS, issued P planes ahead;
  // warps drift apart by up to BAR planes between CTA barriers.
  constexpr int P = WS ? NS : NS - 3 - BAR;  // WS: the producer runs ahead by itself
  static_assert(WS ? NS >= 5 : P >= 1, "need at least one plane of prefetch");
  static_assert(!WS || TY == 8, "the register split of the warp-specialised variants is for 8 compute warps");
  extern __shared__ __align__(128) unsigned char smem[];
  // WTL: the layout holds the w ring (every substep of such a variant); WT:
  // this substep reads w through it
  constexpr bool WTL = WS && x2_wring<TY, NS>() > 0;
  constexpr bool WT = WTL && SUB > 0;
  constexpr int NW = WTL ? x2_wring<TY, NS>() : 1;
  static_assert(!WP || WTL, "the interleaved w layout is read through the w ring");
  unsigned char *wst = smem + NS * SH::STAGE_BYTES;
  uint64_t *bars = reinterpret_cast<uint64_t *>(wst + (WTL ? NW * x2_wstage_bytes<TY>() : 0));
  uint64_t *wfull = bars + 2 * NS, *wempty = bars + 2 * NS + NW;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  __shared__ int ws_abort;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    if constexpr (WS)
      for (int s = 0; s < NS; ++s) mbar_init(&bars[NS + s], TY);
    if constexpr (WTL)
      for (int s = 0; s < NW; ++s) {
        mbar_init(&wfull[s], 1);
        mbar_init(&wempty[s], TY);
      }
    if constexpr (WS) ws_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();
  if constexpr (WS) {
    if (ty >= TY) {
      asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(X2_WS_PRODUCER_REGS));
      if (ty == TY && tx == 0)
        x2_produce<TY, NS, SUB, WT, WP>(runs, tiles, ntiles, smem, bars, bars + NS, wst, wfull, wempty, &ws_abort);
      return;
    }
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(X2_WS_COMPUTE_REGS));
  }

  unsigned long long G = 0;  // planes issued by this CTA before the current tile
  unsigned long long gwc = 0;  // WT: output planes whose w this warp has taken from the ring
  bool failed = false, waits_ok = true;
  int fail_run = -1, fail_p = 0, issued_hi = 0;

  for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
    const Tile tile = tiles[t];
    if (tile.z1 <= tile.z0) continue;  // padding entry of the work split
    const RunDesc &R = runs[tile.run];
    const StepCoeffs &K = *R.coeffs;
    PairCoefs<ISO> c;
    c.load(R);
    const int nx = R.nx, ny = R.ny, nz = R.nz, px = R.px, py = R.py, nzg = R.nzg;
    const bool zper = R.z_open == 0;
    const long long fs = R.fstride;
    const int par = (K.parity + substep) & 1;
    const CUtensorMap *map = &R.tmap[par];
    float *__restrict__ qout = static_cast<float *>(R.q[par ^ 1]);
    float *__restrict__ w = static_cast<float *>(R.w);
    const float2 dt = bc(float(K.dt));
    const float2 alpha = bc(float(RK_ALPHA(substep))), beta = bc(float(RK_BETA(substep)));
    const int x = tile.x0 + 2 * tx, y = tile.y0 + ty;
    const bool act0 = x < nx && y < ny, act1 = x + 1 < nx && y < ny;
    const bool yedge = y < RAD || y >= ny - RAD;
    const bool xn0 = x < RAD || x >= nx - RAD, xn1 = x + 1 < RAD || x + 1 >= nx - RAD;
    const bool edge0 = yedge || xn0, edge1 = yedge || xn1;
    // Every point within RAD of a face has exactly one image per non-empty
    // subset of its non-zero shifts (x +- nx, y +- ny, z +- nz) when each
    // periodic axis has at least 2 RAD + 1 points: the y and z shifts are
    // common to the pair, so those images are stored as pairs too, and only
    // the x images are stored per point.
    const bool shift_images = nx >= 2 * RAD + 1 && ny >= 2 * RAD + 1 && (nz >= 2 * RAD + 1 || !zper);
    const int npl = (tile.z1 - tile.z0) + 2 * RAD;  // lead planes z0-3 .. z1+2

    const bool forcing = K.forcing != 0;
    const bool force_in_rhs = forcing && R.forcing_mode == 0;
    const bool force_at_end = forcing && R.forcing_mode == 1 && substep == 2;
    float2 exr = bc(1.f), exi = bc(0.f);  // e^{i (k_x x + k_y y)} of the two points
    int mz = 0;                            // (k_z * z_out) mod nzg, global plane index
    if (forcing) {
      const Cplx<float> *rx = static_cast<const Cplx<float> *>(R.roots[0]);
      const Cplx<float> *ry = static_cast<const Cplx<float> *>(R.roots[1]);
      if (act0) {
        const Cplx<float> ey = ry[(int)(((long long)K.kmod[1] * y) % ny)];
        const Cplx<float> e0 = cmul(rx[(int)(((long long)K.kmod[0] * x) % nx)], ey);
        const Cplx<float> e1 = act1 ? cmul(rx[(int)(((long long)K.kmod[0] * (x + 1)) % nx)], ey) : e0;
        exr = pk(e0.re, e1.re);
        exi = pk(e0.im, e1.im);
      }
      mz = (int)(((long long)K.kmod[2] * (tile.z0 + R.z_off)) % nzg);
    }
    const int kz = K.kmod[2];
    const Cplx<float> ephi = {float(K.cphi), float(K.sphi)};
    const Cplx<float> *rz = static_cast<const Cplx<float> *>(R.roots[2]);
    // warp-specialised variants: e^{i k_z z} of the next output plane is
    // requested one plane ahead (measured: the barrier variants run slower so)
    Cplx<float> ez_next = {1.f, 0.f};
    if (WS && forcing) ez_next = rz[mz];

    int slot = (int)(G % NS);
    uint32_t phase = (uint32_t)((G / NS) & 1ull);
    auto issue = [&](int p, int sl) {
      uint64_t *bar = &bars[sl];
      mbar_arrive_expect_tx(bar, (uint32_t)(NF * FIELD * sizeof(float)));
      tma_load_4d(smem + sl * SH::STAGE_BYTES, map, bar, tile.x0, tile.y0, tile.z0 + p, 0);
    };
    if (!WS && tid == 0) {
      fence_proxy_async_smem();
      const int first = npl < P ? npl : P;
      for (int p = 0; p < first; ++p) issue(p, (slot + p) % NS);
      issued_hi = first;
    }

    // Registers that follow the sweep: the three planes below the centre
    // plane (pz[f][k]: plane o-3+k), and the halves of the x-z / y-z mixed
    // derivatives contributed by planes below, for output planes o, o+1, o+2
    // (a*[k]).  aX1 = d_x d_z u_z, aY1 = d_y d_z u_z, aZ1 = d_x d_z u_x +
    // d_y d_z u_y; aX2, aY2, aZ2 the same for A.
    float2 pz[NF][3];
    float2 aX1[3], aY1[3], aZ1[3], aX2[3], aY2[3], aZ2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int f = 0; f < NF; ++f) pz[f][k] = bc(0.f);
      aX1[k] = aY1[k] = aZ1[k] = aX2[k] = aY2[k] = aZ2[k] = bc(0.f);
    }
    const int cxy = (ty + RAD) * SX + 2 * tx + 4;  // the pair's first point inside a field plane
    const bool need_w = substep > 0 && act0;
    const long long wplane = (long long)py * px;
    // padded index of the first point of the pair in output plane z0
    long long cidx = ((long long)(tile.z0 + OZ) * py + (y + OY)) * px + (x + OX);
    float fa[3] = {0.f, 0.f, 0.f}, fb[3] = {0.f, 0.f, 0.f};
    if (forcing)
      for (int a = 0; a < 3; ++a) {
        fa[a] = float(K.fa[a]);
        fb[a] = float(K.fb[a]);
      }

    // the halves from planes below: ring update with the differences d_s of
    // the plane that is leaving the centre (output o+s receives -wm_s d_s)
    auto pass1 = [&](float2 a[3], int pr, float2 d1, float2 d2, float2 d3) {
      a[0] = fma2(c.wmn(pr, 1), d1, a[1]);
      a[1] = fma2(c.wmn(pr, 2), d2, a[2]);
      a[2] = mul2(c.wmn(pr, 3), d3);
    };
    auto pass2 = [&](float2 a[3], float2 x1, float2 x2, float2 x3, float2 y1, float2 y2, float2 y3) {
      a[0] = fma2(c.wmn(2, 1), y1, fma2(c.wmn(1, 1), x1, a[1]));
      a[1] = fma2(c.wmn(2, 2), y2, fma2(c.wmn(1, 2), x2, a[2]));
      a[2] = fma2(c.wmn(2, 3), y3, mul2(c.wmn(1, 3), x3));
    };
    auto ydiff = [&](const float *b, int s) { return sub2(ld2(b + s * SX), ld2(b - s * SX)); };

    for (int p = 0; p < npl && !failed; ++p) {
      if (!WS && tid == 0 && p + P < npl) {
        fence_proxy_async_smem();
        int sl = slot + P;
        if (sl >= NS) sl -= NS;
        issue(p + P, sl);
        issued_hi = p + P + 1;
      }
      const int o = p - RAD;       // centre plane (lead index), interior plane z0 + o - 3
      const bool outp = o >= RAD;  // an interior plane of this tile: computed and stored
      float2 wc[NF];
      if (!WT && need_w && outp) {
        const float *wp = w + cidx;
#pragma unroll
        for (int f = 0; f < NF; ++f, wp += fs) wc[f] = ldcs2_pinned(wp);
      }
      const bool ok = mbar_wait(&bars[slot], phase);
      if (o >= 0 && ok) {
        int os = slot - RAD;
        if (os < 0) os += NS;
        auto stage = [&](int k) {  // plane o + k, k = 0..3
          int sl = os + k;
          if (sl >= NS) sl -= NS;
          return reinterpret_cast<const float *>(smem + sl * SH::STAGE_BYTES) + cxy;
        };
        const float *so = stage(0);
        if (!outp) {
          // halo plane below the tile: only its centres and differences enter the registers
          float2 cen[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) cen[f] = ld2(so + f * FIELD);
          const XRow xux = xrow(so + 1 * FIELD), xuz = xrow(so + 3 * FIELD), xAx = xrow(so + 4 * FIELD),
                     xAz = xrow(so + 6 * FIELD);
          const YRow yuy = yrow<SX>(so + 2 * FIELD), yuz = yrow<SX>(so + 3 * FIELD), yAy = yrow<SX>(so + 5 * FIELD),
                     yAz = yrow<SX>(so + 6 * FIELD);
          pass1(aX1, 1, xuz.d1, xuz.d2, xuz.d3);
          pass1(aY1, 2, yuz.d1, yuz.d2, yuz.d3);
          pass2(aZ1, xux.d1, xux.d2, xux.d3, yuy.d1, yuy.d2, yuy.d3);
          pass1(aX2, 1, xAz.d1, xAz.d2, xAz.d3);
          pass1(aY2, 2, yAz.d1, yAz.d2, yAz.d3);
          pass2(aZ2, xAx.d1, xAx.d2, xAx.d3, yAy.d1, yAy.d2, yAy.d3);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            pz[f][0] = pz[f][1];
            pz[f][1] = pz[f][2];
            pz[f][2] = cen[f];
          }
        } else {
          // ---- output plane: the planes above come from shared memory ----
          const float *s1 = stage(1), *s2 = stage(2), *s3 = stage(3);
          auto zrow = [&](int f, float2 &d1, float2 &d2, float2 &d3, float2 &e1, float2 &e2, float2 &e3) {
            const float2 p1 = ld2(s1 + f * FIELD), p2 = ld2(s2 + f * FIELD), p3 = ld2(s3 + f * FIELD);
            d1 = sub2(p1, pz[f][2]);
            e1 = add2(p1, pz[f][2]);
            d2 = sub2(p2, pz[f][1]);
            e2 = add2(p2, pz[f][1]);
            d3 = sub2(p3, pz[f][0]);
            e3 = add2(p3, pz[f][0]);
          };
          // halves of the x-z / y-z mixed derivatives from the planes above
          auto fxz = [&](int f) {
            return fma2(c.wm(1, 3), xdiff<3>(s3 + f * FIELD),
                        fma2(c.wm(1, 2), xdiff<2>(s2 + f * FIELD), mul2(c.wm(1, 1), xdiff<1>(s1 + f * FIELD))));
          };
          auto fyz = [&](int f) {
            return fma2(c.wm(2, 3), ydiff(s3 + f * FIELD, 3),
                        fma2(c.wm(2, 2), ydiff(s2 + f * FIELD, 2), mul2(c.wm(2, 1), ydiff(s1 + f * FIELD, 1))));
          };
          PairDerivs d;
          float2 zd1, zd2, zd3, ze1, ze2, ze3;

          // Each field group is finished -- its differences passed on to the
          // rings of the planes below and its centres pushed into the pencils --
          // as soon as its derivatives are formed, so that its rows need no
          // registers afterwards.
          // vector potential: B = curl A, lap A, j
          {
            const XRow xAx = xrow(so + 4 * FIELD), xAy = xrow(so + 5 * FIELD), xAz = xrow(so + 6 * FIELD);
            const YRow yAx = yrow<SX>(so + 4 * FIELD), yAy = yrow<SX>(so + 5 * FIELD), yAz = yrow<SX>(so + 6 * FIELD);
            zrow(4, zd1, zd2, zd3, ze1, ze2, ze3);
            const float2 dzAx = d1p(c, 2, zd1, zd2, zd3);
            const float2 Axz_ = d2p(c, 2, xAx.c, ze1, ze2, ze3);
            zrow(5, zd1, zd2, zd3, ze1, ze2, ze3);
            const float2 dzAy = d1p(c, 2, zd1, zd2, zd3);
            const float2 Ayz_ = d2p(c, 2, xAy.c, ze1, ze2, ze3);
            zrow(6, zd1, zd2, zd3, ze1, ze2, ze3);
            const float2 Azz = d2p(c, 2, xAz.c, ze1, ze2, ze3);
            d.B[0] = sub2(d1p(c, 1, yAz.d1, yAz.d2, yAz.d3), dzAy);
            d.B[1] = sub2(dzAx, d1p(c, 0, xAz.d1, xAz.d2, xAz.d3));
            d.B[2] = sub2(d1p(c, 0, xAy.d1, xAy.d2, xAy.d3), d1p(c, 1, yAx.d1, yAx.d2, yAx.d3));
            const float2 Axx = d2p(c, 0, xAx.c, xAx.e1, xAx.e2, xAx.e3), Axy_ = d2p(c, 1, xAx.c, yAx.e1, yAx.e2, yAx.e3);
            const float2 Ayx = d2p(c, 0, xAy.c, xAy.e1, xAy.e2, xAy.e3), Ayy = d2p(c, 1, xAy.c, yAy.e1, yAy.e2, yAy.e3);
            const float2 Azx = d2p(c, 0, xAz.c, xAz.e1, xAz.e2, xAz.e3), Azy = d2p(c, 1, xAz.c, yAz.e1, yAz.e2, yAz.e3);
            d.lapA[0] = add2(add2(Axx, Axy_), Axz_);
            d.lapA[1] = add2(add2(Ayx, Ayy), Ayz_);
            d.lapA[2] = add2(add2(Azx, Azy), Azz);
            d.jc[0] = sub2(sub2(add2(dxy_pair<SX>(so + 5 * FIELD, c), add2(fxz(6), aX2[0])), Axy_), Axz_);
            d.jc[1] = sub2(sub2(add2(dxy_pair<SX>(so + 4 * FIELD, c), add2(fyz(6), aY2[0])), Ayx), Ayz_);
            d.jc[2] = sub2(sub2(add2(add2(fxz(4), fyz(5)), aZ2[0]), Azx), Azy);
            pass1(aX2, 1, xAz.d1, xAz.d2, xAz.d3);
            pass1(aY2, 2, yAz.d1, yAz.d2, yAz.d3);
            pass2(aZ2, xAx.d1, xAx.d2, xAx.d3, yAy.d1, yAy.d2, yAy.d3);
            const float2 cen[3] = {xAx.c, xAy.c, xAz.c};
#pragma unroll
            for (int f = 4; f < NF; ++f) {
              pz[f][0] = pz[f][1];
              pz[f][1] = pz[f][2];
              pz[f][2] = cen[f - 4];
            }
          }

          // velocity: grad u, lap u, grad div u
          {
            const XRow xux = xrow(so + 1 * FIELD), xuy = xrow(so + 2 * FIELD), xuz = xrow(so + 3 * FIELD);
            const YRow yux = yrow<SX>(so + 1 * FIELD), yuy = yrow<SX>(so + 2 * FIELD), yuz = yrow<SX>(so + 3 * FIELD);
            d.u[0] = xux.c;
            d.u[1] = xuy.c;
            d.u[2] = xuz.c;
            float2 uz2[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const XRow &xr = a == 0 ? xux : a == 1 ? xuy : xuz;
              const YRow &yr = a == 0 ? yux : a == 1 ? yuy : yuz;
              zrow(1 + a, zd1, zd2, zd3, ze1, ze2, ze3);
              d.G[a][0] = d1p(c, 0, xr.d1, xr.d2, xr.d3);
              d.G[a][1] = d1p(c, 1, yr.d1, yr.d2, yr.d3);
              d.G[a][2] = d1p(c, 2, zd1, zd2, zd3);
              const float2 xx = d2p(c, 0, xr.c, xr.e1, xr.e2, xr.e3), yy = d2p(c, 1, xr.c, yr.e1, yr.e2, yr.e3),
                           zz = d2p(c, 2, xr.c, ze1, ze2, ze3);
              d.lapu[a] = add2(add2(xx, yy), zz);
              uz2[a] = a == 0 ? xx : a == 1 ? yy : zz;  // the d_a d_a u_a term of grad div u
            }
            d.gdu[0] = add2(add2(uz2[0], dxy_pair<SX>(so + 2 * FIELD, c)), add2(fxz(3), aX1[0]));
            d.gdu[1] = add2(add2(dxy_pair<SX>(so + 1 * FIELD, c), uz2[1]), add2(fyz(3), aY1[0]));
            d.gdu[2] = add2(add2(add2(fxz(1), fyz(2)), aZ1[0]), uz2[2]);
            pass1(aX1, 1, xuz.d1, xuz.d2, xuz.d3);
            pass1(aY1, 2, yuz.d1, yuz.d2, yuz.d3);
            pass2(aZ1, xux.d1, xux.d2, xux.d3, yuy.d1, yuy.d2, yuy.d3);
#pragma unroll
            for (int f = 1; f < 4; ++f) {
              pz[f][0] = pz[f][1];
              pz[f][1] = pz[f][2];
              pz[f][2] = d.u[f - 1];
            }
          }

          // density: grad ln rho and the upwinding term
          {
            const XRow xl = xrow(so);
            const YRow yl = yrow<SX>(so);
            zrow(0, zd1, zd2, zd3, ze1, ze2, ze3);
            d.lnr = xl.c;
            d.g[0] = d1p(c, 0, xl.d1, xl.d2, xl.d3);
            d.g[1] = d1p(c, 1, yl.d1, yl.d2, yl.d3);
            d.g[2] = d1p(c, 2, zd1, zd2, zd3);
            d.up = bc(0.f);
            if (c.upwind) {
              // sixth difference (f-3 + f3) - 6 (f-2 + f2) + 15 (f-1 + f1) - 20 f0 per axis
              const float2 m20 = mul2(bc(-20.f), xl.c);
              auto d6 = [&](float2 e1, float2 e2, float2 e3) {
                return add2(fma2(bc(-6.f), e2, e3), fma2(bc(15.f), e1, m20));
              };
              auto absu = [&](float2 u) { return pk(fabsf(u.x), fabsf(u.y)); };
              d.up = fma2(mul2(c.w6(2), absu(d.u[2])), d6(ze1, ze2, ze3),
                          fma2(mul2(c.w6(1), absu(d.u[1])), d6(yl.e1, yl.e2, yl.e3),
                               mul2(mul2(c.w6(0), absu(d.u[0])), d6(xl.e1, xl.e2, xl.e3))));
            }
            pz[0][0] = pz[0][1];
            pz[0][1] = pz[0][2];
            pz[0][2] = xl.c;
          }

          // forcing of the step at the pair (Eqs. 4-6)
          float2 fz[3] = {bc(0.f), bc(0.f), bc(0.f)};
          if (forcing) {
            const Cplx<float> ez = cmul(WS ? ez_next : rz[mz], ephi);  // e^{i (k_z z + phi)}
            const float2 er = fma2(exr, bc(ez.re), mul2(exi, bc(-ez.im)));
            const float2 ei = fma2(exr, bc(ez.im), mul2(exi, bc(ez.re)));
#pragma unroll
            for (int a = 0; a < 3; ++a) fz[a] = fma2(bc(fa[a]), er, mul2(bc(-fb[a]), ei));
          }
          const float2 fr[3] = {force_in_rhs ? fz[0] : bc(0.f), force_in_rhs ? fz[1] : bc(0.f),
                                force_in_rhs ? fz[2] : bc(0.f)};
          float2 r[NF];
          rhs_pair(d, c, fr, r);

          // RK3-2N update: w <- alpha w + dt RHS, q <- q + beta w
          float2 qc[NF];  // centres of the output plane (just pushed into the pencils)
#pragma unroll
          for (int f = 0; f < NF; ++f) qc[f] = pz[f][2];
          float2 wv[NF], qn[NF];
          if constexpr (WT) {
            // w of this output plane from the ring, then the slot goes back
            const int ws = (int)(gwc % NW);
            if (!mbar_wait(&wfull[ws], (uint32_t)((gwc / NW) & 1ull))) {
              ws_abort = 1;
              atomicOr(&R.clock->status, 2);
            }
            const float *wr = reinterpret_cast<const float *>(wst + ws * x2_wstage_bytes<TY>());
            if constexpr (WP) {
#pragma unroll
              for (int m = 0; m < 3; ++m) {
                const float4 v = *reinterpret_cast<const float4 *>(wr + (m * TY + ty) * 128 + 4 * tx);
                wc[2 * m] = make_float2(v.x, v.y);
                wc[2 * m + 1] = make_float2(v.z, v.w);
              }
              wc[6] = ld2(wr + 3 * TY * 128 + ty * 64 + 2 * tx);
            } else {
#pragma unroll
              for (int f = 0; f < NF; ++f) wc[f] = ld2(wr + (f * TY + ty) * 64 + 2 * tx);
            }
            __syncwarp();
            if (tx == 0) mbar_arrive(&wempty[ws]);
            ++gwc;
          }
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            wv[f] = mul2(dt, r[f]);
            if constexpr (SUB > 0) wv[f] = fma2(alpha, wc[f], wv[f]);
            qn[f] = fma2(beta, wv[f], qc[f]);
          }
          if (force_at_end)
#pragma unroll
            for (int a = 0; a < 3; ++a) qn[1 + a] = fma2(dt, fz[a], qn[1 + a]);
          if (act0) {
            const int z = tile.z0 + o - RAD;  // interior index of the output plane
            const bool zn = z < RAD || z >= nz - RAD;
            const bool near0 = edge0 || zn, near1 = edge1 || zn;
            if (act1 && !near0 && !near1) {
              if constexpr (SUB < 2 && WP) {
                float *wb = w + 2 * cidx;
#pragma unroll
                for (int m = 0; m < 3; ++m)
                  __stcs(reinterpret_cast<float4 *>(wb + 2 * m * fs),
                         make_float4(wv[2 * m].x, wv[2 * m].y, wv[2 * m + 1].x, wv[2 * m + 1].y));
                __stcs(reinterpret_cast<float2 *>(w + cidx + 6 * fs), wv[6]);
              }
              float *wp = w + cidx, *qp = qout + cidx;
#pragma unroll
              for (int f = 0; f < NF; ++f, wp += fs, qp += fs) {
                if constexpr (SUB < 2 && !WP) __stcs(reinterpret_cast<float2 *>(wp), wv[f]);
                __stcs(reinterpret_cast<float2 *>(qp), qn[f]);
              }
            } else if (act1 && shift_images) {
              if constexpr (SUB < 2 && WP) {
                float *wb = w + 2 * cidx;
#pragma unroll
                for (int m = 0; m < 3; ++m)
                  __stcs(reinterpret_cast<float4 *>(wb + 2 * m * fs),
                         make_float4(wv[2 * m].x, wv[2 * m].y, wv[2 * m + 1].x, wv[2 * m + 1].y));
                __stcs(reinterpret_cast<float2 *>(w + cidx + 6 * fs), wv[6]);
              }
              float *wp = w + cidx, *qp = qout + cidx;
#pragma unroll
              for (int f = 0; f < NF; ++f, wp += fs, qp += fs) {
                if constexpr (SUB < 2 && !WP) __stcs(reinterpret_cast<float2 *>(wp), wv[f]);
                __stcs(reinterpret_cast<float2 *>(qp), qn[f]);
              }
              {
                // images: the y / z shifts of the pair, then the x images per point
                const long long dy = !yedge ? 0 : (y < RAD ? (long long)ny * px : -(long long)ny * px);
                const long long dz = !(zper && zn) ? 0 : (z < RAD ? (long long)nz * wplane : -(long long)nz * wplane);
                auto put2 = [&](long long o) {
                  float *p = qout + o;
#pragma unroll
                  for (int f = 0; f < NF; ++f, p += fs) __stcs(reinterpret_cast<float2 *>(p), qn[f]);
                };
                auto put1 = [&](long long o, int e) {
                  float *p = qout + o;
#pragma unroll
                  for (int f = 0; f < NF; ++f, p += fs) __stcs(p, e == 0 ? qn[f].x : qn[f].y);
                };
                if (dy != 0) put2(cidx + dy);
                if (dz != 0) put2(cidx + dz);
                if (dy != 0 && dz != 0) put2(cidx + dy + dz);
#pragma unroll
                for (int e = 0; e < 2; ++e)
                  if (e == 0 ? xn0 : xn1) {
                    const int xe = x + e;
                    const long long b = cidx + e + (xe < RAD ? nx : -nx);
                    put1(b, e);
                    if (dy != 0) put1(b + dy, e);
                    if (dz != 0) put1(b + dz, e);
                    if (dy != 0 && dz != 0) put1(b + dy + dz, e);
                  }
              }
            } else {
              float q0[NF], q1[NF];
#pragma unroll
              for (int f = 0; f < NF; ++f) {
                q0[f] = qn[f].x;
                q1[f] = qn[f].y;
                if constexpr (SUB < 2) {
                  // field f of padded point i: interleaved array f / 2 (WP, f < 6) or field f
                  auto wi = [&](long long i) {
                    return WP && f < 6 ? (long long)(f >> 1) * 2 * fs + 4 * (i >> 1) + 2 * (f & 1) + (i & 1)
                                        : f * fs + i;
                  };
                  __stcs(w + wi(cidx), wv[f].x);
                  if (act1) __stcs(w + wi(cidx + 1), wv[f].y);
                }
              }
              store_with_images<float, true>(qout, fs, cidx, q0, near0, x, y, z, nx, ny, nz, px, py, zper);
              if (act1)
                store_with_images<float, true>(qout, fs, cidx + 1, q1, near1, x + 1, y, z, nx, ny, nz, px, py, zper);
            }
          }

        }
      }
      if (outp) {
        cidx += wplane;
        if (forcing) {
          mz += kz;
          if (mz >= nzg) mz -= nzg;
          if constexpr (WS) ez_next = rz[mz];
        }
      }
      if (++slot == NS) {
        slot = 0;
        phase ^= 1u;
      }
      if constexpr (WS) {
        // release the stage of plane p - 3 after its last use; a wait that
        // gave up stops every compute warp of the CTA at its next plane
        if (p >= RAD) {
          int rs = slot - 1 - RAD;  // slot was advanced past plane p just above
          if (rs < 0) rs += NS;
          __syncwarp();
          if (tx == 0) mbar_arrive(&bars[NS + rs]);
        }
        if (!ok) {
          ws_abort = 1;
          atomicOr(&R.clock->status, 2);
        }
        if (*(volatile int *)&ws_abort) {
          failed = true;
          break;
        }
      } else if constexpr (BAR == 1) {
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
    }
    if constexpr (WS) {
      if (!failed) {
        // the last three planes of the tile had no later plane to release them
        for (int q = npl - RAD; q < npl; ++q) {
          __syncwarp();
          if (tx == 0) mbar_arrive(&bars[NS + (int)((G + q) % NS)]);
        }
      }
    }
    if (!failed) G += npl;
  }

  if (!WS && failed && tid == 0) {
    // record the time-out, then wait (bounded) for the copies still in flight
    atomicOr(&runs[fail_run].clock->status, 2);
    for (int p = fail_p; p < issued_hi; ++p) {
      const unsigned long long g = G + p;
      mbar_wait(&bars[(int)(g % NS)], (uint32_t)((g / NS) & 1ull));
    }
  }
}


// Tile rows of a paired-point variant (0 if `tile` is not one).
int x2_rows(int tile) {
#define X(ID, TY, NS, BR, WS, WP) \
  if (tile == ID) return TY;
  MHD_X2_VARIANTS(X)
#undef X
  return 0;
}

// 1 if the variant keeps w's fields 0-5 in the interleaved layout (WP), 0
// otherwise.
int x2_w_pairs(int tile) {
#define X(ID, TY, NS, BR, WS, WP) \
  if (tile == ID) return WP;
  MHD_X2_VARIANTS(X)
#undef X
  return 0;
}

int x2_prepare(int tile) {
  int e = (int)cudaErrorInvalidValue;
#define X(ID, TY, NS, BR, WS, WP)                                                             \
  if (tile == ID) {                                                                           \
    const int sm = x2_smem_bytes<TY, NS, WS>();                                               \
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;                  \
    e = (int)cudaFuncSetAttribute(k_substep_x2<TY, NS, BR, true, 0, WS, WP>, a, sm);          \
    if (!e) e = (int)cudaFuncSetAttribute(k_substep_x2<TY, NS, BR, true, 1, WS, WP>, a, sm);  \
    if (!e) e = (int)cudaFuncSetAttribute(k_substep_x2<TY, NS, BR, true, 2, WS, WP>, a, sm);  \
    if (!e) e = (int)cudaFuncSetAttribute(k_substep_x2<TY, NS, BR, false, 0, WS, WP>, a, sm); \
    if (!e) e = (int)cudaFuncSetAttribute(k_substep_x2<TY, NS, BR, false, 1, WS, WP>, a, sm); \
    if (!e) e = (int)cudaFuncSetAttribute(k_substep_x2<TY, NS, BR, false, 2, WS, WP>, a, sm); \
  }
  MHD_X2_VARIANTS(X)
#undef X
  return e;
}

int x2_occupancy(int tile, int *bps) {
#define X(ID, TY, NS, BR, WS, WP)                                                                             \
  if (tile == ID)                                                                                             \
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_substep_x2<TY, NS, BR, true, 1, WS, WP>, \
                                                              32 * TY + (WS ? 128 : 0),                       \
                                                              x2_smem_bytes<TY, NS, WS>());
  MHD_X2_VARIANTS(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

namespace {
template <int TY, int NS, int BR, bool ISO, bool WS, bool WP>
void x2_go(const RunDesc *runs, const Tile *tiles, int ntiles, int substep, int grid, cudaStream_t s) {
  const dim3 block(32, TY + (WS ? 4 : 0));
  const int sm = x2_smem_bytes<TY, NS, WS>();
  if (substep == 0)
    k_substep_x2<TY, NS, BR, ISO, 0, WS, WP><<<grid, block, sm, s>>>(runs, tiles, ntiles);
  else if (substep == 1)
    k_substep_x2<TY, NS, BR, ISO, 1, WS, WP><<<grid, block, sm, s>>>(runs, tiles, ntiles);
  else
    k_substep_x2<TY, NS, BR, ISO, 2, WS, WP><<<grid, block, sm, s>>>(runs, tiles, ntiles);
}
}  // namespace

int x2_launch(int tile, const RunDesc *runs, const Tile *tiles, int ntiles, int substep, int grid, int iso,
              cudaStream_t s) {
  if (grid <= 0 || grid > ntiles) grid = ntiles;
  if (grid == 0) return 0;
  if (substep < 0 || substep > 2) return (int)cudaErrorInvalidValue;
#define X(ID, TY, NS, BR, WS, WP)                                              \
  if (tile == ID) {                                                            \
    if (iso)                                                                   \
      x2_go<TY, NS, BR, true, WS, WP>(runs, tiles, ntiles, substep, grid, s);  \
    else                                                                       \
      x2_go<TY, NS, BR, false, WS, WP>(runs, tiles, ntiles, substep, grid, s); \
    return (int)cudaGetLastError();                                            \
  }
  MHD_X2_VARIANTS(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

}  // namespace mhd
