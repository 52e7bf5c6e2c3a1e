// Host side of the C ABI declared in include/mhd.h: parameter validation,
// device workspace layout, tile tables, step orchestration and batching.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mhd.h"
#include "../../include/mhd_check.h"
#include "../../include/mhd_plan.h"
#include "mhd_internal.h"

using namespace mhd;

namespace {
thread_local std::string g_err;
}  // namespace

void mhd::set_last_error(const char *msg) { g_err = msg; }

namespace {

constexpr size_t ALIGN = 256;
constexpr int TARGET_CTAS = 2 * 2 * 148;  // ~two waves of two CTAs per SM on 148 SMs
constexpr int RESIDENT_CTAS = 2 * 148;     // reduction blocks resident at once (two per SM)
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Byte offsets of every region of a context's device workspace.
struct Layout {
  int px, py, pz;
  long long fstride;
  size_t esz;
  size_t q[2], w, roots[3], kshell, clock, coeffs, partials, counter, diag, scratch, run, tiles, sub_tiles;
  size_t sub_cap;  // entries reserved for the substep work split
  size_t total;
  int nk;
  int tw, th;    // reduction tiles (prologue, diagnostics): block shape and TMA box of rmap
  int stw, sth;  // substep tiles: TMA box of tmap and the work split's columns
  int wpairs;    // w's fields 0-5 in the interleaved layout of x2_w_pairs
  std::vector<Tile> tiles_host;
};

int shell_vectors(double kmin, double kmax, std::vector<int> *out) {
  // Integer wave vectors with kmin <= |k| <= kmax, kx varying slowest.
  const int K = (int)std::floor(kmax);
  int n = 0;
  for (int a = -K; a <= K; ++a)
    for (int b = -K; b <= K; ++b)
      for (int c = -K; c <= K; ++c) {
        const double m = std::sqrt((double)(a * a + b * b + c * c));
        if (m >= kmin && m <= kmax) {
          if (out) {
            out->push_back(a);
            out->push_back(b);
            out->push_back(c);
          }
          ++n;
        }
      }
  return n;
}

int num_sms() {
  int dev = 0, n = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

// Tiles of one run: TX x TY columns, z split into chunks so that the launch
// covers the GPU with a couple of waves; chunks of at least 8 planes keep the
// re-read z-halo (6 planes per chunk) small.  Among the splits into nch0 ..
// 2 nch0 + 2 chunks (nch0 from the target CTA count) the one with the least
// estimated time is taken: whole waves of RESIDENT_CTAS blocks times the
// planes a block reads (chunk + 6), so the last wave is not left mostly idle.
std::vector<Tile> make_tiles(int nx, int ny, int nz, int tw, int th, int target_ctas) {
  const int ntx = (nx + tw - 1) / tw, nty = (ny + th - 1) / th;
  const long long ncol = (long long)ntx * nty;
  const int nch0 = (int)std::max(1LL, (target_ctas + ncol - 1) / ncol);
  auto chunk_of = [&](int nch) { return std::min(nz, std::max(8, (nz + nch - 1) / nch)); };
  int chunk = chunk_of(nch0);
  long long best = -1;
  for (int nch = nch0; nch <= 2 * nch0 + 2; ++nch) {
    const int c = chunk_of(nch);
    const long long tiles = ncol * ((nz + c - 1) / c);
    const long long cost = (tiles + RESIDENT_CTAS - 1) / RESIDENT_CTAS * (c + 2 * RAD);
    if (best < 0 || cost < best) {
      best = cost;
      chunk = c;
    }
  }
  std::vector<Tile> t;
  int slot = 0;
  for (int z0 = 0; z0 < nz; z0 += chunk)
    for (int j = 0; j < nty; ++j)
      for (int i = 0; i < ntx; ++i) t.push_back(Tile{0, i * tw, j * th, z0, std::min(nz, z0 + chunk), slot++});
  return t;
}

// ---- work split of the fused substep over the persistent CTAs --------------
// The substep kernel is persistent (about one CTA per SM) and walks a table
// of (column, z-range) tiles.  Whole columns keep the z-pipeline long (six
// halo planes per tile) and let concurrently running CTAs sweep neighbouring
// columns at the same z (their shared halo rows meet in L2); an equal number
// of tiles per CTA balances the load.  Both at once: every CTA takes q whole
// columns (q full waves), and the remaining columns, laid end to end, are cut
// into equal shares of work, one per CTA.  A column's work per plane is
// weighted by its active fraction (ragged edge tiles do the TMA and lead-plane
// work for the full tile but compute fewer points).  The table is laid out
// round-robin (entry c + G*j = tile j of CTA c), padded with empty tiles.
// The per-plane weights are a cost model fitted to per-tile clock records of
// the FP32 32x12 kernel at 256^3 (interior 4220 cycles per plane, tiles at an
// x face 4650, at a y face 4426, the ragged last row of 4 active rows 3175):
// the points within RAD of a face also store their periodic images, and a
// partly idle tile keeps the TMA and lead-plane work of a full one.  Each CTA
// then receives remainder work up to an equal total load.
constexpr int GMAX = 4 * 148;   // most persistent CTAs of any variant on a B300
constexpr double MIN_SHARE = 6.0;  // smallest remainder share, in weighted planes

struct SubCol {
  int run, x0, y0, nz;
  double w;    // work per plane relative to a full tile
  int zb = 0;  // first interior plane of the column's z-range
};

// Columns of planes zb .. zb + nz - 1 of one run (zb > 0: the inner or outer
// z-range of a slab of a decomposed domain).
//
// The paired-point kernel (64-wide tiles) has its own face weights, fitted
// the same way at 384^3 - 1024^2 x 256 (x face 1.15-1.25 by substep, y face
// 1.02-1.05), and its columns are listed in bands of two tile rows -- x
// across the band, the band's two rows adjacent -- which spreads the x-face
// columns of the whole-column waves more evenly over the CTAs than a plain
// row-major list (512^3: 2.3% shorter substeps with both changes).
void add_columns(std::vector<SubCol> *cols, int run, int nx, int ny, int nz, int tw, int th, int zb = 0) {
  const bool paired = tw == 64;
  const double wx = paired ? 1.18 : 1.10, wy = paired ? 1.03 : 1.05;
  const int band = paired ? 2 * th : th;
  for (int yb = 0; yb < ny; yb += band)
    for (int x0 = 0; x0 < nx; x0 += tw)
      for (int y0 = yb; y0 < std::min(ny, yb + band); y0 += th) {
        const double act = (double)std::min(tw, nx - x0) * std::min(th, ny - y0) / ((double)tw * th);
        const bool xface = x0 < RAD || x0 + tw > nx - RAD, yface = y0 < RAD || y0 + th > ny - RAD;
        double w = act >= 1.0 ? 1.0 : 0.565 + 0.435 * act;
        if (xface) w *= wx;
        if (yface) w *= wy;
        cols->push_back(SubCol{run, x0, y0, nz, w, zb});
      }
}

// (Leaving CTAs idle to run one or two waves of whole columns was faster
// with the barrier-synchronised paired kernel; with the warp-specialised one
// the split below is: 256^3 3% and 384^3 3% shorter steps.)
std::vector<Tile> split_columns(const std::vector<SubCol> &cols, int G, int *grid_out) {
  G = std::max(1, G);
  std::vector<std::vector<Tile>> per(G);
  // whole-column waves over the full columns of the largest length
  int nzmax = 0;
  for (const SubCol &c : cols) nzmax = std::max(nzmax, c.nz);
  std::vector<size_t> full, rest;
  for (size_t i = 0; i < cols.size(); ++i) (cols[i].nz == nzmax ? full : rest).push_back(i);
  const size_t q = full.size() / G;
  std::vector<double> load(G, 0.0);
  for (size_t k = 0; k < q * G; ++k) {
    const SubCol &c = cols[full[k]];
    per[k % G].push_back(Tile{c.run, c.x0, c.y0, c.zb, c.zb + c.nz, 0});
    load[k % G] += c.w * c.nz;
  }
  for (size_t k = q * G; k < full.size(); ++k) rest.push_back(full[k]);
  std::sort(rest.begin(), rest.end());
  // the rest, end to end: CTA g takes a contiguous share budget[g] that
  // tops its load up to the common total (equal shares when q == 0).  (A
  // z-aligned split of the rest -- piece h of every remaining column on the
  // same planes -- measured 1.27x algorithmic DRAM traffic instead of ~1.5x
  // but 4-5% slower steps: it cannot even out the heavier face columns.)
  double R = 0;
  for (size_t i : rest) R += cols[i].w * cols[i].nz;
  const int Gr = rest.empty() ? 0 : (int)std::max(1.0, std::min((double)G, std::floor(R / MIN_SHARE)));
  std::vector<double> budget(Gr, Gr ? R / Gr : 0.0);
  if (q > 0 && Gr == G) {
    double tot = R;
    for (double l : load) tot += l;
    double bsum = 0;
    for (int g = 0; g < G; ++g) bsum += (budget[g] = std::max(0.0, tot / G - load[g]));
    for (int g = 0; g < G; ++g) budget[g] = bsum > 0 ? budget[g] * R / bsum : R / G;
  }
  auto plane_at = [&](double d, const SubCol &c) {
    return (int)std::min<long>(c.nz, std::max<long>(0, std::lround(d / c.w)));
  };
  size_t ci = 0;
  double S = 0;  // weighted start of column rest[ci]
  double a = 0;
  for (int g = 0; g < Gr; ++g) {
    const double b = (g + 1 == Gr) ? R : a + budget[g];
    while (ci < rest.size() && S + cols[rest[ci]].w * cols[rest[ci]].nz <= a) {
      S += cols[rest[ci]].w * cols[rest[ci]].nz;
      ++ci;
    }
    double Sj = S;
    for (size_t cj = ci; cj < rest.size() && Sj < b; ++cj) {
      const SubCol &c = cols[rest[cj]];
      const double W = c.w * c.nz;
      const int z0 = plane_at(std::max(a, Sj) - Sj, c), z1 = plane_at(std::min(b, Sj + W) - Sj, c);
      if (z1 > z0) per[g].push_back(Tile{c.run, c.x0, c.y0, c.zb + z0, c.zb + z1, 0});
      Sj += W;
    }
    a = b;
  }
  const int used = q > 0 ? G : std::max(Gr, 1);
  size_t k = 0;
  for (int g = 0; g < used; ++g) k = std::max(k, per[g].size());
  std::vector<Tile> t((size_t)used * k, Tile{0, 0, 0, 0, 0, 0});
  for (int g = 0; g < used; ++g)
    for (size_t j = 0; j < per[g].size(); ++j) t[g + (size_t)used * j] = per[g][j];
  *grid_out = used;
  return t;
}

int validate(const mhd_params *p, std::string *why) {
  auto bad = [&](const char *m) {
    *why = m;
    return MHD_EINVAL;
  };
  if (!p) return bad("params is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return bad("nx, ny, nz must be >= 1");
  if (p->nx > 4096 || p->ny > 4096 || p->nz > 4096) return bad("nx, ny, nz must be <= 4096");
  if (!(p->lx > 0 && p->ly > 0 && p->lz > 0)) return bad("box sizes must be > 0");
  if (!(p->cs > 0)) return bad("cs must be > 0");
  if (!(p->nu >= 0 && p->eta >= 0)) return bad("nu and eta must be >= 0");
  if (!(p->f0 >= 0)) return bad("f0 must be >= 0");
  if (p->f0 > 0) {
    if (!(p->kmin > 0 && p->kmax >= p->kmin)) return bad("forcing shell needs 0 < kmin <= kmax");
    if (p->kmax > 64) return bad("kmax must be <= 64");
    if (shell_vectors(p->kmin, p->kmax, nullptr) == 0) return bad("forcing shell holds no integer wave vector");
    if (!(p->sigma >= 0 && p->sigma <= 1)) return bad("sigma must be in [0, 1]");
  }
  if (!(p->dt_fixed >= 0)) return bad("dt_fixed must be >= 0");
  if (p->dt_fixed == 0 && !(p->cfl > 0 && p->cfl_visc > 0)) return bad("cfl and cfl_visc must be > 0");
  if (p->forcing_mode != 0 && p->forcing_mode != 1) return bad("forcing_mode must be 0 or 1");
  if (p->upwind != 0 && p->upwind != 1) return bad("upwind must be 0 or 1");
  if (p->dtype != MHD_F32 && p->dtype != MHD_F64) return bad("dtype must be MHD_F32 or MHD_F64");
  if (p->kernel != MHD_KERNEL_AUTO && p->kernel != MHD_KERNEL_SMEM && p->kernel != MHD_KERNEL_TMA)
    return bad("kernel must be MHD_KERNEL_AUTO, MHD_KERNEL_SMEM or MHD_KERNEL_TMA");
  if (p->kernel == MHD_KERNEL_SMEM && p->tile != 0) return bad("the plane-ring kernel has one tile (tile = 0)");
  if (p->tile < 0 || p->tile > tma_num_tiles(p->dtype)) return bad("tile id out of range");
  return MHD_OK;
}

// AUTO resolves to the TMA kernel; tile 0 to the fastest variant measured on
// B300: FP32 grids take the warp-specialised paired-point kernel with 6
// stages of q and 3 of w, both copied by its producer warpgroup, and w kept
// in interleaved field pairs (tile 28; 512^3: 1.05e10 cell-updates/s against
// 1.02e10 with w field by field (tile 26), 8.66e9 for the barrier-synchronised
// paired tile 18 and 7.6e9 for the 32 x 12 scalar kernel; 256^3 - 1024^3
// 1.5-8.6% faster than tile 26), FP64 the 32 x 8 scalar tile with 6 stages.
mhd_params resolved(const mhd_params *p) {
  mhd_params r = *p;
  if (r.kernel == MHD_KERNEL_AUTO) r.kernel = MHD_KERNEL_TMA;
  if (r.kernel == MHD_KERNEL_TMA && r.tile == 0) r.tile = r.dtype == MHD_F32 ? 28 : 3;
  return r;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  return fn;
}

// 4-D map of one state buffer: (x: px, y: py, z: pz, field: 7), box = one
// z-plane of a (tw+8) x (th+6) tile of all seven fields.
// Padded 4-D field array (x, y, z, field) with a box of bx x by points of one
// z-plane, all fields.
int encode_box_map(CUtensorMap *m, void *base, size_t esz, int px, int py, int pz, int bx, int by,
                   std::string *why);

// The substep / reduction tile of tw x th points with its halo (4 points
// left and right so that rows stay 16-byte aligned, RAD above and below).
int encode_state_map(CUtensorMap *m, void *base, size_t esz, int px, int py, int pz, int tw, int th,
                     std::string *why) {
  return encode_box_map(m, base, esz, px, py, pz, tw + 8, th + 2 * RAD, why);
}

// 4-D array (x: dx values, y: py, z: pz, then nf arrays fs values apart),
// rows dx values apart; box bx x by x 1 x nf.
int encode_map4(CUtensorMap *m, void *base, size_t esz, long long dx, int py, int pz, int nf, long long fs,
                int bx, int by, std::string *why) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    *why = "cuTensorMapEncodeTiled is not available from the driver";
    return MHD_ECUDA;
  }
  const cuuint64_t dims[4] = {(cuuint64_t)dx, (cuuint64_t)py, (cuuint64_t)pz, (cuuint64_t)nf};
  const cuuint64_t strides[3] = {(cuuint64_t)dx * esz, (cuuint64_t)dx * py * esz, (cuuint64_t)fs * esz};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1u, (cuuint32_t)nf};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  CUresult r = fn(m, esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, base,
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *why = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
    return MHD_ECUDA;
  }
  return MHD_OK;
}

int encode_box_map(CUtensorMap *m, void *base, size_t esz, int px, int py, int pz, int bx, int by,
                   std::string *why) {
  return encode_map4(m, base, esz, px, py, pz, NF, (long long)px * py * pz, bx, by, why);
}

// The w maps of the interleaved layout: fields 0-5 as three arrays (2 px
// values per row, 2 fstride apart; box 2 tw x th), and field 6 (box tw x th).
int encode_w_pair_maps(RunDesc *R, const Layout &L, std::string *why) {
  char *w = static_cast<char *>(R->w);
  if (int e = encode_map4(&R->wpmap[0], w, L.esz, 2LL * L.px, L.py, L.pz, 3, 2 * L.fstride, 2 * L.stw, L.sth,
                          why))
    return e;
  return encode_map4(&R->wpmap[1], w + (size_t)6 * L.fstride * L.esz, L.esz, L.px, L.py, L.pz, 1, L.fstride,
                     L.stw, L.sth, why);
}

Layout make_layout(const mhd_params *p_in) {
  const mhd_params rp = resolved(p_in);
  const mhd_params *p = &rp;
  Layout L;
  L.esz = p->dtype == MHD_F32 ? 4 : 8;
  L.px = (int)align_up((size_t)p->nx + OX + RAD, 8);
  L.py = p->ny + 2 * RAD;
  L.pz = p->nz + 2 * RAD;
  L.fstride = (long long)L.px * L.py * L.pz;
  L.nk = p->f0 > 0 ? shell_vectors(p->kmin, p->kmax, nullptr) : 0;
  substep_tile_shape(p->dtype, p->kernel, p->tile, &L.stw, &L.sth);
  L.wpairs = p->dtype == MHD_F32 && p->kernel == MHD_KERNEL_TMA && x2_w_pairs(p->tile);
  reduction_tile_shape(p->dtype, p->kernel, p->tile, &L.tw, &L.th);
  // The tile table is a function of the parameters alone (not of the device
  // it runs on), so per-tile reduction partials -- and hence every reduced
  // value -- come out in the same order on every GPU and in every batch.
  L.tiles_host = make_tiles(p->nx, p->ny, p->nz, L.tw, L.th, TARGET_CTAS);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes, ALIGN);
    return at;
  };
  const size_t field_set = (size_t)NF * L.fstride * L.esz;
  L.q[0] = take(field_set);
  L.q[1] = take(field_set);
  L.w = take(field_set);
  const int n[3] = {p->nx, p->ny, p->nz};
  for (int a = 0; a < 3; ++a) L.roots[a] = take((size_t)n[a] * 2 * L.esz);
  L.kshell = take(sizeof(int) * 3 * std::max(L.nk, 1));
  L.clock = take(sizeof(Clock));
  L.coeffs = take(sizeof(StepCoeffs));
  L.partials = take(sizeof(double) * NPART * L.tiles_host.size());
  L.counter = take(sizeof(unsigned int) * 4);
  L.diag = take(sizeof(double) * NDIAG);
  L.scratch = take(sizeof(double) * 16);
  L.run = take(sizeof(RunDesc));
  L.tiles = take(sizeof(Tile) * L.tiles_host.size());
  const size_t ncols = (size_t)((p->nx + L.stw - 1) / L.stw) * ((p->ny + L.sth - 1) / L.sth);
  L.sub_cap = ncols + 3 * (size_t)GMAX;
  L.sub_tiles = take(sizeof(Tile) * L.sub_cap);
  L.total = o;
  return L;
}

}  // namespace

namespace mhd {
// padding canaries (kernels.cu)
int launch_padding_check(int dtype, const void *q, int nf, long long fstride, int nx, int px, int py, int pz,
                         unsigned long long *bad, cudaStream_t s);
}  // namespace mhd

struct mhd_ctx {
  mhd_params p;
  cudaStream_t stream;
  Layout L;
  char *ws;
  bool owns_ws;
  RunDesc h_run;
  RunDesc *d_run;
  Tile *d_tiles;
  int ntiles;
  int grid;  // substep launch grid (persistent CTAs)
  Tile *d_sub;  // substep work split (split_columns) and its grid
  int nsub, sub_grid;
  int iso;   // equal grid spacings on all axes
  std::string err;
  cufftHandle fft = 0;  // spectrum plan, made by the first mhd_spectrum call
  bool fft_made = false;
};

struct mhd_batch {
  std::vector<mhd_ctx *> runs;
  cudaStream_t stream;
  int dtype, kernel, tile, tw, th;
  RunDesc *d_runs;
  Tile *d_tiles;
  int ntiles, grid, iso;
  Tile *d_sub;  // substep work split over all runs' columns
  int nsub, sub_grid;
  cudaGraphExec_t exec;
  int graph_steps;
};

namespace {

int fail(mhd_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  g_err = buf;
  return code;
}

int cuda_fail(mhd_ctx *ctx, int e, const char *what) {
  return fail(ctx, MHD_ECUDA, "%s: %s", what, cudaGetErrorString((cudaError_t)e));
}

#define CK(ctx, call)                                            \
  do {                                                           \
    int e__ = (int)(call);                                       \
    if (e__ != 0) return cuda_fail((ctx), e__, #call);           \
  } while (0)

int read_clock(mhd_ctx *ctx, Clock *c) {
  CK(ctx, cudaMemcpyAsync(c, ctx->h_run.clock, sizeof(Clock), cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return MHD_OK;
}

int check_status(mhd_ctx *ctx, const Clock &c) {
  if (c.status & 2)
    return fail(ctx, MHD_ETIMEOUT, "a bounded wait for a TMA plane copy gave up by step %lld", c.step);
  if (c.status & 1)
    return fail(ctx, MHD_ENONFINITE, "non-finite time step at step %lld (run blew up)", c.step);
  return MHD_OK;
}

int enqueue_step(cudaStream_t s, int dtype, int kernel, int tile, int tw, int th,
                 const RunDesc *runs, const Tile *tiles, int ntiles, const Tile *sub_tiles, int nsub,
                 int sub_grid, int iso) {
  int e = launch_prologue(dtype, kernel, tile, runs, tiles, ntiles, tw, th, s);
  for (int sub = 0; sub < 3 && e == 0; ++sub)
    e = launch_substep(dtype, kernel, tile, runs, sub_tiles, nsub, sub, sub_grid, iso, s);
  return e;
}

size_t host_esz(int host_dtype) { return host_dtype == MHD_F32 ? 4 : 8; }

// Host <-> device transfer of the interior of the 7 fields of one state
// buffer (dev: its first field) of ctx.  Host field f starts at host + f *
// hfield bytes and holds nz planes of nx * ny values (x fastest), nx, ny, nz
// those of ctx.  Same precision: one strided 3-D copy per field; otherwise a
// dense copy through staging (the RK register, dead between steps) and a
// converting kernel.  Asynchronous on the context's stream.
int upload_fields(mhd_ctx *ctx, const char *host, size_t hfield, int host_dtype, char *dev) {
  const RunDesc &R = ctx->h_run;
  const size_t esz = ctx->L.esz, hb = (size_t)R.nx * R.ny * R.nz * host_esz(host_dtype);
  cudaStream_t s = ctx->stream;
  for (int f = 0; f < NF; ++f) {
    char *field = dev + (size_t)f * R.fstride * esz;
    const char *src = host + f * hfield;
    if (host_dtype == ctx->p.dtype) {
      cudaMemcpy3DParms c3 = {};
      c3.srcPtr = make_cudaPitchedPtr(const_cast<char *>(src), (size_t)R.nx * esz, R.nx, R.ny);
      c3.dstPtr = make_cudaPitchedPtr(field, (size_t)R.px * esz, R.px, R.py);
      c3.dstPos = make_cudaPos((size_t)OX * esz, OY, OZ);
      c3.extent = make_cudaExtent((size_t)R.nx * esz, R.ny, R.nz);
      c3.kind = cudaMemcpyHostToDevice;
      CK(ctx, cudaMemcpy3DAsync(&c3, s));
    } else {
      CK(ctx, cudaMemcpyAsync(R.w, src, hb, cudaMemcpyHostToDevice, s));
      CK(ctx, launch_set_field(ctx->p.dtype, host_dtype, R.w, field, R.nx, R.ny, R.nz, R.px, R.py, s));
    }
  }
  return MHD_OK;
}

int download_fields(mhd_ctx *ctx, const char *dev, int host_dtype, char *host, size_t hfield) {
  const RunDesc &R = ctx->h_run;
  const size_t esz = ctx->L.esz, hb = (size_t)R.nx * R.ny * R.nz * host_esz(host_dtype);
  cudaStream_t s = ctx->stream;
  for (int f = 0; f < NF; ++f) {
    const char *field = dev + (size_t)f * R.fstride * esz;
    char *out = host + f * hfield;
    if (host_dtype == ctx->p.dtype) {
      cudaMemcpy3DParms c3 = {};
      c3.srcPtr = make_cudaPitchedPtr(const_cast<char *>(field), (size_t)R.px * esz, R.px, R.py);
      c3.srcPos = make_cudaPos((size_t)OX * esz, OY, OZ);
      c3.dstPtr = make_cudaPitchedPtr(out, (size_t)R.nx * esz, R.nx, R.ny);
      c3.extent = make_cudaExtent((size_t)R.nx * esz, R.ny, R.nz);
      c3.kind = cudaMemcpyDeviceToHost;
      CK(ctx, cudaMemcpy3DAsync(&c3, s));
    } else {
      CK(ctx, launch_get_field(ctx->p.dtype, host_dtype, field, R.w, R.nx, R.ny, R.nz, R.px, R.py, 0, s));
      CK(ctx, cudaMemcpyAsync(out, R.w, hb, cudaMemcpyDeviceToHost, s));
    }
  }
  return MHD_OK;
}

}  // namespace

extern "C" {

void mhd_default_params(mhd_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nx = p->ny = p->nz = 32;
  p->lx = p->ly = p->lz = 2.0 * M_PI;
  p->cs = 1.0;
  p->nu = p->eta = 5e-3;
  p->f0 = 0.0;
  p->kmin = 2.5;
  p->kmax = 3.5;
  p->sigma = 0.0;
  p->seed = 1;
  p->cfl = 0.4;
  p->cfl_visc = 0.08;
  p->dt_fixed = 0.0;
  p->forcing_mode = 0;
  p->upwind = 0;
  p->dtype = MHD_F32;
  p->kernel = MHD_KERNEL_AUTO;
  p->tile = 0;
}

int mhd_resolve_params(const mhd_params *p, mhd_params *out) {
  std::string why;
  if (validate(p, &why)) return fail(nullptr, MHD_EINVAL, "%s", why.c_str());
  if (!out) return fail(nullptr, MHD_EINVAL, "out is NULL");
  *out = resolved(p);
  return MHD_OK;
}

int mhd_workspace_bytes(const mhd_params *p, size_t *bytes) {
  std::string why;
  if (validate(p, &why)) return fail(nullptr, MHD_EINVAL, "%s", why.c_str());
  if (!bytes) return fail(nullptr, MHD_EINVAL, "bytes is NULL");
  *bytes = make_layout(p).total;
  return MHD_OK;
}

int mhd_create(const mhd_params *p, void *stream, void *workspace, size_t workspace_bytes,
               mhd_ctx **out) {
  std::string why;
  if (!out) return fail(nullptr, MHD_EINVAL, "out is NULL");
  *out = nullptr;
  if (validate(p, &why)) return fail(nullptr, MHD_EINVAL, "%s", why.c_str());
  mhd_ctx *ctx = new mhd_ctx();
  ctx->p = resolved(p);
  p = &ctx->p;
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->L = make_layout(p);
  const Layout &L = ctx->L;
  if (workspace) {
    if (workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) % ALIGN) != 0) {
      delete ctx;
      return fail(nullptr, MHD_ENOMEM, "workspace must be >= %zu bytes and 256-byte aligned", L.total);
    }
    ctx->ws = static_cast<char *>(workspace);
    ctx->owns_ws = false;
  } else {
    cudaError_t e = cudaMalloc(&ctx->ws, L.total);
    if (e != cudaSuccess) {
      delete ctx;
      return fail(nullptr, MHD_ENOMEM, "cudaMalloc(%zu): %s", L.total, cudaGetErrorString(e));
    }
    ctx->owns_ws = true;
  }
  auto cleanup = [&](int code) {
    if (ctx->owns_ws) cudaFree(ctx->ws);
    g_err = ctx->err;
    delete ctx;
    return code;
  };
  char *ws = ctx->ws;
  RunDesc &R = ctx->h_run;
  std::memset(&R, 0, sizeof(R));
  R.nx = p->nx;
  R.ny = p->ny;
  R.nz = p->nz;
  R.nzg = p->nz;  // a whole grid: no z-slab decomposition
  R.z_off = 0;
  R.z_open = 0;
  R.px = L.px;
  R.py = L.py;
  R.pz = L.pz;
  R.fstride = L.fstride;
  R.q[0] = ws + L.q[0];
  R.q[1] = ws + L.q[1];
  R.w = ws + L.w;
  for (int a = 0; a < 3; ++a) R.roots[a] = ws + L.roots[a];
  R.kshell = reinterpret_cast<const int *>(ws + L.kshell);
  R.nk = L.nk;
  R.forcing_mode = p->forcing_mode;
  R.upwind = p->upwind;
  R.clock = reinterpret_cast<Clock *>(ws + L.clock);
  R.coeffs = reinterpret_cast<StepCoeffs *>(ws + L.coeffs);
  R.partials = reinterpret_cast<double *>(ws + L.partials);
  R.counter = reinterpret_cast<unsigned int *>(ws + L.counter);
  R.diag = reinterpret_cast<double *>(ws + L.diag);
  R.cs = p->cs;
  R.cs2 = p->cs * p->cs;
  R.nu = p->nu;
  R.eta = p->eta;
  R.f0 = p->f0;
  R.sigma = p->sigma;
  const double Lb[3] = {p->lx, p->ly, p->lz};
  const int n[3] = {p->nx, p->ny, p->nz};
  R.dmin = 1e300;
  for (int a = 0; a < 3; ++a) {
    const double h = Lb[a] / n[a];
    R.inv_h[a] = 1.0 / h;
    R.kscale[a] = 2.0 * M_PI / Lb[a];
    R.dmin = std::min(R.dmin, h);
  }
  ctx->iso = R.inv_h[0] == R.inv_h[1] && R.inv_h[1] == R.inv_h[2];
  R.cfl = p->cfl;
  R.cfl_visc = p->cfl_visc;
  R.dt_fixed = p->dt_fixed;
  R.seed = p->seed;
  R.ntiles = (int)L.tiles_host.size();
  ctx->ntiles = R.ntiles;
  if (p->kernel == MHD_KERNEL_TMA) {
    std::string why;
    for (int b = 0; b < 2; ++b)
      if (encode_state_map(&R.tmap[b], R.q[b], L.esz, L.px, L.py, L.pz, L.stw, L.sth, &why) ||
          encode_state_map(&R.rmap[b], R.q[b], L.esz, L.px, L.py, L.pz, L.tw, L.th, &why) ||
          (b == 0 && encode_box_map(&R.wmap, R.w, L.esz, L.px, L.py, L.pz, L.stw, L.sth, &why)) ||
          (b == 0 && L.wpairs && encode_w_pair_maps(&R, L, &why))) {
        fail(ctx, MHD_ECUDA, "%s", why.c_str());
        return cleanup(MHD_ECUDA);
      }
  }
  ctx->d_run = reinterpret_cast<RunDesc *>(ws + L.run);
  ctx->d_tiles = reinterpret_cast<Tile *>(ws + L.tiles);
  int bps = 1;
  if (substep_max_grid(p->dtype, p->kernel, p->tile, &bps) != 0 || bps < 1) bps = 1;
  ctx->grid = std::min(ctx->ntiles, bps * num_sms());
  std::vector<SubCol> cols;
  add_columns(&cols, 0, p->nx, p->ny, p->nz, L.stw, L.sth);
  int sub_grid = 1;
  std::vector<Tile> sub_tiles = split_columns(cols, std::min(bps * num_sms(), GMAX), &sub_grid);
  if (sub_tiles.size() <= L.sub_cap) {
    ctx->d_sub = reinterpret_cast<Tile *>(ws + L.sub_tiles);
    ctx->nsub = (int)sub_tiles.size();
    ctx->sub_grid = sub_grid;
  } else {  // cannot happen for columns of one run; keep the reduction tiles
    sub_tiles.clear();
    ctx->d_sub = ctx->d_tiles;
    ctx->nsub = ctx->ntiles;
    ctx->sub_grid = ctx->grid;
  }

  // host tables: roots of unity (FP64 cos/sin, rounded to the working
  // precision), shell list, tiles
  std::vector<char> roots[3];
  for (int a = 0; a < 3; ++a) {
    roots[a].resize((size_t)n[a] * 2 * L.esz);
    for (int m = 0; m < n[a]; ++m) {
      const double ang = 2.0 * M_PI * (double)m / n[a];
      const double c = std::cos(ang), s = std::sin(ang);
      if (L.esz == 4) {
        float *r = reinterpret_cast<float *>(roots[a].data());
        r[2 * m] = (float)c;
        r[2 * m + 1] = (float)s;
      } else {
        double *r = reinterpret_cast<double *>(roots[a].data());
        r[2 * m] = c;
        r[2 * m + 1] = s;
      }
    }
  }
  std::vector<int> shell;
  if (L.nk) shell_vectors(p->kmin, p->kmax, &shell);
  cudaStream_t s = ctx->stream;
  int e = prepare_substep(p->dtype, p->kernel, p->tile);
  if (!e) e = (int)cudaMemsetAsync(ws, 0, L.total, s);
  // state buffers and RK register: all NaN (0xFF bytes), then the zero state at
  // the interior and ghost points of q[0]; the alignment padding keeps its NaN
  // canaries (mhd_padding_check)
  if (!e) e = (int)cudaMemsetAsync(ws + L.q[0], 0xFF, L.w + (size_t)NF * L.fstride * L.esz - L.q[0], s);
  if (!e)
    e = launch_seed_field(p->dtype, ws + L.q[0] + (size_t)4 * L.fstride * L.esz, L.fstride, p->nx, p->ny, p->nz,
                          L.px, L.py, 0ull, 0.0, s);
  if (!e) e = launch_halo(p->dtype, ws + L.q[0], NF, L.fstride, p->nx, p->ny, p->nz, L.px, L.py, s);
  for (int a = 0; a < 3 && !e; ++a)
    e = (int)cudaMemcpyAsync(ws + L.roots[a], roots[a].data(), roots[a].size(), cudaMemcpyHostToDevice, s);
  if (!e && L.nk)
    e = (int)cudaMemcpyAsync(ws + L.kshell, shell.data(), shell.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  if (!e) e = (int)cudaMemcpyAsync(ctx->d_run, &R, sizeof(R), cudaMemcpyHostToDevice, s);
  if (!e)
    e = (int)cudaMemcpyAsync(ctx->d_tiles, L.tiles_host.data(), sizeof(Tile) * L.tiles_host.size(),
                             cudaMemcpyHostToDevice, s);
  if (!e && !sub_tiles.empty())
    e = (int)cudaMemcpyAsync(ctx->d_sub, sub_tiles.data(), sizeof(Tile) * sub_tiles.size(),
                             cudaMemcpyHostToDevice, s);
  if (!e) e = (int)cudaStreamSynchronize(s);
  if (e) {
    cuda_fail(ctx, e, "mhd_create upload");
    return cleanup(MHD_ECUDA);
  }
  *out = ctx;
  return MHD_OK;
}

void mhd_destroy(mhd_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->fft_made) cufftDestroy(ctx->fft);
  if (ctx->owns_ws) cudaFree(ctx->ws);
  delete ctx;
}

int mhd_set_state(mhd_ctx *ctx, const void *host_soa, int host_dtype, double t, int64_t step) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (!host_soa) return fail(ctx, MHD_EINVAL, "host_soa is NULL");
  if (host_dtype != MHD_F32 && host_dtype != MHD_F64) return fail(ctx, MHD_EINVAL, "bad host_dtype");
  if (step < 0) return fail(ctx, MHD_EINVAL, "step must be >= 0");
  const RunDesc &R = ctx->h_run;
  const size_t hb = (size_t)R.nx * R.ny * R.nz * host_esz(host_dtype);
  char *dst = static_cast<char *>(R.q[step & 1]);
  cudaStream_t s = ctx->stream;
  int rc = upload_fields(ctx, static_cast<const char *>(host_soa), hb, host_dtype, dst);
  if (rc) return rc;
  CK(ctx, launch_halo(ctx->p.dtype, dst, NF, R.fstride, R.nx, R.ny, R.nz, R.px, R.py, s));
  Clock c;
  std::memset(&c, 0, sizeof c);
  c.t = t;
  c.step = step;
  CK(ctx, cudaMemcpyAsync(R.clock, &c, sizeof c, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaStreamSynchronize(s));
  return MHD_OK;
}

int mhd_set_seed_field(mhd_ctx *ctx, uint64_t seed, double amp) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (!(amp >= 0.0) || !std::isfinite(amp)) return fail(ctx, MHD_EINVAL, "amp must be finite and >= 0");
  const RunDesc &R = ctx->h_run;
  char *dst = static_cast<char *>(R.q[0]);
  cudaStream_t s = ctx->stream;
  CK(ctx, launch_seed_field(ctx->p.dtype, dst + (size_t)4 * R.fstride * ctx->L.esz, R.fstride, R.nx, R.ny,
                            R.nz, R.px, R.py, seed, amp, s));
  CK(ctx, launch_halo(ctx->p.dtype, dst, NF, R.fstride, R.nx, R.ny, R.nz, R.px, R.py, s));
  Clock c;
  std::memset(&c, 0, sizeof c);
  CK(ctx, cudaMemcpyAsync(R.clock, &c, sizeof c, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaStreamSynchronize(s));
  return MHD_OK;
}

int mhd_get_state(mhd_ctx *ctx, void *host_soa, int host_dtype, double *t, int64_t *step) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (host_dtype != MHD_F32 && host_dtype != MHD_F64) return fail(ctx, MHD_EINVAL, "bad host_dtype");
  Clock c;
  int rc = read_clock(ctx, &c);
  if (rc) return rc;
  if (host_soa) {
    const RunDesc &R = ctx->h_run;
    const size_t hb = (size_t)R.nx * R.ny * R.nz * host_esz(host_dtype);
    rc = download_fields(ctx, static_cast<const char *>(R.q[c.step & 1]), host_dtype,
                         static_cast<char *>(host_soa), hb);
    if (rc) return rc;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (t) *t = c.t;
  if (step) *step = c.step;
  return check_status(ctx, c);
}

int mhd_step(mhd_ctx *ctx, int nsteps) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (nsteps < 0) return fail(ctx, MHD_EINVAL, "nsteps must be >= 0");
  for (int i = 0; i < nsteps; ++i) {
    int e = enqueue_step(ctx->stream, ctx->p.dtype, ctx->p.kernel, ctx->p.tile, ctx->L.tw, ctx->L.th,
                         ctx->d_run, ctx->d_tiles, ctx->ntiles, ctx->d_sub, ctx->nsub, ctx->sub_grid,
                         ctx->iso);
    if (e) return cuda_fail(ctx, e, "mhd_step launch");
  }
  return MHD_OK;
}

int mhd_step_timed(mhd_ctx *ctx, int nsteps, double *stage_ms, double *total_ms) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (nsteps < 0) return fail(ctx, MHD_EINVAL, "nsteps must be >= 0");
  if (!stage_ms || !total_ms) return fail(ctx, MHD_EINVAL, "stage_ms and total_ms must be non-NULL");
  if (nsteps == 0) return MHD_OK;
  std::vector<cudaEvent_t> ev((size_t)4 * nsteps + 1, nullptr);
  int rc = MHD_OK;
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      rc = fail(ctx, MHD_ECUDA, "cudaEventCreate failed");
      break;
    }
  cudaStream_t s = ctx->stream;
  for (int i = 0; i < nsteps && rc == MHD_OK; ++i) {
    int e = (int)cudaEventRecord(ev[4 * i], s);
    if (!e)
      e = launch_prologue(ctx->p.dtype, ctx->p.kernel, ctx->p.tile, ctx->d_run, ctx->d_tiles, ctx->ntiles,
                          ctx->L.tw, ctx->L.th, s);
    for (int sub = 0; sub < 3 && !e; ++sub) {
      e = (int)cudaEventRecord(ev[4 * i + 1 + sub], s);
      if (!e) e = launch_substep(ctx->p.dtype, ctx->p.kernel, ctx->p.tile, ctx->d_run, ctx->d_sub,
                                 ctx->nsub, sub, ctx->sub_grid, ctx->iso, s);
    }
    if (e) rc = cuda_fail(ctx, e, "mhd_step_timed launch");
  }
  if (rc == MHD_OK) {
    int e = (int)cudaEventRecord(ev[4 * nsteps], s);
    if (!e) e = (int)cudaEventSynchronize(ev[4 * nsteps]);
    if (e) rc = cuda_fail(ctx, e, "mhd_step_timed sync");
  }
  if (rc == MHD_OK) {
    for (int i = 0; i < nsteps; ++i)
      for (int st = 0; st < 4; ++st) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[4 * i + st], ev[4 * i + st + 1]);
        stage_ms[st] += ms;
      }
    float tot = 0.f;
    cudaEventElapsedTime(&tot, ev[0], ev[4 * nsteps]);
    *total_ms += tot;
  }
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  return rc;
}

int mhd_diagnostics(mhd_ctx *ctx, double *out) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (!out) return fail(ctx, MHD_EINVAL, "out is NULL");
  CK(ctx, launch_diagnostics(ctx->p.dtype, ctx->d_run, ctx->h_run, ctx->d_tiles, ctx->ntiles,
                             ctx->L.tw, ctx->L.th, ctx->stream));
  CK(ctx, cudaMemcpyAsync(out, ctx->h_run.diag, sizeof(double) * NDIAG, cudaMemcpyDeviceToHost,
                          ctx->stream));
  Clock c;
  int rc = read_clock(ctx, &c);
  if (rc) return rc;
  return check_status(ctx, c);
}

int mhd_reduce(mhd_ctx *ctx, int kind, double *out) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (kind < 0 || kind >= MHD_NREDUCE) return fail(ctx, MHD_EINVAL, "unknown reduction kind %d", kind);
  if (!out) return fail(ctx, MHD_EINVAL, "out is NULL");
  if (kind == MHD_BRMS) {  // one fused pass: no stored B, no halo, no other sums
    // TMA runs: the prologue sweep in B_rms mode, which also caches the CFL
    // maximum of this state, so the next step's prologue sweeps nothing
    if (ctx->p.kernel == MHD_KERNEL_TMA)
      CK(ctx, tma_launch_prologue(ctx->p.dtype, ctx->p.tile, ctx->d_run, ctx->d_tiles, ctx->ntiles, ctx->stream, 1));
    else
      CK(ctx, launch_brms(ctx->p.dtype, ctx->d_run, ctx->d_tiles, ctx->ntiles, ctx->L.tw, ctx->L.th, ctx->stream));
    CK(ctx, cudaMemcpyAsync(out, ctx->h_run.diag + 1, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    Clock c;
    int rc = read_clock(ctx, &c);
    if (rc) return rc;
    return check_status(ctx, c);
  }
  double all[MHD_NREDUCE];
  int rc = mhd_diagnostics(ctx, all);
  if (rc) return rc;
  *out = all[kind];
  return MHD_OK;
}

int mhd_time(mhd_ctx *ctx, double *t, double *dt_last, int64_t *step) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  Clock c;
  int rc = read_clock(ctx, &c);
  if (rc) return rc;
  if (t) *t = c.t;
  if (dt_last) *dt_last = c.dt_last;
  if (step) *step = c.step;
  return check_status(ctx, c);
}

int mhd_sync(mhd_ctx *ctx) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  Clock c;
  int rc = read_clock(ctx, &c);
  if (rc) return rc;
  return check_status(ctx, c);
}

int mhd_forcing_draw(mhd_ctx *ctx, int64_t step, double *out) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (!out) return fail(ctx, MHD_EINVAL, "out is NULL");
  if (ctx->h_run.nk == 0) return fail(ctx, MHD_EINVAL, "run has no forcing (f0 = 0)");
  if (step < 0) return fail(ctx, MHD_EINVAL, "step must be >= 0");
  double *scratch = reinterpret_cast<double *>(ctx->ws + ctx->L.scratch);
  CK(ctx, launch_forcing_draw(ctx->d_run, step, scratch, ctx->stream));
  CK(ctx, cudaMemcpyAsync(out, scratch, sizeof(double) * 13, cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return MHD_OK;
}

int mhd_padding_check(mhd_ctx *ctx, long long *bad) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (!bad) return fail(ctx, MHD_EINVAL, "bad is NULL");
  const RunDesc &R = ctx->h_run;
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(ctx->ws + ctx->L.scratch);
  cudaStream_t s = ctx->stream;
  CK(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  for (int b = 0; b < 2; ++b)
    CK(ctx, launch_padding_check(ctx->p.dtype, R.q[b], NF, R.fstride, R.nx, R.px, R.py, R.pz, cnt, s));
  unsigned long long h = 0;
  CK(ctx, cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  *bad = (long long)h;
  return MHD_OK;
}

int mhd_wait_selftest(void *stream, double *seconds, double *kernel_bound_seconds) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int *d = nullptr;
  int h = -1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0xFF, sizeof(int), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  double scale = 0.0;
  if (e == cudaSuccess) e = (cudaError_t)launch_wait_selftest(d, s, &scale);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return fail(nullptr, MHD_ECUDA, "mhd_wait_selftest: %s", cudaGetErrorString(e));
  if (seconds) *seconds = ms * 1e-3;
  if (kernel_bound_seconds) *kernel_bound_seconds = ms * 1e-3 * scale;
  if (h == 2) return fail(nullptr, MHD_ETIMEOUT, "the bounded wait gave up after %.3f s (expected)", ms * 1e-3);
  return MHD_OK;
}

int mhd_substep_plan(const mhd_params *p, int grid_ctas, int *tiles, int max_tiles, int *ntiles, int *grid) {
  std::string why;
  if (validate(p, &why)) return fail(nullptr, MHD_EINVAL, "%s", why.c_str());
  if (grid_ctas < 1 || !ntiles || !grid) return fail(nullptr, MHD_EINVAL, "grid_ctas < 1 or NULL output");
  const Layout L = make_layout(p);
  std::vector<SubCol> cols;
  add_columns(&cols, 0, p->nx, p->ny, p->nz, L.stw, L.sth);
  const std::vector<Tile> t = split_columns(cols, std::min(grid_ctas, GMAX), grid);
  *ntiles = (int)t.size();
  for (size_t i = 0; tiles && i < t.size() && (int)i < max_tiles; ++i) {
    tiles[5 * i + 0] = t[i].x0;
    tiles[5 * i + 1] = t[i].y0;
    tiles[5 * i + 2] = t[i].z0;
    tiles[5 * i + 3] = t[i].z1;
    tiles[5 * i + 4] = t[i].run;
  }
  return MHD_OK;
}

int mhd_spectrum_shells(const mhd_params *p, int *nshells) {
  std::string why;
  if (validate(p, &why)) return fail(nullptr, MHD_EINVAL, "%s", why.c_str());
  if (!nshells) return fail(nullptr, MHD_EINVAL, "nshells is NULL");
  if (p->lx != p->ly || p->lx != p->lz) return fail(nullptr, MHD_EINVAL, "spectra need a cubic box (lx = ly = lz)");
  if (p->nx < 2) return fail(nullptr, MHD_EINVAL, "spectra need nx >= 2");
  *nshells = spectrum_nshells(p->nx, p->ny, p->nz);
  return MHD_OK;
}

int mhd_spectrum(mhd_ctx *ctx, double *host_out, int max_shells, int *nshells) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (!host_out || max_shells < 0) return fail(ctx, MHD_EINVAL, "host_out is NULL or max_shells < 0");
  const mhd_params &p = ctx->p;
  if (p.lx != p.ly || p.lx != p.lz) return fail(ctx, MHD_EINVAL, "spectra need a cubic box (lx = ly = lz)");
  if (p.nx < 2) return fail(ctx, MHD_EINVAL, "spectra need nx >= 2");
  const RunDesc &R = ctx->h_run;
  const int ns = spectrum_nshells(R.nx, R.ny, R.nz);
  if (nshells) *nshells = ns;
  // scratch: the RK register w, dead between steps (alpha_1 = 0): fields
  // 0..2 hold B, 3..5 the half spectrum, 6 the shell sums
  const long long nh = R.nx / 2 + 1, nrows = (long long)R.ny * R.nz, odist = nrows * nh;
  const size_t esz = ctx->L.esz, fbytes = (size_t)R.fstride * esz;
  char *w = static_cast<char *>(R.w);
  void *bh = w + 3 * fbytes;
  char *scratch = w + 6 * fbytes;
  if ((size_t)(3 * odist) * 2 * esz > 3 * fbytes || spectrum_scratch_bytes(R.nx, R.ny, R.nz) > fbytes)
    return fail(ctx, MHD_ENOMEM, "spectrum scratch does not fit the RK register");
  const size_t rows_bytes = ((size_t)(nrows * nh * 8) + 15) / 16 * 16;
  double *shells = reinterpret_cast<double *>(scratch + rows_bytes + ((size_t)nrows * 8 + 15) / 16 * 16);
  if (!ctx->fft_made) {
    if (cufftCreate(&ctx->fft) != CUFFT_SUCCESS) return fail(ctx, MHD_ECUDA, "cufftCreate failed");
    // axes of one point are left out of the transform (x, the halved
    // axis, always stays); inembed gives each kept axis' stride in units of
    // the next inner kept axis
    long long n[3], inembed[3], onembed[3];
    int rank = 0;
    if (R.nz > 1) {
      n[rank] = R.nz;
      inembed[rank] = R.pz;
      onembed[rank++] = R.nz;
    }
    if (R.ny > 1) {
      n[rank] = R.ny;
      inembed[rank] = R.py;
      onembed[rank++] = R.ny;
    } else if (rank == 1) {
      inembed[0] = R.pz;  // ignored by cuFFT for the outermost axis
    }
    n[rank] = R.nx;
    inembed[rank] = (R.ny > 1 || rank == 0) ? R.px : (long long)R.py * R.px;
    onembed[rank++] = nh;
    size_t work = 0;
    const cufftResult r = cufftMakePlanMany64(ctx->fft, rank, n, inembed, 1, R.fstride, onembed, 1, odist,
                                              p.dtype == MHD_F32 ? CUFFT_R2C : CUFFT_D2Z, 3, &work);
    if (r != CUFFT_SUCCESS) {
      cufftDestroy(ctx->fft);
      return fail(ctx, MHD_ECUDA, "cuFFT plan failed (cufftResult %d)", (int)r);
    }
    ctx->fft_made = true;
  }
  if (cufftSetStream(ctx->fft, ctx->stream) != CUFFT_SUCCESS) return fail(ctx, MHD_ECUDA, "cufftSetStream failed");
  CK(ctx, launch_curl(p.dtype, ctx->d_run, ctx->d_tiles, ctx->ntiles, ctx->L.tw, ctx->L.th, ctx->stream));
  const size_t in_off = ((size_t)OZ * R.py + OY) * R.px + OX;  // first interior point (elements)
  const cufftResult r = p.dtype == MHD_F32
      ? cufftExecR2C(ctx->fft, reinterpret_cast<cufftReal *>(R.w) + in_off, static_cast<cufftComplex *>(bh))
      : cufftExecD2Z(ctx->fft, reinterpret_cast<cufftDoubleReal *>(R.w) + in_off,
                     static_cast<cufftDoubleComplex *>(bh));
  if (r != CUFFT_SUCCESS) return fail(ctx, MHD_ECUDA, "cuFFT transform failed (cufftResult %d)", (int)r);
  CK(ctx, launch_spectrum_bins(p.dtype, bh, odist, R.nx, R.ny, R.nz, scratch, shells, ctx->stream));
  const int ncopy = std::min(ns, max_shells);
  if (ncopy > 0)
    CK(ctx, cudaMemcpyAsync(host_out, shells, sizeof(double) * ncopy, cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return MHD_OK;
}

int mhd_eval_rhs(mhd_ctx *ctx, int64_t step, double dt_forcing, void *host_rhs, int host_dtype) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (!host_rhs) return fail(ctx, MHD_EINVAL, "host_rhs is NULL");
  if (host_dtype != MHD_F32 && host_dtype != MHD_F64) return fail(ctx, MHD_EINVAL, "bad host_dtype");
  if (step < 0) return fail(ctx, MHD_EINVAL, "step must be >= 0");
  Clock c;
  int rc = read_clock(ctx, &c);
  if (rc) return rc;
  const RunDesc &R = ctx->h_run;
  const int par = (int)(c.step & 1);
  cudaStream_t s = ctx->stream;
  // substep 0 with dt = 1 leaves w = RHS; the other state buffer is
  // overwritten (it is dead between steps) and serves as staging.
  CK(ctx, launch_coeffs(ctx->p.dtype, ctx->d_run, step, 1.0, dt_forcing, par, s));
  CK(ctx, launch_substep(ctx->p.dtype, ctx->p.kernel, ctx->p.tile, ctx->d_run, ctx->d_sub,
                         ctx->nsub, 0, ctx->sub_grid, ctx->iso, s));
  const size_t npts = (size_t)R.nx * R.ny * R.nz, hb = npts * host_esz(host_dtype);
  void *staging = R.q[par ^ 1];
  const bool pairs = ctx->L.wpairs;
  for (int f = 0; f < NF; ++f) {
    // field f of w: interleaved array f / 2 from its value 2 (f % 2) on, or field f
    const bool pf = pairs && f < 6;
    const size_t at = pf ? (size_t)(f >> 1) * 2 * R.fstride + 2 * (f & 1) : (size_t)f * R.fstride;
    CK(ctx, launch_get_field(ctx->p.dtype, host_dtype, static_cast<const char *>(R.w) + at * ctx->L.esz,
                             staging, R.nx, R.ny, R.nz, R.px, R.py, pf ? 1 : 0, s));
    CK(ctx, cudaMemcpyAsync(static_cast<char *>(host_rhs) + f * hb, staging, hb,
                            cudaMemcpyDeviceToHost, s));
  }
  // the staging buffer held the other parity's state, which is dead between
  // steps (the next substep rewrites its interior and ghost zones): refill it
  // with NaN so the padding canaries hold again.  The step constants were
  // overwritten too; the next prologue rewrites them.
  CK(ctx, cudaMemsetAsync(staging, 0xFF, (size_t)NF * R.fstride * ctx->L.esz, s));
  CK(ctx, cudaStreamSynchronize(s));
  return MHD_OK;
}

int mhd_eval_rhs_at(mhd_ctx *ctx, int64_t step, double dt_forcing, int npts, const int *ijk, double *host_out) {
  if (!ctx) return fail(nullptr, MHD_EINVAL, "ctx is NULL");
  if (!ijk || !host_out) return fail(ctx, MHD_EINVAL, "ijk and host_out must be non-NULL");
  if (npts < 1 || npts > MHD_EVAL_AT_MAX_POINTS)
    return fail(ctx, MHD_EINVAL, "npts must be in [1, %d]", (int)MHD_EVAL_AT_MAX_POINTS);
  if (step < 0) return fail(ctx, MHD_EINVAL, "step must be >= 0");
  const RunDesc &R = ctx->h_run;
  for (int n = 0; n < npts; ++n)
    if (ijk[3 * n] < 0 || ijk[3 * n] >= R.nx || ijk[3 * n + 1] < 0 || ijk[3 * n + 1] >= R.ny ||
        ijk[3 * n + 2] < 0 || ijk[3 * n + 2] >= R.nz)
      return fail(ctx, MHD_EINVAL, "point %d (%d, %d, %d) is outside the grid", n, ijk[3 * n], ijk[3 * n + 1],
                  ijk[3 * n + 2]);
  Clock c;
  int rc = read_clock(ctx, &c);
  if (rc) return rc;
  const int par = (int)(c.step & 1);
  cudaStream_t s = ctx->stream;
  // as mhd_eval_rhs: substep 0 with dt = 1 leaves w = RHS; the dead state
  // buffer holds the point list and the gathered values, then is re-poisoned
  char *staging = static_cast<char *>(R.q[par ^ 1]);
  const size_t ijk_bytes = align_up((size_t)3 * npts * sizeof(int), ALIGN);
  if (ijk_bytes + (size_t)NF * npts * sizeof(double) > (size_t)NF * R.fstride * ctx->L.esz)
    return fail(ctx, MHD_EINVAL, "%d points do not fit this grid's staging buffer", npts);
  CK(ctx, launch_coeffs(ctx->p.dtype, ctx->d_run, step, 1.0, dt_forcing, par, s));
  CK(ctx, launch_substep(ctx->p.dtype, ctx->p.kernel, ctx->p.tile, ctx->d_run, ctx->d_sub,
                         ctx->nsub, 0, ctx->sub_grid, ctx->iso, s));
  int *d_ijk = reinterpret_cast<int *>(staging);
  double *d_out = reinterpret_cast<double *>(staging + ijk_bytes);
  CK(ctx, cudaMemcpyAsync(d_ijk, ijk, (size_t)3 * npts * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(ctx, launch_gather_points(ctx->p.dtype, R.w, R.fstride, R.px, R.py, d_ijk, npts, d_out, ctx->L.wpairs, s));
  CK(ctx, cudaMemcpyAsync(host_out, d_out, (size_t)NF * npts * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaMemsetAsync(staging, 0xFF, (size_t)NF * R.fstride * ctx->L.esz, s));
  CK(ctx, cudaStreamSynchronize(s));
  return MHD_OK;
}

const char *mhd_last_error(const mhd_ctx *ctx) {
  if (ctx) return ctx->err.c_str();
  return g_err.c_str();
}

// ---- batches ----------------------------------------------------------------

int mhd_batch_create(mhd_ctx *const *runs, int nruns, mhd_batch **out) {
  if (!out) return fail(nullptr, MHD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!runs || nruns < 1) return fail(nullptr, MHD_EINVAL, "need at least one run");
  mhd_ctx *r0 = runs[0];
  if (!r0) return fail(nullptr, MHD_EINVAL, "runs[0] is NULL");
  std::vector<RunDesc> descs;
  std::vector<Tile> tiles;
  double cells_total = 0;
  for (int i = 0; i < nruns; ++i) {
    mhd_ctx *r = runs[i];
    if (!r) return fail(nullptr, MHD_EINVAL, "runs[%d] is NULL", i);
    if (r->p.dtype != r0->p.dtype || r->stream != r0->stream || r->p.kernel != r0->p.kernel ||
        r->p.tile != r0->p.tile)
      return fail(nullptr, MHD_EINVAL,
                  "runs of a batch must share dtype, stream, kernel and tile");
    for (int j = 0; j < i; ++j)
      if (runs[j] == r) return fail(nullptr, MHD_EINVAL, "run %d appears twice", i);
    cells_total += (double)r->p.nx * r->p.ny * r->p.nz;
  }
  // The batch has its own tile table: each run gets a share of about two
  // waves of CTAs in proportion to its size (small runs get whole columns,
  // so few z-halo planes are re-read).  Substep results are pointwise and
  // the dt reduction is a maximum, so the tiling changes no run's result;
  // diagnostics keep using each run's own tiles.
  for (int i = 0; i < nruns; ++i) {
    mhd_ctx *r = runs[i];
    const double share = (double)r->p.nx * r->p.ny * r->p.nz / cells_total;
    const int target = std::max(1, (int)std::lround(TARGET_CTAS * share));
    std::vector<Tile> rt = make_tiles(r->p.nx, r->p.ny, r->p.nz, r->L.tw, r->L.th, target);
    if (rt.size() > r->L.tiles_host.size()) rt = r->L.tiles_host;  // partial slots are sized for these
    RunDesc d = r->h_run;
    d.ntiles = (int)rt.size();
    descs.push_back(d);
    for (Tile t : rt) {
      t.run = i;
      tiles.push_back(t);
    }
  }
  mhd_batch *b = new mhd_batch();
  b->runs.assign(runs, runs + nruns);
  b->iso = 1;
  for (int i = 0; i < nruns; ++i) b->iso &= runs[i]->iso;
  b->stream = r0->stream;
  b->dtype = r0->p.dtype;
  b->kernel = r0->p.kernel;
  b->tile = r0->p.tile;
  b->tw = r0->L.tw;
  b->th = r0->L.th;
  b->ntiles = (int)tiles.size();
  b->exec = nullptr;
  b->graph_steps = 0;
  int bps = 1;
  if (substep_max_grid(b->dtype, b->kernel, b->tile, &bps) != 0 || bps < 1) bps = 1;
  b->grid = std::min(b->ntiles, bps * num_sms());
  std::vector<SubCol> cols;
  for (int i = 0; i < nruns; ++i)
    add_columns(&cols, i, runs[i]->p.nx, runs[i]->p.ny, runs[i]->p.nz, runs[i]->L.stw, runs[i]->L.sth);
  std::vector<Tile> sub_tiles = split_columns(cols, std::min(bps * num_sms(), GMAX), &b->sub_grid);
  b->nsub = (int)sub_tiles.size();
  b->d_runs = nullptr;
  b->d_tiles = nullptr;
  b->d_sub = nullptr;
  cudaError_t e = cudaMalloc(&b->d_runs, sizeof(RunDesc) * descs.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, sizeof(Tile) * tiles.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_sub, sizeof(Tile) * sub_tiles.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_sub, sub_tiles.data(), sizeof(Tile) * sub_tiles.size(), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_runs, descs.data(), sizeof(RunDesc) * descs.size(), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    cudaFree(b->d_runs);
    cudaFree(b->d_tiles);
    cudaFree(b->d_sub);
    delete b;
    return fail(nullptr, MHD_ECUDA, "mhd_batch_create: %s", cudaGetErrorString(e));
  }
  *out = b;
  return MHD_OK;
}

int mhd_batch_step(mhd_batch *b, int nsteps) {
  if (!b) return fail(nullptr, MHD_EINVAL, "batch is NULL");
  if (nsteps < 0) return fail(nullptr, MHD_EINVAL, "nsteps must be >= 0");
  cudaStream_t s = b->stream;
  // Steps are captured once into a graph of graph_steps steps and replayed;
  // a remainder is launched directly.  The device clocks advance on replay,
  // so the same graph serves every later call.
  if (!b->exec && nsteps >= 2 && s != nullptr) {
    const int g = std::min(nsteps, 16);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    int le = 0;
    for (int i = 0; i < g && e == cudaSuccess && !le; ++i)
      le = enqueue_step(s, b->dtype, b->kernel, b->tile, b->tw, b->th, b->d_runs, b->d_tiles,
                        b->ntiles, b->d_sub, b->nsub, b->sub_grid, b->iso);
    cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess && !le && e2 == cudaSuccess) {
      if (cudaGraphInstantiate(&b->exec, graph, 0) == cudaSuccess) b->graph_steps = g;
      else b->exec = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
  }
  int done = 0;
  if (b->exec) {
    for (; done + b->graph_steps <= nsteps; done += b->graph_steps) {
      cudaError_t e = cudaGraphLaunch(b->exec, s);
      if (e != cudaSuccess) return fail(nullptr, MHD_ECUDA, "graph launch: %s", cudaGetErrorString(e));
    }
  }
  for (; done < nsteps; ++done) {
    int e = enqueue_step(s, b->dtype, b->kernel, b->tile, b->tw, b->th, b->d_runs, b->d_tiles,
                         b->ntiles, b->d_sub, b->nsub, b->sub_grid, b->iso);
    if (e) return fail(nullptr, MHD_ECUDA, "batch step launch: %s", cudaGetErrorString((cudaError_t)e));
  }
  return MHD_OK;
}

void mhd_batch_destroy(mhd_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->d_runs);
  cudaFree(b->d_tiles);
  cudaFree(b->d_sub);
  delete b;
}

}  // extern "C"

// ---- z-slab domain decomposition (Sec. 3.3, 3.4) ----------------------------
// Each slab is a context of its own (own workspace, TMA maps and tiles) whose
// run descriptor is patched: the grid spacing, forcing wave-vector scale and
// z roots of unity of the whole grid, its global plane offset, open z faces
// (no periodic z images), and one clock, one set of step constants, one
// partial-sum array and one set of counters shared by all slabs, so that a
// single prologue launch over every slab's tiles reduces the CFL maximum of
// the whole grid, sets one dt and draws one forcing for all slabs.
struct mhd_slabs {
  mhd_params p;  // the whole grid (resolved kernel and tile)
  int n = 0, overlap = 0;
  std::vector<mhd_ctx *> s;
  std::vector<int> z0, nzs;
  cudaStream_t stream = nullptr, side = nullptr;
  cudaEvent_t ev_outer = nullptr, ev_copied = nullptr;
  char *shared = nullptr;    // clock, coefficients, partials, counters, diagnostics, z roots
  Clock *clock = nullptr;
  double *diag = nullptr;
  RunDesc *d_runs = nullptr;  // slab k's patched descriptor at index k
  Tile *d_tab = nullptr;      // all tile tables below, back to back
  int nred = 0;               // reduction tiles of all slabs (slots numbered across slabs)
  int nall = 0, grid_all = 1, nouter = 0, grid_outer = 1, ninner = 0, grid_inner = 1;
  size_t off_all = 0, off_outer = 0, off_inner = 0;
  long long step = 0;  // host copy of the step index: which state buffer is current
  int iso = 1;
};

namespace {

int slabs_fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define SCK(call)                                                                               \
  do {                                                                                          \
    cudaError_t e__ = (cudaError_t)(call);                                                      \
    if (e__ != cudaSuccess) return slabs_fail(MHD_ECUDA, "%s: %s", #call, cudaGetErrorString(e__)); \
  } while (0)

// Halo exchange along z of state buffer `buf` (use_w: the RK register) over
// its first nf fields: slab k's top three interior planes go to the bottom
// ghost planes of slab k+1, and slab k+1's bottom three interior planes to
// the top ghost planes of slab k (periodic in k).  A plane is px * py values
// including its x/y ghost columns; the nf fields of a slab are fstride apart,
// so each face and direction is one 2-D copy of nf rows.
int slab_exchange(mhd_slabs *S, bool use_w, int buf, int nf, cudaStream_t st) {
  for (int k = 0; k < S->n; ++k) {
    mhd_ctx *lo = S->s[k], *hi = S->s[(k + 1) % S->n];
    const RunDesc &A = lo->h_run, &B = hi->h_run;
    const size_t esz = lo->L.esz, plane = (size_t)A.px * A.py * esz;
    char *a = static_cast<char *>(use_w ? A.w : A.q[buf]);
    char *b = static_cast<char *>(use_w ? B.w : B.q[buf]);
    const size_t pa = (size_t)A.fstride * esz, pb = (size_t)B.fstride * esz;
    // up: interior planes nz-3 .. nz-1 of lo (padded nz .. nz+2) -> ghost planes 0 .. 2 of hi
    SCK(cudaMemcpy2DAsync(b, pb, a + (size_t)A.nz * plane, pa, 3 * plane, nf, cudaMemcpyDeviceToDevice, st));
    // down: interior planes 0 .. 2 of hi (padded 3 .. 5) -> ghost planes nz+3 .. nz+5 of lo
    SCK(cudaMemcpy2DAsync(a + (size_t)(A.nz + OZ) * plane, pa, b + (size_t)OZ * plane, pb, 3 * plane, nf,
                          cudaMemcpyDeviceToDevice, st));
  }
  return MHD_OK;
}

int slab_prologue(mhd_slabs *S) {
  const mhd_params &p = S->p;
  const Layout &L = S->s[0]->L;
  return launch_prologue(p.dtype, p.kernel, p.tile, S->d_runs, S->d_tab, S->nred, L.tw, L.th, S->stream);
}

int slab_substep(mhd_slabs *S, size_t off, int ntab, int grid, int sub, cudaStream_t st) {
  if (ntab <= 0) return 0;
  return launch_substep(S->p.dtype, S->p.kernel, S->p.tile, S->d_runs, S->d_tab + off, ntab, sub, grid, S->iso,
                        st);
}

}  // namespace

extern "C" {

void mhd_slabs_destroy(mhd_slabs *S) {
  if (!S) return;
  if (S->stream || S->s.size()) cudaStreamSynchronize(S->stream);
  if (S->side) {
    cudaStreamSynchronize(S->side);
    cudaStreamDestroy(S->side);
  }
  if (S->ev_outer) cudaEventDestroy(S->ev_outer);
  if (S->ev_copied) cudaEventDestroy(S->ev_copied);
  for (mhd_ctx *c : S->s) mhd_destroy(c);
  cudaFree(S->shared);
  cudaFree(S->d_runs);
  cudaFree(S->d_tab);
  delete S;
}

int mhd_slabs_create(const mhd_params *p_in, int nslabs, int overlap, void *stream, mhd_slabs **out) {
  std::string why;
  if (!out) return slabs_fail(MHD_EINVAL, "out is NULL");
  *out = nullptr;
  if (validate(p_in, &why)) return slabs_fail(MHD_EINVAL, "%s", why.c_str());
  const mhd_params p = resolved(p_in);
  if (p.kernel != MHD_KERNEL_TMA) return slabs_fail(MHD_EINVAL, "slabs need the TMA kernel");
  if (nslabs < 1) return slabs_fail(MHD_EINVAL, "nslabs must be >= 1");
  if (p.nz < 3 * nslabs) return slabs_fail(MHD_EINVAL, "%d planes cannot give %d slabs of at least 3", p.nz, nslabs);
  mhd_slabs *S = new mhd_slabs();
  S->p = p;
  S->n = nslabs;
  S->overlap = overlap != 0;
  S->stream = static_cast<cudaStream_t>(stream);
  auto bail = [&](int code) {
    const std::string msg = g_err;
    mhd_slabs_destroy(S);
    g_err = msg;
    return code;
  };
  // slab extents and contexts
  int z = 0;
  for (int k = 0; k < nslabs; ++k) {
    const int nzk = p.nz / nslabs + (k < p.nz % nslabs ? 1 : 0);
    S->z0.push_back(z);
    S->nzs.push_back(nzk);
    z += nzk;
    mhd_params sp = p;
    sp.nz = nzk;
    sp.lz = p.lz * nzk / p.nz;  // spacing and wave vectors are patched to the whole grid's below
    mhd_ctx *c = nullptr;
    const int rc = mhd_create(&sp, stream, nullptr, 0, &c);
    if (rc) return bail(rc);
    S->s.push_back(c);
  }
  const size_t esz = S->s[0]->L.esz;
  int ntot = 0;
  for (mhd_ctx *c : S->s) ntot += c->ntiles;
  S->nred = ntot;
  // shared region: clock, step constants, partials of all slabs' tiles,
  // counters, diagnostics, z roots of unity of the whole grid
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, ALIGN);
    return at;
  };
  const size_t o_clock = take(sizeof(Clock)), o_coeffs = take(sizeof(StepCoeffs)),
               o_part = take(sizeof(double) * NPART * ntot), o_cnt = take(sizeof(unsigned int) * 4),
               o_diag = take(sizeof(double) * NDIAG), o_roots = take((size_t)p.nz * 2 * esz);
  if (cudaMalloc(&S->shared, o) != cudaSuccess) return bail(slabs_fail(MHD_ENOMEM, "cudaMalloc of %zu bytes", o));
  S->clock = reinterpret_cast<Clock *>(S->shared + o_clock);
  S->diag = reinterpret_cast<double *>(S->shared + o_diag);
  // whole-grid spacing, wave-vector scale and minimum spacing, formed as
  // mhd_create forms them for an undecomposed run
  const double Lb[3] = {p.lx, p.ly, p.lz};
  const int ng[3] = {p.nx, p.ny, p.nz};
  double inv_h[3], kscale[3], dmin = 1e300;
  for (int a = 0; a < 3; ++a) {
    const double h = Lb[a] / ng[a];
    inv_h[a] = 1.0 / h;
    kscale[a] = 2.0 * M_PI / Lb[a];
    dmin = std::min(dmin, h);
  }
  S->iso = inv_h[0] == inv_h[1] && inv_h[1] == inv_h[2];
  std::vector<char> roots((size_t)p.nz * 2 * esz);
  for (int m = 0; m < p.nz; ++m) {
    const double ang = 2.0 * M_PI * (double)m / p.nz, c = std::cos(ang), s = std::sin(ang);
    if (esz == 4) {
      reinterpret_cast<float *>(roots.data())[2 * m] = (float)c;
      reinterpret_cast<float *>(roots.data())[2 * m + 1] = (float)s;
    } else {
      reinterpret_cast<double *>(roots.data())[2 * m] = c;
      reinterpret_cast<double *>(roots.data())[2 * m + 1] = s;
    }
  }
  // patched descriptors and the tile tables over all slabs
  std::vector<RunDesc> descs;
  std::vector<Tile> red, all, outer, inner;
  std::vector<SubCol> c_all, c_outer, c_inner;
  int slot0 = 0;
  for (int k = 0; k < nslabs; ++k) {
    mhd_ctx *c = S->s[k];
    RunDesc &R = c->h_run;
    for (int a = 0; a < 3; ++a) {
      R.inv_h[a] = inv_h[a];
      R.kscale[a] = kscale[a];
    }
    R.dmin = dmin;
    R.roots[2] = S->shared + o_roots;
    R.nzg = p.nz;
    R.z_off = S->z0[k];
    R.z_open = 1;
    R.clock = S->clock;
    R.coeffs = reinterpret_cast<StepCoeffs *>(S->shared + o_coeffs);
    R.partials = reinterpret_cast<double *>(S->shared + o_part);
    R.counter = reinterpret_cast<unsigned int *>(S->shared + o_cnt);
    R.diag = S->diag;
    R.ntiles = ntot;
    c->iso = S->iso;
    descs.push_back(R);
    for (Tile t : c->L.tiles_host) {
      t.run = k;
      t.slot += slot0;
      red.push_back(t);
    }
    slot0 += c->ntiles;
    const int nzk = S->nzs[k];
    add_columns(&c_all, k, p.nx, p.ny, nzk, c->L.stw, c->L.sth);
    if (nzk >= 2 * 2 * RAD) {  // outer: the three planes at each face; inner: the rest
      add_columns(&c_outer, k, p.nx, p.ny, RAD, c->L.stw, c->L.sth, 0);
      add_columns(&c_outer, k, p.nx, p.ny, RAD, c->L.stw, c->L.sth, nzk - RAD);
      add_columns(&c_inner, k, p.nx, p.ny, nzk - 2 * RAD, c->L.stw, c->L.sth, RAD);
    } else {  // too thin to split: all of it is outer
      add_columns(&c_outer, k, p.nx, p.ny, nzk, c->L.stw, c->L.sth, 0);
    }
  }
  int bps = 1;
  if (substep_max_grid(p.dtype, p.kernel, p.tile, &bps) != 0 || bps < 1) bps = 1;
  const int G = std::min(bps * num_sms(), GMAX);
  all = split_columns(c_all, G, &S->grid_all);
  if (!c_outer.empty()) outer = split_columns(c_outer, G, &S->grid_outer);
  if (!c_inner.empty()) inner = split_columns(c_inner, G, &S->grid_inner);
  S->nall = (int)all.size();
  S->nouter = (int)outer.size();
  S->ninner = (int)inner.size();
  std::vector<Tile> tab = red;
  S->off_all = tab.size();
  tab.insert(tab.end(), all.begin(), all.end());
  S->off_outer = tab.size();
  tab.insert(tab.end(), outer.begin(), outer.end());
  S->off_inner = tab.size();
  tab.insert(tab.end(), inner.begin(), inner.end());
  cudaStream_t st = S->stream;
  cudaError_t e = cudaMalloc(&S->d_runs, sizeof(RunDesc) * descs.size());
  if (e == cudaSuccess) e = cudaMalloc(&S->d_tab, sizeof(Tile) * tab.size());
  if (e == cudaSuccess) e = cudaMemsetAsync(S->shared, 0, o, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->shared + o_roots, roots.data(), roots.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->d_runs, descs.data(), sizeof(RunDesc) * descs.size(), cudaMemcpyHostToDevice, st);
  for (int k = 0; k < nslabs && e == cudaSuccess; ++k)  // each slab's own descriptor too
    e = cudaMemcpyAsync(S->s[k]->d_run, &descs[k], sizeof(RunDesc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->d_tab, tab.data(), sizeof(Tile) * tab.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_outer, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_copied, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bail(slabs_fail(MHD_ECUDA, "mhd_slabs_create: %s", cudaGetErrorString(e)));
  // the zero state: fill the z ghost planes from the neighbours
  int rc = slab_exchange(S, false, 0, NF, st);
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = slabs_fail(MHD_ECUDA, "mhd_slabs_create sync");
  if (rc) return bail(rc);
  *out = S;
  return MHD_OK;
}

int mhd_slabs_extent(const mhd_slabs *S, int slab, int *z0, int *nz) {
  if (!S || slab < 0 || slab >= S->n) return slabs_fail(MHD_EINVAL, "no such slab");
  if (z0) *z0 = S->z0[slab];
  if (nz) *nz = S->nzs[slab];
  return MHD_OK;
}

int mhd_slabs_set_state(mhd_slabs *S, const void *host_soa, int host_dtype, double t, int64_t step) {
  if (!S || !host_soa) return slabs_fail(MHD_EINVAL, "slabs and host_soa must be non-NULL");
  if (host_dtype != MHD_F32 && host_dtype != MHD_F64) return slabs_fail(MHD_EINVAL, "bad host_dtype");
  if (step < 0) return slabs_fail(MHD_EINVAL, "step must be >= 0");
  const size_t plane = (size_t)S->p.nx * S->p.ny * host_esz(host_dtype), hfield = plane * S->p.nz;
  const int b = (int)(step & 1);
  for (int k = 0; k < S->n; ++k) {
    mhd_ctx *c = S->s[k];
    const char *src = static_cast<const char *>(host_soa) + (size_t)S->z0[k] * plane;
    int rc = upload_fields(c, src, hfield, host_dtype, static_cast<char *>(c->h_run.q[b]));
    if (rc) return slabs_fail(rc, "%s", c->err.c_str());
    // x/y ghost columns (the z ghost planes it fills by local wrap are
    // replaced by the exchange below)
    SCK(launch_halo(S->p.dtype, c->h_run.q[b], NF, c->h_run.fstride, c->h_run.nx, c->h_run.ny, c->h_run.nz,
                    c->h_run.px, c->h_run.py, S->stream));
  }
  int rc = slab_exchange(S, false, b, NF, S->stream);
  if (rc) return rc;
  Clock c;
  std::memset(&c, 0, sizeof c);
  c.t = t;
  c.step = step;
  SCK(cudaMemcpyAsync(S->clock, &c, sizeof c, cudaMemcpyHostToDevice, S->stream));
  SCK(cudaStreamSynchronize(S->stream));
  S->step = step;
  return MHD_OK;
}

static int slabs_read_clock(mhd_slabs *S, Clock *c) {
  SCK(cudaMemcpyAsync(c, S->clock, sizeof(Clock), cudaMemcpyDeviceToHost, S->stream));
  SCK(cudaStreamSynchronize(S->stream));
  if (c->status & 2) return slabs_fail(MHD_ETIMEOUT, "a bounded wait for a TMA plane copy gave up by step %lld", c->step);
  if (c->status & 1) return slabs_fail(MHD_ENONFINITE, "non-finite time step at step %lld (run blew up)", c->step);
  return MHD_OK;
}

int mhd_slabs_get_state(mhd_slabs *S, void *host_soa, int host_dtype, double *t, int64_t *step) {
  if (!S) return slabs_fail(MHD_EINVAL, "slabs is NULL");
  if (host_dtype != MHD_F32 && host_dtype != MHD_F64) return slabs_fail(MHD_EINVAL, "bad host_dtype");
  Clock c;
  SCK(cudaMemcpyAsync(&c, S->clock, sizeof(Clock), cudaMemcpyDeviceToHost, S->stream));
  SCK(cudaStreamSynchronize(S->stream));
  if (host_soa) {
    const size_t plane = (size_t)S->p.nx * S->p.ny * host_esz(host_dtype), hfield = plane * S->p.nz;
    for (int k = 0; k < S->n; ++k) {
      mhd_ctx *x = S->s[k];
      char *dst = static_cast<char *>(host_soa) + (size_t)S->z0[k] * plane;
      int rc = download_fields(x, static_cast<const char *>(x->h_run.q[c.step & 1]), host_dtype, dst, hfield);
      if (rc) return slabs_fail(rc, "%s", x->err.c_str());
    }
    SCK(cudaStreamSynchronize(S->stream));
  }
  if (t) *t = c.t;
  if (step) *step = c.step;
  return slabs_read_clock(S, &c);
}

int mhd_slabs_step(mhd_slabs *S, int nsteps) {
  if (!S) return slabs_fail(MHD_EINVAL, "slabs is NULL");
  if (nsteps < 0) return slabs_fail(MHD_EINVAL, "nsteps must be >= 0");
  cudaStream_t st = S->stream;
  for (int i = 0; i < nsteps; ++i) {
    SCK(slab_prologue(S));
    for (int sub = 0; sub < 3; ++sub) {
      // substep `sub` of step n writes state buffer (n + sub + 1) mod 2
      const int b = (int)((S->step + sub + 1) & 1);
      if (S->overlap && S->ninner > 0) {
        SCK(slab_substep(S, S->off_outer, S->nouter, S->grid_outer, sub, st));
        SCK(cudaEventRecord(S->ev_outer, st));
        SCK(cudaStreamWaitEvent(S->side, S->ev_outer, 0));
        int rc = slab_exchange(S, false, b, NF, S->side);
        if (rc) return rc;
        SCK(cudaEventRecord(S->ev_copied, S->side));
        SCK(slab_substep(S, S->off_inner, S->ninner, S->grid_inner, sub, st));
        SCK(cudaStreamWaitEvent(st, S->ev_copied, 0));
      } else {
        SCK(slab_substep(S, S->off_all, S->nall, S->grid_all, sub, st));
        int rc = slab_exchange(S, false, b, NF, st);
        if (rc) return rc;
      }
    }
    ++S->step;
  }
  return MHD_OK;
}

int mhd_slabs_diagnostics(mhd_slabs *S, double *out) {
  if (!S || !out) return slabs_fail(MHD_EINVAL, "slabs and out must be non-NULL");
  cudaStream_t st = S->stream;
  const int dt = S->p.dtype;
  for (mhd_ctx *c : S->s) {
    const RunDesc &R = c->h_run;
    SCK(launch_curl(dt, c->d_run, c->d_tiles, c->ntiles, c->L.tw, c->L.th, st));
    SCK(launch_halo(dt, R.w, 3, R.fstride, R.nx, R.ny, R.nz, R.px, R.py, st));
  }
  int rc = slab_exchange(S, true, 0, 3, st);
  if (rc) return rc;
  const Layout &L = S->s[0]->L;
  SCK(launch_diag_pass(dt, S->d_runs, S->d_tab, S->nred, L.tw, L.th, st));
  SCK(cudaMemcpyAsync(out, S->diag, sizeof(double) * NDIAG, cudaMemcpyDeviceToHost, st));
  Clock c;
  return slabs_read_clock(S, &c);
}

}  // extern "C"
