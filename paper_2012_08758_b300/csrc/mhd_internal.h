// Internal structures shared by the host side of the C ABI and the kernels.
// Not part of the public interface (include/mhd.h is).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mhd {

constexpr int NF = 7;            // ln rho, u_x, u_y, u_z, A_x, A_y, A_z
constexpr int RAD = 3;           // stencil radius r of the 6th-order scheme (Sec. 3.1)
constexpr int OX = 4;            // padded x index of interior point 0 (one spare column
                                 // keeps interior rows 16-byte aligned)
constexpr int OY = 3, OZ = 3;    // padded y / z index of interior point 0
constexpr int NDIAG = 9;         // quantities of mhd_diagnostics
constexpr int NPART = 8;         // doubles per reduction tile
constexpr int MAX_TILE_THREADS = 512;  // largest tile (block) of any substep variant

// Device-resident clock of one run: time, last dt and index of the state
// currently held in q[step & 1].  Advanced on the device by the step
// prologue, so a captured sequence of steps can be replayed.
struct Clock {
  double t;
  double dt_last;
  long long step;
  int status;   // bit 0: the time-step reduction saw a non-finite value;
                // bit 1: a bounded wait for a TMA copy gave up
  int pad;
  // The CFL maximum of the state at the start of step cache_tag - 1, taken by
  // a B_rms reduction of that state (the same sweep); 0 = nothing cached.
  // Every write of the state zeroes the clock, and with it the tag.
  long long cache_tag;
  double cache_vmax;
};

// Per-step constants written by the prologue and read by every substep of
// that step: dt and the forcing realisation of Eqs. 4-6 (amplitude already
// folded in: fa = N a, fb = N b).
struct StepCoeffs {
  double dt;
  double fa[3], fb[3];
  double cphi, sphi;   // e^{i phi}
  int kmod[3];         // k mod N per axis, in [0, N)
  int forcing;         // 1: apply the forcing this step
  int parity;          // state of this step lives in q[parity] at substep 0
  int pad;
};

// Everything a kernel needs to know about one run, resident in device memory.
struct RunDesc {
  CUtensorMap tmap[2];      // TMA maps of q[0], q[1]: 4-D (x, y, z, field), box of one z-plane
                            // of a substep tile with its halo
  CUtensorMap rmap[2];      // the same for the reduction tiles (step prologue, B_rms sweep);
                            // equal to tmap unless the substep tile is wider
  CUtensorMap wmap;         // TMA maps of w for the paired variants with a w ring; boxes: the
  CUtensorMap wpmap[2];     // substep tile's interior points of one z-plane.  wmap: all fields;
                            // wpmap (variants with the layout of x2_w_pairs): fields 0-5 as
                            // (2 px, py, pz, array), and field 6
  int nx, ny, nz;
  int px, py, pz;           // padded extents; px is the row pitch
  long long fstride;        // elements per field (px * py * pz)
  void *q[2];               // state buffers, NF fields each
  void *w;                  // RK3-2N register, NF fields
  const void *roots[3];     // e^{2 pi i m / N_a}, m < N_a, working precision
  const int *kshell;        // forcing shell, 3 ints per vector
  int nk;
  int forcing_mode;
  Clock *clock;
  StepCoeffs *coeffs;
  double *partials;         // NPART doubles per reduction tile of this run
  unsigned int *counter;    // last-tile-done counters [0]: dt, [1]: diagnostics
  double *diag;             // NDIAG doubles
  double cs, cs2, nu, eta, f0, sigma;
  double inv_h[3];          // 1 / grid spacing per axis
  double kscale[3];         // 2 pi / L per axis (physical wave vector)
  double cfl, cfl_visc, dt_fixed, dmin;
  unsigned long long seed;
  int ntiles;               // reduction tiles of this run
  int upwind;               // 1: upwind-biased ln rho advection (Sec. 4)
  // z-slab of a decomposed domain (Sec. 3.3): the slab holds global planes
  // z_off .. z_off + nz - 1 of a grid of nzg planes.  z_open = 1: the z ghost
  // planes come from the neighbouring slabs (halo exchange), so no periodic
  // z images are stored.  An undecomposed run has z_off = 0, nzg = nz, z_open = 0.
  int z_off, nzg, z_open;
};

static_assert(alignof(RunDesc) >= 64 && sizeof(RunDesc) % 64 == 0,
              "tensor maps inside RunDesc arrays must stay 64-byte aligned");

// A unit of work: an x-y tile of one run and a range [z0, z1) of interior
// planes.  slot = index of this tile among the run's tiles.
struct Tile {
  int run, x0, y0, z0, z1, slot;
};

// Records msg as the calling thread's last error (mhd_last_error(NULL)).
void set_last_error(const char *msg);

// ---- launchers (kernels.cu / reduce.cu) -------------------------------------
// dtype: 0 = float, 1 = double.  All return a cudaError_t as int.
// Step prologue (max-speed reduction, dt, forcing draw, clock) for runs of
// the given kernel variant (TMA runs use the TMA prologue).
int launch_prologue(int dtype, int kernel, int tile, const RunDesc *runs, const Tile *tiles, int ntiles,
                    int tw, int th, cudaStream_t s);
int launch_prologue_plain(int dtype, const RunDesc *runs, const Tile *tiles, int ntiles, int tw, int th,
                          cudaStream_t s);
// iso != 0: every run of the launch has equal grid spacings on all axes
int launch_substep(int dtype, int kernel, int tile, const RunDesc *runs, const Tile *tiles,
                   int ntiles, int substep, int grid, int iso, cudaStream_t s);
int prepare_substep(int dtype, int kernel, int tile);
// TMA variant (kernels_tma.cu); tile ids start at 1
// Bounded-wait self-test kernel (mhd_wait_selftest): out[0] = 2 on give-up;
// *scale = the kernels' poll bound over the self-test's.
int launch_wait_selftest(int *out, cudaStream_t s, double *scale);
int tma_num_tiles(int dtype);
int tma_tile_shape(int dtype, int tile, int *tx, int *ty);
int tma_prepare(int dtype, int tile);
int tma_occupancy(int dtype, int tile, int *bps);
// mode 0: the step prologue (takes the cached CFL maximum when the clock
// holds one for this step); mode 1: B_rms of the current state into diag[1],
// caching the CFL maximum of the same sweep for the next step's prologue.
int tma_launch_prologue(int dtype, int tile, const RunDesc *runs, const Tile *tiles, int ntiles,
                        cudaStream_t s, int mode = 0);
int tma_launch(int dtype, int tile, const RunDesc *runs, const Tile *tiles, int ntiles, int substep,
               int grid, int iso, cudaStream_t s);
// Paired-point FP32 substep variants (kernels_x2.cu): x2_rows(tile) is the
// tile's row count (0: not such a variant); tiles are 64 points wide.
int x2_rows(int tile);
// 1 if the variant keeps w's fields 0-5 as three interleaved arrays (field
// 2m + c of padded point i at w[2 m fstride + 4 (i / 2) + 2 c + i % 2]), 0
// otherwise
int x2_w_pairs(int tile);
int x2_prepare(int tile);
int x2_occupancy(int tile, int *bps);
int x2_launch(int tile, const RunDesc *runs, const Tile *tiles, int ntiles, int substep, int grid, int iso,
              cudaStream_t s);
int substep_tile_shape(int dtype, int kernel, int tile, int *tx, int *ty);
// block shape of the reduction kernels and the step prologue for this variant
int reduction_tile_shape(int dtype, int kernel, int tile, int *tx, int *ty);
int substep_max_grid(int dtype, int kernel, int tile, int *blocks_per_sm);
int launch_halo(int dtype, void *fields, int nfields, long long fstride, int nx, int ny, int nz,
                int px, int py, cudaStream_t s);
// A = amp * N(0,1) per component and interior point (counter-based, see kernels.cu)
int launch_seed_field(int dtype, void *A, long long fstride, int nx, int ny, int nz, int px, int py,
                      unsigned long long seed, double amp, cudaStream_t s);
int launch_set_field(int dtype, int host_dtype, const void *src, void *dst_field, int nx, int ny,
                     int nz, int px, int py, cudaStream_t s);
// out[7 n + f] = field f of the NF-field array q at padded point of ijk[3n ..];
// wpairs: q's fields 0-5 are in the interleaved layout of x2_w_pairs
int launch_gather_points(int dtype, const void *q, long long fstride, int px, int py, const int *ijk, int npts,
                         double *out, int wpairs, cudaStream_t s);
// dense copy of a padded field whose padded point i is src_field[i], or
// (pairs) src_field[4 (i / 2) + i % 2]: one field of x2_w_pairs' layout, with
// src_field at its array's first value of that field
int launch_get_field(int dtype, int host_dtype, const void *src_field, void *dst, int nx, int ny,
                     int nz, int px, int py, int pairs, cudaStream_t s);
// B_rms of the run's current state into diag[1] (curl and sum in one pass)
int launch_brms(int dtype, const RunDesc *run_dev, const Tile *tiles, int ntiles, int tw, int th,
                cudaStream_t s);
// B = curl A of the run's current state into fields 0..2 of its w buffer
// (interior points only).
int launch_curl(int dtype, const RunDesc *run_dev, const Tile *tiles, int ntiles, int tw, int th,
                cudaStream_t s);
// Magnetic spectrum shells (spectrum.cu): shell count of an nx x ny x nz
// grid, device scratch bytes of the shell sum, and the shell sum itself from
// the half-spectrum bh (3 components, odist complex values apart) into
// shells_out[spectrum_nshells] (device doubles).
int spectrum_nshells(int nx, int ny, int nz);
size_t spectrum_scratch_bytes(int nx, int ny, int nz);
int launch_spectrum_bins(int dtype, const void *bh, long long odist, int nx, int ny, int nz, void *scratch,
                         double *shells_out, cudaStream_t s);
int launch_diagnostics(int dtype, const RunDesc *run_dev, const RunDesc &run_host,
                       const Tile *tiles, int ntiles, int tw, int th, cudaStream_t s);
// the reduction pass of the diagnostics alone (B with its halo in w)
int launch_diag_pass(int dtype, const RunDesc *runs, const Tile *tiles, int ntiles, int tw, int th,
                     cudaStream_t s);
int launch_coeffs(int dtype, const RunDesc *run, int64_t draw_step, double dt_update,
                  double dt_forcing, int parity, cudaStream_t s);
int launch_forcing_draw(const RunDesc *run, int64_t step, double *out13, cudaStream_t s);

}  // namespace mhd
