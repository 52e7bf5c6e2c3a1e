/*
 * mhd.h -- C ABI of the B300 (sm_103a) isothermal MHD stepper.
 *
 * One time step of compressible isothermal resistive MHD on a triply
 * periodic box (Vaisala et al. 2020, arXiv:2012.08758): continuity
 * (Sec. 4, Eq. 1), momentum (Eq. 2) and induction in the diffusive gauge
 * (Eq. 3) with the random helical/non-helical forcing of Eqs. 4-6,
 * discretised with 6th-order central finite differences and advanced by
 * third-order 2N-storage Runge-Kutta (Sec. 2).  Periodic boundaries are
 * wrapped ghost zones of radius 3 (Sec. 3.1).
 *
 * Conventions for every entry point:
 *  - return 0 (MHD_OK) on success, a negative MHD_E* code on failure; the
 *    message is then available from mhd_last_error(ctx) (ctx may be NULL
 *    for failures that happen before a context exists).
 *  - host pointers belong to the caller and are only read/written during
 *    the call; device memory belongs to the context (or to the caller, when
 *    the caller passes a workspace to mhd_create).
 *  - a failed call leaves the context as it was (no half-built state).
 *  - all device work of a context is ordered on the CUDA stream given to
 *    mhd_create; calls documented as asynchronous return before the GPU
 *    has finished, calls documented as synchronising wait for that stream.
 *  - host state arrays are SoA: 7 fields of nx*ny*nz values each, x
 *    fastest, in the order ln rho, u_x, u_y, u_z, A_x, A_y, A_z.
 *
 * Not thread-safe per context: one host thread at a time per mhd_ctx.
 */
#ifndef MHD_H
#define MHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhd_ctx mhd_ctx;
typedef struct mhd_batch mhd_batch;

/* Working precision of fields and stencil arithmetic (Sec. 3.2: the
 * precision of reals is a build-time choice in the paper; here both
 * instantiations ship and the choice is per context). */
typedef enum { MHD_F32 = 0, MHD_F64 = 1 } mhd_dtype;

enum {
  MHD_OK = 0,
  MHD_EINVAL = -1,     /* bad argument or parameter                       */
  MHD_ENOMEM = -2,     /* device or host allocation failed / too small    */
  MHD_ECUDA = -3,      /* a CUDA runtime call failed                      */
  MHD_ETIMEOUT = -4,   /* a bounded device-side wait gave up              */
  MHD_ENONFINITE = -5, /* the time-step reduction saw NaN/Inf (run blew up)*/
  MHD_ESTATE = -6      /* call not valid in the current state             */
};

/* Quantities of mhd_reduce / mhd_diagnostics (volume means over the
 * nx*ny*nz interior points; B = curl A with the first-derivative stencil).
 * Global averages of this kind are the run-time diagnostics of Sec. 4. */
enum {
  MHD_URMS = 0,     /* sqrt(<|u|^2>)                                     */
  MHD_BRMS = 1,     /* sqrt(<|B|^2>)                                     */
  MHD_UMAX = 2,     /* max |u|                                           */
  MHD_BMAX = 3,     /* max |B|                                           */
  MHD_EKIN = 4,     /* <rho |u|^2> / 2                                   */
  MHD_EMAG = 5,     /* <|B|^2> / 2   (mu0 = 1, Sec. 4 units)             */
  MHD_DIVB_MAX = 6, /* max |div B| (zero up to rounding)                 */
  MHD_MASS = 7,     /* <rho>                                             */
  MHD_VMAX = 8,     /* max(|u| + sqrt(cs^2 + |B|^2/rho)), the CFL speed  */
  MHD_NREDUCE = 9
};

/* Kernel variants of the fused RHS + RK substep. */
enum {
  MHD_KERNEL_AUTO = 0,  /* fastest measured variant for this grid          */
  MHD_KERNEL_SMEM = 1,  /* plane ring in shared memory, plain loads        */
  MHD_KERNEL_TMA = 2    /* TMA-staged planes + register pencils along z    */
};

typedef struct {
  int nx, ny, nz;           /* interior points per axis, each >= 1           */
  double lx, ly, lz;        /* box size (default 2 pi, Sec. 4)               */
  double cs;                /* isothermal sound speed                        */
  double nu, eta;           /* viscosity and resistivity (>= 0)              */
  double f0;                /* forcing scale factor of Eq. 5 (0: no forcing) */
  double kmin, kmax;        /* forcing shell kmin <= |k| <= kmax (integer k) */
  double sigma;             /* forcing helicity in [0, 1] (Eq. 6)            */
  uint64_t seed;            /* forcing random stream of this run             */
  double cfl;               /* advective Courant number (default 0.4)        */
  double cfl_visc;          /* diffusive number (default 0.08)               */
  double dt_fixed;          /* > 0: constant dt instead of the CFL rule      */
  int forcing_mode;         /* 0: f in every substep; 1: dt*f once per step  */
  int dtype;                /* mhd_dtype                                     */
  int kernel;               /* MHD_KERNEL_*                                  */
  int tile;                 /* 0: automatic tile choice, else a tile id      */
  int upwind;               /* 0: central ln rho advection (default); 1: the */
                            /* high-order upwinding of the continuity        */
                            /* equation (Sec. 4): per axis the fifth-order   */
                            /* upwind-biased first derivative, i.e. the      */
                            /* central one minus |u_a| h_a^5/60 d^6/dx_a^6   */
} mhd_params;

/* Fills p with the defaults: 32^3, L = 2 pi, cs = 1, nu = eta = 5e-3,
 * no forcing (f0 = 0), shell [2.5, 3.5], sigma = 0, seed = 1, cfl = 0.4,
 * cfl_visc = 0.08, CFL time step, forcing in every substep, FP32, automatic
 * kernel and tile, no upwinding.  p must be non-NULL. */
void mhd_default_params(mhd_params *p);

/* The parameters a context created with p runs with: p with the automatic
 * choices made (kernel MHD_KERNEL_AUTO -> MHD_KERNEL_TMA; on that kernel tile
 * 0 -> FP32: 28, the warp-specialised paired-point kernel with w in the
 * interleaved layout; FP64: 3).  Host-only.  Errors: MHD_EINVAL (invalid p,
 * NULL out). */
int mhd_resolve_params(const mhd_params *p, mhd_params *out);

/* Device bytes a context with parameters p needs when the caller supplies
 * the workspace (mhd_create with workspace != NULL).  Returns MHD_EINVAL on
 * invalid parameters. */
int mhd_workspace_bytes(const mhd_params *p, size_t *bytes);

/* Creates a context on the current CUDA device.
 *   p          parameters (validated; copied).
 *   stream     cudaStream_t to order all work on (NULL: legacy stream).
 *   workspace  device buffer of >= mhd_workspace_bytes bytes, 256-byte
 *              aligned, owned by the caller and kept alive until
 *              mhd_destroy; or NULL, and the context allocates its own.
 *   out        receives the context.
 * The state is zero (ln rho = 0, u = A = 0) at t = 0, step 0.
 * Synchronising.  Errors: MHD_EINVAL, MHD_ENOMEM, MHD_ECUDA. */
int mhd_create(const mhd_params *p, void *stream, void *workspace, size_t workspace_bytes,
               mhd_ctx **out);

/* Releases the context and any device memory it allocated itself.
 * Waits for the context's stream.  NULL is ignored. */
void mhd_destroy(mhd_ctx *ctx);

/* Uploads a state: host_soa holds 7*nx*ny*nz values of type host_dtype
 * (converted to the working precision on the device), t is the time and
 * step the step index (it selects the forcing draws that follow).  Fills the
 * periodic ghost zones.  Synchronising. */
int mhd_set_state(mhd_ctx *ctx, const void *host_soa, int host_dtype, double t, int64_t step);

/* Sets the state to the paper's initial condition (Sec. 4) at t = 0, step 0:
 * ln rho = 0, u = 0 and a weak delta-correlated seed field A = amp * N(0,1),
 * independent per component and interior point, generated on the device
 * (no host arrays): normal number n = c * nx*ny*nz + e of component c and
 * point e = (k*ny + j)*nx + i is sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller, FP64),
 * u1 = ((SplitMix64(seed, 2n) >> 11) + 1) 2^-53, u2 = (SplitMix64(seed, 2n+1)
 * >> 11) 2^-53, SplitMix64(key, c) being output c of the stream keyed by key
 * (as in the forcing draw), rounded to the context's precision.  Use a seed
 * other than the forcing seed of mhd_params for independent streams.
 * Synchronising.  Errors: MHD_EINVAL (NULL ctx, amp < 0 or not finite),
 * MHD_ECUDA. */
int mhd_set_seed_field(mhd_ctx *ctx, uint64_t seed, double amp);

/* Downloads the state into host_soa (7*nx*ny*nz values of host_dtype) and
 * the time and step index (either pointer may be NULL).  Synchronising;
 * returns MHD_ENONFINITE if the run has produced a non-finite time step. */
int mhd_get_state(mhd_ctx *ctx, void *host_soa, int host_dtype, double *t, int64_t *step);

/* Enqueues nsteps time steps (nsteps >= 0) on the context's stream and
 * returns without waiting.  Each step: time-step reduction (CFL rule, or
 * dt_fixed) and forcing draw on the device, then three fused RHS + RK3-2N
 * substeps (Sec. 2) with the ghost zones refilled by each substep.  No
 * host<->device traffic.  Errors of the launches are reported here;
 * numerical blow-up is reported by the next synchronising call. */
int mhd_step(mhd_ctx *ctx, int nsteps);

/* mhd_step with CUDA events recorded on the context's stream around every
 * kernel stage; waits for the steps to finish and adds the device time of
 * each stage, summed over the nsteps steps, to stage_ms[0..3] = step
 * prologue (time-step reduction + forcing draw), substeps 1, 2 and 3; the
 * total elapsed time (first to last event) is added to *total_ms.  The
 * work done is exactly that of mhd_step.  Synchronising. */
int mhd_step_timed(mhd_ctx *ctx, int nsteps, double *stage_ms, double *total_ms);

/* Reads one quantity (MHD_URMS ... MHD_VMAX) of the current state into
 * *out, accumulated in FP64 in a fixed order.  MHD_BRMS (sampled after every
 * step by growth-rate runs) takes a single fused pass with the same per-point
 * B, tiles and summation order as mhd_diagnostics.  On the TMA kernel that
 * pass is the time-step sweep of the next step's prologue: its CFL maximum is
 * kept on the device and that prologue reuses it instead of sweeping again
 * (results are bit-for-bit those of a run that is never sampled; any write of
 * the state discards the kept value).  Synchronising. */
int mhd_reduce(mhd_ctx *ctx, int kind, double *out);

/* All MHD_NREDUCE quantities at once into out[MHD_NREDUCE].  Synchronising. */
int mhd_diagnostics(mhd_ctx *ctx, double *out);

/* Time, last time step and step index of the current state (any pointer
 * may be NULL).  Synchronising; MHD_ENONFINITE after a blow-up. */
int mhd_time(mhd_ctx *ctx, double *t, double *dt_last, int64_t *step);

/* Waits for the context's stream; MHD_ENONFINITE after a blow-up. */
int mhd_sync(mhd_ctx *ctx);

/* The forcing draw of step index `step` (Sec. 4, Eqs. 4 and 6) as computed
 * on the device: out[0..2] = integer k, out[3] = phi, out[4..6] = e,
 * out[7..9] = Re f_k, out[10..12] = Im f_k.  Does not change the run.
 * Synchronising.  MHD_EINVAL when the run has no forcing. */
int mhd_forcing_draw(mhd_ctx *ctx, int64_t step, double *out);

/* Right-hand side of Eqs. 1-3 for the current state, evaluated by the same
 * fused kernel as a substep: host_rhs (7*nx*ny*nz values of host_dtype)
 * receives dq/dt, including the forcing of step index `step` normalised
 * with time step dt_forcing (dt_forcing <= 0: no forcing).  Does not
 * change the state.  Synchronising. */
int mhd_eval_rhs(mhd_ctx *ctx, int64_t step, double dt_forcing, void *host_rhs, int host_dtype);

/* The same right-hand side at npts listed grid points only, for grids whose
 * full dq/dt is too large to bring to the host (the whole field is still
 * evaluated on the device; only the listed values are copied back).
 *   ijk       host array of 3*npts ints: (i, j, k) of each point,
 *             0 <= i < nx, 0 <= j < ny, 0 <= k < nz (caller-owned).
 *   host_out  host array of 7*npts doubles (caller-owned): point-major,
 *             host_out[7*n + f] = dq_f/dt at point n, fields in state order.
 * 1 <= npts <= MHD_EVAL_AT_MAX_POINTS, and the list and values must fit the
 * context's spare state buffer (12 + 56 bytes per point against 7 padded
 * fields: any npts up to a third of the grid's points).  Does not change the
 * state.  Synchronising.  Errors: MHD_EINVAL (NULL pointers, npts out of
 * range, a point outside the grid), MHD_ECUDA. */
enum { MHD_EVAL_AT_MAX_POINTS = 1 << 16 };
int mhd_eval_rhs_at(mhd_ctx *ctx, int64_t step, double dt_forcing, int npts, const int *ijk,
                    double *host_out);

/* ---- magnetic energy spectrum (Sec. 5, power spectra) ----------------------
 * E_B(m) for shells m = 0 .. nshells-1 of the current state:
 *   B = curl A with the first-derivative stencil (the B of mhd_diagnostics),
 *   B^(k) = N^-3 sum_x B(x) exp(-i k.x) over the N = nx*ny*nz points, k the
 *   integer wave vector (units of 2 pi / L),
 *   E_B(m) = 1/2 sum of |B^(k)|^2 over the k with m - 1/2 <= |k| < m + 1/2,
 * so sum_m E_B(m) = <|B|^2>/2 = MHD_EMAG (energy per unit volume; the paper's
 * normalisation, the integral of B^2/2 over the box, is this times lx*ly*lz).
 * Shell m = 0 is the mean field (zero for a periodic A).  Needs a cubic box
 * (lx = ly = lz; the grid sizes may differ) and nx >= 2; nshells =
 * floor(sqrt((nx/2)^2 + (ny/2)^2 + (nz/2)^2) + 1/2) + 1 (integer halves). */

/* Number of shells for parameters p (host only).  Errors: MHD_EINVAL
 * (invalid parameters, non-cubic box, nx < 2, NULL nshells). */
int mhd_spectrum_shells(const mhd_params *p, int *nshells);

/* Computes E_B of the current state into host_out[0 .. min(nshells,
 * max_shells) - 1] (host doubles owned by the caller); *nshells (may be
 * NULL) receives the shell count.  The transform is cuFFT's real-to-complex
 * FFT in the context's precision; the shell sums are FP64 in a fixed order
 * (bitwise reproducible).  Uses the RK register as scratch (free between
 * steps); the first call makes a cuFFT plan, whose work area cuFFT allocates
 * and mhd_destroy frees.  Synchronising.  Errors: MHD_EINVAL (NULL
 * arguments, non-cubic box, nx < 2), MHD_ECUDA (CUDA or cuFFT failure). */
int mhd_spectrum(mhd_ctx *ctx, double *host_out, int max_shells, int *nshells);

/* Message of the last failure on ctx (or of the calling thread when ctx is
 * NULL); never NULL. */
const char *mhd_last_error(const mhd_ctx *ctx);

/* ---- batched stepping of independent runs ------------------------------
 * A batch steps several contexts (same device, stream and dtype; any grid
 * sizes) with one launch per kernel stage over a combined tile table, the
 * k-step sequence captured once in a CUDA graph and replayed.  Every run
 * gives bit-for-bit the result it gives when stepped alone (per-run
 * reductions have a fixed order that does not depend on the batch). */

/* Creates a batch over runs[0..nruns-1] (the contexts must outlive it).
 * Synchronising.  Errors: MHD_EINVAL (mixed dtype/stream), MHD_ENOMEM,
 * MHD_ECUDA. */
int mhd_batch_create(mhd_ctx *const *runs, int nruns, mhd_batch **out);

/* Enqueues nsteps steps of every run of the batch.  Asynchronous. */
int mhd_batch_step(mhd_batch *b, int nsteps);

/* Releases the batch (not the contexts).  NULL is ignored. */
void mhd_batch_destroy(mhd_batch *b);

/* ---- z-slab domain decomposition (Sec. 3.3 and 3.4) -----------------------
 * The grid is cut along z into nslabs slabs of nz/nslabs planes (the first
 * nz mod nslabs slabs one plane more), each a context of its own, as the
 * paper decomposes its domain over GPUs.  Every substep, each slab sends its
 * three planes nearest a face -- all seven fields, with their x/y ghost
 * columns -- into the ghost planes of the neighbour across that face
 * (periodically: the last slab's top neighbour is the first slab); the time
 * step is the minimum over all slabs (one reduction of the CFL maxima of all
 * slabs), and the forcing is evaluated at global z.  With overlap = 1 each
 * substep first computes the slabs' outer planes (within three of a face),
 * then the exchange runs on a second stream while the inner planes are
 * computed, as in the paper's inner/outer split; overlap = 0 computes all
 * planes, then exchanges.  The substep arithmetic per point is that of the
 * undecomposed run, so the decomposed state equals it bit for bit; the
 * diagnostics are summed over the slabs' tiles in another order (equal up to
 * rounding).  All slabs live on the current device (one GPU); the exchange
 * is one cudaMemcpy2DAsync per face and direction.  Requires the TMA kernel
 * (MHD_KERNEL_AUTO or MHD_KERNEL_TMA) and at least 3 planes per slab.
 * Errors are reported by mhd_last_error(NULL). */
typedef struct mhd_slabs mhd_slabs;

/* Creates the decomposition of the grid of p into nslabs z-slabs on the
 * current device, ordered on `stream` (NULL: legacy stream).  The state is
 * zero at t = 0, step 0.  Synchronising.  Errors: MHD_EINVAL (bad parameters,
 * nslabs < 1, fewer than 3 planes per slab, the plane-ring kernel),
 * MHD_ENOMEM, MHD_ECUDA. */
int mhd_slabs_create(const mhd_params *p, int nslabs, int overlap, void *stream, mhd_slabs **out);

/* First global plane *z0 and plane count *nz of slab `slab`.  Host only. */
int mhd_slabs_extent(const mhd_slabs *s, int slab, int *z0, int *nz);

/* As mhd_set_state / mhd_get_state for the whole grid: host_soa holds 7 *
 * nx*ny*nz values (SoA, x fastest); each slab takes or gives its planes.
 * Synchronising. */
int mhd_slabs_set_state(mhd_slabs *s, const void *host_soa, int host_dtype, double t, int64_t step);
int mhd_slabs_get_state(mhd_slabs *s, void *host_soa, int host_dtype, double *t, int64_t *step);

/* Enqueues nsteps steps of the decomposed run.  Asynchronous. */
int mhd_slabs_step(mhd_slabs *s, int nsteps);

/* The MHD_NREDUCE diagnostics of the whole grid into out[MHD_NREDUCE]
 * (B = curl A per slab, B's ghost planes exchanged, one reduction over all
 * slabs' tiles).  Synchronising. */
int mhd_slabs_diagnostics(mhd_slabs *s, double *out);

/* Releases the slabs and their device memory.  NULL is ignored. */
void mhd_slabs_destroy(mhd_slabs *s);

/* ---- diagnostics without device allocation ---------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory: a plugin inside an application whose own
 * memory pool already owns every byte of the GPU, code that must run within a
 * memory budget fixed before it starts, and code on a latency-critical path,
 * where cudaMalloc is unwelcome because it can synchronise the whole device
 * and can fail once another allocator has reserved the memory.
 *
 * Computes the MHD_NREDUCE quantities of mhd_diagnostics (same order, same
 * definitions; per-point values formed in the working precision and summed
 * in FP64, as mhd_diagnostics does) for a state the caller already holds on
 * the device; no context of this library is involved.
 *   state_dev  device pointer, read only: 7*nx*ny*nz values of `dtype`
 *              (MHD_F32 or MHD_F64), dense SoA without ghost zones, x fastest,
 *              fields ln rho, u_x, u_y, u_z, A_x, A_y, A_z (periodic box).
 *   nx..cs     grid, box lengths and sound speed, as in mhd_params.
 *   out_dev    device pointer to MHD_NREDUCE doubles, written by the kernel.
 *   stream     cudaStream_t the work is ordered on (NULL: legacy stream).
 * Asynchronous: out_dev holds the result once the stream reaches this work.
 * Allocates nothing.  Its scratch -- per-block partial sums and a counter --
 * is one static device array of 256 KiB inside this library, which every GPU
 * that loads the library keeps until the process exits.  That bounds the grid
 * to MHD_NOALLOC_MAX_POINTS points (2^24, e.g. 256^3); larger grids are
 * rejected with MHD_EINVAL and a message saying so.  The array exists once
 * per CUDA context: the first call in a context (the calling thread's current
 * one; the device's primary context if none is current) looks up the array's
 * device address there and caches it under the context's unique id, so a
 * device reset or another context gets its own lookup at its first call.
 * Make that first call before any stream capture.  All calls share the one
 * array, which keeps the last call's partials: the counter is cleared at the
 * start of every call, but calls whose work overlaps on the GPU (different
 * streams or threads without ordering) race and give wrong results -- order
 * them on one stream or synchronise in between.
 * Errors: MHD_EINVAL (NULL pointer, bad size, grid above the limit),
 * MHD_ECUDA; the message is returned by mhd_last_error(NULL). */
enum { MHD_NOALLOC_MAX_POINTS = 1 << 24 };
int mhd_diagnostics_noalloc(const void *state_dev, int dtype, int nx, int ny, int nz, double lx,
                            double ly, double lz, double cs, double *out_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MHD_H */
