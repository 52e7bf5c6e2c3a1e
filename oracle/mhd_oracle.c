/*
 * mhd_oracle.c -- plain, slow, FP64 CPU oracle of one time step of
 * compressible isothermal resistive MHD on a triply periodic box
 * (Vaisala et al. 2020, arXiv:2012.08758, Sec. 4 Eqs. 1-6; numerical
 * method named in Sec. 2: 6th-order finite differences, 3rd-order
 * 2N-storage Runge-Kutta).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product:
 * only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may build, load or call it.  It shares no code, header,
 * table or constant with the CUDA library.
 *
 * Everything is evaluated literally, point by point, with periodic index
 * wrap (no halo arrays, no blocking, no fusion): the state q is seven
 * arrays of nx*ny*nz doubles, x fastest, in the order
 *   q0 = ln rho, q1..q3 = u_x,u_y,u_z, q4..q6 = A_x,A_y,A_z.
 *
 * Readings of the paper where it is silent (each also listed in the
 * design notes of the repository):
 *  R1  stencil weights: standard 6th-order central first and second
 *      derivatives; mixed derivatives use the diagonal points drawn in the
 *      stencil figure of Sec. 3.1 (weights 270, -27, 2 over 720 h_a h_b).
 *  R2  j = curl curl A = grad(div A) - lap A, built from the second and
 *      mixed stencils (mu0 = 1, Sec. 4).
 *  R3  RK3-2N coefficients: Williamson (1980) low-storage third order,
 *      alpha = (0, -5/9, -153/128), beta = (1/3, 15/16, 8/15).
 *  R4  forcing held fixed within a step and included in every substep's
 *      right-hand side (forcing_mode 0); mode 1 adds dt*f once after the
 *      third substep instead.
 *  R5  forcing draw: counter-based SplitMix64 (Steele, Lea & Flood 2014);
 *      draw j of step n uses counter n*64+j; k uniform over the integer
 *      shell list ordered lexicographically (kx slowest, each from -K..K);
 *      phi uniform in [-pi, pi); e an isotropic unit vector, redrawn while
 *      |k.e| > 0.99|k|.
 *  R6  time step: dt = min(cfl*dmin/max(|u| + sqrt(cs^2 + B^2/rho)),
 *      cfl_visc*dmin^2/max(nu, eta)); dt_fixed > 0 overrides it.
 *  R7  grid points x_i = i*L/N (vertex centred).
 *  R8  upwinding (Sec. 4 names a high-order upwinding of the continuity
 *      equation without giving it): with upwind = 1 the advection term
 *      u . grad ln rho takes, along each axis a, the fifth-order
 *      upwind-biased first derivative, i.e. the six-point stencil from three
 *      points upstream to two downstream of the centre, chosen by the sign
 *      of u_a.  Only the continuity equation is upwinded.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define PI_D 3.14159265358979323846

typedef struct {
  int nx, ny, nz;
  double lx, ly, lz;
  double cs, nu, eta;
  double f0, kmin, kmax, sigma;
  uint64_t seed;
  double cfl, cfl_visc, dt_fixed;
  int forcing_mode; /* R4: 0 = in every substep, 1 = once per step */
  int upwind;       /* R8: 0 = central ln rho advection, 1 = upwind-biased */
} orc_params;

/* One realisation of the forcing of Sec. 4 Eqs. 4-6 for one step.
 * f(x) = amp * (a cos(theta) - b sin(theta)), theta = kp.x + phi. */
typedef struct {
  int k[3];         /* integer wave vector (units of 2 pi / L)          */
  double kp[3];     /* physical wave vector 2 pi k / L                  */
  double phi;       /* random phase                                     */
  double e[3];      /* random unit vector                               */
  double a[3], b[3];/* Re and Im of f_k, Eq. 6                          */
  double amp;       /* normalisation N of Eq. 5 (depends on dt)         */
} orc_forcing;

/* Threads used by the OpenMP loop of orc_rhs (1 when built without it);
 * returns the count actually in effect. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Grid helpers (Sec. 3.1: periodic boundaries = wrapped ghost zones)  */
/* ------------------------------------------------------------------ */
static int wrapi(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

static long at(const orc_params *p, int i, int j, int k) {
  return ((long)wrapi(k, p->nz) * p->ny + wrapi(j, p->ny)) * p->nx + wrapi(i, p->nx);
}

static double spacing(const orc_params *p, int axis) {
  if (axis == 0) return p->lx / p->nx;
  if (axis == 1) return p->ly / p->ny;
  return p->lz / p->nz;
}

/* ------------------------------------------------------------------ */
/* Stencils on raw samples (Sec. 2: 6th-order finite differences; R1)  */
/* ------------------------------------------------------------------ */

/* First derivative from f(-3..3) (line7[3] is the centre). */
double orc_stencil_d1(const double *line7, double h) {
  const double *f = line7 + 3;
  return (45.0 * (f[1] - f[-1]) - 9.0 * (f[2] - f[-2]) + (f[3] - f[-3])) / (60.0 * h);
}

/* Second derivative from f(-3..3). */
double orc_stencil_d2(const double *line7, double h) {
  const double *f = line7 + 3;
  return (-490.0 * f[0] + 270.0 * (f[1] + f[-1]) - 27.0 * (f[2] + f[-2]) +
          2.0 * (f[3] + f[-3])) / (180.0 * h * h);
}

/* R8: fifth-order upwind-biased first derivative from f(-3..3).  For a
 * flow towards +axis (direction >= 0) the upstream side is -axis and the
 * stencil uses f(-3..2); otherwise it is mirrored and uses f(-2..3).  The
 * weights are the unique ones exact on polynomials of degree <= 5 over
 * those six points. */
double orc_stencil_up(const double *line7, double h, int direction) {
  const double *f = line7 + 3;
  if (direction >= 0)
    return (-2.0 * f[-3] + 15.0 * f[-2] - 60.0 * f[-1] + 20.0 * f[0] + 30.0 * f[1] - 3.0 * f[2]) /
           (60.0 * h);
  return (3.0 * f[-2] - 30.0 * f[-1] - 20.0 * f[0] + 60.0 * f[1] - 15.0 * f[2] + 2.0 * f[3]) / (60.0 * h);
}

/* Mixed derivative d2f/(da db) from a 7x7 patch, patch[(sb+3)*7 + (sa+3)]
 * holding f(a + sa*ha, b + sb*hb); only the two diagonals are used:
 * S_s = f(+s,+s) + f(-s,-s) - f(+s,-s) - f(-s,+s). */
double orc_stencil_dmix(const double *patch, double ha, double hb) {
#define P(sa, sb) patch[((sb) + 3) * 7 + ((sa) + 3)]
  double S[4];
  for (int s = 1; s <= 3; ++s) S[s] = P(s, s) + P(-s, -s) - P(s, -s) - P(-s, s);
#undef P
  return (270.0 * S[1] - 27.0 * S[2] + 2.0 * S[3]) / (720.0 * ha * hb);
}

/* ------------------------------------------------------------------ */
/* Stencils on a periodic field: gather with wrap, then the raw stencil */
/* ------------------------------------------------------------------ */
static void offset(int axis, int s, int *di, int *dj, int *dk) {
  *di = axis == 0 ? s : 0;
  *dj = axis == 1 ? s : 0;
  *dk = axis == 2 ? s : 0;
}

double orc_d1(const orc_params *p, const double *f, int i, int j, int k, int axis) {
  double line[7];
  for (int s = -3; s <= 3; ++s) {
    int di, dj, dk;
    offset(axis, s, &di, &dj, &dk);
    line[s + 3] = f[at(p, i + di, j + dj, k + dk)];
  }
  return orc_stencil_d1(line, spacing(p, axis));
}

double orc_dup(const orc_params *p, const double *f, int i, int j, int k, int axis, int direction) {
  double line[7];
  for (int s = -3; s <= 3; ++s) {
    int di, dj, dk;
    offset(axis, s, &di, &dj, &dk);
    line[s + 3] = f[at(p, i + di, j + dj, k + dk)];
  }
  return orc_stencil_up(line, spacing(p, axis), direction);
}

double orc_d2(const orc_params *p, const double *f, int i, int j, int k, int axis) {
  double line[7];
  for (int s = -3; s <= 3; ++s) {
    int di, dj, dk;
    offset(axis, s, &di, &dj, &dk);
    line[s + 3] = f[at(p, i + di, j + dj, k + dk)];
  }
  return orc_stencil_d2(line, spacing(p, axis));
}

double orc_dmix(const orc_params *p, const double *f, int i, int j, int k, int a, int b) {
  double patch[49];
  for (int sb = -3; sb <= 3; ++sb)
    for (int sa = -3; sa <= 3; ++sa) {
      int ai, aj, ak, bi, bj, bk;
      offset(a, sa, &ai, &aj, &ak);
      offset(b, sb, &bi, &bj, &bk);
      patch[(sb + 3) * 7 + (sa + 3)] = f[at(p, i + ai + bi, j + aj + bj, k + ak + bk)];
    }
  return orc_stencil_dmix(patch, spacing(p, a), spacing(p, b));
}

/* Second derivative d2f/(da db): pure stencil when a == b. */
static double dd(const orc_params *p, const double *f, int i, int j, int k, int a, int b) {
  return a == b ? orc_d2(p, f, i, j, k, a) : orc_dmix(p, f, i, j, k, a, b);
}

/* ------------------------------------------------------------------ */
/* Forcing (Sec. 4 Eqs. 4-6)                                            */
/* ------------------------------------------------------------------ */

/* Integer wave vectors with kmin <= |k| <= kmax, kx slowest (R5).
 * Returns the count; writes at most max vectors into out[3*n]. */
int orc_kshell(double kmin, double kmax, int *out, int max) {
  int K = (int)floor(kmax);
  int n = 0;
  for (int kx = -K; kx <= K; ++kx)
    for (int ky = -K; ky <= K; ++ky)
      for (int kz = -K; kz <= K; ++kz) {
        double m = sqrt((double)(kx * kx + ky * ky + kz * kz));
        if (m >= kmin && m <= kmax) {
          if (out && n < max) {
            out[3 * n + 0] = kx;
            out[3 * n + 1] = ky;
            out[3 * n + 2] = kz;
          }
          ++n;
        }
      }
  return n;
}

/* SplitMix64 output number c of the stream started at seed:
 * state = seed + (c+1) * 0x9E3779B97F4A7C15, then the published mixer. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double uniform01(uint64_t seed, uint64_t c) {
  return (double)(orc_splitmix64(seed, c) >> 11) * (1.0 / 9007199254740992.0);
}

static void cross3(const double *x, const double *y, double *r) {
  r[0] = x[1] * y[2] - x[2] * y[1];
  r[1] = x[2] * y[0] - x[0] * y[2];
  r[2] = x[0] * y[1] - x[1] * y[0];
}

/* Draw k, phi and e for step `step` (R5) and build f_k of Eq. 6.
 * The amplitude (Eq. 5) needs dt and is set by orc_forcing_amplitude. */
void orc_forcing_draw(const orc_params *p, int64_t step, orc_forcing *F) {
  memset(F, 0, sizeof(*F));
  int nk = orc_kshell(p->kmin, p->kmax, NULL, 0);
  if (nk <= 0) return;
  int *shell = (int *)malloc(sizeof(int) * 3 * nk);
  orc_kshell(p->kmin, p->kmax, shell, nk);
  uint64_t base = (uint64_t)step * 64u;
  int idx = (int)(uniform01(p->seed, base + 0) * nk);
  if (idx > nk - 1) idx = nk - 1;
  for (int d = 0; d < 3; ++d) F->k[d] = shell[3 * idx + d];
  free(shell);
  F->phi = PI_D * (2.0 * uniform01(p->seed, base + 1) - 1.0);
  double L[3] = {p->lx, p->ly, p->lz};
  for (int d = 0; d < 3; ++d) F->kp[d] = 2.0 * PI_D * F->k[d] / L[d];
  double kk = sqrt(F->kp[0] * F->kp[0] + F->kp[1] * F->kp[1] + F->kp[2] * F->kp[2]);
  for (int attempt = 0; attempt < 31; ++attempt) {
    double cz = 2.0 * uniform01(p->seed, base + 2 + 2 * attempt) - 1.0;
    double psi = 2.0 * PI_D * uniform01(p->seed, base + 3 + 2 * attempt);
    double sz = sqrt(fmax(0.0, 1.0 - cz * cz));
    F->e[0] = sz * cos(psi);
    F->e[1] = sz * sin(psi);
    F->e[2] = cz;
    double ke = F->kp[0] * F->e[0] + F->kp[1] * F->e[1] + F->kp[2] * F->e[2];
    if (fabs(ke) <= 0.99 * kk) break;
  }
  /* Eq. 6: f_k = [k x (k x e) - i sigma |k| (k x e)] /
   *              [sqrt(1 + sigma^2) k^2 sqrt(1 - (k.e)^2 / k^2)]        */
  double kxe[3], kxkxe[3];
  cross3(F->kp, F->e, kxe);
  cross3(F->kp, kxe, kxkxe);
  double ke = F->kp[0] * F->e[0] + F->kp[1] * F->e[1] + F->kp[2] * F->e[2];
  double k2 = kk * kk;
  double den = sqrt(1.0 + p->sigma * p->sigma) * k2 * sqrt(1.0 - ke * ke / k2);
  for (int d = 0; d < 3; ++d) {
    F->a[d] = kxkxe[d] / den;
    F->b[d] = -p->sigma * kk * kxe[d] / den;
  }
}

/* Eq. 5: N = f0 cs sqrt(|k| cs / dt). */
void orc_forcing_amplitude(const orc_params *p, double dt, orc_forcing *F) {
  double kk = sqrt(F->kp[0] * F->kp[0] + F->kp[1] * F->kp[1] + F->kp[2] * F->kp[2]);
  F->amp = (p->f0 > 0.0 && kk > 0.0) ? p->f0 * p->cs * sqrt(kk * p->cs / dt) : 0.0;
}

/* Eq. 4: f(x) = Re{ N f_k exp(i k.x + i phi) } = N (a cos th - b sin th). */
void orc_forcing_at(const orc_params *p, const orc_forcing *F, int i, int j, int k, double *f) {
  double th = F->kp[0] * (i * spacing(p, 0)) + F->kp[1] * (j * spacing(p, 1)) +
              F->kp[2] * (k * spacing(p, 2)) + F->phi;
  double c = cos(th), s = sin(th);
  for (int d = 0; d < 3; ++d) f[d] = F->amp * (F->a[d] * c - F->b[d] * s);
}

/* ------------------------------------------------------------------ */
/* Right-hand side (Sec. 4 Eqs. 1-3)                                    */
/* ------------------------------------------------------------------ */

/* d q / dt of Eqs. 1-3 at grid point (i, j, k): out[0..6].
 * F == NULL or F->amp == 0: no forcing. */
void orc_rhs_at(const orc_params *p, const double *q, const orc_forcing *F, int i, int j, int k,
          double *out) {
  const long n = (long)p->nx * p->ny * p->nz;
  const double *lnrho = q;
  const double *u[3] = {q + n, q + 2 * n, q + 3 * n};
  const double *A[3] = {q + 4 * n, q + 5 * n, q + 6 * n};
  const double cs2 = p->cs * p->cs;
  const long c = ((long)k * p->ny + j) * p->nx + i;
  double g[3], G[3][3], gA[3][3], uu[3];
  for (int a = 0; a < 3; ++a) {
    g[a] = orc_d1(p, lnrho, i, j, k, a);          /* grad ln rho       */
    uu[a] = u[a][c];
    for (int b = 0; b < 3; ++b) {
      G[a][b] = orc_d1(p, u[a], i, j, k, b);       /* d u_a / d x_b     */
      gA[a][b] = orc_d1(p, A[a], i, j, k, b);      /* d A_a / d x_b     */
    }
  }
  const double rho = exp(lnrho[c]);
  const double divu = G[0][0] + G[1][1] + G[2][2];
  /* B = curl A */
  double B[3] = {gA[2][1] - gA[1][2], gA[0][2] - gA[2][0], gA[1][0] - gA[0][1]};
  /* Laplacians, grad(div u), grad(div A) from second/mixed stencils */
  double lapu[3], lapA[3], gdu[3], gdA[3];
  for (int a = 0; a < 3; ++a) {
    lapu[a] = lapA[a] = gdu[a] = gdA[a] = 0.0;
    for (int b = 0; b < 3; ++b) {
      lapu[a] += orc_d2(p, u[a], i, j, k, b);
      lapA[a] += orc_d2(p, A[a], i, j, k, b);
      gdu[a] += dd(p, u[b], i, j, k, a, b);        /* d_a d_b u_b       */
      gdA[a] += dd(p, A[b], i, j, k, a, b);        /* d_a d_b A_b       */
    }
  }
  /* R2: j = grad(div A) - lap A (mu0 = 1) */
  double J[3] = {gdA[0] - lapA[0], gdA[1] - lapA[1], gdA[2] - lapA[2]};
  double JxB[3], uxB[3];
  cross3(J, B, JxB);
  cross3(uu, B, uxB);
  /* traceless rate of strain S_ab = (G_ab + G_ba)/2 - delta_ab div u / 3 */
  double S[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      S[a][b] = 0.5 * (G[a][b] + G[b][a]) - (a == b ? divu / 3.0 : 0.0);
  double f[3] = {0.0, 0.0, 0.0};
  if (F && F->amp != 0.0 && p->forcing_mode == 0) orc_forcing_at(p, F, i, j, k, f);

  /* Eq. 1: D ln rho / Dt = -div u; R8: upwind-biased advection if asked */
  double adv_lnrho = 0.0;
  for (int a = 0; a < 3; ++a)
    adv_lnrho += uu[a] * (p->upwind ? orc_dup(p, lnrho, i, j, k, a, uu[a] >= 0.0 ? 1 : -1) : g[a]);
  out[0] = -adv_lnrho - divu;
  for (int a = 0; a < 3; ++a) {
    /* Eq. 2: Du/Dt = -cs^2 grad ln rho + j x B / rho
     *         + nu [lap u + grad(div u)/3 + 2 S.grad ln rho] + f */
    double adv = uu[0] * G[a][0] + uu[1] * G[a][1] + uu[2] * G[a][2];
    double Sg = S[a][0] * g[0] + S[a][1] * g[1] + S[a][2] * g[2];
    out[1 + a] = -adv - cs2 * g[a] + JxB[a] / rho +
                 p->nu * (lapu[a] + gdu[a] / 3.0 + 2.0 * Sg) + f[a];
    /* Eq. 3: dA/dt = u x B + eta lap A (diffusive gauge) */
    out[4 + a] = uxB[a] + p->eta * lapA[a];
  }
}

/* rhs[7*n] = d q / dt for state q at every grid point. */
void orc_rhs(const orc_params *p, const double *q, const orc_forcing *F, double *rhs) {
  const long n = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        const long c = ((long)k * p->ny + j) * p->nx + i;
        double out[7];
        orc_rhs_at(p, q, F, i, j, k, out);
        for (int f = 0; f < 7; ++f) rhs[f * n + c] = out[f];
      }
}

/* ------------------------------------------------------------------ */
/* Time step (R6)                                                       */
/* ------------------------------------------------------------------ */
double orc_max_speed(const orc_params *p, const double *q) {
  const long n = (long)p->nx * p->ny * p->nz;
  const double cs2 = p->cs * p->cs;
  double vmax = 0.0;
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        const long c = ((long)k * p->ny + j) * p->nx + i;
        double gA[3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) gA[a][b] = orc_d1(p, q + (4 + a) * n, i, j, k, b);
        double B[3] = {gA[2][1] - gA[1][2], gA[0][2] - gA[2][0], gA[1][0] - gA[0][1]};
        double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
        double ux = q[n + c], uy = q[2 * n + c], uz = q[3 * n + c];
        double v = sqrt(ux * ux + uy * uy + uz * uz) + sqrt(cs2 + B2 / exp(q[c]));
        if (!(v <= vmax)) vmax = v; /* NaN propagates */
      }
  return vmax;
}

double orc_dt(const orc_params *p, const double *q) {
  if (p->dt_fixed > 0.0) return p->dt_fixed;
  double dmin = fmin(spacing(p, 0), fmin(spacing(p, 1), spacing(p, 2)));
  double dt = p->cfl * dmin / orc_max_speed(p, q);
  double diff = fmax(p->nu, p->eta);
  if (diff > 0.0) dt = fmin(dt, p->cfl_visc * dmin * dmin / diff);
  return dt;
}

/* ------------------------------------------------------------------ */
/* One time step: RK3-2N (Sec. 2; R3), forcing per R4                   */
/* ------------------------------------------------------------------ */
static const double RK_ALPHA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double RK_BETA[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

/* Advances q (7*n doubles) by one step with index `step` (selects the
 * forcing draw).  w and rhs are caller scratch of 7*n doubles each.
 * Returns dt; writes the step's forcing to F_out when non-NULL. */
double orc_step(const orc_params *p, double *q, int64_t step, double *w, double *rhs,
                orc_forcing *F_out) {
  const long n7 = 7L * p->nx * p->ny * p->nz;
  const long n = (long)p->nx * p->ny * p->nz;
  orc_forcing F;
  memset(&F, 0, sizeof(F));
  const double dt = orc_dt(p, q);
  if (p->f0 > 0.0) {
    orc_forcing_draw(p, step, &F);
    orc_forcing_amplitude(p, dt, &F);
  }
  for (int s = 0; s < 3; ++s) {
    orc_rhs(p, q, &F, rhs);
    for (long c = 0; c < n7; ++c) {
      w[c] = RK_ALPHA[s] * w[c] + dt * rhs[c];
      q[c] = q[c] + RK_BETA[s] * w[c];
    }
  }
  if (p->forcing_mode == 1 && F.amp != 0.0) {
    for (int k = 0; k < p->nz; ++k)
      for (int j = 0; j < p->ny; ++j)
        for (int i = 0; i < p->nx; ++i) {
          const long c = ((long)k * p->ny + j) * p->nx + i;
          double f[3];
          orc_forcing_at(p, &F, i, j, k, f);
          for (int a = 0; a < 3; ++a) q[(1 + a) * n + c] += dt * f[a];
        }
  }
  if (F_out) *F_out = F;
  return dt;
}

/* n steps starting at step index step0; dts[] (n doubles) gets each
 * step's dt when non-NULL.  Returns the final time. */
double orc_run(const orc_params *p, double *q, int64_t step0, int nsteps, double t0,
               double *dts) {
  const long n7 = 7L * p->nx * p->ny * p->nz;
  double *w = (double *)calloc((size_t)n7, sizeof(double));
  double *rhs = (double *)calloc((size_t)n7, sizeof(double));
  double t = t0;
  for (int s = 0; s < nsteps; ++s) {
    double dt = orc_step(p, q, step0 + s, w, rhs, NULL);
    t += dt;
    if (dts) dts[s] = dt;
  }
  free(w);
  free(rhs);
  return t;
}

/* ------------------------------------------------------------------ */
/* Diagnostics: volume means over the N^3 points (Sec. 4, Sec. 5)       */
/* ------------------------------------------------------------------ */

/* Neumaier compensated sum, so the oracle's means are accurate to a few
 * ulp regardless of the grid size. */
typedef struct { double s, c; } ksum;
static void kadd(ksum *k, double x) {
  double t = k->s + x;
  if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
  else k->c += (x - t) + k->s;
  k->s = t;
}
static double kval(const ksum *k) { return k->s + k->c; }

/* B = curl A with the first-derivative stencil at every point:
 * B[3*n], component-major, x fastest (the B of the diagnostics and of the
 * magnetic spectrum). */
void orc_curl(const orc_params *p, const double *q, double *B) {
  const long n = (long)p->nx * p->ny * p->nz;
  const double *A[3] = {q + 4 * n, q + 5 * n, q + 6 * n};
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        const long c = ((long)k * p->ny + j) * p->nx + i;
        B[c] = orc_d1(p, A[2], i, j, k, 1) - orc_d1(p, A[1], i, j, k, 2);
        B[n + c] = orc_d1(p, A[0], i, j, k, 2) - orc_d1(p, A[2], i, j, k, 0);
        B[2 * n + c] = orc_d1(p, A[1], i, j, k, 0) - orc_d1(p, A[0], i, j, k, 1);
      }
}

/* out[0..8] = u_rms, B_rms, max|u|, max|B|, E_kin = <rho u^2>/2,
 * E_mag = <B^2>/2, max|div B|, <rho>, max(|u| + sqrt(cs^2 + B^2/rho)). */
void orc_diagnostics(const orc_params *p, const double *q, double *out) {
  const long n = (long)p->nx * p->ny * p->nz;
  double *B = (double *)malloc(sizeof(double) * 3 * n);
  ksum su = {0, 0}, sb = {0, 0}, sk = {0, 0}, sm = {0, 0};
  double umax = 0.0, bmax = 0.0, vmax = 0.0;
  const double cs2 = p->cs * p->cs;
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        const long c = ((long)k * p->ny + j) * p->nx + i;
        double gA[3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) gA[a][b] = orc_d1(p, q + (4 + a) * n, i, j, k, b);
        B[c] = gA[2][1] - gA[1][2];
        B[n + c] = gA[0][2] - gA[2][0];
        B[2 * n + c] = gA[1][0] - gA[0][1];
        double u2 = q[n + c] * q[n + c] + q[2 * n + c] * q[2 * n + c] + q[3 * n + c] * q[3 * n + c];
        double b2 = B[c] * B[c] + B[n + c] * B[n + c] + B[2 * n + c] * B[2 * n + c];
        double rho = exp(q[c]);
        kadd(&su, u2);
        kadd(&sb, b2);
        kadd(&sk, rho * u2);
        kadd(&sm, rho);
        if (sqrt(u2) > umax) umax = sqrt(u2);
        if (sqrt(b2) > bmax) bmax = sqrt(b2);
        double v = sqrt(u2) + sqrt(cs2 + b2 / rho);
        if (v > vmax) vmax = v;
      }
  double divmax = 0.0;
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        double d = orc_d1(p, B, i, j, k, 0) + orc_d1(p, B + n, i, j, k, 1) +
                   orc_d1(p, B + 2 * n, i, j, k, 2);
        if (fabs(d) > divmax) divmax = fabs(d);
      }
  free(B);
  out[0] = sqrt(kval(&su) / n);
  out[1] = sqrt(kval(&sb) / n);
  out[2] = umax;
  out[3] = bmax;
  out[4] = 0.5 * kval(&sk) / n;
  out[5] = 0.5 * kval(&sb) / n;
  out[6] = divmax;
  out[7] = kval(&sm) / n;
  out[8] = vmax;
}
