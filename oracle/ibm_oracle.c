/*
 * Plain FP64 CPU oracle of the distribution-function-correction IB-LBM
 * (Tao, He, Chen, Huang, arXiv 1803.09380).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -std=c11 -fPIC -shared, one thread.  The
 * same file built with -fopenmp spreads the node loops that have no
 * summation order (collision, streaming, moments, marker interpolation,
 * adding the spread correction) over host threads; every sum whose order
 * matters (spreading in ascending marker order, force sums) stays serial, so
 * both builds give bitwise the same results.  Everything is double
 * precision.  Loops follow the paper's equations in the paper's order;
 * nothing is fused or reordered.
 *
 * What one time step computes (section 2, Eqs. 1-8 and 22-29; section 3.3,
 * Eqs. 37-42):
 *   1. IB correction loop, n = 0..N-1, Jacobi over markers (section 2.3):
 *      interpolate the nodal equilibria to every marker (Eq. 22b with Eq. 28),
 *      form the deviation (Eqs. 24, 25 simplified to Eq. 28), spread it with
 *      the 4-point cosine delta function (Eqs. 15c, 26) and correct f (Eq. 27).
 *      Force and torque on each body are summed from the deviations (Eq. 29,
 *      Eqs. 37-38 without the internal-mass terms).
 *   2. One more interpolation gives the final no-slip residual r^N.
 *   3. Free bodies: Newton-Euler update in FP64 (Eqs. 37-42).
 *   4. Extrapolation boundary columns are rebuilt from their inner neighbours
 *      (ora_open_boundaries).  Moments of the corrected state (Eq. 7) are
 *      recorded; collision with
 *      the equilibrium of Eq. 3: BGK (Eq. 1 with the single-relaxation
 *      operator named in section 2.1) or the MRT operator of Eqs. 2, 5, 6.
 *   5. Streaming (Eq. 1) with the domain boundary rules.
 *
 * Readings of places where the paper is silent or garbled (each is listed
 * with its reason in the design notes of the repository):
 *   - D2Q9 ordering: e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1)
 *     e6=(-1,1) e7=(-1,-1) e8=(1,-1), the order fixed by the rows of the
 *     transform matrix of Eq. 5 (Eq. 4 is garbled in the extracted text).
 *   - (f^eq)* in Eq. 28 interpolates the NODAL equilibria f^eq(rho(x),u(x)).
 *   - The boundary density in f^eq(rho, U) of Eq. 24 is the interpolated
 *     density rho* = sum_x D rho(x) (= sum_i (f_i^eq)*), so the correction
 *     conserves mass, and the density parts of f^eq(rho*, U) and (f^eq)*
 *     cancel exactly.
 *   - Markers are corrected simultaneously (Jacobi): every marker of
 *     iteration n reads the same f^n.
 *   - The correction acts on the post-stream populations, before the moments
 *     and the collision of the step.
 *   - Stencil nodes outside a non-periodic domain are skipped (no
 *     renormalisation).
 *   - Lattice units: dx = dt = 1, so D = delta(dx) delta(dy) (Eq. 15).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_Q 9

/* Eq. 4 (ordering from the rows of Eq. 5), weights of Eq. 4. */
static const int ora_ex[ORA_Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ora_ey[ORA_Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double ora_w[ORA_Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                                    1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                                    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

enum { ORA_PERIODIC = 0, ORA_BOUNCEBACK = 1, ORA_FREESLIP = 2,
       ORA_INLET_EQ = 3, ORA_OUTLET_ZEROGRAD = 4, ORA_INLET_NEE = 5,
       ORA_OUTLET_NEE = 6 };
enum { ORA_BODY_FIXED = 0, ORA_BODY_PRESCRIBED = 1, ORA_BODY_FREE = 2 };

typedef struct {
  int kind;
  int m0, m1;               /* marker index range [m0, m1) */
  double xc[2], u[2], omega, theta;
  double u_prev[2], omega_prev;
  double rho_s, rho_f, volume, inertia, radius, mass;
  double gravity[2];
  double F_ib[2], T_ib;     /* Eq. 29 sums of the last step */
  double F_c[2];            /* Eq. 39 collision force of the last step */
  double theta0;            /* angle at which the marker offsets were taken */
} ora_body;

typedef struct {
  int nx, ny;
  double tau, rho0;
  int bc[4];                /* sides -x, +x, -y, +y */
  double wall_u[4][2];
  double inlet_u[2];
  int n_corr;
  int mrt;                  /* 0: BGK, 1: MRT (Eqs. 2, 5, 6) */
  int delta_points;         /* 2, 3 or 4: the delta function of Eq. 15a-c */
  /* Alternative readings of section 2.3 (all 0 = the readings above); used
   * only to show how the Couette convergence order depends on them. */
  int rd_interp_moments;    /* (f^eq)* = f^eq(rho*, j* / rho*), interpolated moments */
  int rd_rho_b_ref;         /* boundary density rho_b = rho0 instead of rho* */
  int rd_post_collision;    /* correct the post-collision populations */
  int rd_unit_ds;           /* spread without the arc length ds (Eq. 26 weight 1) */
  double s_rate[ORA_Q];     /* diagonal of S in Eq. 6 */
  double *f;                /* [9][ny][nx], post-stream state */
  double *g;                /* streaming scratch */
  double *df;               /* spreading scratch, [9][ny][nx] */
  double *rho, *ux, *uy;    /* moments of the last corrected state */
  int nm, mcap;
  double *X, *Y, *ds, *dX, *dY; /* marker positions, arc lengths, offsets */
  double *Uset;             /* prescribed marker velocities [2 nm], or NULL */
  int *mbody;
  int nb, bcap;
  ora_body *bodies;
  double *resid;            /* r^0 .. r^N of the last step */
  double F_euler[2];        /* Eulerian-side force sum of the last step */
  double *rowF;             /* its per-row partial sums [ny][2] */
  long steps;
} ora_lattice;

/* ---------------------------------------------------------------- kernels */

/* Eq. 15c: 4-point cosine delta function, zero for |r| >= 2. */
double ora_delta4(double r) {
  double a = fabs(r);
  if (a >= 2.0) return 0.0;
  return 0.25 * (1.0 + cos(M_PI * a / 2.0));
}

/* Eq. 15a: 2-point (linear hat) delta function, zero for |r| >= 1. */
double ora_delta2(double r) {
  double a = fabs(r);
  return a >= 1.0 ? 0.0 : 1.0 - a;
}

/* Eq. 15b: 3-point delta function, zero for |r| >= 1.5. */
double ora_delta3(double r) {
  double a = fabs(r);
  if (a < 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
  if (a < 1.5) return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))) / 6.0;
  return 0.0;
}

/* Eq. 3 with c_s^2 = 1/3. */
void ora_feq(double rho, double ux, double uy, double *feq) {
  double uu = ux * ux + uy * uy;
  for (int i = 0; i < ORA_Q; ++i) {
    double eu = ora_ex[i] * ux + ora_ey[i] * uy;
    feq[i] = ora_w[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
  }
}

/* Eq. 7, in a fixed summation order with antisymmetric pairs first, so that
 * a mirror-symmetric state gives exactly zero momentum. */
void ora_moments(const double *p, double *rho, double *jx, double *jy) {
  *rho = ((p[0] + (p[1] + p[3])) + (p[2] + p[4])) + ((p[5] + p[7]) + (p[6] + p[8]));
  *jx = ((p[1] - p[3]) + (p[5] - p[7])) + (p[8] - p[6]);
  *jy = ((p[2] - p[4]) + (p[5] - p[7])) + (p[6] - p[8]);
}

/* Eq. 5: the transform matrix M.  Row k maps the populations to moment k:
 * density, energy e, energy square epsilon, x-momentum, x energy flux q_x,
 * y-momentum, y energy flux q_y, and the stress moments p_xx, p_xy. */
static const double ora_M[ORA_Q][ORA_Q] = {
    { 1,  1,  1,  1,  1, 1,  1,  1,  1},
    {-4, -1, -1, -1, -1, 2,  2,  2,  2},
    { 4, -2, -2, -2, -2, 1,  1,  1,  1},
    { 0,  1,  0, -1,  0, 1, -1, -1,  1},
    { 0, -2,  0,  2,  0, 1, -1, -1,  1},
    { 0,  0,  1,  0, -1, 1,  1, -1, -1},
    { 0,  0, -2,  0,  2, 1,  1, -1, -1},
    { 0,  1, -1,  1, -1, 0,  0,  0,  0},
    { 0,  0,  0,  0,  0, 1, -1,  1, -1}};

void ora_mrt_matrix(double *out) {
  for (int k = 0; k < ORA_Q; ++k)
    for (int i = 0; i < ORA_Q; ++i) out[k * ORA_Q + i] = ora_M[k][i];
}

/* Eq. 2 at one node: ps = p - M^-1 S M (p - feq), with S = diag(s) of
 * Eq. 6.  The rows of M are mutually orthogonal, so M^-1 = M^T N^-1 with
 * N = diag(|row k|^2); the norms are summed from M itself. */
void ora_mrt_collide(const double *s, const double *p, const double *feq, double *ps) {
  double r[ORA_Q];
  for (int k = 0; k < ORA_Q; ++k) {
    double mk = 0.0, nk = 0.0;
    for (int i = 0; i < ORA_Q; ++i) {
      mk += ora_M[k][i] * (p[i] - feq[i]);
      nk += ora_M[k][i] * ora_M[k][i];
    }
    r[k] = s[k] * mk / nk;
  }
  for (int i = 0; i < ORA_Q; ++i) {
    double acc = 0.0;
    for (int k = 0; k < ORA_Q; ++k) acc += ora_M[k][i] * r[k];
    ps[i] = p[i] - acc;
  }
}

static size_t idx(const ora_lattice *L, int i, int x, int y) {
  return ((size_t)i * L->ny + (size_t)y) * L->nx + (size_t)x;
}

static void node_pops(const ora_lattice *L, const double *a, int x, int y,
                      double *p) {
  for (int i = 0; i < ORA_Q; ++i) p[i] = a[idx(L, i, x, y)];
}

/* ---------------------------------------------------------------- setup */

ora_lattice *ora_create(int nx, int ny, double tau, double rho0, const int *bc,
                        const double *wall_u, const double *inlet_u,
                        int n_corr) {
  ora_lattice *L = (ora_lattice *)calloc(1, sizeof(ora_lattice));
  if (!L) return NULL;
  L->nx = nx;
  L->ny = ny;
  L->tau = tau;
  L->rho0 = rho0;
  for (int s = 0; s < 4; ++s) {
    L->bc[s] = bc ? bc[s] : ORA_PERIODIC;
    L->wall_u[s][0] = wall_u ? wall_u[2 * s] : 0.0;
    L->wall_u[s][1] = wall_u ? wall_u[2 * s + 1] : 0.0;
  }
  L->inlet_u[0] = inlet_u ? inlet_u[0] : 0.0;
  L->inlet_u[1] = inlet_u ? inlet_u[1] : 0.0;
  L->n_corr = n_corr;
  L->delta_points = 4;
  size_t n = (size_t)nx * ny;
  L->f = (double *)malloc(sizeof(double) * ORA_Q * n);
  L->g = (double *)malloc(sizeof(double) * ORA_Q * n);
  L->df = (double *)malloc(sizeof(double) * ORA_Q * n);
  L->rho = (double *)malloc(sizeof(double) * n);
  L->ux = (double *)malloc(sizeof(double) * n);
  L->uy = (double *)malloc(sizeof(double) * n);
  L->resid = (double *)calloc((size_t)n_corr + 1, sizeof(double));
  L->rowF = (double *)calloc(2 * (size_t)ny, sizeof(double));
  /* rest equilibrium at rho0 */
  double feq[ORA_Q];
  ora_feq(rho0, 0.0, 0.0, feq);
  for (int i = 0; i < ORA_Q; ++i)
    for (size_t k = 0; k < n; ++k) L->f[(size_t)i * n + k] = feq[i];
  for (size_t k = 0; k < n; ++k) {
    L->rho[k] = rho0;
    L->ux[k] = 0.0;
    L->uy[k] = 0.0;
  }
  return L;
}

/* Switch the collision to MRT (Eqs. 2, 5, 6) with rates s_e, s_eps, s_q for
 * the energy, energy-square and energy-flux moments; the stress moments
 * relax at 1/tau (Eq. 8).  The conserved moments (density, momentum) have
 * zero non-equilibrium part, so their rates are immaterial; they are set to
 * 1/tau, which makes the operator BGK when every rate is 1/tau. */
void ora_set_mrt(ora_lattice *L, double s_e, double s_eps, double s_q) {
  double sn = 1.0 / L->tau;
  double s[ORA_Q] = {sn, s_e, s_eps, sn, s_q, sn, s_q, sn, sn};
  L->mrt = 1;
  for (int k = 0; k < ORA_Q; ++k) L->s_rate[k] = s[k];
}

/* Choose the delta function of Eq. 15 (2, 3 or 4 points; 4 by default).
 * Every support lies inside the 4 x 4 node window floor(X)-1 .. floor(X)+2,
 * so interpolation and spreading keep that window; nodes outside the
 * chosen support get weight zero. */
void ora_set_delta(ora_lattice *L, int points) { L->delta_points = points; }

static double delta_of(const ora_lattice *L, double r) {
  if (L->delta_points == 2) return ora_delta2(r);
  if (L->delta_points == 3) return ora_delta3(r);
  return ora_delta4(r);
}

void ora_destroy(ora_lattice *L) {
  if (!L) return;
  free(L->f); free(L->g); free(L->df);
  free(L->rho); free(L->ux); free(L->uy); free(L->resid); free(L->rowF);
  free(L->X); free(L->Y); free(L->ds); free(L->dX); free(L->dY);
  free(L->mbody); free(L->bodies); free(L->Uset);
  free(L);
}

/* body: kind, xc[2], u[2], omega, theta, rho_s, rho_f, volume, inertia,
 * radius, gravity[2] -- packed as 14 doubles after the kind. */
int ora_add_body(ora_lattice *L, int kind, const double *bd, const double *xy,
                 const double *ds, int n) {
  free(L->Uset);            /* prescribed velocities are reset by new markers */
  L->Uset = NULL;
  if (L->nm + n > L->mcap) {
    int cap = (L->nm + n) * 2;
    L->X = (double *)realloc(L->X, sizeof(double) * cap);
    L->Y = (double *)realloc(L->Y, sizeof(double) * cap);
    L->ds = (double *)realloc(L->ds, sizeof(double) * cap);
    L->dX = (double *)realloc(L->dX, sizeof(double) * cap);
    L->dY = (double *)realloc(L->dY, sizeof(double) * cap);
    L->mbody = (int *)realloc(L->mbody, sizeof(int) * cap);
    L->mcap = cap;
  }
  if (L->nb + 1 > L->bcap) {
    L->bcap = (L->nb + 1) * 2;
    L->bodies = (ora_body *)realloc(L->bodies, sizeof(ora_body) * L->bcap);
  }
  ora_body *B = &L->bodies[L->nb];
  memset(B, 0, sizeof(*B));
  B->kind = kind;
  B->xc[0] = bd[0]; B->xc[1] = bd[1];
  B->u[0] = bd[2]; B->u[1] = bd[3];
  B->omega = bd[4]; B->theta = bd[5];
  B->rho_s = bd[6]; B->rho_f = bd[7];
  B->volume = bd[8]; B->inertia = bd[9]; B->radius = bd[10];
  B->gravity[0] = bd[11]; B->gravity[1] = bd[12];
  B->mass = B->rho_s * B->volume;
  B->u_prev[0] = B->u[0]; B->u_prev[1] = B->u[1];
  B->omega_prev = B->omega;
  B->theta0 = B->theta;
  B->m0 = L->nm;
  B->m1 = L->nm + n;
  for (int k = 0; k < n; ++k) {
    int l = L->nm + k;
    L->X[l] = xy[2 * k];
    L->Y[l] = xy[2 * k + 1];
    L->ds[l] = ds[k];
    L->dX[l] = L->X[l] - B->xc[0];
    L->dY[l] = L->Y[l] - B->xc[1];
    L->mbody[l] = L->nb;
  }
  L->nm += n;
  return L->nb++;
}

/* ---------------------------------------------------------------- IB loop */

/* Velocity of marker l: rigid motion of its body, U + omega x (X - xc). */
static void marker_velocity(const ora_lattice *L, int l, double *U) {
  const ora_body *B = &L->bodies[L->mbody[l]];
  if (L->Uset && B->kind == ORA_BODY_FIXED) {
    U[0] = L->Uset[2 * l];
    U[1] = L->Uset[2 * l + 1];
    return;
  }
  U[0] = B->u[0] - B->omega * (L->Y[l] - B->xc[1]);
  U[1] = B->u[1] + B->omega * (L->X[l] - B->xc[0]);
}

/* Prescribe the velocity U_l of Eq. 24 marker by marker (interleaved u_x,
 * u_y for all markers) for markers of fixed bodies, from the next step on;
 * a time-dependent boundary sets it before every step. */
int ora_set_marker_velocities(ora_lattice *L, const double *uv, int n) {
  if (n != L->nm) return -1;
  double *u = (double *)realloc(L->Uset, sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
  if (!u) return -1;
  L->Uset = u;
  for (int k = 0; k < 2 * n; ++k) L->Uset[k] = uv[k];
  return 0;
}

/* Lattice index of stencil coordinate c along an axis of length n, or -1
 * when it falls outside a non-periodic domain (skipped). */
static int axis_node(int c, int n, int periodic) {
  if (periodic) {
    int r = c % n;
    return r < 0 ? r + n : r;
  }
  return (c < 0 || c >= n) ? -1 : c;
}

/* The velocity part of Eq. 3: f_i^eq(rho, u) = w_i rho (1 + psi_i(u)). */
static double psi(int i, double ux, double uy) {
  double eu = ora_ex[i] * ux + ora_ey[i] * uy;
  return 3.0 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy);
}

/* Eq. 22b with Eq. 28: interpolation of the nodal equilibria
 * f_i^eq(rho(x), u(x)) = w_i rho(x) + w_i rho(x) psi_i(u(x)) over the 4 x 4
 * support, in row-major node order.  Returns the interpolated density
 * rho* = sum_x D rho(x) and fills phi_i = sum_x D w_i rho(x) psi_i(u(x)),
 * so that (f_i^eq)* = w_i rho* + phi_i.  (Alternative reading
 * rd_interp_moments: the equilibrium of the interpolated moments,
 * phi_i = w_i rho* psi_i(j* / rho*) with j* = sum_x D j(x).) */
static double interpolate_feq(const ora_lattice *L, int l, double *phi) {
  int px = L->bc[0] == ORA_PERIODIC, py = L->bc[2] == ORA_PERIODIC;
  int bx = (int)floor(L->X[l]) - 1, by = (int)floor(L->Y[l]) - 1;
  double rs = 0.0, jsx = 0.0, jsy = 0.0;
  for (int i = 0; i < ORA_Q; ++i) phi[i] = 0.0;
  for (int b = 0; b < 4; ++b) {
    int y = axis_node(by + b, L->ny, py);
    if (y < 0) continue;
    double wy = delta_of(L, L->Y[l] - (double)(by + b));
    for (int a = 0; a < 4; ++a) {
      int x = axis_node(bx + a, L->nx, px);
      if (x < 0) continue;
      double wx = delta_of(L, L->X[l] - (double)(bx + a));
      double p[ORA_Q], rho, jx, jy;
      node_pops(L, L->f, x, y, p);
      ora_moments(p, &rho, &jx, &jy);
      double W = wx * wy;
      rs += W * rho;
      if (L->rd_interp_moments) {
        jsx += W * jx;
        jsy += W * jy;
      } else {
        for (int i = 0; i < ORA_Q; ++i)
          phi[i] += W * (ora_w[i] * rho * psi(i, jx / rho, jy / rho));
      }
    }
  }
  if (L->rd_interp_moments)
    for (int i = 0; i < ORA_Q; ++i) phi[i] = ora_w[i] * rs * psi(i, jsx / rs, jsy / rs);
  return rs;
}

/* Residual of marker l: | (rho u)* / rho* - U_l | from interpolated equilibria. */
static double marker_residual(const double *fs, const double *U) {
  double rho = 0.0, jx = 0.0, jy = 0.0;
  for (int i = 0; i < ORA_Q; ++i) {
    rho += fs[i];
    jx += ora_ex[i] * fs[i];
    jy += ora_ey[i] * fs[i];
  }
  double dx = jx / rho - U[0], dy = jy / rho - U[1];
  return sqrt(dx * dx + dy * dy);
}

/* Interpolation at marker l: fills (f_i^eq)*_l and, when dfm is given, the
 * deviation of Eq. 28 there; returns the marker's residual.
 *   delta f_i = f_i^eq(rho_b, U_l) - (f_i^eq)*
 *             = w_i (rho_b - rho*) + w_i rho_b psi_i(U_l) - phi_i.
 * With rho_b = rho* (the interpolated density of Eq. 24) the density parts
 * of the two equilibria are the same number and cancel exactly, so a state
 * at rest with markers at rest gets no correction at all. */
static double marker_deviation(const ora_lattice *L, int l, double *dfm) {
  double phi[ORA_Q], fs[ORA_Q], U[2];
  double rs = interpolate_feq(L, l, phi);
  for (int i = 0; i < ORA_Q; ++i) fs[i] = ora_w[i] * rs + phi[i];
  marker_velocity(L, l, U);
  double rl = marker_residual(fs, U);
  if (dfm) {
    double rho_b = L->rd_rho_b_ref ? L->rho0 : rs;   /* Eq. 24 */
    for (int i = 0; i < ORA_Q; ++i)                  /* Eq. 28 */
      dfm[i] = ora_w[i] * (rho_b - rs) + ora_w[i] * rho_b * psi(i, U[0], U[1]) - phi[i];
  }
  return rl;
}

/* Arc-length weight of marker l in Eq. 26 (and in the force of Eq. 29). */
static double marker_ds(const ora_lattice *L, int l) {
  return L->rd_unit_ds ? 1.0 : L->ds[l];
}

/* One correction iteration n (Eqs. 22-27 with Eq. 28), all markers at once.
 * Returns r^n, the largest marker residual before the correction. */
static double ib_iteration(ora_lattice *L, double *dfm) {
  int px = L->bc[0] == ORA_PERIODIC, py = L->bc[2] == ORA_PERIODIC;
  size_t n = (size_t)L->nx * L->ny;
  double r = 0.0;
  /* Interpolation and deviation at every marker, all from the same f^n. */
#pragma omp parallel for schedule(static) reduction(max : r)
  for (int l = 0; l < L->nm; ++l) {
    double rl = marker_deviation(L, l, dfm + (size_t)l * ORA_Q);
    if (rl > r) r = rl;
  }
  /* Eq. 26: spread every deviation, markers in ascending order. */
#pragma omp parallel for schedule(static)
  for (size_t k = 0; k < ORA_Q * n; ++k) L->df[k] = 0.0;
  for (int l = 0; l < L->nm; ++l) {
    int bx = (int)floor(L->X[l]) - 1, by = (int)floor(L->Y[l]) - 1;
    for (int b = 0; b < 4; ++b) {
      int y = axis_node(by + b, L->ny, py);
      if (y < 0) continue;
      double wy = delta_of(L, L->Y[l] - (double)(by + b));
      for (int a = 0; a < 4; ++a) {
        int x = axis_node(bx + a, L->nx, px);
        if (x < 0) continue;
        double wx = delta_of(L, L->X[l] - (double)(bx + a));
        double W = wx * wy * marker_ds(L, l);
        for (int i = 0; i < ORA_Q; ++i)
          L->df[idx(L, i, x, y)] += W * dfm[(size_t)l * ORA_Q + i];
      }
    }
  }
  /* Eq. 27: correct the distribution functions once. */
#pragma omp parallel for schedule(static)
  for (size_t k = 0; k < ORA_Q * n; ++k) L->f[k] += L->df[k];
  /* Eq. 29, read along its sums: force on each body from the marker
   * deviations (sum over directions of e_i delta f, weighted by the arc
   * length that the spreading gave them), and the same sum taken over the
   * Eulerian nodes as a cross-check. */
  for (int l = 0; l < L->nm; ++l) {
    ora_body *B = &L->bodies[L->mbody[l]];
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < ORA_Q; ++i) {
      sx += ora_ex[i] * dfm[(size_t)l * ORA_Q + i];
      sy += ora_ey[i] * dfm[(size_t)l * ORA_Q + i];
    }
    double Fx = -marker_ds(L, l) * sx, Fy = -marker_ds(L, l) * sy;
    B->F_ib[0] += Fx;
    B->F_ib[1] += Fy;
    /* Eq. 38: torque of the same force about the mass centre */
    B->T_ib += (L->X[l] - B->xc[0]) * Fy - (L->Y[l] - B->xc[1]) * Fx;
  }
#pragma omp parallel for schedule(static)
  for (int y = 0; y < L->ny; ++y) {
    double sx = 0.0, sy = 0.0;
    for (int x = 0; x < L->nx; ++x)
      for (int i = 0; i < ORA_Q; ++i) {
        sx -= ora_ex[i] * L->df[idx(L, i, x, y)];
        sy -= ora_ey[i] * L->df[idx(L, i, x, y)];
      }
    L->rowF[2 * y] = sx;
    L->rowF[2 * y + 1] = sy;
  }
  for (int y = 0; y < L->ny; ++y) {   /* rows added in order */
    L->F_euler[0] += L->rowF[2 * y];
    L->F_euler[1] += L->rowF[2 * y + 1];
  }
  return r;
}

/* The whole correction loop of one step; records r^0..r^N. */
void ora_ib_correct(ora_lattice *L) {
  for (int b = 0; b < L->nb; ++b) {
    L->bodies[b].F_ib[0] = L->bodies[b].F_ib[1] = 0.0;
    L->bodies[b].T_ib = 0.0;
  }
  L->F_euler[0] = L->F_euler[1] = 0.0;
  if (L->nm == 0) {
    for (int k = 0; k <= L->n_corr; ++k) L->resid[k] = 0.0;
    return;
  }
  double *dfm = (double *)malloc(sizeof(double) * ORA_Q * (size_t)L->nm);
  for (int it = 0; it < L->n_corr; ++it) L->resid[it] = ib_iteration(L, dfm);
  /* final residual from one more interpolation, no correction */
  double r = 0.0;
#pragma omp parallel for schedule(static) reduction(max : r)
  for (int l = 0; l < L->nm; ++l) {
    double rl = marker_deviation(L, l, NULL);
    if (rl > r) r = rl;
  }
  L->resid[L->n_corr] = r;
  free(dfm);
}

/* ---------------------------------------------------------------- bodies */

/* Wall coordinate of side s for the mirror particle of Eq. 39: half-way
 * walls sit half a spacing outside the first and last nodes. */
static double wall_coord(const ora_lattice *L, int s) {
  switch (s) {
    case 0: return -0.5;
    case 1: return (double)L->nx - 0.5;
    case 2: return -0.5;
    default: return (double)L->ny - 0.5;
  }
}

/* Eq. 39: repulsive force on body i from a partner at distance vector d
 * (x_i - x_j), with threshold xi = 0.05 D_i and force scale c_ij the net
 * buoyancy-reduced weight of body i. */
static void collision_force(const ora_body *Bi, double Rj, double dx,
                            double dy, double *F) {
  double eps_c = 0.01;
  double xi = 0.05 * 2.0 * Bi->radius;
  double gmag = sqrt(Bi->gravity[0] * Bi->gravity[0] +
                     Bi->gravity[1] * Bi->gravity[1]);
  double c = Bi->mass * (1.0 - Bi->rho_f / Bi->rho_s) * gmag;
  double d = sqrt(dx * dx + dy * dy);
  if (d > Bi->radius + Rj + xi || d <= 0.0) return;
  double s = (d - Bi->radius - Rj - xi) / xi;
  F[0] += c / eps_c * s * s * dx / d;
  F[1] += c / eps_c * s * s * dy / d;
}

/* Eqs. 37-42 for every free body, then rigid motion of all moving markers. */
void ora_move_bodies(ora_lattice *L) {
  for (int b = 0; b < L->nb; ++b) {
    ora_body *B = &L->bodies[b];
    B->F_c[0] = B->F_c[1] = 0.0;
    if (B->kind != ORA_BODY_FREE) continue;
    for (int o = 0; o < L->nb; ++o) {
      if (o == b || L->bodies[o].kind != ORA_BODY_FREE) continue;
      collision_force(B, L->bodies[o].radius, B->xc[0] - L->bodies[o].xc[0],
                      B->xc[1] - L->bodies[o].xc[1], B->F_c);
    }
    for (int s = 0; s < 4; ++s) {
      if (L->bc[s] != ORA_BOUNCEBACK && L->bc[s] != ORA_FREESLIP) continue;
      double w = wall_coord(L, s);
      if (s < 2) { /* mirror across x = w */
        double xm = 2.0 * w - B->xc[0];
        collision_force(B, B->radius, B->xc[0] - xm, 0.0, B->F_c);
      } else {
        double ym = 2.0 * w - B->xc[1];
        collision_force(B, B->radius, 0.0, B->xc[1] - ym, B->F_c);
      }
    }
  }
  for (int b = 0; b < L->nb; ++b) {
    ora_body *B = &L->bodies[b];
    if (B->kind == ORA_BODY_FREE) {
      /* Eq. 37: hydrodynamic force plus the internal-mass term (lagged
       * explicit derivative); Eq. 40: collision force and net weight. */
      double Ft[2], Tt;
      for (int d = 0; d < 2; ++d)
        Ft[d] = B->F_ib[d] + B->rho_f * B->volume * (B->u[d] - B->u_prev[d]) +
                B->F_c[d] + B->mass * (1.0 - B->rho_f / B->rho_s) * B->gravity[d];
      /* Eq. 38 */
      Tt = B->T_ib + B->rho_f / B->rho_s * B->inertia * (B->omega - B->omega_prev);
      double un[2] = {B->u[0], B->u[1]}, wn = B->omega;
      /* Eq. 42 (uses u^n) then Eq. 41 */
      for (int d = 0; d < 2; ++d) B->xc[d] += un[d] + 0.5 * Ft[d] / B->mass;
      B->theta += wn + 0.5 * Tt / B->inertia;
      for (int d = 0; d < 2; ++d) {
        B->u_prev[d] = un[d];
        B->u[d] = un[d] + Ft[d] / B->mass;
      }
      B->omega_prev = wn;
      B->omega = wn + Tt / B->inertia;
    } else if (B->kind == ORA_BODY_PRESCRIBED) {
      for (int d = 0; d < 2; ++d) B->xc[d] += B->u[d];
      B->theta += B->omega;
    } else {
      continue;
    }
    double c = cos(B->theta - B->theta0), s = sin(B->theta - B->theta0);
    for (int l = B->m0; l < B->m1; ++l) {
      L->X[l] = B->xc[0] + c * L->dX[l] - s * L->dY[l];
      L->Y[l] = B->xc[1] + s * L->dX[l] + c * L->dY[l];
    }
  }
}

/* ---------------------------------------------------------------- LBM */

static int is_open(int bc) {
  return bc == ORA_INLET_EQ || bc == ORA_OUTLET_ZEROGRAD || bc == ORA_INLET_NEE ||
         bc == ORA_OUTLET_NEE;
}

/* Non-equilibrium extrapolation (the velocity and pressure boundary scheme
 * the paper uses at the inlet and outlet of section 3.2): the whole
 * post-stream state of a boundary node x_b is rebuilt from its inner
 * neighbour x_f as
 *     f_i(x_b) = f_i^eq(rho_b, u_b) + [f_i(x_f) - f_i^eq(rho(x_f), u(x_f))].
 * Inlet (-x side, column 0 from column 1): u_b = U_in, rho_b = rho(x_f).
 * Outlet (+x side, column nx-1 from column nx-2): rho_b = rho0,
 * u_b = u(x_f).  The rebuilt node then collides and streams like any other;
 * populations it would receive from outside are never read. */
void ora_open_boundaries(ora_lattice *L) {
  int nx = L->nx;
  for (int side = 0; side < 2; ++side) {
    if (L->bc[side] != (side == 0 ? ORA_INLET_NEE : ORA_OUTLET_NEE)) continue;
    int xb = side == 0 ? 0 : nx - 1, xf = side == 0 ? 1 : nx - 2;
    for (int y = 0; y < L->ny; ++y) {
      double p[ORA_Q], rho, jx, jy, fe_f[ORA_Q], fe_b[ORA_Q];
      node_pops(L, L->f, xf, y, p);
      ora_moments(p, &rho, &jx, &jy);
      ora_feq(rho, jx / rho, jy / rho, fe_f);
      if (side == 0)
        ora_feq(rho, L->inlet_u[0], L->inlet_u[1], fe_b);
      else
        ora_feq(L->rho0, jx / rho, jy / rho, fe_b);
      for (int i = 0; i < ORA_Q; ++i) L->f[idx(L, i, xb, y)] = fe_b[i] + (p[i] - fe_f[i]);
    }
  }
}

static int find_dir(int ex, int ey) {
  for (int i = 0; i < ORA_Q; ++i)
    if (ora_ex[i] == ex && ora_ey[i] == ey) return i;
  return -1;
}

/* Records the moments of the current (corrected) state, Eq. 7. Inlet
 * nodes are held at the inlet equilibrium. */
void ora_record_moments(ora_lattice *L) {
  size_t n = (size_t)L->nx * L->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < L->ny; ++y)
    for (int x = 0; x < L->nx; ++x) {
      size_t k = (size_t)y * L->nx + x;
      if (x == 0 && L->bc[0] == ORA_INLET_EQ) {
        L->rho[k] = L->rho0;
        L->ux[k] = L->inlet_u[0];
        L->uy[k] = L->inlet_u[1];
        continue;
      }
      double p[ORA_Q], rho, jx, jy;
      node_pops(L, L->f, x, y, p);
      ora_moments(p, &rho, &jx, &jy);
      L->rho[k] = rho;
      L->ux[k] = jx / rho;
      L->uy[k] = jy / rho;
    }
  (void)n;
}

/* BGK collision (Eq. 1 with Omega_i = -(f_i - f_i^eq)/tau), or MRT (Eq. 2)
 * after ora_set_mrt, followed by
 * streaming with the boundary rules:
 *   periodic: wrap;
 *   bounce-back (half-way): a population leaving through the wall returns
 *     to the same node reversed, minus 6 w_i rho0 (e_i . U_w) for a moving
 *     wall;
 *   free-slip: specular reflection of the normal component;
 *   inlet (-x side): the first column is held at f^eq(rho0, U_in);
 *   outlet (+x side): the populations entering from outside are copied from
 *     column nx-2;
 *   extrapolation sides: nothing here (ora_open_boundaries rebuilds the
 *     boundary column before the collision).
 * Populations leaving through an open side are dropped. */
/* Post-collision populations of node (x, y): BGK (Eq. 1) or MRT (Eq. 2)
 * toward the equilibrium of Eq. 3; an equilibrium-inlet node is held at
 * f^eq(rho0, U_in). */
static void collide_node(const ora_lattice *L, const double *feq_in, int x, int y,
                         double *ps) {
  if (x == 0 && L->bc[0] == ORA_INLET_EQ) {
    for (int i = 0; i < ORA_Q; ++i) ps[i] = feq_in[i];
    return;
  }
  double p[ORA_Q], rho, jx, jy, feq[ORA_Q];
  node_pops(L, L->f, x, y, p);
  ora_moments(p, &rho, &jx, &jy);
  ora_feq(rho, jx / rho, jy / rho, feq);
  if (L->mrt)
    ora_mrt_collide(L->s_rate, p, feq, ps);
  else
    for (int i = 0; i < ORA_Q; ++i) ps[i] = p[i] - (p[i] - feq[i]) / L->tau;
}

/* Streaming (Eq. 1) of the post-collision populations ps of node (x, y)
 * into L->g with the boundary rules listed above ora_collide_stream.  Every
 * target slot has exactly one source, so nodes may stream in any order. */
static void stream_node(ora_lattice *L, int x, int y, const double *ps) {
  int nx = L->nx, ny = L->ny;
  for (int i = 0; i < ORA_Q; ++i) {
    int tx = x + ora_ex[i], ty = y + ora_ey[i];
    int sx = tx < 0 ? 0 : (tx >= nx ? 1 : -1);
    int sy = ty < 0 ? 2 : (ty >= ny ? 3 : -1);
    if (sx >= 0 && L->bc[sx] == ORA_PERIODIC) { tx = (tx + nx) % nx; sx = -1; }
    if (sy >= 0 && L->bc[sy] == ORA_PERIODIC) { ty = (ty + ny) % ny; sy = -1; }
    if (sx < 0 && sy < 0) {
      L->g[idx(L, i, tx, ty)] = ps[i];
    } else if ((sx >= 0 && is_open(L->bc[sx])) || (sy >= 0 && is_open(L->bc[sy]))) {
      /* leaves through an open side */
    } else if (sx < 0 && L->bc[sy] == ORA_FREESLIP) {
      L->g[idx(L, find_dir(ora_ex[i], -ora_ey[i]), tx, y)] = ps[i];
    } else if (sy < 0 && L->bc[sx] == ORA_FREESLIP) {
      L->g[idx(L, find_dir(-ora_ex[i], ora_ey[i]), x, ty)] = ps[i];
    } else {
      int s = sy >= 0 ? sy : sx;
      double eu = ora_ex[i] * L->wall_u[s][0] + ora_ey[i] * L->wall_u[s][1];
      L->g[idx(L, find_dir(-ora_ex[i], -ora_ey[i]), x, y)] =
          ps[i] - 6.0 * ora_w[i] * L->rho0 * eu;
    }
  }
}

static void stream_begin(ora_lattice *L) {
  size_t n = (size_t)L->nx * L->ny;
#pragma omp parallel for schedule(static)
  for (size_t k = 0; k < ORA_Q * n; ++k) L->g[k] = NAN;
}

/* Outlet copy and inlet hold after streaming, then g becomes f. */
static void stream_end(ora_lattice *L, const double *feq_in) {
  int nx = L->nx, ny = L->ny;
  if (L->bc[1] == ORA_OUTLET_ZEROGRAD && nx >= 2)
    for (int y = 0; y < ny; ++y)
      for (int i = 0; i < ORA_Q; ++i)
        if (ora_ex[i] < 0) L->g[idx(L, i, nx - 1, y)] = L->g[idx(L, i, nx - 2, y)];
  if (L->bc[0] == ORA_INLET_EQ)
    for (int y = 0; y < ny; ++y)
      for (int i = 0; i < ORA_Q; ++i) L->g[idx(L, i, 0, y)] = feq_in[i];
  double *t = L->f;
  L->f = L->g;
  L->g = t;
}

/* BGK collision (Eq. 1 with Omega_i = -(f_i - f_i^eq)/tau), or MRT (Eq. 2)
 * after ora_set_mrt, followed by
 * streaming with the boundary rules:
 *   periodic: wrap;
 *   bounce-back (half-way): a population leaving through the wall returns
 *     to the same node reversed, minus 6 w_i rho0 (e_i . U_w) for a moving
 *     wall;
 *   free-slip: specular reflection of the normal component;
 *   inlet (-x side): the first column is held at f^eq(rho0, U_in);
 *   outlet (+x side): the populations entering from outside are copied from
 *     column nx-2;
 *   extrapolation sides: nothing here (ora_open_boundaries rebuilds the
 *     boundary column before the collision).
 * Populations leaving through an open side are dropped. */
void ora_collide_stream(ora_lattice *L) {
  double feq_in[ORA_Q];
  ora_feq(L->rho0, L->inlet_u[0], L->inlet_u[1], feq_in);
  stream_begin(L);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < L->ny; ++y)
    for (int x = 0; x < L->nx; ++x) {
      double ps[ORA_Q];
      collide_node(L, feq_in, x, y, ps);
      stream_node(L, x, y, ps);
    }
  stream_end(L, feq_in);
}

/* Alternative reading rd_post_collision: the correction loop acts on the
 * post-collision populations, between the collision and the streaming. */
static void step_post_collision(ora_lattice *L) {
  double feq_in[ORA_Q];
  ora_feq(L->rho0, L->inlet_u[0], L->inlet_u[1], feq_in);
  ora_open_boundaries(L);
  ora_record_moments(L);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < L->ny; ++y)
    for (int x = 0; x < L->nx; ++x) {
      double ps[ORA_Q];
      collide_node(L, feq_in, x, y, ps);
      for (int i = 0; i < ORA_Q; ++i) L->f[idx(L, i, x, y)] = ps[i];
    }
  ora_ib_correct(L);
  ora_move_bodies(L);
  stream_begin(L);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < L->ny; ++y)
    for (int x = 0; x < L->nx; ++x) {
      double ps[ORA_Q];
      node_pops(L, L->f, x, y, ps);
      stream_node(L, x, y, ps);
    }
  stream_end(L, feq_in);
}

/* One full time step in the order stated at the top of this file. */
void ora_step(ora_lattice *L, int nsteps) {
  for (int s = 0; s < nsteps; ++s) {
    if (L->rd_post_collision) {
      step_post_collision(L);
    } else {
      ora_ib_correct(L);
      ora_move_bodies(L);
      ora_open_boundaries(L);
      ora_record_moments(L);
      ora_collide_stream(L);
    }
    L->steps++;
  }
}

/* Selects alternative readings of section 2.3 (each 0 or 1; all 0 is the
 * default reading): equilibria of interpolated moments, rho_b = rho0,
 * correction of the post-collision populations, spreading without ds. */
void ora_set_reading(ora_lattice *L, int interp_moments, int rho_b_ref,
                     int post_collision, int unit_ds) {
  L->rd_interp_moments = interp_moments;
  L->rd_rho_b_ref = rho_b_ref;
  L->rd_post_collision = post_collision;
  L->rd_unit_ds = unit_ds;
}

/* Host threads of the -fopenmp build (0: all cores); returns the count in
 * use, always 1 in the serial build. */
int ora_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ---------------------------------------------------------------- access */

void ora_get_f(const ora_lattice *L, double *out) {
  memcpy(out, L->f, sizeof(double) * ORA_Q * (size_t)L->nx * L->ny);
}
void ora_set_f(ora_lattice *L, const double *in) {
  memcpy(L->f, in, sizeof(double) * ORA_Q * (size_t)L->nx * L->ny);
}
/* f := f^eq(rho, u) node by node (Eq. 3); the moments are recorded too. */
void ora_init_equilibrium(ora_lattice *L, const double *rho, const double *ux,
                          const double *uy) {
  size_t n = (size_t)L->nx * L->ny;
  for (size_t k = 0; k < n; ++k) {
    double feq[ORA_Q];
    ora_feq(rho[k], ux[k], uy[k], feq);
    for (int i = 0; i < ORA_Q; ++i) L->f[(size_t)i * n + k] = feq[i];
    L->rho[k] = rho[k];
    L->ux[k] = ux[k];
    L->uy[k] = uy[k];
  }
}
void ora_get_moments(const ora_lattice *L, double *rho, double *ux, double *uy) {
  size_t n = (size_t)L->nx * L->ny;
  memcpy(rho, L->rho, sizeof(double) * n);
  memcpy(ux, L->ux, sizeof(double) * n);
  memcpy(uy, L->uy, sizeof(double) * n);
}
void ora_get_resid(const ora_lattice *L, double *out) {
  memcpy(out, L->resid, sizeof(double) * ((size_t)L->n_corr + 1));
}
/* Per body: xc, yc, ux, uy, omega, theta, Fx, Fy, T (the Eq. 29 sums of the
 * last step, without the internal-mass terms). */
void ora_get_bodies(const ora_lattice *L, double *out) {
  for (int b = 0; b < L->nb; ++b) {
    const ora_body *B = &L->bodies[b];
    double *o = out + 9 * b;
    o[0] = B->xc[0]; o[1] = B->xc[1]; o[2] = B->u[0]; o[3] = B->u[1];
    o[4] = B->omega; o[5] = B->theta; o[6] = B->F_ib[0]; o[7] = B->F_ib[1];
    o[8] = B->T_ib;
  }
}
void ora_get_markers(const ora_lattice *L, double *xy) {
  for (int l = 0; l < L->nm; ++l) {
    xy[2 * l] = L->X[l];
    xy[2 * l + 1] = L->Y[l];
  }
}
void ora_get_force_euler(const ora_lattice *L, double *out) {
  out[0] = L->F_euler[0];
  out[1] = L->F_euler[1];
}
int ora_num_markers(const ora_lattice *L) { return L->nm; }
int ora_num_bodies(const ora_lattice *L) { return L->nb; }
