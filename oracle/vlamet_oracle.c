/*
 * FP64 CPU oracle of the metric semi-Lagrangian Vlasov-Poisson step.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  Plain, serial
 * (optional OpenMP over independent sites), FP64 throughout, written from
 * the paper in its order and notation:
 *   Sec. 2.1    elements of metric, second-order forward/inverse map
 *   Sec. 2.2.1  six-point quadratic interpolation (transport)
 *   Sec. 2.2.2  cubic B-spline interpolation, f = 0 and df = 0 at the edges
 *   Sec. 2.3.1  percolation (influence map), alpha ranges, unexplored sites
 *   Sec. 2.3.2  smooth blended map Q_r with the Monaghan kernel, beta ranges
 *   Sec. 2.4    equations of motion and the drift-kick-drift scheme
 *   Sec. 2.5    pixel masses, mass-scan force, finite differences, TSC
 *   Sec. 3.2    energy diagnostic
 *
 * Floating-point evaluation order is fixed and documented at each formula
 * (build with -ffp-contract=off so no multiply-add is fused): decisions
 * that turn a double into an integer (nearest node, ranges, the d
 * comparisons of the percolation) are exactly reproducible this way.
 *
 * Readings where the paper is silent or garbled (each is listed with its
 * justification in the design notes of the repository):
 *   node-centred fixed box; lattice centred on the box; distance normalised
 *   by the element spacing; minus-neighbour terms of the quadratic formula
 *   use the Lagrange form on {-1,0,1}; a' uses 2*dx (parabola fit); T kick
 *   adds to T_v (not T_x); per-element "processed" set; overlaps resolved by
 *   min d, then min element index; holes filled by Jacobi rounds from the
 *   4-neighbours; the spline is the finite B-spline sum evaluated
 *   everywhere (no cut at the box edge); force factor 2*pi*G.
 *
 * Parity status: every function here is pinned by a test against a closed
 * form, an invariant or brute force.  The smooth map Q_r and E_map are
 * pinned on hand-built states of displaced isotropic elements, whose
 * blended positions and mismatches are simple fractions worked out by hand,
 * and Q_r's continuity across ownership boundaries is checked under grid
 * refinement for a curved flow.
 */
#include "vlamet_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

typedef struct {
  double x, v, Txx, Txv, Tvx, Tvv;
  double Hx[3]; /* Hx_xx, Hx_xv, Hx_vv */
  double Hv[3]; /* Hv_xx, Hv_xv, Hv_vv */
} elem_t;

typedef struct {
  double x, v;          /* P_m */
  double Ti[4];         /* T^-1 row major: Ti00 Ti01 Ti10 Ti11 */
  double Gx[3], Gv[3];  /* [T^-1]^T H_l T^-1, symmetric: 00 01 11 */
  double Qx, Qv;        /* Q_m */
} taylor_t;

struct vo_state {
  vo_config c;
  double dx, dv, dxm, dvm, inv_dx, inv_dv, inv_dxm, inv_dvm, cx, cv;
  int32_t Kx, Kv, Lx, Lv, ne;
  double *fini, *eta, *f;
  elem_t* el;
  taylor_t* tay;
  int32_t* map;
  double *M, *a, *da, *d2a;
  double Mtot;
  int64_t nstep;
  int32_t cyc;
  int32_t have_f;
  double c_dyn;  /* > 0: variable time step (Sec. 2.4), Delta t = min(dt, c_dyn / sqrt(rho_max)) */
  double time;   /* sum of the steps taken since vo_set_f */
  double last_dt;
  /* adaptive computing domain (Sec. 2.2.1, eq. constrf; Sec. 2.3): f_th > 0
   * restricts f_ini to the rectangle of nodes where |f_ini| > f_th; elements
   * exist on the lattice rows klo..khi and columns llo..lhi covering it plus
   * one extra layer; each map's sites are those of the rectangle spanned by
   * the existing elements' positions (rect: i_lo, i_hi, j_lo, j_hi) */
  double f_th;
  int32_t klo, khi, llo, lhi;
  int32_t rect[4];
  /* percolation scratch */
  int32_t* stamp;
  int32_t* queue;
  uint64_t* bestkey;
  int32_t* prevmap;
  int64_t stat_multi, stat_holes;
  int32_t stat_rounds;
  int32_t* bbox; /* per element: i_min, i_max, j_min, j_max of its component */
};

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static uint64_t dbits(double d) {
  uint64_t u;
  memcpy(&u, &d, sizeof u);
  return u;
}

/* Nearest integer with halves rounded up: floor(u + 0.5). */
static int64_t nearest(double u) { return (int64_t)floor(u + 0.5); }

/* ------------------------------------------------------------------ */
/* Sec. 2.2.1: six-point quadratic interpolation                        */
/* ------------------------------------------------------------------ */

static double Fat(const double* F, int32_t nx, int32_t nv, int64_t i, int64_t j) {
  if (i < 0 || j < 0 || i >= nx || j >= nv) return 0.0;
  return F[i * nv + j];
}

/* Interpolate the node values F at index coordinates (u, w): nearest node
 * (i_n, j_n), its 5-point cross, and the corner of the square that contains
 * the point, found from the integer parts (i_c, j_c).  The minus-neighbour
 * terms use the Lagrange weights dq(dq-1)/2 on {-1,0,1} (the printed sign
 * and the printed (i_n-1, j_n) in the v term are read as typesetting slips:
 * with them the formula does not pass through F at dq = -1).  Nodes outside
 * the grid read 0. */
double vo_qinterp(const double* F, int32_t nx, int32_t nv, double u, double w) {
  if (!(u > -2.0 && u < (double)nx + 1.0 && w > -2.0 && w < (double)nv + 1.0)) return 0.0;
  int64_t in = nearest(u), jn = nearest(w);
  int64_t ic = (int64_t)floor(u), jc = (int64_t)floor(w);
  double dqx = u - (double)in;
  double dqv = w - (double)jn;
  double f = Fat(F, nx, nv, in, jn) * ((1.0 - dqx * dqx) - dqv * dqv);
  f = f + ((0.5 * Fat(F, nx, nv, in + 1, jn)) * dqx) * (1.0 + dqx);
  f = f + ((0.5 * Fat(F, nx, nv, in - 1, jn)) * dqx) * (dqx - 1.0);
  f = f + ((0.5 * Fat(F, nx, nv, in, jn + 1)) * dqv) * (1.0 + dqv);
  f = f + ((0.5 * Fat(F, nx, nv, in, jn - 1)) * dqv) * (dqv - 1.0);
  double cross = ((Fat(F, nx, nv, ic + 1, jc + 1) + Fat(F, nx, nv, ic, jc)) -
                  Fat(F, nx, nv, ic + 1, jc)) - Fat(F, nx, nv, ic, jc + 1);
  f = f + (cross * dqx) * dqv;
  return f;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2.2: cubic B-splines with f' = 0 at both end nodes            */
/* ------------------------------------------------------------------ */

/* Uniform cubic B-spline centred at 0, support [-2, 2]. */
double vo_bspline3(double t) {
  t = fabs(t);
  if (t < 1.0) return (2.0 / 3.0 - t * t) + 0.5 * (t * t * t);
  if (t < 2.0) {
    double r = 2.0 - t;
    return (r * r * r) / 6.0;
  }
  return 0.0;
}

/* Coefficients eta_0..eta_{n-1} such that sum_k eta_k B(i-k) = f_i at every
 * node, with ghosts eta_{-1} = eta_1 and eta_n = eta_{n-2} (zero slope at both
 * end nodes).  Rows, multiplied by 6: 4 eta_0 + 2 eta_1 = 6 f_0;
 * eta_{i-1} + 4 eta_i + eta_{i+1} = 6 f_i; 2 eta_{n-2} + 4 eta_{n-1} = 6 f_{n-1}.
 * Solved by the Thomas algorithm (the matrix is strictly diagonally
 * dominant). */
void vo_spline_solve_1d(int32_t n, const double* f, double* eta) {
  if (n < 1) return;
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  double* dp = (double*)malloc(sizeof(double) * (size_t)n);
  for (int32_t i = 0; i < n; i++) {
    double sub = (i == 0) ? 0.0 : ((i == n - 1) ? 2.0 : 1.0);
    double sup = (i == n - 1) ? 0.0 : ((i == 0) ? 2.0 : 1.0);
    double dia = 4.0;
    double rhs = 6.0 * f[i];
    if (i == 0) {
      cp[i] = sup / dia;
      dp[i] = rhs / dia;
    } else {
      double den = dia - sub * cp[i - 1];
      cp[i] = sup / den;
      dp[i] = (rhs - sub * dp[i - 1]) / den;
    }
  }
  eta[n - 1] = dp[n - 1];
  for (int32_t i = n - 2; i >= 0; i--) eta[i] = dp[i] - cp[i] * eta[i + 1];
  free(cp);
  free(dp);
}

/* Tensor product: solve along v for every x row, then along x for every v
 * column. */
void vo_spline_solve_2d(int32_t nx, int32_t nv, const double* f, double* eta) {
  double* tmp = (double*)malloc(sizeof(double) * (size_t)nx * nv);
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < nx; i++) vo_spline_solve_1d(nv, f + (size_t)i * nv, tmp + (size_t)i * nv);
#pragma omp parallel for schedule(static)
  for (int32_t j = 0; j < nv; j++) {
    double* col = (double*)malloc(sizeof(double) * (size_t)nx);
    double* out = (double*)malloc(sizeof(double) * (size_t)nx);
    for (int32_t i = 0; i < nx; i++) col[i] = tmp[(size_t)i * nv + j];
    vo_spline_solve_1d(nx, col, out);
    for (int32_t i = 0; i < nx; i++) eta[(size_t)i * nv + j] = out[i];
    free(col);
    free(out);
  }
  free(tmp);
}

/* Mirror ghost index of the coefficients: -1 -> 1, n -> n-2; anything else
 * outside [0, n) has no coefficient (returns -1). */
static int64_t ghost(int64_t k, int32_t n) {
  if (k >= 0 && k < n) return k;
  if (k == -1) return 1;
  if (k == n) return n - 2;
  return -1;
}

/* f(u, w) = sum_k sum_l eta_kl B(u-k) B(w-l), the finite sum over the
 * coefficients -1..n (ghosts by the zero-slope mirror).  It is evaluated
 * everywhere: it is C2 in (u, w) and vanishes for u <= -3 or u >= n+2, so a
 * point that rounding puts just outside an edge node gets the same value as
 * one just inside (the paper's f = 0 at the edge then holds to the
 * truncation of the initial condition). */
double vo_spline_eval(const double* eta, int32_t nx, int32_t nv, double u, double w) {
  if (!(u > -3.0 && u < (double)(nx + 2) && w > -3.0 && w < (double)(nv + 2))) return 0.0;
  int64_t ku = (int64_t)floor(u), kw = (int64_t)floor(w);
  double sum = 0.0;
  for (int64_t k = ku - 1; k <= ku + 2; k++) {
    int64_t gk = ghost(k, nx);
    if (gk < 0) continue;
    double bu = vo_bspline3(u - (double)k);
    for (int64_t l = kw - 1; l <= kw + 2; l++) {
      int64_t gl = ghost(l, nv);
      if (gl < 0) continue;
      sum = sum + (eta[gk * nv + gl] * bu) * vo_bspline3(w - (double)l);
    }
  }
  return sum;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1: Taylor terms of the inverse map                             */
/* ------------------------------------------------------------------ */

static void taylor_of(const elem_t* e, double Qx, double Qv, taylor_t* t) {
  /* det T (eq. of |T|), inverse by the adjugate times 1/det T */
  double det = e->Txx * e->Tvv - e->Txv * e->Tvx;
  double id = 1.0 / det;
  double Ti00 = e->Tvv * id, Ti01 = -e->Txv * id;
  double Ti10 = -e->Tvx * id, Ti11 = e->Txx * id;
  t->x = e->x;
  t->v = e->v;
  t->Ti[0] = Ti00;
  t->Ti[1] = Ti01;
  t->Ti[2] = Ti10;
  t->Ti[3] = Ti11;
  for (int l = 0; l < 2; l++) {
    const double* h = (l == 0) ? e->Hx : e->Hv;
    double* G = (l == 0) ? t->Gx : t->Gv;
    /* A = H_l T^-1, then G_l = [T^-1]^T A */
    double A00 = h[0] * Ti00 + h[1] * Ti10;
    double A01 = h[0] * Ti01 + h[1] * Ti11;
    double A10 = h[1] * Ti00 + h[2] * Ti10;
    double A11 = h[1] * Ti01 + h[2] * Ti11;
    G[0] = Ti00 * A00 + Ti10 * A10;
    G[1] = Ti00 * A01 + Ti10 * A11;
    G[2] = Ti01 * A01 + Ti11 * A11;
  }
  t->Qx = Qx;
  t->Qv = Qv;
}

/* Second-order inverse map, Sec. 2.1:
 *   Q - Q_m = y - (1/2) T^-1 s,  y = T^-1 dP,  s_l = dP^T G_l dP,
 * returned as the offset dQ = Q - Q_m. */
static void qofp_t(const taylor_t* t, double Px, double Pv, double* dqx, double* dqv) {
  double dPx = Px - t->x;
  double dPv = Pv - t->v;
  double yx = t->Ti[0] * dPx + t->Ti[1] * dPv;
  double yv = t->Ti[2] * dPx + t->Ti[3] * dPv;
  double g0 = t->Gx[0] * dPx + t->Gx[1] * dPv;
  double g1 = t->Gx[1] * dPx + t->Gx[2] * dPv;
  double sx = dPx * g0 + dPv * g1;
  g0 = t->Gv[0] * dPx + t->Gv[1] * dPv;
  g1 = t->Gv[1] * dPx + t->Gv[2] * dPv;
  double sv = dPx * g0 + dPv * g1;
  double cx = t->Ti[0] * sx + t->Ti[1] * sv;
  double cv = t->Ti[2] * sx + t->Ti[3] * sv;
  *dqx = yx - 0.5 * cx;
  *dqv = yv - 0.5 * cv;
}

static void elem_from12(const double* p, elem_t* e) {
  e->x = p[0];
  e->v = p[1];
  e->Txx = p[2];
  e->Txv = p[3];
  e->Tvx = p[4];
  e->Tvv = p[5];
  for (int k = 0; k < 3; k++) {
    e->Hx[k] = p[6 + k];
    e->Hv[k] = p[9 + k];
  }
}

static void elem_to12(const elem_t* e, double* p) {
  p[0] = e->x;
  p[1] = e->v;
  p[2] = e->Txx;
  p[3] = e->Txv;
  p[4] = e->Tvx;
  p[5] = e->Tvv;
  for (int k = 0; k < 3; k++) {
    p[6 + k] = e->Hx[k];
    p[9 + k] = e->Hv[k];
  }
}

static void taylor_to14(const taylor_t* t, double* p) {
  p[0] = t->x;
  p[1] = t->v;
  for (int k = 0; k < 4; k++) p[2 + k] = t->Ti[k];
  for (int k = 0; k < 3; k++) {
    p[6 + k] = t->Gx[k];
    p[9 + k] = t->Gv[k];
  }
  p[12] = t->Qx;
  p[13] = t->Qv;
}

static void taylor_from14(const double* p, taylor_t* t) {
  t->x = p[0];
  t->v = p[1];
  for (int k = 0; k < 4; k++) t->Ti[k] = p[2 + k];
  for (int k = 0; k < 3; k++) {
    t->Gx[k] = p[6 + k];
    t->Gv[k] = p[9 + k];
  }
  t->Qx = p[12];
  t->Qv = p[13];
}

void vo_taylor_one(const double* el12, double Qx, double Qv, double* tay14) {
  elem_t e;
  taylor_t t;
  elem_from12(el12, &e);
  taylor_of(&e, Qx, Qv, &t);
  taylor_to14(&t, tay14);
}

void vo_qofp(const double* tay14, double Px, double Pv, double* dqx, double* dqv) {
  taylor_t t;
  taylor_from14(tay14, &t);
  qofp_t(&t, Px, Pv, dqx, dqv);
}

/* Monaghan (1992) M4 kernel, unnormalised, Sec. 2.3.2. */
double vo_W(double x) {
  if (x <= 1.0) return (1.0 - 1.5 * (x * x)) + 0.75 * (x * x * x);
  if (x <= 2.0) {
    double r = 2.0 - x;
    return 0.25 * (r * r * r);
  }
  return 0.0;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.5: force from the pixel masses                                 */
/* ------------------------------------------------------------------ */

/* a(i) = 2 pi G [M_total - M_left(i) - M_left(i-1)], M_left(i) = sum_{m<=i} M(m).
 * Derivatives by centred differences on the parabola through i-1, i, i+1,
 * with a(-1) = +2 pi G M_total and a(nx) = -2 pi G M_total beyond the grid. */
void vo_force_from_mass(const double* M, int32_t nx, double dx, double G, int32_t literal_fd,
                        double* a, double* da, double* d2a) {
  double A = 2.0 * PI * G;
  double Mtot = 0.0;
  for (int32_t i = 0; i < nx; i++) Mtot = Mtot + M[i];
  double left_prev = 0.0, left = 0.0;
  for (int32_t i = 0; i < nx; i++) {
    left = left_prev + M[i];
    a[i] = A * ((Mtot - left) - left_prev);
    left_prev = left;
  }
  double alo = A * Mtot, ahi = -(A * Mtot);
  double twodx = literal_fd ? dx : 2.0 * dx;
  double dx2 = dx * dx;
  for (int32_t i = 0; i < nx; i++) {
    double am = (i > 0) ? a[i - 1] : alo;
    double ap = (i < nx - 1) ? a[i + 1] : ahi;
    da[i] = (ap - am) / twodx;
    d2a[i] = ((ap + am) - 2.0 * a[i]) / dx2;
  }
}

/* Dual TSC interpolation of a grid quantity at index coordinate u; values
 * beyond the grid are ext_lo (i < 0) and ext_hi (i > nx-1). */
double vo_tsc(const double* A, int32_t nx, double ext_lo, double ext_hi, double u) {
  if (!(u > -1e9 && u < 1e9)) return (u < 0.0) ? ext_lo : ext_hi;
  int64_t i = nearest(u);
  double w = u - (double)i;
  double v[3];
  for (int k = -1; k <= 1; k++) {
    int64_t ii = i + k;
    v[k + 1] = (ii < 0) ? ext_lo : ((ii >= nx) ? ext_hi : A[ii]);
  }
  double wl = 0.5 * ((0.5 - w) * (0.5 - w));
  double wc = 0.75 - w * w;
  double wr = 0.5 * ((0.5 + w) * (0.5 + w));
  return (wl * v[0] + wc * v[1]) + wr * v[2];
}

/* ------------------------------------------------------------------ */
/* state                                                               */
/* ------------------------------------------------------------------ */

static double lattice_qx(const vo_state* S, int32_t k) {
  return S->cx + (double)(k - S->Kx - 1) * S->dxm;
}
static double lattice_qv(const vo_state* S, int32_t l) {
  return S->cv + (double)(l - S->Kv - 1) * S->dvm;
}

/* Does element (k, l) exist (is it on the part of the lattice that covers
 * the computing domain)? */
static int exists(const vo_state* S, int32_t k, int32_t l) {
  return k >= S->klo && k <= S->khi && l >= S->llo && l <= S->lhi;
}

static int64_t floor_div(int64_t a, int64_t b) { /* b > 0 */
  int64_t q = a / b;
  return (q * b > a) ? q - 1 : q;
}
static int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }

/* Sec. 2.2.1, eq. constrf: the Lagrangian computing domain is the smallest
 * rectangle of nodes holding every node where |f_ini| > f_th; f_ini is cut
 * to it, and elements exist on the lattice lines that cover it (the last
 * lattice line at or before its first node and the first at or after its
 * last node, in index units (nx-1)/2 + (k-Kx-1) s, exact in integers) plus
 * one extra layer on every side (Sec. 2.3).  f_th = 0: the whole box and
 * the whole lattice. */
static void computing_domain(vo_state* S) {
  const int32_t nx = S->c.nx, nv = S->c.nv, s = S->c.s;
  if (!(S->f_th > 0.0)) {
    S->klo = 0;
    S->khi = S->Lx - 1;
    S->llo = 0;
    S->lhi = S->Lv - 1;
    return;
  }
  int32_t ilo = nx, ihi = -1, jlo = nv, jhi = -1;
  for (int32_t i = 0; i < nx; i++)
    for (int32_t j = 0; j < nv; j++)
      if (fabs(S->fini[(size_t)i * nv + j]) > S->f_th) {
        if (i < ilo) ilo = i;
        if (i > ihi) ihi = i;
        if (j < jlo) jlo = j;
        if (j > jhi) jhi = j;
      }
  for (int32_t i = 0; i < nx; i++)
    for (int32_t j = 0; j < nv; j++)
      if (i < ilo || i > ihi || j < jlo || j > jhi) S->fini[(size_t)i * nv + j] = 0.0;
  if (ihi < 0) { /* nothing above the threshold: no element */
    S->klo = S->llo = 0;
    S->khi = S->lhi = -1;
    return;
  }
  int64_t klo = S->Kx + 1 + floor_div(2 * (int64_t)ilo - (nx - 1), 2 * (int64_t)s) - 1;
  int64_t khi = S->Kx + 1 + ceil_div(2 * (int64_t)ihi - (nx - 1), 2 * (int64_t)s) + 1;
  int64_t llo = S->Kv + 1 + floor_div(2 * (int64_t)jlo - (nv - 1), 2 * (int64_t)s) - 1;
  int64_t lhi = S->Kv + 1 + ceil_div(2 * (int64_t)jhi - (nv - 1), 2 * (int64_t)s) + 1;
  S->klo = (int32_t)(klo < 0 ? 0 : klo);
  S->khi = (int32_t)(khi > S->Lx - 1 ? S->Lx - 1 : khi);
  S->llo = (int32_t)(llo < 0 ? 0 : llo);
  S->lhi = (int32_t)(lhi > S->Lv - 1 ? S->Lv - 1 : lhi);
}

/* Sec. 2.3: the Eulerian computing domain of a map is the rectangle spanned
 * by the positions of the existing elements, as grid sites: i from
 * ceil((min x_m - x_lo)/dx) to floor((max x_m - x_lo)/dx), clamped to the
 * grid, same along v.  f_th = 0: the whole grid. */
static void euler_rect(vo_state* S) {
  const int32_t nx = S->c.nx, nv = S->c.nv;
  if (!(S->f_th > 0.0)) {
    S->rect[0] = 0;
    S->rect[1] = nx - 1;
    S->rect[2] = 0;
    S->rect[3] = nv - 1;
    return;
  }
  double xmin = INFINITY, xmax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
  for (int32_t k = S->klo; k <= S->khi; k++)
    for (int32_t l = S->llo; l <= S->lhi; l++) {
      const elem_t* e = &S->el[k * S->Lv + l];
      if (e->x < xmin) xmin = e->x;
      if (e->x > xmax) xmax = e->x;
      if (e->v < vmin) vmin = e->v;
      if (e->v > vmax) vmax = e->v;
    }
  if (!(xmin <= xmax) || !(vmin <= vmax)) {
    S->rect[0] = S->rect[2] = 0;
    S->rect[1] = S->rect[3] = -1;
    return;
  }
  double a = ceil((xmin - S->c.x_lo) * S->inv_dx), b = floor((xmax - S->c.x_lo) * S->inv_dx);
  double c = ceil((vmin - S->c.v_lo) * S->inv_dv), d = floor((vmax - S->c.v_lo) * S->inv_dv);
  S->rect[0] = (int32_t)(a < 0.0 ? 0.0 : (a > nx ? nx : a));
  S->rect[1] = (int32_t)(b > nx - 1 ? nx - 1 : (b < -1.0 ? -1.0 : b));
  S->rect[2] = (int32_t)(c < 0.0 ? 0.0 : (c > nv ? nv : c));
  S->rect[3] = (int32_t)(d > nv - 1 ? nv - 1 : (d < -1.0 ? -1.0 : d));
}

static int in_rect(const vo_state* S, int64_t i, int64_t j) {
  return i >= S->rect[0] && i <= S->rect[1] && j >= S->rect[2] && j <= S->rect[3];
}

void vo_set_fth(vo_state* S, double f_th) { S->f_th = f_th; }
void vo_domain(const vo_state* S, int32_t* act4, int32_t* rect4) {
  act4[0] = S->klo;
  act4[1] = S->khi;
  act4[2] = S->llo;
  act4[3] = S->lhi;
  memcpy(rect4, S->rect, sizeof S->rect);
}

vo_state* vo_create(const vo_config* c) {
  if (c->nx < 4 || c->nv < 4 || c->s < 1 || c->pad < 0 || !(c->x_hi > c->x_lo) ||
      !(c->v_hi > c->v_lo) || c->n_s < 1)
    return NULL;
  vo_state* S = (vo_state*)calloc(1, sizeof(vo_state));
  S->c = *c;
  if (S->c.max_hole_rounds <= 0) S->c.max_hole_rounds = c->nx + c->nv;
  S->dx = (c->x_hi - c->x_lo) / (double)(c->nx - 1);
  S->dv = (c->v_hi - c->v_lo) / (double)(c->nv - 1);
  S->dxm = (double)c->s * S->dx;
  S->dvm = (double)c->s * S->dv;
  S->inv_dx = 1.0 / S->dx;
  S->inv_dv = 1.0 / S->dv;
  S->inv_dxm = 1.0 / S->dxm;
  S->inv_dvm = 1.0 / S->dvm;
  S->cx = 0.5 * (c->x_lo + c->x_hi);
  S->cv = 0.5 * (c->v_lo + c->v_hi);
  S->Kx = (c->nx - 1 + 2 * c->s - 1) / (2 * c->s);
  S->Kv = (c->nv - 1 + 2 * c->s - 1) / (2 * c->s);
  S->Lx = 2 * S->Kx + 3;
  S->Lv = 2 * S->Kv + 3;
  S->ne = S->Lx * S->Lv;
  size_t n = (size_t)c->nx * c->nv;
  size_t np = (size_t)(c->nx + 2 * c->pad) * (c->nv + 2 * c->pad);
  S->fini = (double*)calloc(n, sizeof(double));
  S->eta = (double*)calloc(n, sizeof(double));
  S->f = (double*)calloc(n, sizeof(double));
  S->el = (elem_t*)calloc((size_t)S->ne, sizeof(elem_t));
  S->tay = (taylor_t*)calloc((size_t)S->ne, sizeof(taylor_t));
  S->map = (int32_t*)malloc(sizeof(int32_t) * n);
  S->prevmap = (int32_t*)malloc(sizeof(int32_t) * n);
  S->bestkey = (uint64_t*)malloc(sizeof(uint64_t) * n);
  S->stamp = (int32_t*)malloc(sizeof(int32_t) * np);
  S->queue = (int32_t*)malloc(sizeof(int32_t) * np);
  S->bbox = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)S->ne);
  S->M = (double*)calloc((size_t)c->nx, sizeof(double));
  S->a = (double*)calloc((size_t)c->nx, sizeof(double));
  S->da = (double*)calloc((size_t)c->nx, sizeof(double));
  S->d2a = (double*)calloc((size_t)c->nx, sizeof(double));
  for (size_t p = 0; p < n; p++) S->map[p] = -1;
  S->klo = S->llo = 0;
  S->khi = S->Lx - 1;
  S->lhi = S->Lv - 1;
  S->rect[0] = S->rect[2] = 0;
  S->rect[1] = c->nx - 1;
  S->rect[3] = c->nv - 1;
  return S;
}

void vo_destroy(vo_state* S) {
  if (!S) return;
  free(S->fini);
  free(S->eta);
  free(S->f);
  free(S->el);
  free(S->tay);
  free(S->map);
  free(S->prevmap);
  free(S->bestkey);
  free(S->stamp);
  free(S->queue);
  free(S->bbox);
  free(S->M);
  free(S->a);
  free(S->da);
  free(S->d2a);
  free(S);
}

int32_t vo_num_elements(const vo_state* S) { return S->ne; }
int32_t vo_lattice_dims(const vo_state* S, int32_t* Lx, int32_t* Lv) {
  *Lx = S->Lx;
  *Lv = S->Lv;
  return S->ne;
}

/* Sec. 2.3, lattice of isotropic elements: P_m = Q_m on the lattice, T = I,
 * H = 0. */
static void reset_elements(vo_state* S) {
  for (int32_t k = 0; k < S->Lx; k++)
    for (int32_t l = 0; l < S->Lv; l++) {
      elem_t* e = &S->el[k * S->Lv + l];
      memset(e, 0, sizeof *e);
      e->x = lattice_qx(S, k);
      e->v = lattice_qv(S, l);
      e->Txx = 1.0;
      e->Tvv = 1.0;
    }
  S->cyc = 0;
}

int32_t vo_set_f(vo_state* S, const double* f0) {
  size_t n = (size_t)S->c.nx * S->c.nv;
  memcpy(S->fini, f0, n * sizeof(double));
  computing_domain(S);
  memcpy(S->f, S->fini, n * sizeof(double));
  vo_spline_solve_2d(S->c.nx, S->c.nv, S->fini, S->eta);
  reset_elements(S);
  S->nstep = 0;
  S->time = 0.0;
  S->last_dt = 0.0;
  S->have_f = 1;
  return VO_OK;
}

/* Variable time step (Sec. 2.4, eq. of Delta t): each step takes
 * min(dt, c_dyn / sqrt(rho_max)), rho_max the largest projected density
 * rho(x_i) = sum_j f(i, j) dv of the last reconstructed f (f0 before the
 * first step); c_dyn = 0 keeps the constant dt of the configuration. */
void vo_set_cdyn(vo_state* S, double c_dyn) { S->c_dyn = c_dyn; }
double vo_time(const vo_state* S) { return S->time; }
double vo_last_dt(const vo_state* S) { return S->last_dt; }

static double step_dt(vo_state* S, double dt_cap) {
  if (!(S->c_dyn > 0.0)) return dt_cap;
  const int32_t nx = S->c.nx, nv = S->c.nv;
  double rmax = 0.0;
  for (int32_t i = 0; i < nx; i++) {
    double r = 0.0;
    for (int32_t j = 0; j < nv; j++) r = r + S->f[(size_t)i * nv + j];
    r = r * S->dv;
    if (r > rmax) rmax = r;
  }
  if (rmax > 0.0) {
    const double lim = S->c_dyn / sqrt(rmax);
    if (lim < dt_cap) return lim;
  }
  return dt_cap;
}

void vo_get_elements(const vo_state* S, double* out) {
  for (int32_t m = 0; m < S->ne; m++) elem_to12(&S->el[m], out + (size_t)m * 12);
}
void vo_set_elements(vo_state* S, const double* in) {
  for (int32_t m = 0; m < S->ne; m++) elem_from12(in + (size_t)m * 12, &S->el[m]);
}

static void compute_taylor(vo_state* S) {
  for (int32_t k = 0; k < S->Lx; k++)
    for (int32_t l = 0; l < S->Lv; l++) {
      int32_t m = k * S->Lv + l;
      taylor_of(&S->el[m], lattice_qx(S, k), lattice_qv(S, l), &S->tay[m]);
    }
}

void vo_get_taylor(vo_state* S, double* out) {
  compute_taylor(S);
  for (int32_t m = 0; m < S->ne; m++) taylor_to14(&S->tay[m], out + (size_t)m * 14);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3.1: percolation                                               */
/* ------------------------------------------------------------------ */

static double site_x(const vo_state* S, int64_t i) { return S->c.x_lo + (double)i * S->dx; }
static double site_v(const vo_state* S, int64_t j) { return S->c.v_lo + (double)j * S->dv; }

/* Lagrangian distance of eq. "d[dQ]" with the element spacing as unit,
 * squared: d^2 = (dq_x/dx_m)^2 + (dq_v/dv_m)^2. */
static double dist2(const vo_state* S, int32_t m, double Px, double Pv, double* xi_o,
                    double* ze_o) {
  double dqx, dqv;
  qofp_t(&S->tay[m], Px, Pv, &dqx, &dqv);
  double xi = dqx * S->inv_dxm;
  double ze = dqv * S->inv_dvm;
  if (xi_o) *xi_o = xi;
  if (ze_o) *ze_o = ze;
  return xi * xi + ze * ze;
}

/* Ranges of neighbour offsets to investigate, from the position of Q
 * relative to the element, in units of the element spacing (alpha ranges:
 * below -alpha -> {-1,0}; [-alpha, alpha) -> {0}; from alpha -> {0,1}). */
static void alpha_range(double r, double alpha, int* lo, int* hi) {
  if (r < -alpha) {
    *lo = -1;
    *hi = 0;
  } else if (r < alpha) {
    *lo = 0;
    *hi = 0;
  } else {
    *lo = 0;
    *hi = 1;
  }
}

/* Neighbour offsets (a, b) != (0, 0) investigated by the percolation test
 * (the rectangle of alpha ranges of both axes, minus the centre). */
int32_t vo_alpha_offsets(double xi, double ze, double alpha, int32_t* ab) {
  int a0, a1, b0, b1, n = 0;
  alpha_range(xi, alpha, &a0, &a1);
  alpha_range(ze, alpha, &b0, &b1);
  for (int a = a0; a <= a1; a++)
    for (int b = b0; b <= b1; b++) {
      if (a == 0 && b == 0) continue;
      ab[2 * n] = a;
      ab[2 * n + 1] = b;
      n++;
    }
  return n;
}

/* The percolation test of a site for element m: it passes unless one of the
 * investigated neighbours proposes a strictly smaller distance. */
static int passes(const vo_state* S, int32_t m, double Px, double Pv, double* d2_o) {
  double xi, ze;
  double d2 = dist2(S, m, Px, Pv, &xi, &ze);
  *d2_o = d2;
  int32_t ab[18];
  int32_t n = vo_alpha_offsets(xi, ze, S->c.alpha, ab);
  int32_t k = m / S->Lv, l = m % S->Lv;
  for (int32_t q = 0; q < n; q++) {
    int32_t kk = k + ab[2 * q], ll = l + ab[2 * q + 1];
    if (kk < 0 || kk >= S->Lx || ll < 0 || ll >= S->Lv || !exists(S, kk, ll)) continue;
    double d2n = dist2(S, kk * S->Lv + ll, Px, Pv, NULL, NULL);
    if (d2n < d2) return 0;
  }
  return 1;
}

/* Claim rule for a site reached by several elements: smaller d wins, then
 * the smaller element index.  d^2 >= 0 is compared through its IEEE bit
 * pattern, which orders non-negative doubles numerically (NaN last). */
static void claim(vo_state* S, int64_t i, int64_t j, int32_t m, double d2) {
  if (i < 0 || j < 0 || i >= S->c.nx || j >= S->c.nv || !in_rect(S, i, j)) return;
  size_t p = (size_t)i * S->c.nv + (size_t)j;
  uint64_t key = dbits(d2);
  if (S->map[p] < 0) {
    S->map[p] = m;
    S->bestkey[p] = key;
    return;
  }
  S->stat_multi++;
  if (key < S->bestkey[p] || (key == S->bestkey[p] && m < S->map[p])) {
    S->map[p] = m;
    S->bestkey[p] = key;
  }
}

static int32_t percolate(vo_state* S) {
  const int32_t nx = S->c.nx, nv = S->c.nv, pad = S->c.pad;
  const int64_t PW = nx + 2 * pad, PH = nv + 2 * pad;
  size_t n = (size_t)nx * nv;
  for (size_t p = 0; p < n; p++) S->map[p] = -1;
  for (int64_t p = 0; p < PW * PH; p++) S->stamp[p] = -1;
  S->stat_multi = 0;
  for (int32_t m = 0; m < S->ne; m++) {
    int32_t* bb = S->bbox + 4 * (size_t)m;
    bb[0] = bb[2] = 1;
    bb[1] = bb[3] = 0;
    if (!exists(S, m / S->Lv, m % S->Lv)) continue;
    /* start from the grid site nearest to P_m */
    double us = (S->el[m].x - S->c.x_lo) * S->inv_dx;
    double ws = (S->el[m].v - S->c.v_lo) * S->inv_dv;
    if (!(us > -1e9 && us < 1e9 && ws > -1e9 && ws < 1e9)) continue;
    int64_t i0 = nearest(us), j0 = nearest(ws);
    if (i0 < -pad || i0 >= nx + pad || j0 < -pad || j0 >= nv + pad) continue;
    int64_t p0 = (i0 + pad) * PH + (j0 + pad);
    S->stamp[p0] = m;
    double d2;
    if (!passes(S, m, site_x(S, i0), site_v(S, j0), &d2)) continue;
    claim(S, i0, j0, m, d2);
    bb[0] = bb[1] = (int32_t)i0;
    bb[2] = bb[3] = (int32_t)j0;
    int64_t qh = 0, qt = 0;
    S->queue[qt++] = (int32_t)p0;
    while (qh < qt) {
      int64_t p = S->queue[qh++];
      int64_t i = p / PH - pad, j = p % PH - pad;
      static const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
      for (int q = 0; q < 4; q++) {
        int64_t ii = i + di[q], jj = j + dj[q];
        if (ii < -pad || ii >= nx + pad || jj < -pad || jj >= nv + pad) continue;
        int64_t pp = (ii + pad) * PH + (jj + pad);
        if (S->stamp[pp] == m) continue;
        S->stamp[pp] = m;
        if (passes(S, m, site_x(S, ii), site_v(S, jj), &d2)) {
          claim(S, ii, jj, m, d2);
          if (ii < bb[0]) bb[0] = (int32_t)ii;
          if (ii > bb[1]) bb[1] = (int32_t)ii;
          if (jj < bb[2]) bb[2] = (int32_t)jj;
          if (jj > bb[3]) bb[3] = (int32_t)jj;
          S->queue[qt++] = (int32_t)pp;
        }
      }
    }
  }
  /* Unexplored sites: repeated local rounds.  In each round every hole takes,
   * among the elements assigned to its in-grid 4-neighbours at the end of the
   * previous round, the one with the smallest d at the hole (then the
   * smaller index). */
  int64_t holes = 0;
  for (size_t p = 0; p < n; p++) holes += (S->map[p] < 0 && in_rect(S, (int64_t)(p / nv), (int64_t)(p % nv)));
  S->stat_holes = holes;
  int32_t rounds = 0;
  while (holes > 0) {
    if (rounds >= S->c.max_hole_rounds) {
      S->stat_rounds = rounds;
      return VO_E_NOT_CONVERGED;
    }
    memcpy(S->prevmap, S->map, n * sizeof(int32_t));
#pragma omp parallel for schedule(dynamic, 64)
    for (int32_t i = 0; i < nx; i++)
      for (int32_t j = 0; j < nv; j++) {
        size_t p = (size_t)i * nv + j;
        if (S->prevmap[p] >= 0 || !in_rect(S, i, j)) continue;
        int32_t best = -1;
        uint64_t bestk = 0;
        static const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
        for (int q = 0; q < 4; q++) {
          int32_t ii = i + di[q], jj = j + dj[q];
          if (ii < 0 || ii >= nx || jj < 0 || jj >= nv) continue;
          int32_t cand = S->prevmap[(size_t)ii * nv + jj];
          if (cand < 0) continue;
          uint64_t key = dbits(dist2(S, cand, site_x(S, i), site_v(S, j), NULL, NULL));
          if (best < 0 || key < bestk || (key == bestk && cand < best)) {
            best = cand;
            bestk = key;
          }
        }
        S->map[p] = best;
      }
    holes = 0;
    for (size_t p = 0; p < n; p++) holes += (S->map[p] < 0 && in_rect(S, (int64_t)(p / nv), (int64_t)(p % nv)));
    rounds++;
  }
  S->stat_rounds = rounds;
  return VO_OK;
}

int32_t vo_compute_map(vo_state* S, int32_t* map_out) {
  compute_taylor(S);
  euler_rect(S);
  int32_t st = percolate(S);
  if (map_out) memcpy(map_out, S->map, sizeof(int32_t) * (size_t)S->c.nx * S->c.nv);
  return st;
}

/* Bounding box (i_min, i_max, j_min, j_max, padded-lattice indices) of each
 * element's connected component in the last percolation; empty components
 * have min > max. */
void vo_component_bbox(const vo_state* S, int32_t* out4xne) {
  memcpy(out4xne, S->bbox, sizeof(int32_t) * 4 * (size_t)S->ne);
}

int32_t vo_map_stats(const vo_state* S, int64_t* multi, int64_t* holes, int32_t* rounds) {
  *multi = S->stat_multi;
  *holes = S->stat_holes;
  *rounds = S->stat_rounds;
  return 0;
}

/* ------------------------------------------------------------------ */
/* transport reconstruction, pixel masses and force                      */
/* ------------------------------------------------------------------ */

/* f(P) = f_ini(Q(P)) with Q from the element that owns P (Liouville), the
 * quadratic interpolation of Sec. 2.2.1; then the pixel masses
 * M(i) = (sum_j f(i,j)) dx dv and the force of Sec. 2.5. */
static void reconstruct_and_force(vo_state* S) {
  const int32_t nx = S->c.nx, nv = S->c.nv;
  double dxdv = S->dx * S->dv;
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < nx; i++) {
    double Px = site_x(S, i);
    double rowsum = 0.0;
    for (int32_t j = 0; j < nv; j++) {
      size_t p = (size_t)i * nv + j;
      int32_t m = S->map[p];
      double fv = 0.0;
      if (m >= 0) {
        double dqx, dqv;
        const taylor_t* t = &S->tay[m];
        qofp_t(t, Px, site_v(S, j), &dqx, &dqv);
        double u = ((t->Qx + dqx) - S->c.x_lo) * S->inv_dx;
        double w = ((t->Qv + dqv) - S->c.v_lo) * S->inv_dv;
        fv = vo_qinterp(S->fini, nx, nv, u, w);
      }
      S->f[p] = fv;
      rowsum = rowsum + fv;
    }
    S->M[i] = rowsum * dxdv;
  }
  vo_force_from_mass(S->M, nx, S->dx, S->c.G, S->c.literal_fd, S->a, S->da, S->d2a);
  double Mtot = 0.0;
  for (int32_t i = 0; i < nx; i++) Mtot = Mtot + S->M[i];
  S->Mtot = Mtot;
}

int32_t vo_reconstruct(vo_state* S, double* f_out) {
  int32_t st = vo_compute_map(S, NULL);
  reconstruct_and_force(S);
  if (f_out) memcpy(f_out, S->f, sizeof(double) * (size_t)S->c.nx * S->c.nv);
  return st;
}

void vo_density_force(const vo_state* S, double* M, double* a, double* da, double* d2a,
                      double* Mtot) {
  size_t b = sizeof(double) * (size_t)S->c.nx;
  if (M) memcpy(M, S->M, b);
  if (a) memcpy(a, S->a, b);
  if (da) memcpy(da, S->da, b);
  if (d2a) memcpy(d2a, S->d2a, b);
  if (Mtot) *Mtot = S->Mtot;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.4: drift-kick-drift                                            */
/* ------------------------------------------------------------------ */

/* Half drift: only positions (and the x rows of T and H) change. */
static void drift_half(vo_state* S) {
  double h = 0.5 * S->c.dt;
  for (int32_t m = 0; m < S->ne; m++) {
    elem_t* e = &S->el[m];
    e->x = e->x + e->v * h;
    e->Txx = e->Txx + e->Tvx * h;
    e->Txv = e->Txv + e->Tvv * h;
    for (int k = 0; k < 3; k++) e->Hx[k] = e->Hx[k] + e->Hv[k] * h;
  }
}

/* Kick over a full step with a, a', a'' interpolated (dual TSC) at the
 * drifted positions: dv = a dt, dT_v. = a' T_x. dt,
 * dH_v.. = (a' H_x.. + a'' T_x. T_x.) dt. */
static void kick(vo_state* S, const double* a, const double* da, const double* d2a,
                 double a_lo, double a_hi) {
  double dt = S->c.dt;
  for (int32_t m = 0; m < S->ne; m++) {
    elem_t* e = &S->el[m];
    double u = (e->x - S->c.x_lo) * S->inv_dx;
    double am = vo_tsc(a, S->c.nx, a_lo, a_hi, u);
    double dam = vo_tsc(da, S->c.nx, 0.0, 0.0, u);
    double d2am = vo_tsc(d2a, S->c.nx, 0.0, 0.0, u);
    e->v = e->v + am * dt;
    e->Tvx = e->Tvx + (dam * e->Txx) * dt;
    e->Tvv = e->Tvv + (dam * e->Txv) * dt;
    e->Hv[0] = e->Hv[0] + (dam * e->Hx[0] + (d2am * e->Txx) * e->Txx) * dt;
    e->Hv[1] = e->Hv[1] + (dam * e->Hx[1] + (d2am * e->Txx) * e->Txv) * dt;
    e->Hv[2] = e->Hv[2] + (dam * e->Hx[2] + (d2am * e->Txv) * e->Txv) * dt;
  }
}

/* Sec. 2.3.2, beta ranges: per axis, below -beta -> {-1,0}; [-beta, beta)
 * -> {-1,0,1}; from beta -> {0,1}; when either axis takes all three, the
 * diagonal offsets are dropped (a*b = 0).  Writes the offsets, centre
 * included, and returns their number (4 or 5). */
int32_t vo_beta_offsets(double xi, double ze, double beta, int32_t* ab) {
  int a0 = (xi < -beta) ? -1 : ((xi < beta) ? -1 : 0);
  int a1 = (xi < -beta) ? 0 : 1;
  int b0 = (ze < -beta) ? -1 : ((ze < beta) ? -1 : 0);
  int b1 = (ze < -beta) ? 0 : 1;
  int full = (a0 == -1 && a1 == 1) || (b0 == -1 && b1 == 1);
  int n = 0;
  for (int a = a0; a <= a1; a++)
    for (int b = b0; b <= b1; b++) {
      if (full && a != 0 && b != 0) continue;
      ab[2 * n] = a;
      ab[2 * n + 1] = b;
      n++;
    }
  return n;
}

/* Sec. 2.3.2: blended Lagrangian position Q_r at site P owned by m,
 * Q_r = sum W(2 d_m') Q(P, m') / sum W(2 d_m') over the beta set. */
static void blended_q(const vo_state* S, int32_t m, double Px, double Pv, double* Qx,
                      double* Qv) {
  double xi, ze;
  dist2(S, m, Px, Pv, &xi, &ze);
  int32_t ab[18];
  int32_t n = vo_beta_offsets(xi, ze, S->c.beta, ab);
  int32_t k = m / S->Lv, l = m % S->Lv;
  double nx_ = 0.0, nv_ = 0.0, den = 0.0;
  for (int32_t q = 0; q < n; q++) {
    int32_t kk = k + ab[2 * q], ll = l + ab[2 * q + 1];
    if (kk < 0 || kk >= S->Lx || ll < 0 || ll >= S->Lv || !exists(S, kk, ll)) continue;
    int32_t mm = kk * S->Lv + ll;
    double dqx, dqv;
    const taylor_t* t = &S->tay[mm];
    qofp_t(t, Px, Pv, &dqx, &dqv);
    double x1 = dqx * S->inv_dxm, z1 = dqv * S->inv_dvm;
    double d = sqrt(x1 * x1 + z1 * z1);
    double wgt = vo_W(2.0 * d);
    nx_ = nx_ + wgt * (t->Qx + dqx);
    nv_ = nv_ + wgt * (t->Qv + dqv);
    den = den + wgt;
  }
  if (den > 0.0) {
    *Qx = nx_ / den;
    *Qv = nv_ / den;
  } else {
    double dqx, dqv;
    qofp_t(&S->tay[m], Px, Pv, &dqx, &dqv);
    *Qx = S->tay[m].Qx + dqx;
    *Qv = S->tay[m].Qv + dqv;
  }
}

/* Remap resample (Secs. 2.2.2 and 2.3.2): with the map of the current
 * elements, f_new(P) = spline[f_ini](Q_r(P)). */
int32_t vo_remap_resample(vo_state* S, double* fnew, double* Qr) {
  const int32_t nx = S->c.nx, nv = S->c.nv;
  int32_t st = vo_compute_map(S, NULL);
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < nx; i++)
    for (int32_t j = 0; j < nv; j++) {
      size_t p = (size_t)i * nv + j;
      int32_t m = S->map[p];
      double Qx = 0.0, Qv = 0.0, val = 0.0;
      if (m >= 0) {
        blended_q(S, m, site_x(S, i), site_v(S, j), &Qx, &Qv);
        double u = (Qx - S->c.x_lo) * S->inv_dx;
        double w = (Qv - S->c.v_lo) * S->inv_dv;
        val = vo_spline_eval(S->eta, nx, nv, u, w);
      }
      fnew[p] = val;
      if (Qr) {
        Qr[2 * p] = Qx;
        Qr[2 * p + 1] = Qv;
      }
    }
  return st;
}

/* Full remap: the resampled f becomes the new f_ini, its spline coefficients
 * are recomputed and new isotropic elements are laid on the lattice. */
int32_t vo_remap(vo_state* S) {
  size_t n = (size_t)S->c.nx * S->c.nv;
  double* fnew = (double*)malloc(sizeof(double) * n);
  int32_t st = vo_remap_resample(S, fnew, NULL);
  memcpy(S->fini, fnew, n * sizeof(double));
  free(fnew);
  computing_domain(S);
  vo_spline_solve_2d(S->c.nx, S->c.nv, S->fini, S->eta);
  reset_elements(S);
  return st;
}

/* One step t -> t + dt (Sec. 2.4): half drift; map with the predicted
 * elements; f(t + dt/2) by transport; masses and force; kick; half drift;
 * remap at the end of every n_s-th step of a cycle. */
int32_t vo_step(vo_state* S, int32_t nsteps) {
  int32_t st = VO_OK;
  const double dt_cap = S->c.dt;
  for (int32_t it = 0; it < nsteps; it++) {
    S->c.dt = step_dt(S, dt_cap);
    S->last_dt = S->c.dt;
    drift_half(S);
    int32_t s1 = vo_compute_map(S, NULL);
    if (s1 != VO_OK) st = s1;
    reconstruct_and_force(S);
    double A = 2.0 * PI * S->c.G;
    kick(S, S->a, S->da, S->d2a, A * S->Mtot, -(A * S->Mtot));
    drift_half(S);
    S->nstep++;
    S->time = S->time + S->c.dt;
    S->cyc++;
    if (S->cyc >= S->c.n_s) {
      int32_t s2 = vo_remap(S);
      if (s2 != VO_OK) st = s2;
    }
  }
  S->c.dt = dt_cap;
  return st;
}

void vo_push_frozen(vo_state* S, const double* a, const double* da, const double* d2a,
                    double ext_lo, double ext_hi, int32_t nsteps) {
  for (int32_t it = 0; it < nsteps; it++) {
    drift_half(S);
    kick(S, a, da, d2a, ext_lo, ext_hi);
    drift_half(S);
  }
}

void vo_get_fini(const vo_state* S, double* out) {
  memcpy(out, S->fini, sizeof(double) * (size_t)S->c.nx * S->c.nv);
}
void vo_get_eta(const vo_state* S, double* out) {
  memcpy(out, S->eta, sizeof(double) * (size_t)S->c.nx * S->c.nv);
}
void vo_get_last_f(const vo_state* S, double* out) {
  memcpy(out, S->f, sizeof(double) * (size_t)S->c.nx * S->c.nv);
}
int64_t vo_step_count(const vo_state* S) { return S->nstep; }
int32_t vo_cycle_step(const vo_state* S) { return S->cyc; }

/* Sec. 3.2: mass and total energy of the last reconstructed f and force,
 * E = 1/2 sum v^2 f dx dv - 1/(8 pi G) sum (a^2 - (2 pi G M)^2) dx, plus the
 * range of det T over the elements (Sec. 2.1, |T| = 1). */
void vo_diagnostics(const vo_state* S, double* mass, double* energy, double* dmin,
                    double* dmax) {
  const int32_t nx = S->c.nx, nv = S->c.nv;
  double dxdv = S->dx * S->dv;
  double ek = 0.0, ms = 0.0;
  for (int32_t i = 0; i < nx; i++)
    for (int32_t j = 0; j < nv; j++) {
      double v = site_v(S, j);
      double fv = S->f[(size_t)i * nv + j];
      ek = ek + 0.5 * (v * v) * fv * dxdv;
      ms = ms + fv * dxdv;
    }
  double ep = 0.0;
  if (S->c.G != 0.0) {
    double A = 2.0 * PI * S->c.G;
    double a8 = A * S->Mtot;
    for (int32_t i = 0; i < nx; i++) ep = ep + (S->a[i] * S->a[i] - a8 * a8) * S->dx;
    ep = -ep / (8.0 * PI * S->c.G);
  }
  *mass = ms;
  *energy = ek + ep;
  double lo = INFINITY, hi = -INFINITY;
  for (int32_t m = 0; m < S->ne; m++) {
    if (!exists(S, m / S->Lv, m % S->Lv)) continue;
    const elem_t* e = &S->el[m];
    double d = e->Txx * e->Tvv - e->Txv * e->Tvx;
    if (d < lo) lo = d;
    if (d > hi) hi = d;
  }
  *dmin = lo;
  *dmax = hi;
}

/* Sec. 3.2: the Casimir S = -sum f log|f| dx dv (0 where f = 0) and the L1
 * and L2 norms sum |f| dx dv, sum f^2 dx dv of the last reconstructed f. */
void vo_casimirs(const vo_state* S, double* entropy, double* l1, double* l2) {
  const size_t n = (size_t)S->c.nx * S->c.nv;
  const double dxdv = S->dx * S->dv;
  double se = 0.0, s1 = 0.0, s2 = 0.0;
  for (size_t p = 0; p < n; p++) {
    const double fv = S->f[p];
    if (fv != 0.0) se = se - fv * log(fabs(fv)) * dxdv;
    s1 = s1 + fabs(fv) * dxdv;
    s2 = s2 + fv * fv * dxdv;
  }
  *entropy = se;
  *l1 = s1;
  *l2 = s2;
}

/* Sec. 2.3.2: E_map, the largest mismatch, in element spacings, between the
 * Lagrangian position Q(P) the owner m of a site proposes and the one a
 * neighbour n investigated by the percolation test proposes:
 *   ((a + xi_n) - xi_m, (b + ze_n) - ze_m),  (a, b) = n - m,
 * since Q_n - Q_m = (a dx_m, b dv_m) on the lattice; E_map is the largest
 * Euclidean norm over the grid's sites, from the last influence map and the
 * Taylor terms it used. */
double vo_emap(const vo_state* S) {
  const int32_t nx = S->c.nx, nv = S->c.nv;
  double worst = 0.0;
  for (int32_t i = 0; i < nx; i++)
    for (int32_t j = 0; j < nv; j++) {
      const int32_t m = S->map[(size_t)i * nv + j];
      if (m < 0) continue;
      const double Px = site_x(S, i), Pv = site_v(S, j);
      double xi, ze;
      dist2(S, m, Px, Pv, &xi, &ze);
      int32_t ab[18];
      const int32_t nn = vo_alpha_offsets(xi, ze, S->c.alpha, ab);
      const int32_t k = m / S->Lv, l = m % S->Lv;
      for (int32_t q = 0; q < nn; q++) {
        const int32_t kk = k + ab[2 * q], ll = l + ab[2 * q + 1];
        if (kk < 0 || kk >= S->Lx || ll < 0 || ll >= S->Lv || !exists(S, kk, ll)) continue;
        double xn, zn;
        dist2(S, kk * S->Lv + ll, Px, Pv, &xn, &zn);
        const double mx = ((double)ab[2 * q] + xn) - xi, mv = ((double)ab[2 * q + 1] + zn) - ze;
        const double e2 = mx * mx + mv * mv;
        if (e2 > worst) worst = e2;
      }
    }
  return sqrt(worst);
}
