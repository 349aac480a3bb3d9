/*
 * FP64 CPU oracle of the metric semi-Lagrangian Vlasov-Poisson step in 4D
 * phase space (x, y, vx, vy).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's
 * CPU-baseline leg; never by the product path.  Plain and serial, FP64
 * throughout, written from the paper in its order and notation, each piece
 * generalised from two to four phase-space dimensions where the paper says
 * how (Sec. 2.1: 4+16+40 = 60 numbers per element and the inverse map of
 * eq. QofP; Sec. 2.2.1: the 15-point quadratic hypersurface through the
 * nearest node, its 9-point cross and one corner per pair of axes; Sec. 2.3:
 * percolation with alpha ranges per axis; Sec. 2.5: Poisson in 2D space on
 * a fixed grid, field gradient and Hessian by finite differences).
 *
 * Readings where the paper gives only the two-dimensional case (listed with
 * their justification in the repository's design notes):
 *   - the alpha ranges of the percolation test and the beta ranges of Q_r
 *     are taken per axis, as in 2D; the beta set drops an offset with two or
 *     more non-zero components as soon as one of them lies on an axis whose
 *     range is {-1,0,1} (in 2D this is the paper's rule i'j' = 0; in 4D it is
 *     the same geometric bound (1-beta)^2 + 1/4 >= 1 of the kernel support);
 *   - Poisson in 2D space, lap(phi) = 4 pi G rho, solved on the grid as the
 *     sum over the pixel masses of the 2D Green function 2 G ln r, the
 *     node's own pixel excluded (as in 1D, where a pixel's own mass does not
 *     act on it); the paper names FFT for this convolution, which computes
 *     the same discrete sum;
 *   - the field's gradient and Hessian by centred differences of the nodal
 *     acceleration, and the kick interpolates the acceleration, gradient
 *     and Hessian at the element by the 2D tensor product of the 1D TSC
 *     weights; the same direct sum defines the field at nodes outside the
 *     grid;
 *   - the 4D cubic spline is the tensor product of the 1D zero-slope spline,
 *     solved along vy, vx, y, then x.
 *
 * Floating-point evaluation order is fixed at each formula (built with
 * -ffp-contract=off) so that the integer decisions are reproducible.
 *
 * Parity status: the 15-point interpolation, the inverse map, the 4D spline,
 * the field and the element push are pinned by closed forms (tests); the
 * percolation map is pinned by its closed form right after a remap and by
 * brute force on tiny grids; the Q_r blend by hand-built displaced elements.
 */
#include "vlamet4d_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "vlamet_oracle.h" /* the 1D pieces pinned in 2D: B-spline, spline solve, W */

#define NE 60
#define NT 64

/* symmetric index of (b, c) in the order 00,01,02,03,11,12,13,22,23,33 */
static int sym(int b, int c) {
  static const int tab[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
  return tab[b][c];
}

static uint64_t dbits(double d) {
  uint64_t u;
  memcpy(&u, &d, sizeof u);
  return u;
}

static int64_t nearest(double u) { return (int64_t)floor(u + 0.5); }

/* ------------------------------------------------------------------ */
/* Sec. 2.2.1: 15-point quadratic interpolation                         */
/* ------------------------------------------------------------------ */

static double F4(const double* F, const int32_t* n, const int64_t* g) {
  for (int a = 0; a < 4; a++)
    if (g[a] < 0 || g[a] >= n[a]) return 0.0;
  return F[((g[0] * n[1] + g[1]) * n[2] + g[2]) * n[3] + g[3]];
}

/* The nearest node G_n, its cross of 3-point segments along the four axes
 * (9 nodes), and for each of the 6 pairs of axes the corner of the square
 * of the pair's plane through G_n that holds the projection of Q (found from
 * the integer parts c = floor(u)); the quadratic through these 15 nodes is
 * the Lagrange form on {-1,0,1} along each axis plus the mixed differences
 * of the squares.  Nodes outside the grid read 0. */
double vo4_qinterp(const double* F, const int32_t* n, const double* u) {
  for (int a = 0; a < 4; a++)
    if (!(u[a] > -2.0 && u[a] < (double)n[a] + 1.0)) return 0.0;
  int64_t gn[4], gc[4];
  double dq[4];
  for (int a = 0; a < 4; a++) {
    gn[a] = nearest(u[a]);
    gc[a] = (int64_t)floor(u[a]);
    dq[a] = u[a] - (double)gn[a];
  }
  double w0 = (((1.0 - dq[0] * dq[0]) - dq[1] * dq[1]) - dq[2] * dq[2]) - dq[3] * dq[3];
  double f = F4(F, n, gn) * w0;
  for (int a = 0; a < 4; a++) {
    int64_t g[4] = {gn[0], gn[1], gn[2], gn[3]};
    g[a] = gn[a] + 1;
    f = f + ((0.5 * F4(F, n, g)) * dq[a]) * (1.0 + dq[a]);
    g[a] = gn[a] - 1;
    f = f + ((0.5 * F4(F, n, g)) * dq[a]) * (dq[a] - 1.0);
  }
  for (int a = 0; a < 4; a++)
    for (int b = a + 1; b < 4; b++) {
      int64_t g11[4] = {gn[0], gn[1], gn[2], gn[3]}, g00[4], g10[4], g01[4];
      memcpy(g00, g11, sizeof g00);
      g11[a] = gc[a] + 1;
      g11[b] = gc[b] + 1;
      g00[a] = gc[a];
      g00[b] = gc[b];
      memcpy(g10, g00, sizeof g10);
      g10[a] = gc[a] + 1;
      memcpy(g01, g00, sizeof g01);
      g01[b] = gc[b] + 1;
      double cross = ((F4(F, n, g11) + F4(F, n, g00)) - F4(F, n, g10)) - F4(F, n, g01);
      f = f + (cross * dq[a]) * dq[b];
    }
  return f;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2.2: 4D tensor-product cubic B-spline                          */
/* ------------------------------------------------------------------ */

/* Coefficients of the tensor-product spline through the node values: the
 * 1D zero-slope solve along every line of axis 3, then 2, 1, 0. */
void vo4_spline_solve(const int32_t* n, const double* f, double* eta) {
  const int64_t N = (int64_t)n[0] * n[1] * n[2] * n[3];
  memcpy(eta, f, sizeof(double) * (size_t)N);
  int64_t stride[4] = {(int64_t)n[1] * n[2] * n[3], (int64_t)n[2] * n[3], n[3], 1};
  int32_t nmax = n[0];
  for (int a = 1; a < 4; a++)
    if (n[a] > nmax) nmax = n[a];
  double* in = (double*)malloc(sizeof(double) * (size_t)nmax);
  double* out = (double*)malloc(sizeof(double) * (size_t)nmax);
  for (int a = 3; a >= 0; a--) {
    for (int64_t base = 0; base < N; base++) {
      /* base is the first node of a line of axis a when its coordinate a is 0 */
      if ((base / stride[a]) % n[a] != 0) continue;
      for (int32_t i = 0; i < n[a]; i++) in[i] = eta[base + i * stride[a]];
      vo_spline_solve_1d(n[a], in, out);
      for (int32_t i = 0; i < n[a]; i++) eta[base + i * stride[a]] = out[i];
    }
  }
  free(in);
  free(out);
}

/* ghost coefficient index: -1 -> 1, n -> n-2, else outside -> -1 */
static int64_t ghost(int64_t k, int32_t n) {
  if (k >= 0 && k < n) return k;
  if (k == -1) return 1;
  if (k == n) return n - 2;
  return -1;
}

/* f(u) = sum over the 4^4 coefficients around u of eta_k prod_a B(u_a - k_a),
 * the finite B-spline sum evaluated everywhere (zero beyond its support). */
double vo4_spline_eval(const double* eta, const int32_t* n, const double* u) {
  for (int a = 0; a < 4; a++)
    if (!(u[a] > -3.0 && u[a] < (double)(n[a] + 2))) return 0.0;
  int64_t k0[4];
  double B[4][4];
  int64_t gk[4][4];
  for (int a = 0; a < 4; a++) {
    k0[a] = (int64_t)floor(u[a]) - 1;
    for (int q = 0; q < 4; q++) {
      B[a][q] = vo_bspline3(u[a] - (double)(k0[a] + q));
      gk[a][q] = ghost(k0[a] + q, n[a]);
    }
  }
  double sum = 0.0;
  for (int q0 = 0; q0 < 4; q0++) {
    if (gk[0][q0] < 0) continue;
    for (int q1 = 0; q1 < 4; q1++) {
      if (gk[1][q1] < 0) continue;
      for (int q2 = 0; q2 < 4; q2++) {
        if (gk[2][q2] < 0) continue;
        for (int q3 = 0; q3 < 4; q3++) {
          if (gk[3][q3] < 0) continue;
          int64_t p = ((gk[0][q0] * n[1] + gk[1][q1]) * n[2] + gk[2][q2]) * n[3] + gk[3][q3];
          sum = sum + (((eta[p] * B[0][q0]) * B[1][q1]) * B[2][q2]) * B[3][q3];
        }
      }
    }
  }
  return sum;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1: Taylor terms of the inverse map                             */
/* ------------------------------------------------------------------ */

/* T^-1 = adj(T) / det T, the adjugate from the 2x2 minors of the first two
 * rows (s) and of the last two rows (c) (Laplace expansion). */
static void inverse4(const double* A, double* B) {
  const double a00 = A[0], a01 = A[1], a02 = A[2], a03 = A[3];
  const double a10 = A[4], a11 = A[5], a12 = A[6], a13 = A[7];
  const double a20 = A[8], a21 = A[9], a22 = A[10], a23 = A[11];
  const double a30 = A[12], a31 = A[13], a32 = A[14], a33 = A[15];
  const double s0 = a00 * a11 - a10 * a01, s1 = a00 * a12 - a10 * a02;
  const double s2 = a00 * a13 - a10 * a03, s3 = a01 * a12 - a11 * a02;
  const double s4 = a01 * a13 - a11 * a03, s5 = a02 * a13 - a12 * a03;
  const double c5 = a22 * a33 - a32 * a23, c4 = a21 * a33 - a31 * a23;
  const double c3 = a21 * a32 - a31 * a22, c2 = a20 * a33 - a30 * a23;
  const double c1 = a20 * a32 - a30 * a22, c0 = a20 * a31 - a30 * a21;
  const double det = ((((s0 * c5 - s1 * c4) + s2 * c3) + s3 * c2) - s4 * c1) + s5 * c0;
  const double id = 1.0 / det;
  B[0] = ((a11 * c5 - a12 * c4) + a13 * c3) * id;
  B[1] = ((a02 * c4 - a01 * c5) - a03 * c3) * id;
  B[2] = ((a31 * s5 - a32 * s4) + a33 * s3) * id;
  B[3] = ((a22 * s4 - a21 * s5) - a23 * s3) * id;
  B[4] = ((a12 * c2 - a10 * c5) - a13 * c1) * id;
  B[5] = ((a00 * c5 - a02 * c2) + a03 * c1) * id;
  B[6] = ((a32 * s2 - a30 * s5) - a33 * s1) * id;
  B[7] = ((a20 * s5 - a22 * s2) + a23 * s1) * id;
  B[8] = ((a10 * c4 - a11 * c2) + a13 * c0) * id;
  B[9] = ((a01 * c2 - a00 * c4) - a03 * c0) * id;
  B[10] = ((a30 * s4 - a31 * s2) + a33 * s0) * id;
  B[11] = ((a21 * s2 - a20 * s4) - a23 * s0) * id;
  B[12] = ((a11 * c1 - a10 * c3) - a12 * c0) * id;
  B[13] = ((a00 * c3 - a01 * c1) + a02 * c0) * id;
  B[14] = ((a31 * s1 - a30 * s3) - a32 * s0) * id;
  B[15] = ((a20 * s3 - a21 * s1) + a22 * s0) * id;
}

static double det4(const double* A) {
  const double s0 = A[0] * A[5] - A[4] * A[1], s1 = A[0] * A[6] - A[4] * A[2];
  const double s2 = A[0] * A[7] - A[4] * A[3], s3 = A[1] * A[6] - A[5] * A[2];
  const double s4 = A[1] * A[7] - A[5] * A[3], s5 = A[2] * A[7] - A[6] * A[3];
  const double c5 = A[10] * A[15] - A[14] * A[11], c4 = A[9] * A[15] - A[13] * A[11];
  const double c3 = A[9] * A[14] - A[13] * A[10], c2 = A[8] * A[15] - A[12] * A[11];
  const double c1 = A[8] * A[14] - A[12] * A[10], c0 = A[8] * A[13] - A[12] * A[9];
  return ((((s0 * c5 - s1 * c4) + s2 * c3) + s3 * c2) - s4 * c1) + s5 * c0;
}

/* Taylor record of one element: P_m, T^-1, G_l = [T^-1]^T H_l T^-1 for
 * l = 0..3 (through A = H_l T^-1), Q_m. */
void vo4_taylor_one(const double* e, const double* Qm, double* t) {
  const double* T = e + 4;
  const double* H = e + 20;
  double* Ti = t + 4;
  for (int a = 0; a < 4; a++) t[a] = e[a];
  inverse4(T, Ti);
  for (int l = 0; l < 4; l++) {
    const double* h = H + 10 * l;
    double A[4][4];
    for (int b = 0; b < 4; b++)
      for (int c = 0; c < 4; c++)
        A[b][c] = ((h[sym(b, 0)] * Ti[0 * 4 + c] + h[sym(b, 1)] * Ti[1 * 4 + c]) +
                   h[sym(b, 2)] * Ti[2 * 4 + c]) + h[sym(b, 3)] * Ti[3 * 4 + c];
    double* G = t + 20 + 10 * l;
    for (int b = 0; b < 4; b++)
      for (int c = b; c < 4; c++)
        G[sym(b, c)] = ((Ti[0 * 4 + b] * A[0][c] + Ti[1 * 4 + b] * A[1][c]) +
                        Ti[2 * 4 + b] * A[2][c]) + Ti[3 * 4 + b] * A[3][c];
  }
  for (int a = 0; a < 4; a++) t[60 + a] = Qm[a];
}

/* Second-order inverse map (Sec. 2.1, eq. QofP): dQ = y - T^-1 s / 2 with
 * y = T^-1 dP and s_l = dP^T G_l dP. */
void vo4_qofp(const double* t, const double* P, double* dQ) {
  const double* Ti = t + 4;
  double dP[4], y[4], s[4];
  for (int a = 0; a < 4; a++) dP[a] = P[a] - t[a];
  for (int a = 0; a < 4; a++)
    y[a] = ((Ti[a * 4 + 0] * dP[0] + Ti[a * 4 + 1] * dP[1]) + Ti[a * 4 + 2] * dP[2]) +
           Ti[a * 4 + 3] * dP[3];
  for (int l = 0; l < 4; l++) {
    const double* G = t + 20 + 10 * l;
    double g[4];
    for (int b = 0; b < 4; b++)
      g[b] = ((G[sym(b, 0)] * dP[0] + G[sym(b, 1)] * dP[1]) + G[sym(b, 2)] * dP[2]) +
             G[sym(b, 3)] * dP[3];
    s[l] = ((dP[0] * g[0] + dP[1] * g[1]) + dP[2] * g[2]) + dP[3] * g[3];
  }
  for (int a = 0; a < 4; a++) {
    double c = ((Ti[a * 4 + 0] * s[0] + Ti[a * 4 + 1] * s[1]) + Ti[a * 4 + 2] * s[2]) +
               Ti[a * 4 + 3] * s[3];
    dQ[a] = y[a] - 0.5 * c;
  }
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3: ranges of neighbouring elements                             */
/* ------------------------------------------------------------------ */

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

/* Offsets investigated by the percolation test: the product of the four
 * per-axis alpha ranges, minus the centre.  Writes 4 ints per offset. */
int32_t vo4_alpha_offsets(const double* xi, double alpha, int32_t* off) {
  int lo[4], hi[4], n = 0;
  for (int a = 0; a < 4; a++) alpha_range(xi[a], alpha, &lo[a], &hi[a]);
  for (int o0 = lo[0]; o0 <= hi[0]; o0++)
    for (int o1 = lo[1]; o1 <= hi[1]; o1++)
      for (int o2 = lo[2]; o2 <= hi[2]; o2++)
        for (int o3 = lo[3]; o3 <= hi[3]; o3++) {
          if (o0 == 0 && o1 == 0 && o2 == 0 && o3 == 0) continue;
          off[4 * n] = o0;
          off[4 * n + 1] = o1;
          off[4 * n + 2] = o2;
          off[4 * n + 3] = o3;
          n++;
        }
  return n;
}

/* Offsets blended into Q_r (Sec. 2.3.2): per axis, below -beta -> {-1,0};
 * [-beta, beta) -> {-1,0,1} ("full"); from beta -> {0,1}; an offset with two
 * or more non-zero components is dropped when one of them is on a full
 * axis.  Centre included. */
int32_t vo4_beta_offsets(const double* xi, double beta, int32_t* off) {
  int lo[4], hi[4], full[4], n = 0;
  for (int a = 0; a < 4; a++) {
    lo[a] = (xi[a] < -beta) ? -1 : ((xi[a] < beta) ? -1 : 0);
    hi[a] = (xi[a] < -beta) ? 0 : 1;
    full[a] = (lo[a] == -1 && hi[a] == 1);
  }
  for (int o0 = lo[0]; o0 <= hi[0]; o0++)
    for (int o1 = lo[1]; o1 <= hi[1]; o1++)
      for (int o2 = lo[2]; o2 <= hi[2]; o2++)
        for (int o3 = lo[3]; o3 <= hi[3]; o3++) {
          int o[4] = {o0, o1, o2, o3}, nz = 0, onfull = 0;
          for (int a = 0; a < 4; a++)
            if (o[a] != 0) {
              nz++;
              if (full[a]) onfull = 1;
            }
          if (nz >= 2 && onfull) continue;
          for (int a = 0; a < 4; a++) off[4 * n + a] = o[a];
          n++;
        }
  return n;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.5: Poisson in 2D space, field, gradient and Hessian            */
/* ------------------------------------------------------------------ */

/* g(r_ij) = -2 G sum_{pixels p != (i,j)} M_p (r_ij - r_p) / |r_ij - r_p|^2,
 * r_ij - r_p = ((i - i_p) dx, (j - j_p) dy). */
void vo4_accel_at_node(const double* M, int32_t n0, int32_t n1, double dx, double dy, double G,
                       int64_t i, int64_t j, double* g2) {
  double gx = 0.0, gy = 0.0;
  for (int64_t p = 0; p < n0; p++)
    for (int64_t q = 0; q < n1; q++) {
      if (p == i && q == j) continue;
      double m = M[p * n1 + q];
      double rx = (double)(i - p) * dx;
      double ry = (double)(j - q) * dy;
      double r2 = rx * rx + ry * ry;
      double c = m / r2;
      gx = gx + c * rx;
      gy = gy + c * ry;
    }
  g2[0] = -(2.0 * G) * gx;
  g2[1] = -(2.0 * G) * gy;
}

/* Field record at node (i, j) from the accelerations at its 3x3 block
 * (ga[3][3][2], centre [1][1]): g, centred first differences J and second
 * differences K. */
static void field_from_block(const double ga[3][3][2], double dx, double dy, double* o) {
  o[0] = ga[1][1][0];
  o[1] = ga[1][1][1];
  for (int a = 0; a < 2; a++) {
    o[2 + 2 * a] = (ga[2][1][a] - ga[0][1][a]) / (2.0 * dx);
    o[3 + 2 * a] = (ga[1][2][a] - ga[1][0][a]) / (2.0 * dy);
    o[6 + 3 * a] = ((ga[2][1][a] + ga[0][1][a]) - 2.0 * ga[1][1][a]) / (dx * dx);
    o[7 + 3 * a] = (((ga[2][2][a] - ga[2][0][a]) - ga[0][2][a]) + ga[0][0][a]) / ((4.0 * dx) * dy);
    o[8 + 3 * a] = ((ga[1][2][a] + ga[1][0][a]) - 2.0 * ga[1][1][a]) / (dy * dy);
  }
}

void vo4_field_at_node(const double* M, int32_t n0, int32_t n1, double dx, double dy, double G,
                       int64_t i, int64_t j, double* out12) {
  double ga[3][3][2];
  for (int p = 0; p < 3; p++)
    for (int q = 0; q < 3; q++) vo4_accel_at_node(M, n0, n1, dx, dy, G, i + p - 1, j + q - 1, ga[p][q]);
  field_from_block(ga, dx, dy, out12);
}

/* ------------------------------------------------------------------ */
/* state                                                               */
/* ------------------------------------------------------------------ */

struct vo4_state {
  vo4_config c;
  double d[4], inv_d[4], dm[4], inv_dm[4], ctr[4];
  int32_t K[4], L[4], ne;
  int64_t nsite, npad, pstride[4], gstride[4];
  double *fini, *eta, *f;
  double* el;  /* NE x ne */
  double* tay; /* NT x ne */
  int32_t *map, *prevmap, *stamp, *queue;
  uint64_t* bestkey;
  double* M; /* n0 x n1 pixel masses */
  double Mtot;
  /* accelerations cached on the nodes [-E, n0-1+E] x [-E, n1-1+E] */
  int32_t E;
  double* gcache;
  const double* frozen; /* non-NULL: frozen polynomial field (12 coefficients) */
  int64_t stat_multi, stat_holes;
  int32_t stat_rounds;
  int64_t nstep;
  int32_t cyc;
};

static void lattice_q(const vo4_state* S, int64_t m, double* Q) {
  int64_t k[4];
  for (int a = 3; a >= 0; a--) {
    k[a] = m % S->L[a];
    m /= S->L[a];
  }
  for (int a = 0; a < 4; a++) Q[a] = S->ctr[a] + (double)(k[a] - S->K[a] - 1) * S->dm[a];
}

vo4_state* vo4_create(const vo4_config* c) {
  for (int a = 0; a < 4; a++)
    if (c->n[a] < 4 || !(c->hi[a] > c->lo[a])) return NULL;
  if (c->s < 1 || c->pad < 0 || c->n_s < 1) return NULL;
  vo4_state* S = (vo4_state*)calloc(1, sizeof(vo4_state));
  S->c = *c;
  int32_t nsum = 0;
  for (int a = 0; a < 4; a++) nsum += c->n[a];
  if (S->c.max_hole_rounds <= 0) S->c.max_hole_rounds = nsum;
  S->nsite = 1;
  S->npad = 1;
  S->ne = 1;
  for (int a = 0; a < 4; a++) {
    S->d[a] = (c->hi[a] - c->lo[a]) / (double)(c->n[a] - 1);
    S->dm[a] = (double)c->s * S->d[a];
    S->inv_d[a] = 1.0 / S->d[a];
    S->inv_dm[a] = 1.0 / S->dm[a];
    S->ctr[a] = 0.5 * (c->lo[a] + c->hi[a]);
    S->K[a] = (c->n[a] - 1 + 2 * c->s - 1) / (2 * c->s);
    S->L[a] = 2 * S->K[a] + 3;
    S->ne *= S->L[a];
    S->nsite *= c->n[a];
    S->npad *= c->n[a] + 2 * c->pad;
  }
  S->gstride[3] = 1;
  S->pstride[3] = 1;
  for (int a = 2; a >= 0; a--) {
    S->gstride[a] = S->gstride[a + 1] * c->n[a + 1];
    S->pstride[a] = S->pstride[a + 1] * (c->n[a + 1] + 2 * c->pad);
  }
  size_t n = (size_t)S->nsite;
  S->fini = (double*)calloc(n, sizeof(double));
  S->eta = (double*)calloc(n, sizeof(double));
  S->f = (double*)calloc(n, sizeof(double));
  S->el = (double*)calloc((size_t)S->ne * NE, sizeof(double));
  S->tay = (double*)calloc((size_t)S->ne * NT, sizeof(double));
  S->map = (int32_t*)malloc(sizeof(int32_t) * n);
  S->prevmap = (int32_t*)malloc(sizeof(int32_t) * n);
  S->bestkey = (uint64_t*)malloc(sizeof(uint64_t) * n);
  S->stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)S->npad);
  S->queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)S->npad);
  S->M = (double*)calloc((size_t)c->n[0] * c->n[1], sizeof(double));
  S->E = c->pad + 3;
  S->gcache = (double*)calloc((size_t)(c->n[0] + 2 * S->E) * (c->n[1] + 2 * S->E) * 2, sizeof(double));
  for (size_t p = 0; p < n; p++) S->map[p] = -1;
  return S;
}

void vo4_destroy(vo4_state* S) {
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
  free(S->M);
  free(S->gcache);
  free(S);
}

int32_t vo4_num_elements(const vo4_state* S) { return S->ne; }
void vo4_lattice_dims(const vo4_state* S, int32_t* L4) {
  for (int a = 0; a < 4; a++) L4[a] = S->L[a];
}

/* Sec. 2.3.2 (end of a cycle): isotropic elements on the lattice, T = I, H = 0. */
static void reset_elements(vo4_state* S) {
  memset(S->el, 0, sizeof(double) * NE * (size_t)S->ne);
  for (int64_t m = 0; m < S->ne; m++) {
    double* e = S->el + NE * m;
    lattice_q(S, m, e);
    for (int a = 0; a < 4; a++) e[4 + 5 * a] = 1.0;
  }
  S->cyc = 0;
}

int32_t vo4_set_f(vo4_state* S, const double* f0) {
  memcpy(S->fini, f0, sizeof(double) * (size_t)S->nsite);
  memcpy(S->f, f0, sizeof(double) * (size_t)S->nsite);
  vo4_spline_solve(S->c.n, S->fini, S->eta);
  reset_elements(S);
  S->nstep = 0;
  return 0;
}

void vo4_get_elements(const vo4_state* S, double* out) {
  memcpy(out, S->el, sizeof(double) * NE * (size_t)S->ne);
}
void vo4_set_elements(vo4_state* S, const double* in) {
  memcpy(S->el, in, sizeof(double) * NE * (size_t)S->ne);
}

static void compute_taylor(vo4_state* S) {
  for (int64_t m = 0; m < S->ne; m++) {
    double Q[4];
    lattice_q(S, m, Q);
    vo4_taylor_one(S->el + NE * m, Q, S->tay + NT * m);
  }
}

void vo4_get_taylor(vo4_state* S, double* out) {
  compute_taylor(S);
  memcpy(out, S->tay, sizeof(double) * NT * (size_t)S->ne);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3.1: percolation on the 4D lattice                             */
/* ------------------------------------------------------------------ */

static void site_pos(const vo4_state* S, const int64_t* g, double* P) {
  for (int a = 0; a < 4; a++) P[a] = S->c.lo[a] + (double)g[a] * S->d[a];
}

/* d^2 = sum_a (dQ_a / dm_a)^2 of element m at P (Sec. 2.3.1, eq. distdef). */
static double dist2(const vo4_state* S, int64_t m, const double* P, double* xi) {
  double dQ[4], x[4];
  vo4_qofp(S->tay + NT * m, P, dQ);
  for (int a = 0; a < 4; a++) x[a] = dQ[a] * S->inv_dm[a];
  if (xi)
    for (int a = 0; a < 4; a++) xi[a] = x[a];
  return ((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]) + x[3] * x[3];
}

static int64_t elem_offset(const vo4_state* S, int64_t m, const int32_t* o) {
  int64_t k[4], r = m;
  for (int a = 3; a >= 0; a--) {
    k[a] = r % S->L[a];
    r /= S->L[a];
  }
  int64_t mm = 0;
  for (int a = 0; a < 4; a++) {
    int64_t kk = k[a] + o[a];
    if (kk < 0 || kk >= S->L[a]) return -1;
    mm = mm * S->L[a] + kk;
  }
  return mm;
}

/* The site passes for m unless a neighbour in the alpha ranges proposes a
 * strictly smaller distance. */
static int passes(const vo4_state* S, int64_t m, const double* P, double* d2o) {
  double xi[4];
  double d2 = dist2(S, m, P, xi);
  *d2o = d2;
  int32_t off[4 * 16];
  int32_t n = vo4_alpha_offsets(xi, S->c.alpha, off);
  for (int32_t q = 0; q < n; q++) {
    int64_t mm = elem_offset(S, m, off + 4 * q);
    if (mm < 0) continue;
    if (dist2(S, mm, P, NULL) < d2) return 0;
  }
  return 1;
}

static void claim(vo4_state* S, const int64_t* g, int64_t m, double d2) {
  for (int a = 0; a < 4; a++)
    if (g[a] < 0 || g[a] >= S->c.n[a]) return;
  int64_t p = ((g[0] * S->c.n[1] + g[1]) * S->c.n[2] + g[2]) * S->c.n[3] + g[3];
  uint64_t key = dbits(d2);
  if (S->map[p] < 0) {
    S->map[p] = (int32_t)m;
    S->bestkey[p] = key;
    return;
  }
  S->stat_multi++;
  if (key < S->bestkey[p] || (key == S->bestkey[p] && m < S->map[p])) {
    S->map[p] = (int32_t)m;
    S->bestkey[p] = key;
  }
}

static void pad_coords(const vo4_state* S, int64_t pp, int64_t* g) {
  for (int a = 3; a >= 0; a--) {
    int64_t w = S->c.n[a] + 2 * S->c.pad;
    g[a] = pp % w - S->c.pad;
    pp /= w;
  }
}

static int64_t pad_index(const vo4_state* S, const int64_t* g) {
  int64_t pp = 0;
  for (int a = 0; a < 4; a++) pp = pp * (S->c.n[a] + 2 * S->c.pad) + (g[a] + S->c.pad);
  return pp;
}

static int in_pad(const vo4_state* S, const int64_t* g) {
  for (int a = 0; a < 4; a++)
    if (g[a] < -S->c.pad || g[a] >= S->c.n[a] + S->c.pad) return 0;
  return 1;
}

static int32_t percolate(vo4_state* S) {
  const int64_t n = S->nsite;
  for (int64_t p = 0; p < n; p++) S->map[p] = -1;
  for (int64_t p = 0; p < S->npad; p++) S->stamp[p] = -1;
  S->stat_multi = 0;
  for (int64_t m = 0; m < S->ne; m++) {
    const double* e = S->el + NE * m;
    int64_t g0[4];
    int ok = 1;
    for (int a = 0; a < 4; a++) {
      double u = (e[a] - S->c.lo[a]) * S->inv_d[a];
      if (!(u > -1e9 && u < 1e9)) ok = 0;
      else g0[a] = nearest(u);
    }
    if (!ok || !in_pad(S, g0)) continue;
    int64_t p0 = pad_index(S, g0);
    S->stamp[p0] = (int32_t)m;
    double P[4], d2;
    site_pos(S, g0, P);
    if (!passes(S, m, P, &d2)) continue;
    claim(S, g0, m, d2);
    int64_t qh = 0, qt = 0;
    S->queue[qt++] = (int32_t)p0;
    while (qh < qt) {
      int64_t g[4];
      pad_coords(S, S->queue[qh++], g);
      for (int a = 0; a < 4; a++)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          int64_t h[4] = {g[0], g[1], g[2], g[3]};
          h[a] += sgn;
          if (!in_pad(S, h)) continue;
          int64_t pp = pad_index(S, h);
          if (S->stamp[pp] == m) continue;
          S->stamp[pp] = (int32_t)m;
          site_pos(S, h, P);
          if (passes(S, m, P, &d2)) {
            claim(S, h, m, d2);
            S->queue[qt++] = (int32_t)pp;
          }
        }
    }
  }
  /* unexplored sites: Jacobi rounds over the 8 in-grid face neighbours */
  int64_t holes = 0;
  for (int64_t p = 0; p < n; p++) holes += (S->map[p] < 0);
  S->stat_holes = holes;
  int32_t rounds = 0;
  while (holes > 0) {
    if (rounds >= S->c.max_hole_rounds) {
      S->stat_rounds = rounds;
      return 4;
    }
    memcpy(S->prevmap, S->map, sizeof(int32_t) * (size_t)n);
    for (int64_t p = 0; p < n; p++) {
      if (S->prevmap[p] >= 0) continue;
      int64_t g[4], r = p;
      for (int a = 3; a >= 0; a--) {
        g[a] = r % S->c.n[a];
        r /= S->c.n[a];
      }
      double P[4];
      site_pos(S, g, P);
      int32_t best = -1;
      uint64_t bestk = 0;
      for (int a = 0; a < 4; a++)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          int64_t ga = g[a] + sgn;
          if (ga < 0 || ga >= S->c.n[a]) continue;
          int32_t cand = S->prevmap[p + sgn * S->gstride[a]];
          if (cand < 0) continue;
          uint64_t key = dbits(dist2(S, cand, P, NULL));
          if (best < 0 || key < bestk || (key == bestk && cand < best)) {
            best = cand;
            bestk = key;
          }
        }
      S->map[p] = best;
    }
    holes = 0;
    for (int64_t p = 0; p < n; p++) holes += (S->map[p] < 0);
    rounds++;
  }
  S->stat_rounds = rounds;
  return 0;
}

int32_t vo4_compute_map(vo4_state* S, int32_t* map_out) {
  compute_taylor(S);
  int32_t st = percolate(S);
  if (map_out) memcpy(map_out, S->map, sizeof(int32_t) * (size_t)S->nsite);
  return st;
}

void vo4_get_map(const vo4_state* S, int32_t* out) {
  memcpy(out, S->map, sizeof(int32_t) * (size_t)S->nsite);
}

void vo4_map_stats(const vo4_state* S, int64_t* multi, int64_t* holes, int32_t* rounds) {
  *multi = S->stat_multi;
  *holes = S->stat_holes;
  *rounds = S->stat_rounds;
}

/* ------------------------------------------------------------------ */
/* transport reconstruction, pixel masses and the field                  */
/* ------------------------------------------------------------------ */

/* acceleration at node (i, j): frozen polynomial, cache, or direct sum */
static void node_accel(const vo4_state* S, int64_t i, int64_t j, double* g2) {
  if (S->frozen) {
    const double* c = S->frozen;
    double x = S->c.lo[0] + (double)i * S->d[0];
    double y = S->c.lo[1] + (double)j * S->d[1];
    for (int a = 0; a < 2; a++) {
      const double* B = c + 6 + 3 * a;
      double q = ((B[0] * x) * x + ((2.0 * B[1]) * x) * y) + (B[2] * y) * y;
      g2[a] = ((c[a] + c[2 + 2 * a] * x) + c[3 + 2 * a] * y) + 0.5 * q;
    }
    return;
  }
  const int32_t E = S->E, W1 = S->c.n[1] + 2 * E;
  if (i >= -E && i < S->c.n[0] + E && j >= -E && j < S->c.n[1] + E) {
    const double* q = S->gcache + 2 * ((i + E) * W1 + (j + E));
    g2[0] = q[0];
    g2[1] = q[1];
    return;
  }
  vo4_accel_at_node(S->M, S->c.n[0], S->c.n[1], S->d[0], S->d[1], S->c.G, i, j, g2);
}

static void node_field(const vo4_state* S, int64_t i, int64_t j, double* out12) {
  double ga[3][3][2];
  for (int p = 0; p < 3; p++)
    for (int q = 0; q < 3; q++) node_accel(S, i + p - 1, j + q - 1, ga[p][q]);
  field_from_block(ga, S->d[0], S->d[1], out12);
}

static void fill_gcache(vo4_state* S) {
  const int32_t E = S->E, W0 = S->c.n[0] + 2 * E, W1 = S->c.n[1] + 2 * E;
  for (int32_t a = 0; a < W0; a++)
    for (int32_t b = 0; b < W1; b++)
      vo4_accel_at_node(S->M, S->c.n[0], S->c.n[1], S->d[0], S->d[1], S->c.G, a - E, b - E,
                        S->gcache + 2 * ((int64_t)a * W1 + b));
}

/* f(P) = f_ini(Q(P)) through the owner's inverse map and the 15-point
 * interpolation; pixel masses M(i, j) = (sum_{k,l} f) dx dy dvx dvy. */
static void reconstruct_and_field(vo4_state* S) {
  const int32_t* n = S->c.n;
  const double dV = ((S->d[0] * S->d[1]) * S->d[2]) * S->d[3];
  double Mtot = 0.0;
  for (int64_t i = 0; i < n[0]; i++)
    for (int64_t j = 0; j < n[1]; j++) {
      double sum = 0.0;
      for (int64_t k = 0; k < n[2]; k++)
        for (int64_t l = 0; l < n[3]; l++) {
          int64_t g[4] = {i, j, k, l};
          int64_t p = ((i * n[1] + j) * n[2] + k) * n[3] + l;
          int32_t m = S->map[p];
          double fv = 0.0;
          if (m >= 0) {
            const double* t = S->tay + NT * (int64_t)m;
            double P[4], dQ[4], u[4];
            site_pos(S, g, P);
            vo4_qofp(t, P, dQ);
            for (int a = 0; a < 4; a++) u[a] = ((t[60 + a] + dQ[a]) - S->c.lo[a]) * S->inv_d[a];
            fv = vo4_qinterp(S->fini, n, u);
          }
          S->f[p] = fv;
          sum = sum + fv;
        }
      S->M[i * n[1] + j] = sum * dV;
      Mtot = Mtot + S->M[i * n[1] + j];
    }
  S->Mtot = Mtot;
  fill_gcache(S);
}

int32_t vo4_reconstruct(vo4_state* S, double* f_out) {
  int32_t st = vo4_compute_map(S, NULL);
  reconstruct_and_field(S);
  if (f_out) memcpy(f_out, S->f, sizeof(double) * (size_t)S->nsite);
  return st;
}

void vo4_density_force(vo4_state* S, double* M, double* field12, double* Mtot) {
  const int32_t n0 = S->c.n[0], n1 = S->c.n[1];
  if (M) memcpy(M, S->M, sizeof(double) * (size_t)n0 * n1);
  if (field12)
    for (int64_t i = 0; i < n0; i++)
      for (int64_t j = 0; j < n1; j++) node_field(S, i, j, field12 + 12 * (i * n1 + j));
  if (Mtot) *Mtot = S->Mtot;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.4: drift-kick-drift                                            */
/* ------------------------------------------------------------------ */

static void drift_half(vo4_state* S) {
  const double h = 0.5 * S->c.dt;
  for (int64_t m = 0; m < S->ne; m++) {
    double* e = S->el + NE * m;
    double* T = e + 4;
    double* H = e + 20;
    for (int a = 0; a < 2; a++) {
      e[a] = e[a] + e[a + 2] * h;
      for (int b = 0; b < 4; b++) T[a * 4 + b] = T[a * 4 + b] + T[(a + 2) * 4 + b] * h;
      for (int q = 0; q < 10; q++) H[10 * a + q] = H[10 * a + q] + H[10 * (a + 2) + q] * h;
    }
  }
}

/* 1D TSC weights at offset w from the nearest node */
static void tsc_w(double w, double* o) {
  o[0] = 0.5 * ((0.5 - w) * (0.5 - w));
  o[1] = 0.75 - w * w;
  o[2] = 0.5 * ((0.5 + w) * (0.5 + w));
}

/* Kick over a full step with the field interpolated at the drifted element
 * position by the 2D TSC weights: dv_a = g_a dt,
 * dT_{2+a,j} = sum_b J_ab T_bj dt,
 * dH_{2+a,jk} = (sum_b J_ab H_b,jk + sum_bc K_a,bc T_bj T_ck) dt. */
static void kick(vo4_state* S) {
  const double dt = S->c.dt;
  for (int64_t m = 0; m < S->ne; m++) {
    double* e = S->el + NE * m;
    double* T = e + 4;
    double* H = e + 20;
    double ux = (e[0] - S->c.lo[0]) * S->inv_d[0];
    double uy = (e[1] - S->c.lo[1]) * S->inv_d[1];
    if (!(ux > -1e9 && ux < 1e9 && uy > -1e9 && uy < 1e9)) continue;
    int64_t i = nearest(ux), j = nearest(uy);
    double wx[3], wy[3];
    tsc_w(ux - (double)i, wx);
    tsc_w(uy - (double)j, wy);
    double nf[3][3][12];
    for (int p = 0; p < 3; p++)
      for (int q = 0; q < 3; q++) node_field(S, i + p - 1, j + q - 1, nf[p][q]);
    double F[12];
    for (int c = 0; c < 12; c++) {
      double row[3];
      for (int p = 0; p < 3; p++) row[p] = (wy[0] * nf[p][0][c] + wy[1] * nf[p][1][c]) + wy[2] * nf[p][2][c];
      F[c] = (wx[0] * row[0] + wx[1] * row[1]) + wx[2] * row[2];
    }
    const double* J = F + 2;  /* Jxx Jxy Jyx Jyy */
    const double* Kf = F + 6; /* Kx_xx Kx_xy Kx_yy Ky_xx Ky_xy Ky_yy */
    double Tx[2][4];
    double Hx[2][10];
    for (int b = 0; b < 2; b++) {
      for (int q = 0; q < 4; q++) Tx[b][q] = T[b * 4 + q];
      for (int q = 0; q < 10; q++) Hx[b][q] = H[10 * b + q];
    }
    for (int a = 0; a < 2; a++) {
      const double Ja0 = J[2 * a], Ja1 = J[2 * a + 1];
      const double Kxx = Kf[3 * a], Kxy = Kf[3 * a + 1], Kyy = Kf[3 * a + 2];
      e[2 + a] = e[2 + a] + F[a] * dt;
      for (int q = 0; q < 4; q++)
        T[(2 + a) * 4 + q] = T[(2 + a) * 4 + q] + (Ja0 * Tx[0][q] + Ja1 * Tx[1][q]) * dt;
      for (int b = 0; b < 4; b++)
        for (int c = b; c < 4; c++) {
          double t1 = Ja0 * Hx[0][sym(b, c)] + Ja1 * Hx[1][sym(b, c)];
          double t2 = (((Kxx * Tx[0][b]) * Tx[0][c] + (Kxy * Tx[0][b]) * Tx[1][c]) +
                       (Kxy * Tx[1][b]) * Tx[0][c]) + (Kyy * Tx[1][b]) * Tx[1][c];
          H[10 * (2 + a) + sym(b, c)] = H[10 * (2 + a) + sym(b, c)] + (t1 + t2) * dt;
        }
    }
  }
}

/* ------------------------------------------------------------------ */
/* Secs. 2.2.2 and 2.3.2: remap                                          */
/* ------------------------------------------------------------------ */

/* Q_r = sum W(2 d_m') Q(P, m') / sum W(2 d_m') over the beta set of the
 * owner m; Q(P, m) when the weights vanish. */
static void blended_q(const vo4_state* S, int64_t m, const double* P, double* Qr) {
  double xi[4];
  dist2(S, m, P, xi);
  int32_t off[4 * 81];
  int32_t n = vo4_beta_offsets(xi, S->c.beta, off);
  double num[4] = {0.0, 0.0, 0.0, 0.0}, den = 0.0;
  for (int32_t q = 0; q < n; q++) {
    int64_t mm = elem_offset(S, m, off + 4 * q);
    if (mm < 0) continue;
    const double* t = S->tay + NT * mm;
    double dQ[4], x[4];
    vo4_qofp(t, P, dQ);
    for (int a = 0; a < 4; a++) x[a] = dQ[a] * S->inv_dm[a];
    double d = sqrt(((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]) + x[3] * x[3]);
    double w = vo_W(2.0 * d);
    for (int a = 0; a < 4; a++) num[a] = num[a] + w * (t[60 + a] + dQ[a]);
    den = den + w;
  }
  if (den > 0.0) {
    for (int a = 0; a < 4; a++) Qr[a] = num[a] / den;
  } else {
    const double* t = S->tay + NT * m;
    double dQ[4];
    vo4_qofp(t, P, dQ);
    for (int a = 0; a < 4; a++) Qr[a] = t[60 + a] + dQ[a];
  }
}

int32_t vo4_remap_resample(vo4_state* S, double* fnew, double* Qr_out) {
  const int32_t* n = S->c.n;
  int32_t st = vo4_compute_map(S, NULL);
  for (int64_t p = 0; p < S->nsite; p++) {
    int32_t m = S->map[p];
    double val = 0.0;
    if (m >= 0) {
      int64_t g[4], r = p;
      for (int a = 3; a >= 0; a--) {
        g[a] = r % n[a];
        r /= n[a];
      }
      double P[4], Qr[4], u[4];
      site_pos(S, g, P);
      blended_q(S, m, P, Qr);
      for (int a = 0; a < 4; a++) u[a] = (Qr[a] - S->c.lo[a]) * S->inv_d[a];
      val = vo4_spline_eval(S->eta, n, u);
      if (Qr_out)
        for (int a = 0; a < 4; a++) Qr_out[4 * p + a] = Qr[a];
    } else if (Qr_out) {
      for (int a = 0; a < 4; a++) Qr_out[4 * p + a] = 0.0;
    }
    fnew[p] = val;
  }
  return st;
}

int32_t vo4_remap(vo4_state* S) {
  double* fnew = (double*)malloc(sizeof(double) * (size_t)S->nsite);
  int32_t st = vo4_remap_resample(S, fnew, NULL);
  memcpy(S->fini, fnew, sizeof(double) * (size_t)S->nsite);
  free(fnew);
  vo4_spline_solve(S->c.n, S->fini, S->eta);
  reset_elements(S);
  return st;
}

/* One step (Sec. 2.4): half drift; map; f(t + dt/2); masses and field;
 * kick; half drift; remap at the end of every n_s-th step of a cycle. */
int32_t vo4_step(vo4_state* S, int32_t nsteps) {
  int32_t st = 0;
  for (int32_t it = 0; it < nsteps; it++) {
    drift_half(S);
    int32_t s1 = vo4_compute_map(S, NULL);
    if (s1) st = s1;
    reconstruct_and_field(S);
    kick(S);
    drift_half(S);
    S->nstep++;
    S->cyc++;
    if (S->cyc >= S->c.n_s) {
      int32_t s2 = vo4_remap(S);
      if (s2) st = s2;
    }
  }
  return st;
}

void vo4_push_frozen(vo4_state* S, const double* coef12, int32_t nsteps) {
  S->frozen = coef12;
  for (int32_t it = 0; it < nsteps; it++) {
    drift_half(S);
    kick(S);
    drift_half(S);
  }
  S->frozen = NULL;
}

void vo4_get_fini(const vo4_state* S, double* out) {
  memcpy(out, S->fini, sizeof(double) * (size_t)S->nsite);
}
void vo4_get_eta(const vo4_state* S, double* out) {
  memcpy(out, S->eta, sizeof(double) * (size_t)S->nsite);
}
void vo4_get_last_f(const vo4_state* S, double* out) {
  memcpy(out, S->f, sizeof(double) * (size_t)S->nsite);
}
int64_t vo4_step_count(const vo4_state* S) { return S->nstep; }

/* mass sum f dV; kinetic energy sum (vx^2 + vy^2)/2 f dV; potential energy
 * (1/2) sum_p M_p phi_p with phi_p = 2 G sum_{q != p} M_q ln|r_p - r_q|. */
void vo4_diagnostics(vo4_state* S, double* mass, double* ekin, double* epot, double* dmin,
                     double* dmax) {
  const int32_t* n = S->c.n;
  const double dV = ((S->d[0] * S->d[1]) * S->d[2]) * S->d[3];
  double ms = 0.0, ek = 0.0;
  for (int64_t p = 0; p < S->nsite; p++) {
    int64_t l = p % n[3], k = (p / n[3]) % n[2];
    double vx = S->c.lo[2] + (double)k * S->d[2];
    double vy = S->c.lo[3] + (double)l * S->d[3];
    ms = ms + S->f[p] * dV;
    ek = ek + ((0.5 * (vx * vx + vy * vy)) * S->f[p]) * dV;
  }
  double ep = 0.0;
  if (S->c.G != 0.0) {
    /* pixel masses of the last f (the reconstruction's, or f0's before a step) */
    const int64_t np = (int64_t)n[0] * n[1], nvel = (int64_t)n[2] * n[3];
    double* Mp = (double*)malloc(sizeof(double) * (size_t)np);
    for (int64_t q = 0; q < np; q++) {
      double sum = 0.0;
      for (int64_t r = 0; r < nvel; r++) sum = sum + S->f[q * nvel + r];
      Mp[q] = sum * dV;
    }
    for (int64_t i = 0; i < n[0]; i++)
      for (int64_t j = 0; j < n[1]; j++) {
        double phi = 0.0;
        for (int64_t a = 0; a < n[0]; a++)
          for (int64_t b = 0; b < n[1]; b++) {
            if (a == i && b == j) continue;
            double rx = (double)(i - a) * S->d[0], ry = (double)(j - b) * S->d[1];
            phi = phi + Mp[a * n[1] + b] * log(sqrt(rx * rx + ry * ry));
          }
        ep = ep + 0.5 * (Mp[i * n[1] + j] * ((2.0 * S->c.G) * phi));
      }
    free(Mp);
  }
  *mass = ms;
  *ekin = ek;
  *epot = ep;
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t m = 0; m < S->ne; m++) {
    double d = det4(S->el + NE * m + 4);
    if (d < lo) lo = d;
    if (d > hi) hi = d;
  }
  *dmin = lo;
  *dmax = hi;
}
