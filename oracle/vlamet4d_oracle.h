/*
 * FP64 CPU oracle of the metric semi-Lagrangian step in four-dimensional
 * phase space (two space dimensions x, y and two velocity dimensions
 * vx, vy): the generalisation of the method that Secs. 2.1, 2.2.1, 2.3 and
 * 2.5 describe for 4D (60-number elements, 15-point quadratic
 * interpolation, percolation on a 4D lattice, Poisson in 2D space).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests and the CPU-baseline leg of
 * the benchmark; the product path never links, loads or calls it, and it
 * shares no header, helper or table with the CUDA sources.
 *
 * Conventions (the readings that this oracle fixes):
 *   - node-centred fixed box per axis a = 0..3 (x, y, vx, vy):
 *     node i of axis a sits at lo[a] + i*d[a], d[a] = (hi[a]-lo[a])/(n[a]-1);
 *     f is stored f[((i0*n1 + i1)*n2 + i2)*n3 + i3] (vy fastest);
 *   - the element lattice is centred on the box, spacing s*d[a], with one
 *     extra layer on every side: L[a] = 2*K[a]+3 elements along axis a,
 *     K[a] = ceil(((n[a]-1)/2)/s); element m = ((k0*L1 + k1)*L2 + k2)*L3 + k3;
 *   - element state, 60 doubles: P[4]; T[16] row major, T[a*4+b] = dP_a/dQ_b;
 *     H[40], H[a*10 + sym(b,c)] = d2P_a/dQ_b dQ_c with the symmetric index
 *     order (00,01,02,03,11,12,13,22,23,33);
 *   - Taylor record, 64 doubles: P[4], Ti[16] (T^-1 row major),
 *     G[40] (G_l = [T^-1]^T H_l T^-1, same symmetric order), Q_m[4];
 *   - pixel masses M[i0*n1 + i1] over the (x, y) nodes; the field at a node
 *     is 12 doubles: gx, gy, Jxx, Jxy, Jyx, Jyy (J_ab = dg_a/dx_b),
 *     Kx_xx, Kx_xy, Kx_yy, Ky_xx, Ky_xy, Ky_yy (K_a,bc = d2g_a/dx_b dx_c).
 */
#ifndef VLAMET4D_ORACLE_H
#define VLAMET4D_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n[4];
  double lo[4], hi[4];
  int32_t s;               /* element spacing in grid sites (every axis) */
  double dt;
  int32_t n_s;             /* transport steps between remaps */
  double G;                /* Poisson in 2D space: lap(phi) = 4 pi G rho */
  double alpha, beta;      /* range margins of the percolation and of Q_r */
  int32_t pad;             /* connectivity margin around the grid, in sites */
  int32_t max_hole_rounds; /* cap on the unexplored-site repair rounds */
} vo4_config;

typedef struct vo4_state vo4_state;

/* ---- low-level pieces (each pinned separately by the tests) ---- */
double vo4_qinterp(const double* F, const int32_t* n, const double* u);
void vo4_spline_solve(const int32_t* n, const double* f, double* eta);
double vo4_spline_eval(const double* eta, const int32_t* n, const double* u);
void vo4_taylor_one(const double* el60, const double* Qm, double* tay64);
void vo4_qofp(const double* tay64, const double* P, double* dQ);
int32_t vo4_alpha_offsets(const double* xi, double alpha, int32_t* off);
int32_t vo4_beta_offsets(const double* xi, double beta, int32_t* off);
/* pixel masses M (n0 x n1) -> field of 12 doubles at node (i, j), any
 * integers (nodes outside the grid included) */
void vo4_field_at_node(const double* M, int32_t n0, int32_t n1, double dx, double dy, double G,
                       int64_t i, int64_t j, double* out12);
/* gravitational acceleration at node (i, j) by the direct sum over the
 * pixel masses, the node's own pixel excluded */
void vo4_accel_at_node(const double* M, int32_t n0, int32_t n1, double dx, double dy, double G,
                       int64_t i, int64_t j, double* g2);

/* ---- solver state ---- */
vo4_state* vo4_create(const vo4_config* c);
void vo4_destroy(vo4_state* S);
int32_t vo4_num_elements(const vo4_state* S);
void vo4_lattice_dims(const vo4_state* S, int32_t* L4);
int32_t vo4_set_f(vo4_state* S, const double* f0);
void vo4_get_elements(const vo4_state* S, double* out60xne);
void vo4_set_elements(vo4_state* S, const double* in60xne);
void vo4_get_taylor(vo4_state* S, double* out64xne);
int32_t vo4_compute_map(vo4_state* S, int32_t* map_out);
/* the last map (of vo4_compute_map, vo4_reconstruct, a step or a remap) */
void vo4_get_map(const vo4_state* S, int32_t* out);
void vo4_map_stats(const vo4_state* S, int64_t* claimed_multi, int64_t* holes, int32_t* rounds);
int32_t vo4_reconstruct(vo4_state* S, double* f_out);
/* pixel masses of the last reconstruction and the field at the grid nodes */
void vo4_density_force(vo4_state* S, double* M, double* field12, double* Mtot);
int32_t vo4_step(vo4_state* S, int32_t nsteps);
int32_t vo4_remap(vo4_state* S);
/* f_new at every site and, when Qr_out is not NULL, the blended Q_r (4 per site) */
int32_t vo4_remap_resample(vo4_state* S, double* fnew_out, double* Qr_out);
void vo4_get_fini(const vo4_state* S, double* out);
void vo4_get_eta(const vo4_state* S, double* out);
void vo4_get_last_f(const vo4_state* S, double* out);
int64_t vo4_step_count(const vo4_state* S);
/* mass, kinetic and potential energy of the last f; min and max det T */
void vo4_diagnostics(vo4_state* S, double* mass, double* ekin, double* epot, double* detT_min,
                     double* detT_max);
/* element push (drift-kick-drift) under a frozen polynomial acceleration
 * g_a(x, y) = c_a + A_a0 x + A_a1 y + (B_a,xx x^2 + 2 B_a,xy x y + B_a,yy y^2)/2
 * sampled on the nodes (any node, also outside the grid); coef12 = c[2],
 * A[4] row major, B[6] (xx, xy, yy for a = x, then for a = y) */
void vo4_push_frozen(vo4_state* S, const double* coef12, int32_t nsteps);

#ifdef __cplusplus
}
#endif
#endif
