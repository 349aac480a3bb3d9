/*
 * FP64 CPU oracle of the metric semi-Lagrangian Vlasov-Poisson step
 * (Colombi & Alard, "A 'metric' semi-Lagrangian Vlasov-Poisson solver").
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists so that the tests, the smoke
 * check and the CPU-baseline leg of the benchmark can compare the CUDA path
 * against a plain, slow, serial restatement of the paper.  The product path
 * never links, loads or calls it, and it shares no header, helper or table
 * with the CUDA sources.
 *
 * Conventions (the readings of the paper that this oracle fixes):
 *   - node-centred fixed box: x_i = x_lo + i*dx, dx = (x_hi-x_lo)/(nx-1),
 *     same for v; f is stored f[i*nv + j] (v fastest);
 *   - the element lattice is centred on the box, spacing s*dx by s*dv, with
 *     one extra layer on every side: Lx = 2*Kx+3 elements along x where
 *     Kx = ceil(((nx-1)/2)/s); element m = k*Lv + l;
 *   - element state, 12 doubles, in this order:
 *     x, v, Txx, Txv, Tvx, Tvv, Hx_xx, Hx_xv, Hx_vv, Hv_xx, Hv_xv, Hv_vv
 *     with T_ab = dP_a/dQ_b and H_a,bc = d2P_a/dQ_b dQ_c;
 *   - Taylor record, 14 doubles: x, v, Ti00, Ti01, Ti10, Ti11,
 *     Gx00, Gx01, Gx11, Gv00, Gv01, Gv11, Qx, Qv.
 */
#ifndef VLAMET_ORACLE_H
#define VLAMET_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t nx, nv;
  double x_lo, x_hi, v_lo, v_hi;
  int32_t s;               /* element spacing in grid sites (both axes) */
  double dt;
  int32_t n_s;             /* transport steps between remaps */
  double G;                /* gravitational constant; force = 2*pi*G*(M_right-M_left) */
  double alpha, beta;      /* range margins of the percolation and of Q_r */
  int32_t pad;             /* connectivity margin around the grid, in sites */
  int32_t literal_fd;      /* 1: a' = (a(i+1)-a(i-1))/dx exactly as printed */
  int32_t max_hole_rounds; /* cap on the unexplored-site repair rounds */
} vo_config;

typedef struct vo_state vo_state;

enum { VO_OK = 0, VO_E_INVALID = 1, VO_E_NOT_CONVERGED = 4 };

/* ---- low-level pieces (each pinned separately by the tests) ---- */
double vo_qinterp(const double* F, int32_t nx, int32_t nv, double u, double w);
void vo_spline_solve_1d(int32_t n, const double* f, double* eta);
void vo_spline_solve_2d(int32_t nx, int32_t nv, const double* f, double* eta);
double vo_bspline3(double t);
double vo_spline_eval(const double* eta, int32_t nx, int32_t nv, double u, double w);
void vo_taylor_one(const double* el12, double Qx, double Qv, double* tay14);
void vo_qofp(const double* tay14, double Px, double Pv, double* dqx, double* dqv);
double vo_W(double x);
void vo_force_from_mass(const double* M, int32_t nx, double dx, double G,
                        int32_t literal_fd, double* a, double* da, double* d2a);
double vo_tsc(const double* A, int32_t nx, double ext_lo, double ext_hi, double u);
int32_t vo_alpha_offsets(double xi, double ze, double alpha, int32_t* ab18);
int32_t vo_beta_offsets(double xi, double ze, double beta, int32_t* ab18);

/* ---- solver state ---- */
vo_state* vo_create(const vo_config* c);
void vo_destroy(vo_state* S);
int32_t vo_num_elements(const vo_state* S);
int32_t vo_lattice_dims(const vo_state* S, int32_t* Lx, int32_t* Lv);
int32_t vo_set_f(vo_state* S, const double* f0);
void vo_get_elements(const vo_state* S, double* out12xne_aos);
void vo_set_elements(vo_state* S, const double* in12xne_aos);
void vo_get_taylor(vo_state* S, double* out14xne_aos);
int32_t vo_compute_map(vo_state* S, int32_t* map_out);
void vo_component_bbox(const vo_state* S, int32_t* out4xne);
int32_t vo_map_stats(const vo_state* S, int64_t* claimed_multi, int64_t* holes, int32_t* rounds);
int32_t vo_reconstruct(vo_state* S, double* f_out);
void vo_density_force(const vo_state* S, double* M, double* a, double* da, double* d2a,
                      double* Mtot);
int32_t vo_step(vo_state* S, int32_t nsteps);
int32_t vo_remap(vo_state* S);
int32_t vo_remap_resample(vo_state* S, double* fnew_out, double* Qr_out);
void vo_get_fini(const vo_state* S, double* out);
void vo_get_eta(const vo_state* S, double* out);
void vo_get_last_f(const vo_state* S, double* out);
int64_t vo_step_count(const vo_state* S);
int32_t vo_cycle_step(const vo_state* S);
void vo_diagnostics(const vo_state* S, double* mass, double* energy, double* detT_min,
                    double* detT_max);
/* Sec. 3.2: S = -sum f log|f| dx dv, L1 and L2 norms of the last f. */
void vo_casimirs(const vo_state* S, double* entropy, double* l1, double* l2);
/* Sec. 2.3.2: E_map of the last influence map, in element spacings. */
double vo_emap(const vo_state* S);
/* Sec. 2.4: variable time step min(dt, c_dyn / sqrt(rho_max)); 0: constant. */
void vo_set_cdyn(vo_state* S, double c_dyn);
/* Sec. 2.2.1 eq. constrf and Sec. 2.3: adaptive computing domain with
 * threshold f_th (0: the fixed box); takes effect at the next vo_set_f or
 * remap.  vo_domain: existing lattice rows/columns (klo, khi, llo, lhi) and
 * the last map's site rectangle (i_lo, i_hi, j_lo, j_hi). */
void vo_set_fth(vo_state* S, double f_th);
void vo_domain(const vo_state* S, int32_t* act4, int32_t* rect4);
double vo_time(const vo_state* S);
double vo_last_dt(const vo_state* S);
/* element push under a frozen grid force (a, a', a'' given on the x nodes) */
void vo_push_frozen(vo_state* S, const double* a, const double* da, const double* d2a,
                    double ext_lo, double ext_hi, int32_t nsteps);

#ifdef __cplusplus
}
#endif
#endif
