/*
 * vlamet4d.h -- C ABI of the 4D phase-space (two space dimensions) form of
 * the metric semi-Lagrangian Vlasov-Poisson solver (Colombi & Alard).
 *
 * The paper implements 2D phase space and describes how each piece carries
 * over to 4D: elements of 4 + 16 + 40 = 60 numbers (Sec. 2.1), the inverse
 * map of eq. QofP with 4x4 matrices, the second-order hypersurface through
 * 15 grid points (Sec. 2.2.1), percolation with per-axis ranges on a 4D
 * lattice (Sec. 2.3), and Poisson's equation in the space dimensions on a
 * fixed grid (Sec. 2.5).  This library runs that method, FP64 throughout,
 * in its own CUDA kernels on the caller's stream.
 *
 * Grid and storage conventions:
 *   - axes a = 0..3 are x, y, vx, vy; node i of axis a sits at
 *     lo[a] + i*d[a], d[a] = (hi[a] - lo[a])/(n[a] - 1);
 *   - f, f_ini, eta and the map are n0 x n1 x n2 x n3 arrays, vy fastest
 *     (site (i0, i1, i2, i3) at offset ((i0*n1 + i1)*n2 + i2)*n3 + i3);
 *   - elements sit on a lattice centred on the box with spacing s*d[a] and one
 *     extra layer on every side: L[a] = 2*K[a] + 3, K[a] = ceil(((n[a]-1)/2)/s);
 *     element m = ((k0*L1 + k1)*L2 + k2)*L3 + k3;
 *   - element state exchanged as 60 doubles per element (element-major):
 *     P[4]; T[16] row major, T[a*4+b] = dP_a/dQ_b; H[40], H[a*10 + q] =
 *     d2P_a/dQ_b dQ_c with q the symmetric index of (b, c) in the order
 *     00,01,02,03,11,12,13,22,23,33;
 *   - pixel masses M are n0 x n1 (y fastest); the field at a node is 12
 *     doubles: gx, gy, Jxx, Jxy, Jyx, Jyy (J_ab = dg_a/dx_b), Kx_xx, Kx_xy,
 *     Kx_yy, Ky_xx, Ky_xy, Ky_yy (K_a,bc = d2g_a/dx_b dx_c).
 *
 * Ownership, errors and threads follow vlamet.h: one caller workspace
 * (vm_4d_workspace_bytes) kept alive until vm_4d_destroy; every call returns
 * a vm_status; device-side failures set an error word that the synchronising
 * calls (vm_4d_sync and every copy to the host) read and clear; calls on one
 * solver must not overlap.
 */
#ifndef VLAMET4D_H
#define VLAMET4D_H

#include <stddef.h>
#include <stdint.h>

#include "vlamet.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n[4];            /* nodes per axis (x, y, vx, vy), each >= 4 */
  double lo[4], hi[4];     /* box per axis */
  int32_t elem_stride;     /* s: element spacing in grid sites on every axis, 1..8 */
  double dt;               /* time step (Sec. 2.4) */
  int32_t n_s;             /* transport steps between remaps */
  double G;                /* Poisson in 2D space: lap(phi) = 4 pi G rho (Sec. 2.5) */
  double alpha, beta;      /* percolation and Q_r margins (Sec. 2.3.3); 0 -> the paper's */
  int32_t pad;             /* connectivity margin around the grid, sites; 0 -> s */
  int32_t max_hole_rounds; /* cap on unexplored-site repair rounds; 0 -> n0+n1+n2+n3 */
} vm_4d_config;

typedef struct vm_4d_solver vm_4d_solver;

typedef struct {
  double mass;      /* sum f dx dy dvx dvy of the last f */
  double ekin;      /* (1/2) sum (vx^2 + vy^2) f dx dy dvx dvy */
  double epot;      /* (1/2) sum_p M_p phi_p, phi_p = 2 G sum_{q != p} M_q ln|r_p - r_q| over the
                       pixel masses M of the last f (the discrete energy of Sec. 2.5's Poisson
                       solution in 2D space) */
  double detT_min;  /* range of det T over the elements (Sec. 2.1, |T| = 1) */
  double detT_max;
} vm_4d_diag;

/* Device bytes a solver of config *c needs (0 if *c is invalid). */
size_t vm_4d_workspace_bytes(const vm_4d_config* c);

/* Create a solver on the caller's workspace (device, 256-byte aligned, at
 * least vm_4d_workspace_bytes(c) bytes) and stream (NULL: the legacy default
 * stream).  VM_E_INVALID_ARG for a bad config or workspace pointer,
 * VM_E_OOM for a workspace too small. */
vm_status vm_4d_create(const vm_4d_config* c, void* d_workspace, size_t workspace_bytes,
                       void* cuda_stream, vm_4d_solver** out);
void vm_4d_destroy(vm_4d_solver* s);

/* Initial condition (Sec. 2.2.2 and 2.3.2 at t = 0): f_ini <- f, spline
 * coefficients eta of f_ini (tensor product of the 1D zero-slope solve along
 * vy, vx, y, x), isotropic elements on the lattice (T = I, H = 0).  f: host
 * or device (on_device) FP64 array of n0*n1*n2*n3 values. */
vm_status vm_4d_set_f(vm_4d_solver* s, const double* f, int on_device);

/* nsteps drift-kick-drift steps (Sec. 2.4): half drift of the elements;
 * Taylor terms T^-1 and [T^-1]^T H_l T^-1 (Sec. 2.1); influence map by
 * percolation (Sec. 2.3.1); f(t + dt/2) = f_ini(Q(P)) by the 15-point
 * quadratic interpolation (Sec. 2.2.1); pixel masses; the field of the 2D
 * Poisson equation with its gradient and Hessian (Sec. 2.5); kick; half
 * drift; a remap (Sec. 2.3.2: f_ini <- spline(f_ini)(Q_r(P)), new eta,
 * isotropic elements) after every n_s-th step.  Asynchronous.  VM_E_STATE
 * before the first vm_4d_set_f. */
vm_status vm_4d_step(vm_4d_solver* s, int32_t nsteps);

/* The map and the transport reconstruction (f, pixel masses, field) of the
 * current elements, without moving them.  Asynchronous. */
vm_status vm_4d_reconstruct(vm_4d_solver* s);

/* A remap at the current elements now (resample, new eta, isotropic
 * elements).  Asynchronous. */
vm_status vm_4d_remap(vm_4d_solver* s);

/* Copies out (synchronise; host or device destinations).  f: the last
 * reconstructed f (f0 after vm_4d_set_f); fini and eta: the current f_ini
 * and its spline coefficients; map: the last influence map (int32, -1 where
 * no element); M: n0*n1 pixel masses and field: n0*n1*12 node fields of the
 * last reconstruction (either may be NULL). */
vm_status vm_4d_read_f(vm_4d_solver* s, double* out, int on_device);
vm_status vm_4d_read_fini(vm_4d_solver* s, double* out, int on_device);
vm_status vm_4d_read_eta(vm_4d_solver* s, double* out, int on_device);
vm_status vm_4d_read_map(vm_4d_solver* s, int32_t* out, int on_device);
vm_status vm_4d_density_force(vm_4d_solver* s, double* M, double* field, int on_device);

/* Element state in and out (60 doubles per element, layout above). */
vm_status vm_4d_get_elements(vm_4d_solver* s, double* out, int on_device);
vm_status vm_4d_set_elements(vm_4d_solver* s, const double* in, int on_device);

/* Conservation diagnostics of the last f (f0 after vm_4d_set_f, else the last
 * reconstruction's f(t + dt/2)) and of the elements (synchronises). */
vm_status vm_4d_diagnostics(vm_4d_solver* s, vm_4d_diag* out);

/* Number of elements, lattice dimensions (L[4]) and kernel launches so far. */
int32_t vm_4d_num_elements(const vm_4d_solver* s, int32_t* L4);
int64_t vm_4d_launches(const vm_4d_solver* s);

/* Statistics of the last influence map (synchronises): out3[0] elements whose
 * component outgrew the shared-memory flood window of side 2*min(2s, 12)+1
 * and were filled again over the whole padded lattice, out3[1] unexplored
 * sites left by the percolation, out3[2] repair rounds (Sec. 2.3.1);
 * *d2_evals (may be NULL): the FP64 distance evaluations d^2 = |Q(P) - Q_m|^2
 * in the fixed order since creation (219 FP64 operations each), the ones the
 * percolation ran where an FP32 bound left a decision open or a site was
 * claimed by more than one element. */
vm_status vm_4d_map_stats(vm_4d_solver* s, int32_t* out3, int64_t* d2_evals);

/* Per-kernel timing: while on, CUDA events on the solver's stream bracket
 * every launch; vm_4d_profile_read (synchronises) writes, per kernel id
 * 0..n-1 (names from vm_4d_kernel_name), the launches and milliseconds since
 * the last read, and returns the number of kernel ids. */
vm_status vm_4d_profile(vm_4d_solver* s, int on);
int32_t vm_4d_profile_read(vm_4d_solver* s, int64_t* launches, double* ms, int32_t nmax);
const char* vm_4d_kernel_name(int32_t id);

/* Wait for the solver's stream and report (and clear) its error word:
 * VM_E_NOT_CONVERGED (hole repair hit its cap), VM_E_PATCH_OVERFLOW (one
 * breadth-first wave of an element's whole-lattice flood fill held more than
 * 2^18 sites), VM_E_INTERNAL (an index read from device state failed its
 * check). */
vm_status vm_4d_sync(vm_4d_solver* s);

#ifdef __cplusplus
}
#endif
#endif
