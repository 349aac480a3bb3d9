/*
 * vlamet.h -- C ABI of the GB300 (sm_103a) metric semi-Lagrangian
 * Vlasov-Poisson solver (Colombi & Alard, "A 'metric' semi-Lagrangian
 * Vlasov-Poisson solver", 1D space / 2D phase space).
 *
 * The library advances one solve (one phase-space grid) per vm_solver.  Every
 * step of the method runs in the library's own CUDA kernels on the caller's
 * stream; the host only launches.  Pointers are plain host or device
 * pointers; no C++ or framework types cross this boundary.
 *
 * Grid and storage conventions (fixed for every call):
 *   - node-centred fixed box: x_i = x_lo + i*dx, dx = (x_hi - x_lo)/(nx - 1),
 *     v_j = v_lo + j*dv; f, f_ini, eta and the map are [nx][nv], v fastest
 *     (element (i, j) at offset i*nv + j);
 *   - elements of metric sit on a lattice centred on the box with spacing
 *     s*dx by s*dv and one extra layer on every side: Lx = 2*Kx + 3 with
 *     Kx = ceil(((nx-1)/2)/s), same for v; element m = k*Lv + l;
 *   - element state exchanged as 12 arrays of ne doubles (structure of
 *     arrays, row r at offset r*ne): x, v, Txx, Txv, Tvx, Tvv,
 *     Hx_xx, Hx_xv, Hx_vv, Hv_xx, Hv_xv, Hv_vv, where T_ab = dP_a/dQ_b and
 *     H_a,bc = d2P_a/dQ_b dQ_c (Sec. 2.1).
 *
 * Ownership: the caller provides one device workspace (vm_workspace_bytes)
 * at vm_create and keeps it alive until vm_destroy; the solver keeps all of
 * its state there.  Buffers passed to other calls are borrowed for the
 * duration of the call only.
 *
 * Errors: every call returns a vm_status; nothing aborts, throws or traps.
 * Device-side failures (a percolation that does not converge, a flood-fill
 * window that overflows) set an error word on the device, which is read and
 * cleared by the calls that synchronise (vm_sync and every call that copies
 * results to the host).
 *
 * Threads and streams: calls on one solver must not run concurrently; calls
 * are asynchronous on the solver's stream unless they say they synchronise.
 * Distinct solvers on distinct streams are independent.
 */
#ifndef VLAMET_H
#define VLAMET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VM_OK = 0,
  VM_E_INVALID_ARG = 1,
  VM_E_OOM = 2,            /* workspace too small */
  VM_E_CUDA = 3,           /* a CUDA runtime call failed */
  VM_E_NOT_CONVERGED = 4,  /* unexplored-site repair hit its round cap */
  VM_E_PATCH_OVERFLOW = 5, /* an element's influence region exceeded the largest window */
  VM_E_BUDGET = 6,         /* admission refused by a memory budget (batch/serve layer) */
  VM_E_STATE = 7,          /* call out of order (e.g. a step before vm_set_f) */
  VM_E_INTERNAL = 8,       /* an index a kernel read from device state failed its bounds check
                              (the access was skipped; vm_diag.bad_where says which check) */
  VM_E_IO = 9              /* a checkpoint file could not be written or read, or is not one */
} vm_status;

typedef enum { VM_FP64 = 0, VM_FP32_MIXED = 1 } vm_precision;
typedef enum { VM_DTYPE_F64 = 0, VM_DTYPE_F32 = 1 } vm_dtype;

typedef struct {
  int32_t nx, nv;             /* grid nodes along x and v, each >= 4 */
  double x_lo, x_hi;          /* box along x */
  double v_lo, v_hi;          /* box along v */
  int32_t elem_stride;        /* s: element spacing in grid sites (Sec. 2.3, Delta_m = s*Delta) */
  double dt;                  /* constant time step (Sec. 2.4) */
  int32_t n_s;                /* transport steps between remaps (Table 1, n_s) */
  double G;                   /* gravitational constant: a = 2 pi G (M_right - M_left) (Sec. 2.5) */
  int32_t precision;          /* vm_precision */
  double alpha;               /* percolation margin, default sqrt(3)/4 (Sec. 2.3.3) */
  double beta;                /* Q_r margin, default (1 - sqrt(3)/2)/2 (Sec. 2.3.3) */
  int32_t pad;                /* connectivity margin around the grid, sites; 0 -> s */
  int32_t literal_fd;         /* 1: a' = (a(i+1)-a(i-1))/dx as printed; 0: /(2 dx) */
  int32_t max_hole_rounds;    /* cap on unexplored-site repair rounds; 0 -> nx + nv */
  int32_t map_windows;        /* 0: every influence-map tier; 1: components that leave the
                                 32 x 64 window go straight to the whole-lattice window
                                 (the last tier), for testing that tier on small grids */
  double emap_remap;          /* 0: remap every n_s steps only; > 0: also remap after a step
                                 whose map's E_map (Sec. 2.3.2, element spacings; see
                                 vm_diag.emap) exceeds this value.  Each step then computes
                                 E_map, and the decision is taken on the device: the remap's
                                 launches are queued after every step and return at once
                                 unless the decision kernel opens them, so vm_step does not
                                 wait (with f_th > 0 the host decides and vm_step synchronises
                                 once per step).  Batches and servers accept it */
  double c_dyn;               /* 0: constant dt; > 0: each step takes min(dt, c_dyn /
                                 sqrt(rho_max)) (Sec. 2.4), rho_max the largest
                                 rho(x_i) = sum_j f(i, j) dv of the last reconstructed f
                                 (f0 before the first step); vm_step then synchronises once
                                 per step; batches refuse it */
  double f_th;                /* 0: fixed box (every element, every site); > 0: adaptive
                                 computing domain (Sec. 2.2.1, eq. constrf; Sec. 2.3).  At
                                 vm_set_f and at every remap f_ini is cut to the smallest
                                 node rectangle holding every |f_ini| > f_th, and elements
                                 exist only on the lattice lines covering it plus one extra
                                 layer on every side; each map then claims and repairs only
                                 the sites of the rectangle spanned by the existing
                                 elements' positions (f = 0 elsewhere).  The remap reads
                                 the rectangle back (vm_step synchronises once per remap);
                                 batches refuse it */
  int32_t recon_mode;         /* FP32-mixed path's transport reconstruction: 0 one block per x
                                 row, f_ini gathered through the caches; 1 tiles of 4 x rows by
                                 256 v columns whose f_ini patch is staged in shared memory by
                                 bulk copies (cp.async.bulk, the TMA engine).  Results agree to
                                 rounding (the pixel masses are summed in another order) */
} vm_config;

typedef struct {
  double mass;      /* sum f dx dv of the last reconstructed f */
  double energy;    /* 1/2 sum v^2 f dx dv - 1/(8 pi G) sum (a^2 - (2 pi G M)^2) dx (Sec. 3.2) */
  double detT_min;  /* range of det T over the elements (Sec. 2.1, |T| = 1) */
  double detT_max;
  int64_t step;     /* steps taken since vm_set_f */
  int32_t cycle;    /* steps since the last remap */
  int32_t holes;    /* unexplored sites repaired by the last map */
  int32_t hole_rounds;
  int32_t overflow_elements; /* elements that needed the large flood-fill window */
  int32_t tier1_more;        /* elements whose small-window fill tested sites beyond
                                the region predicted from the linear part of the map */
  int32_t last_tier_elements; /* elements filled in the whole-lattice window */
  int32_t exact_tests;       /* small-window site tests the FP32 bound could not settle
                                (run again in FP64) */
  int32_t bad_where;         /* first failed bounds check since creation (0: none) */
  double entropy;   /* S = -sum f log|f| dx dv of the last f (Sec. 3.2; 0 where f = 0) */
  double l1;        /* sum |f| dx dv */
  double l2;        /* sum f^2 dx dv */
  double emap;      /* E_map of the last influence map (Sec. 2.3.2), in element spacings: the
                       largest |((a + xi_n) - xi_m, (b + ze_n) - ze_m)| over grid sites P with
                       owner m and neighbours n = m + (a, b) of the percolation test's alpha
                       ranges, xi, ze = (Q(P) - Q_elem) / (dx_m, dv_m) from each element's
                       second-order map; FP64 in the oracle's order (0 before any map) */
  int64_t emap_remaps; /* remaps that vm_config.emap_remap forced since vm_set_f */
  double time;         /* sum of the steps taken since vm_set_f */
  double last_dt;      /* the last step's time step */
  int32_t lattice_range[4]; /* existing elements: lattice rows k_lo..k_hi, columns l_lo..l_hi */
  int32_t site_rect[4];     /* the last map's sites: rows i_lo..i_hi, columns j_lo..j_hi
                               (the whole grid with vm_config.f_th = 0) */
} vm_diag;

typedef struct vm_solver vm_solver;
typedef struct vm_server vm_server;

/* Fill *c with the paper's defaults (alpha, beta) and zeros elsewhere. */
void vm_config_default(vm_config* c);

/* Device bytes the solver needs for config *c (0 if *c is invalid). */
size_t vm_workspace_bytes(const vm_config* c);

/* Create a solver.  d_workspace: device buffer of at least
 * vm_workspace_bytes(c) bytes, 256-byte aligned, owned by the caller until
 * vm_destroy.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Returns VM_E_INVALID_ARG for a bad config, VM_E_OOM if the workspace is too
 * small.  The state is empty until vm_set_f. */
vm_status vm_create(const vm_config* c, void* d_workspace, size_t workspace_bytes,
                    void* cuda_stream, vm_solver** out);
void vm_destroy(vm_solver* s);  /* waits for the solver's stream first */
const char* vm_status_string(vm_status st);

/* Lattice shape: number of elements, Lx and Lv. */
vm_status vm_lattice(const vm_solver* s, int32_t* ne, int32_t* Lx, int32_t* Lv);

/* New initial condition (Sec. 1 and 2.3): f_ini <- f0 ([nx][nv] doubles,
 * host if on_device == 0, else device), its cubic B-spline coefficients
 * (Sec. 2.2.2), and isotropic elements on the lattice (T = I, H = 0). */
vm_status vm_set_f(vm_solver* s, const double* f0, int32_t on_device);

/* Replace / read the element state (12 x ne doubles, layout above).  Used
 * to inject identical states into two implementations. */
vm_status vm_set_elements(vm_solver* s, const double* soa12, int32_t on_device);
vm_status vm_get_elements(vm_solver* s, double* soa12, int32_t on_device);

/* Influence map of the current elements (Sec. 2.3.1): Taylor terms of the
 * inverse map, percolation, overlap and unexplored-site rules.  Result read
 * with vm_read_map. */
vm_status vm_compute_map(vm_solver* s);

/* Transport-mode f at the current elements (Sec. 2.2.1 with the map of
 * Sec. 2.3.1), its pixel masses and the force (Sec. 2.5).  Results read with
 * vm_read_f and vm_density_force. */
vm_status vm_reconstruct(vm_solver* s);

/* Advance nsteps steps of dt (Sec. 2.4): half drift; map; f(t + dt/2);
 * pixel masses, mass scan, force, a', a''; kick; half drift; and, after
 * every n_s-th step of a cycle, a remap (Secs. 2.2.2, 2.3.2).  Asynchronous. */
vm_status vm_step(vm_solver* s, int32_t nsteps);

/* Remap now, at the current elements: Q_r blend, spline of f_ini at Q_r,
 * new f_ini and coefficients, isotropic elements.  Asynchronous. */
vm_status vm_remap(vm_solver* s);

/* Pixel masses M(i) = sum_j f(i,j) dx dv, and a, a', a'' on the x nodes,
 * from the last reconstruction ([nx] doubles each; any pointer may be
 * NULL).  a(i) = 2 pi G (M_tot - M_left(i) - M_left(i-1)) (Sec. 2.5) with the
 * prefix sums M_left exact (128-bit fixed point at a common scale of 2^-112
 * max|M|): the bracket is correctly rounded once, then multiplied by 2 pi G.
 * Synchronises when on_device == 0. */
vm_status vm_density_force(vm_solver* s, double* M, double* a, double* da, double* d2a,
                           int32_t on_device);

/* Copy out [nx][nv] arrays: the last reconstructed f, the current f_ini,
 * the current spline coefficients eta, the current map (int32).  dtype is a
 * vm_dtype (conversion happens on the device).  Synchronise when
 * on_device == 0. */
vm_status vm_read_f(vm_solver* s, void* out, int32_t dtype, int32_t on_device);
vm_status vm_read_fini(vm_solver* s, void* out, int32_t dtype, int32_t on_device);
vm_status vm_read_eta(vm_solver* s, void* out, int32_t dtype, int32_t on_device);
vm_status vm_read_map(vm_solver* s, int32_t* out, int32_t on_device);

/* Mass, energy and det T range of the last reconstruction (Sec. 3.2, 2.1),
 * plus step counters and map statistics.  Synchronises. */
vm_status vm_diagnostics(vm_solver* s, vm_diag* d);

/* Wait for the solver's stream; return and clear any device-side error. */
vm_status vm_sync(vm_solver* s);

/* Checkpoint of the state the steps carry from one to the next (Sec. 2.4:
 * the elements' P_m, T, H; Secs. 2.2.2, 2.3.2: f_ini and the spline
 * coefficients of the last remap; the step count and the position in the
 * remap cycle), plus the last reconstructed f, to the binary file `path`
 * (native byte order; a header with the grid, precision and step constants,
 * then the arrays).  vm_save synchronises the solver's stream first and
 * returns VM_E_STATE before vm_set_f.  vm_load replaces the state of a
 * solver created with the same grid, element stride, precision, dt, G,
 * alpha and beta (VM_E_INVALID_ARG otherwise); the steps that follow are
 * bit for bit those the saved solver would have taken.  VM_E_IO: the file
 * cannot be opened, written or read, or is not a checkpoint.  Both calls
 * synchronise; the path is borrowed for the call. */
vm_status vm_save(vm_solver* s, const char* path);
vm_status vm_load(vm_solver* s, const char* path);

/* The CUDA error code behind the last VM_E_CUDA returned to this host thread
 * (cudaSuccess = 0 if none), and its name.  Calls that launch work first
 * drop an error that earlier CUDA calls of other code in the thread left
 * unread, so VM_E_CUDA reports this library's launches (or a context that an
 * earlier fault made unusable). */
int32_t vm_last_cuda_error(void);
const char* vm_cuda_error_name(int32_t code);

/* Number of kernel launches the solver has issued since creation (a count
 * kept on the host, for launch accounting). */
int64_t vm_launch_count(const vm_solver* s);

/* Optional per-kernel timing: when enabled, every launch is bracketed by a
 * pair of CUDA events on the solver's stream; vm_profile_read waits for
 * them and returns, per kernel that ran, its launch count and total device
 * time since the last vm_profile call (at most `max` entries written to
 * `out`; the return value is the number of kernels that ran, or -1).
 * Intended for measurement runs; off by default. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
} vm_kernel_stat;
vm_status vm_profile(vm_solver* s, int32_t enable);
int32_t vm_profile_read(vm_solver* s, vm_kernel_stat* out, int32_t max);

/* ---- many independent solves (batching) ----
 *
 * A batch advances many solves together (Sec. 2.4 for each; the solves are
 * independent problems).  Every phase of a step (drift and Taylor terms, the
 * map's tiers, the reconstruction, the mass scan, the kick; and the remap's)
 * is ONE launch for the whole batch, whose persistent blocks walk a work
 * list of (solve, unit) items; the work of the map's later tiers is listed
 * on the device from each solve's counters.  vm_batch_create records a
 * transport step, and a transport step followed by a remap, into two CUDA
 * graphs; vm_batch_step then launches one graph per step on cuda_stream.
 * Results are those of the same solves stepped one by one, bit for bit.
 * The solvers stay owned by the caller and must outlive the batch; they must
 * all have received vm_set_f, share the precision, n_s and their position in
 * the remap cycle (VM_E_STATE otherwise; solves with emap_remap > 0 keep
 * their own cycles on the device and are exempt), not use c_dyn or f_th
 * (VM_E_INVALID_ARG: those take host decisions per step), and must not be
 * profiling.  Every step of a batch with emap_remap solves ends with their
 * E_map, each one's decision and their remap launches, which skip the solves
 * that do not remap this step.  The batch allocates its work tables (about 360 bytes per solve)
 * with cudaMalloc and frees them in vm_batch_destroy.  nstreams is not used
 * (kept for compatibility; pass 0 or any positive count).  Creation
 * synchronises each solver's stream; vm_batch_step orders itself after work
 * queued on the solvers' streams and before later work on them.  Results are
 * read per solver with the single-solve calls. */
typedef struct vm_batch vm_batch;
vm_status vm_batch_create(vm_solver* const* solvers, int32_t n, int32_t nstreams, void* cuda_stream,
                          vm_batch** out);
vm_status vm_batch_step(vm_batch* b, int32_t nsteps);
/* Tune the persistent blocks of each phase on the run's own steps: for each
 * of 1, 2, 4 and 8 blocks per SM, `trials` transport steps of the batch are
 * taken (real steps: the solves advance, and a step that ends a remap cycle
 * is taken with its remap, untimed), each phase timed with CUDA events; each
 * phase then keeps its fastest shape and the graphs are recorded again.  The
 * shape changes no result.  Synchronises. */
vm_status vm_batch_autotune(vm_batch* b, int32_t trials);
/* The tuned shape: blocks per SM and ms per step of the five timed phases
 * (drift + Taylor, map, reconstruction, mass scan + force, kick + drift);
 * returns 1 if vm_batch_autotune ran, 0 if not, -1 for a NULL batch. */
int32_t vm_batch_tuning(const vm_batch* b, int32_t* blocks_per_sm5, double* ms5);
/* Graph nodes (kernel launches) per batch step, without or with the remap. */
int64_t vm_batch_launches_per_step(const vm_batch* b, int32_t with_remap);
void vm_batch_destroy(vm_batch* b);

/* ---- serving: continuous batching of submitted solves ----
 *
 * A server advances many requested solves (Sec. 2.4 for each; independent
 * problems) with continuous batching.  Requests are admitted first come,
 * first served as soon as a slot and enough of the server's device pool are
 * free (each solve's exact vm_workspace_bytes, first-fit in the pool), their
 * state stays resident, and every step of a tick is ONE group step for all
 * active solves (one launch per phase for the whole set, plus one group
 * remap for the solves whose cycle ends), so a request that arrives while
 * others run joins the next step's launches.  The caller drives the server
 * with vm_server_poll, which never waits for the device: it retires
 * finished solves (their result is copied to host memory behind an event),
 * admits waiting ones, and queues one more tick unless two are already in
 * flight.  Results equal those of the same solve stepped alone, bit for bit.
 *
 * Memory: the caller passes one device pool (256-byte aligned), owned by the
 * caller until vm_server_destroy; the server uses its first
 * vm_server_pool_bytes(c) bytes for its work tables and at most
 * c->budget_bytes after them for solver workspaces; it allocates no device
 * memory, and pinned host memory only for staging (initial conditions,
 * results, tables).  Every request must use c->precision and no per-step host
 * decision (c_dyn, f_th: VM_E_INVALID_ARG; emap_remap is decided on the
 * device, its remaps behind each solve's own decision); one whose workspace
 * exceeds the whole budget is refused (VM_E_BUDGET).  Calls on one server
 * must not run concurrently. */
typedef struct {
  size_t budget_bytes;     /* device bytes for solver workspaces (after the tables) */
  int32_t max_active;      /* solves resident at most */
  int32_t steps_per_tick;  /* steps every active solve takes per tick (>= 1) */
  int32_t precision;       /* vm_precision of every request */
} vm_server_config;

typedef struct {
  int64_t id;              /* from vm_server_submit */
  int32_t status;          /* VM_OK, or why the solve failed */
  double submit_s, admit_s, finish_s;  /* host clock, seconds since vm_server_create */
} vm_server_done;

typedef struct {
  int32_t waiting, active, finished, peak_active;
  int64_t used_bytes, peak_bytes;  /* workspace bytes in use, and the most at once */
  int64_t ticks, group_steps, remap_groups;
} vm_server_stat;

/* Bytes of the pool the server keeps for its work tables. */
size_t vm_server_pool_bytes(const vm_server_config* c);
vm_status vm_server_create(const vm_server_config* c, void* d_pool, size_t pool_bytes, void* cuda_stream,
                           vm_server** out);
/* Queue a solve: the grid, box and method constants of *cfg, the initial
 * condition f0 ([nx][nv] doubles, host memory, copied before the call
 * returns) and the number of steps.  *id identifies the request. */
vm_status vm_server_submit(vm_server* s, const vm_config* cfg, const double* f0, int32_t nsteps, int64_t* id);
/* One round of the serving loop (see above); the requests finished since
 * the last report are written to done[0 .. *n_done) (at most max_done). */
vm_status vm_server_poll(vm_server* s, vm_server_done* done, int32_t max_done, int32_t* n_done);
/* The result of a finished request: M, a, a', a'' of its last step ([nx]
 * doubles each, host memory; any pointer may be NULL).  VM_E_STATE while the
 * request is not finished. */
vm_status vm_server_result(vm_server* s, int64_t id, double* M, double* a, double* da, double* d2a);
vm_status vm_server_stats(const vm_server* s, vm_server_stat* out);
/* Waits for the server's stream, then frees its host state; the caller may
 * then free the pool. */
void vm_server_destroy(vm_server* s);

/* Measured FP64 arithmetic rate of the current device, in FLOP/s (2 per
 * fused multiply-add): one launch of eight independent FMA chains of
 * `iters` rounds per thread over 8 blocks of 256 threads per SM, timed with
 * CUDA events on cuda_stream (synchronises).  The denominator of the FP64
 * path's arithmetic roofline; not part of the method.  VM_E_INVALID_ARG for
 * iters < 1 or a NULL result pointer. */
vm_status vm_measure_fp64_peak(int32_t iters, void* cuda_stream, double* flops_per_s);

/* Pixel masses and force from a caller's f, allocating nothing.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory (a plugin whose host application owns the
 * device heap and forbids cudaMalloc, or a loop that must never pay the
 * device-wide synchronisation cudaMalloc and cudaFree can cause).  It
 * computes what vm_reconstruct + vm_density_force produce for an f given on
 * the device: M(i) = sum_j f(i,j) dx dv, then a, a', a'' on the x nodes by
 * the solver's error-free mass scan (the prefix sums of M carried exactly
 * in 128-bit fixed point; same grid conventions as vm_config).
 *
 * f: device pointer, [nx][nv], v fastest, dtype a vm_dtype.  M_out (may be
 * NULL), a, da, d2a: device pointers to [nx] doubles.  cuda_stream: the
 * stream the work is queued on (asynchronous; nothing is synchronised).
 * The only scratch is a file-scope device array holding up to
 * VM_STATIC_FORCE_MAX_NX pixel masses, which every GPU that loads the library
 * keeps until the process exits; nx above that limit returns
 * VM_E_INVALID_ARG.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array and it keeps the last call's
 * contents (every entry used is rewritten by each call); calls whose work
 * overlaps on the GPU race on it, so serialise them (one stream, or events). */
#define VM_STATIC_FORCE_MAX_NX 16384
vm_status vm_force_from_f_static(const void* f, int32_t dtype, int32_t nx, int32_t nv, double x_lo, double x_hi,
                                 double v_lo, double v_hi, double G, int32_t literal_fd, double* M_out, double* a,
                                 double* da, double* d2a, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
