// Internal declarations shared by the CUDA translation units of libvlamet.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vlamet.h"

namespace vm {

// Device error word bits.
enum : int32_t {
  ERR_NOT_CONVERGED = 1,
  ERR_PATCH_OVERFLOW = 2,  // an element outgrew every window, or the contested-site records ran out
  ERR_INTERNAL = 4,        // an index read from device state failed its bounds check (the access was skipped)
};

// Bounds checks on indices that kernels read from device state (lists,
// records, owner tags): a failed check sets ERR_INTERNAL, records which
// check (its number) in DevState::bad_where, and skips the access.
#define VM_BAD(ds, where)                                 \
  do {                                                    \
    atomicOr(&(ds)->err, ERR_INTERNAL);                   \
    atomicCAS(&(ds)->bad_where, 0, (where));              \
  } while (0)

// Grid, lattice and method constants, passed by value to every kernel.  All
// derived doubles are computed once on the host in a fixed order (no fused
// multiply-add), so the percolation decisions see the same operands as any
// other FP64 restatement of the method that uses this order.
struct Grid {
  int32_t nx, nv, s, pad, Kx, Kv, Lx, Lv, ne;
  double x_lo, v_lo, dx, dv, dxm, dvm, inv_dx, inv_dv, inv_dxm, inv_dvm, cx, cv, dxdv;
  double alpha, beta;
  double dt, half_dt, A;  // A = 2 pi G
  double r_vx, r_xv;      // dv_m/dx_m and dx_m/dv_m
  int32_t literal_fd;
  int32_t max_hole_rounds;
  // adaptive computing domain (Sec. 2.2.1, eq. constrf; Sec. 2.3): fth_on
  // restricts each map to the site rectangle DevState::rect spanned by the
  // existing elements; elements exist on lattice rows klo..khi and columns
  // llo..lhi (the whole lattice when fth_on is 0)
  int32_t fth_on;
  int32_t klo, khi, llo, lhi;
  int32_t recon_tiles;  // FP32-mixed path: 1 = reconstruction in tiles staged by bulk copies
  // Remap decided on the device (Sec. 2.3.2): when set, every kernel of a
  // remap enqueued with this Grid returns at once while *gate is 0
  const int32_t* gate;
};

// True when the remap this Grid was enqueued for is not to run (read by
// every thread of a kernel before any barrier, so all return together).
__device__ __forceinline__ bool gate_shut(const Grid& g) { return g.gate != nullptr && __ldcg(g.gate) == 0; }

// Small device-resident control block.
struct DevState {
  int32_t err;
  // counters of one influence map (cleared together at its start)
  int32_t nholes;        // holes in the working list
  int32_t holes_found;   // holes left by the claims (statistics)
  int32_t hole_rounds;   // repair rounds of the last map (statistics)
  int32_t noverflow;     // elements queued for the first large-window attempt
  int32_t overflow_stat;
  int32_t noverflow2;    // ... second attempt
  int32_t overflow2_stat;
  int32_t noverflow3;    // ... third attempt
  int32_t overflow3_stat;
  int32_t nrec;          // records of sites claimed by two or more elements
  int32_t t1_more;       // tier-1 elements that needed tests beyond their predicted region
  int32_t n_exact;       // tests the FP32 bound left to the exact FP64 test (statistics)
  int32_t bad_where;     // first failed bounds check (0: none); kept until read by vm_sync
  int32_t take[3];       // next item of each large-window launch (blocks fetch work dynamically)
  int32_t noverflow_back; // tier-1 escapes of elements with all eight neighbours (listed from the end)
  int32_t nseed;          // tier-1 mask records written for the next tier
  int32_t n_pair_esc;     // tier-0 escapes listed for tier 1
  uint32_t epoch;        // epoch of the current influence map (0..kEpochs-1)
  double Mtot;           // total mass of the last reconstruction
  double sum_mass, sum_kin, sum_pot;
  unsigned long long det_min_key, det_max_key;
  double sum_ent, sum_l1, sum_l2;   // Casimirs of the last f (Sec. 3.2)
  unsigned long long emap2_bits;     // bits of the largest squared E_map term (>= 0)
  unsigned long long rho_max_bits;   // bits of the largest positive projected density
  // adaptive computing domain: the current map's site rectangle (i_lo, i_hi,
  // j_lo, j_hi; empty when lo > hi), the node rectangle of |f_ini| > f_th
  // (same order, atomics), and the completion counter of the rectangle's
  // block reduction
  int32_t rect[4];
  int32_t fbox[4];
  uint32_t rect_done;
  // Remap cycle kept on the device when the remap is decided there (E_map
  // criterion, Sec. 2.3.2): the remaps E_map forced since vm_set_f, steps
  // since the last remap, and the decision of the last step (1: remap now)
  long long emap_remaps;
  int32_t cyc;
  int32_t gate;
  int32_t emap_hit;  // the current map's E_map exceeds the threshold (set by the test, cleared at map start)
};

// Owner slots of the influence map: (epoch << 24) | element index.  A slot
// whose epoch is not the current map's is empty; every site is rewritten
// each map (claimed or repaired), so stale values are never more than one
// map old.  The second slot of a contested site holds (epoch << 24) while
// the site is listed for resolution, and is cleared when it is resolved.
constexpr uint32_t SLOT_EMPTY = 0xFFFFFFFFu;

// Whole-lattice flood-fill windows of the last map tier: blocks working at
// once, and 64-bit words of one window (three masks over the padded lattice).
constexpr int kGlobalBlocks = 16;
constexpr int kSeedRecords = 8192;  // tier-1 mask records kept per map (96 words each)
inline size_t global_window_words(long long nx, long long nv, long long pad) {
  return 3 * (size_t)(nx + 2 * pad) * (size_t)((nv + 2 * pad + 63) / 64);
}
constexpr uint32_t SLOT_MASK = 0x00FFFFFFu;
// Element field of an owner slot marking a site outside the computing
// domain of the current map (never an element: the lattice has fewer than
// 2^24 - 1 elements).
constexpr uint32_t SLOT_OUTSIDE = SLOT_MASK;
// Blocks of the domain-rectangle reduction (partials kept in the workspace).
constexpr int kRectBlocks = 256;
constexpr int kEpochs = 255;  // epochs 0..254; 255 never current

// Element state: 12 doubles per element, structure of arrays.
enum { EL_X = 0, EL_V, EL_TXX, EL_TXV, EL_TVX, EL_TVV, EL_HXXX, EL_HXXV, EL_HXVV, EL_HVXX, EL_HVXV, EL_HVVV, EL_N };
// Taylor record: 16 doubles (128 bytes) per element, array of structures so
// that one element's terms are one cache line for the per-site gathers.
enum { TY_X = 0, TY_V, TY_TI00, TY_TI01, TY_TI10, TY_TI11, TY_GX00, TY_GX01, TY_GX11,
       TY_GV00, TY_GV01, TY_GV11, TY_QX, TY_QV, TY_U, TY_W, TY_N = 16 };
// FP32 record of the inverse map in element units (32 words = 128 bytes):
// with p = (P - P_m)/Delta_m and q = (Q - Q_m)/Delta_m,
//   q_a = sum_b T[a][b] p_b - 1/2 sum_l K[a][l] s_l,  s_l = p^T G_l p
//       = p_x (T[a][0] + A_a p_x + B_a p_v) + p_v (T[a][1] + C_a p_v),
// the second-order coefficients A, B, C combined from K and G in FP64; and
// |each term| of q_a bounded by C1_a |p|_inf + C2_a |p|_inf^2, C2_a from the
// uncombined terms (the coefficients of the bound are rounded up).  UF/WF
// and UI/WI split the element's index position u_m = (x_m - x_lo)/dx into
// integer and fraction.
// Words 20-23 repeat u_m and w_m in FP64 (a 16-byte aligned pair), so that
// the map's first tiers read one 128-byte line per neighbour.
enum { TF_T00 = 0, TF_T01, TF_T10, TF_T11, TF_AX, TF_BX, TF_CX, TF_AV, TF_BV, TF_CV,
       TF_C1X, TF_C2X, TF_C1V, TF_C2V, TF_UF, TF_WF, TF_UI, TF_WI, TF_UD = 20, TF_N = 32 };
// the reconstruction reads words 0-15 of the FP32 record as four float4
static_assert(TF_T00 == 0 && TF_AX == 4 && TF_BV == 8 && TF_C1V == 12 && TF_WF == 15, "FP32 record layout");
static_assert(TF_UD % 4 == 0 && TF_UD >= TF_WI + 1 && TF_UD + 4 <= TF_N, "FP64 index positions in the FP32 record");

constexpr unsigned long long KEY_EMPTY = ~0ull;

// Kernel identities for the optional per-launch timing (vm_profile).
enum KernelId {
  KID_DRIFT = 0, KID_TAYLOR, KID_KICK_DRIFT, KID_RESET, KID_SCAN_FORCE, KID_DIAG,
  KID_MAP_CLEAR, KID_CLAIM_SMALL, KID_CLAIM_LARGE, KID_FINALIZE, KID_HOLES,
  KID_RESOLVE, KID_READ_MAP,
  KID_RECON, KID_REMAP, KID_CONVERT, KID_SPLINE_ROWS, KID_SPLINE_COLS, KID_CLAIM_PAIR, KID_EMAP, KID_N
};
constexpr int PROF_CAP = 1024;

}  // namespace vm

struct vm_solver {
  vm_config cfg;
  vm::Grid g;
  cudaStream_t stream;
  int32_t fp32;            // 1: f_ini, eta, f stored as float
  size_t sreal;            // bytes per stored real
  size_t n;                // nx * nv
  // device buffers (carved from the caller's workspace)
  void* fini;
  void* eta;
  void* f;
  void* tmp;
  uint32_t* map;            // owner slot 0: the influence map (epoch-tagged)
  uint32_t* slot1;          // (epoch << 24): the site is listed as contested in that map
  unsigned long long* rec_key;  // per site: {element index, bits of d^2}, 128-bit minimum; empty between maps
  int32_t* rec_site;        // contested sites of the current map
  int32_t rec_cap;
  int32_t* holes_a;
  int32_t* holes_b;         // also the 8 B/site staging buffer of the copy calls
  int2* overflow_list;      // (element, window mode) for the second tier
  int2* overflow_list2;     // for the last-resort tier
  unsigned long long* gwin; // bit masks of the whole-lattice windows (kGlobalBlocks of them), kept zeroed
  unsigned long long* t1seed; // tier-1 masks of escaped elements: t1seed_cap records of 3 x 32 words
  int32_t t1seed_cap;
  double* el;               // 12 x ne
  double* tay;              // ne x 16
  float* tayf;              // ne x 32 (FP32 record, element units)
  double* M;                // pixel masses of the last step
  double* a;
  double* da;
  double* d2a;
  double* thomas_x;         // 2 x nx: c'_i and 1/den_i of the spline system along x
  double* thomas_v;         // 2 x nv
  float* thomas_xf;
  float* thomas_vf;
  double* rect_part;        // kRectBlocks x 4 partial minima/maxima of the element positions
  double* Mpart;            // nx x ceil(nv / 256) row sums of the reconstruction's tiles
  double* diag_part;        // kRectBlocks x 6 partial sums of the diagnostics
  vm::DevState* ds;
  // host-side bookkeeping
  int32_t have_f;
  int64_t nstep;
  int64_t emap_remaps;      // remaps forced by cfg.emap_remap since vm_set_f
  double time;              // sum of the steps since vm_set_f
  double last_dt;
  int32_t cyc;
  int64_t launches;
  // optional per-launch timing: event pairs around each launch
  int32_t prof;
  int32_t prof_n;
  int32_t prof_created;
  int32_t prof_kind[vm::PROF_CAP];
  cudaEvent_t prof_ev[2 * vm::PROF_CAP];
  int64_t prof_count[vm::KID_N];
  double prof_ms[vm::KID_N];
};

namespace vm {
// A solve whose remap cycle lives on the device (DevState cyc, gate,
// emap_remaps): the E_map criterion decided without a host round trip.  The
// adaptive domain reads its rectangle back at each remap, so with f_th > 0
// the host keeps the decision.
inline bool device_cycle(const vm_solver* s) { return s->cfg.emap_remap > 0.0 && s->cfg.f_th == 0.0; }
cudaError_t cycle_to_device(vm_solver* s);  // host (cyc, emap_remaps) -> device, gate shut
cudaError_t cycle_to_host(vm_solver* s);    // device -> host when device_cycle (synchronises)
}  // namespace vm

namespace vm {

// ---- per-launch timing (no-ops unless vm_profile enabled it) ----
int prof_begin(vm_solver* s, int kid);
void prof_end(vm_solver* s, int slot);
void prof_flush(vm_solver* s);

// ---- solver creation without the final synchronisation (api.cu) ----
vm_status solver_create(const vm_config* c, void* d_workspace, size_t bytes, cudaStream_t stream, bool sync,
                        vm_solver** out);

// ---- one step, enqueue only (api.cu) ----
void step_transport(vm_solver* s);
cudaError_t step_remap(vm_solver* s);

// ---- launchers (each in the translation unit of its kernels) ----
// elements.cu
void launch_drift(vm_solver* s, bool taylor);
void launch_taylor(vm_solver* s);
void launch_kick_drift(vm_solver* s);
void launch_reset_elements(vm_solver* s);
void launch_scan_force(vm_solver* s);
void launch_scan_force_raw(const Grid& g, const double* M, double* a, double* da, double* d2a, DevState* ds,
                           cudaStream_t stream);
void launch_diagnostics(vm_solver* s);
// E_map of the last influence map (Sec. 2.3.2) into ds->emap2_bits (zeroed by the caller)
void launch_emap(vm_solver* s);
// E_map of the step's map and the remap decision on the device (DevState
// cyc, gate, emap_remaps); the gated remap's tmp -> f_ini copy
void launch_remap_gate(vm_solver* s);
void launch_copy_gated(vm_solver* s);
// largest projected density sum_j f(i, j) dv of s->f into ds->rho_max_bits (zeroed by the caller)
void launch_rho_max(vm_solver* s);
// map.cu
bool map_prepare(const Grid& g);
void launch_map(vm_solver* s);
void launch_read_map(vm_solver* s, int32_t* dst);
// recon.cu
void launch_reconstruct(vm_solver* s);
int recon_tiles_of(const Grid& g);
bool recon_prepare();
void launch_remap_resample(vm_solver* s, void* out);
void launch_convert(vm_solver* s, const void* src, void* dst, int32_t dst_dtype, size_t count);
void launch_store_real(vm_solver* s, const double* src, void* dst, size_t count);
// spline.cu
void launch_spline_solve(vm_solver* s, const void* src, void* dst);

// ---- many solves in one launch per phase (group.cu drives them) ----
//
// A group is a set of solves of one precision whose steps are launched
// together: each phase of a step is one launch whose blocks walk a work
// list of (solve, unit) items, a unit being what one block of the
// single-solve launch does (a row, a chunk of elements, an escaped element's
// window...).  Solve sv owns units [off[sv], off[sv + 1]) of a phase; for
// phases whose work is only known on the device (the map's escape lists,
// contested sites, holes) the offsets are computed on the device from each
// solve's counters.  Each unit runs the single-solve kernel's body with its
// virtual block index, so the results are those of the single-solve
// launches, bit for bit, whatever the number of blocks.
struct SolveDesc {
  Grid g;
  float alo, ahi;  // alpha rounded down and up to FP32
  float blo, bhi;  // beta rounded down and up to FP32
  int32_t map_windows;
  void* fini;
  void* eta;
  void* f;
  void* tmp;
  uint32_t* map;
  uint32_t* slot1;
  unsigned long long* rec_key;
  int32_t* rec_site;
  int32_t rec_cap;
  int32_t* holes_a;
  int32_t* holes_b;
  int2* ovf1;
  int2* ovf2;
  unsigned long long* gwin;
  size_t gwin_words;
  unsigned long long* t1seed;
  int32_t t1seed_cap;
  double* el;
  double* tay;
  float* tayf;
  double* M;
  double* a;
  double* da;
  double* d2a;
  double* thx;
  double* thv;
  float* thxf;
  float* thvf;
  double* Mpart;  // tile row sums of the staged reconstruction
  DevState* ds;
  int32_t n_s;      // steps per remap cycle
  double emap_thr;  // E_map remap threshold (0: the cycle alone decides)
};

// Solve owning unit u: the largest sv with off[sv] <= u (off[0] = 0,
// off[ns] = total).
__device__ __forceinline__ int unit_solve(const int* __restrict__ off, int ns, int u) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Device-side unit counts: which per-solve counter a dynamic phase reads.
enum GroupCount : int {
  GC_PAIR_ESC = 0,   // tier-0 escapes (tier 1's list), TE per unit
  GC_OVF1,           // first large-window list (front + back), one element per unit
  GC_OVF2,           // second large-window list
  GC_OVF3,           // last tier's list (front, and the back in map_windows mode)
  GC_REC,            // contested sites, 256 per unit
  GC_HOLES           // one unit per solve that has holes
};

// Launch shape of one group launch: grid size (persistent blocks).
struct GroupShape {
  int blocks;
};

// The host side of a group: the descriptor table and the unit offsets of
// each phase on the device (group.cu).
struct GroupPlan {
  const SolveDesc* D;  // device, ns entries
  int ns;
  int fp32;
  cudaStream_t stream;
  // host-known offsets (device arrays of ns + 1 ints) and totals
  const int* off_elem64; int tot_elem64;   // 64-element chunks
  const int* off_pair; int tot_pair;       // tier-0 blocks (2 * TP elements)
  const int* off_rows; int tot_rows;       // x rows
  const int* off_diff; int tot_diff;       // 128 x-node chunks
  const int* off_sites; int tot_sites;     // 1024-site chunks (4 per thread)
  const int* off_copy; int tot_copy;       // 4096-value chunks of an [nx][nv] array
  const int* off_rows4; int tot_rows4;     // 4-row chunks (row spline sweeps)
  const int* off_cols; int tot_cols;       // 32-column chunks (column spline sweeps)
  const int* off_solve;                    // one unit per solve
  const int* off_tiles; int tot_tiles;     // reconstruction tiles (4 x rows by 256 v columns)
  int recon_tiles;                         // the group's reconstruction kernel (all solves alike)
  // device-computed offsets (ns + 1 ints each; the total at [ns])
  int* off_dyn;                            // scratch for one dynamic phase at a time
  int big_blocks_cap;                      // virtual blocks per solve of the large windows
  size_t big_smem;                         // dynamic shared memory of the large windows
  GroupShape shape[32];                    // per phase (GroupPhase)
};

enum GroupPhase : int {
  GP_DRIFT = 0, GP_TAYLOR, GP_MAP_BEGIN, GP_PAIR, GP_SMALL, GP_BIG1, GP_BIG2, GP_BIG3, GP_RESOLVE,
  GP_FIND_HOLES, GP_HOLES, GP_RECON, GP_SCAN, GP_DIFF, GP_KICK, GP_REMAP, GP_COPY, GP_ROWS, GP_COLS,
  GP_RESET, GP_UNITS, GP_EMAP, GP_N
};

// The solve of unit u, its Grid in shared memory (read by every thread of
// the block), and the unit's index within its solve.  GROUP_LOOP also skips
// the solves whose gated remap is not to run (gate_shut): a block that meets
// one moves on to its first unit past that solve.  GROUP_LOOP_ALL visits
// every unit (the phases that take the decision).
#define GROUP_LOOP_GATED_(off, ns, total, gated)                     \
  __shared__ Grid gsh;                                               \
  __shared__ int svsh, skipsh;                                       \
  for (int u = blockIdx.x; u < (total); u += gridDim.x) {            \
    if (threadIdx.x == 0) {                                          \
      const int sv_ = unit_solve((off), (ns), u);                    \
      svsh = sv_;                                                    \
      skipsh = -1;                                                   \
      if ((gated) && gate_shut(D[sv_].g)) {                          \
        const int nx_ = __ldg((off) + sv_ + 1), G_ = (int)gridDim.x; \
        skipsh = nx_ + ((int)blockIdx.x - nx_ % G_ + G_) % G_;       \
      } else {                                                       \
        gsh = D[sv_].g;                                              \
      }                                                              \
    }                                                                \
    __syncthreads();                                                 \
    if (skipsh >= 0) {                                               \
      u = skipsh - (int)gridDim.x;                                   \
      __syncthreads();                                               \
      continue;                                                      \
    }                                                                \
    const int sv = svsh;                                             \
    const SolveDesc& d = D[sv];                                      \
    const int vb = u - __ldg((off) + sv);                            \
    if (vb >= __ldg((off) + sv + 1) - __ldg((off) + sv)) {           \
      /* (a table and its totals out of step: never expected) */     \
      if (threadIdx.x == 0) VM_BAD(d.ds, 50);                        \
      __syncthreads();                                               \
      continue;                                                      \
    }
#define GROUP_LOOP(off, ns, total) GROUP_LOOP_GATED_(off, ns, total, true)
#define GROUP_LOOP_ALL(off, ns, total) GROUP_LOOP_GATED_(off, ns, total, false)
#define GROUP_END \
    __syncthreads(); \
  }

// Blocks of a group launch: the phase's tuned shape, capped by its units.
unsigned group_grid(const GroupPlan& G, GroupPhase ph, int total);

// group launchers (each in the translation unit of its kernels)
void group_drift(const GroupPlan& G, bool taylor);
void group_taylor(const GroupPlan& G);
void group_kick(const GroupPlan& G);
void group_reset(const GroupPlan& G);
void group_scan_force(const GroupPlan& G);
void group_map(const GroupPlan& G);
void group_reconstruct(const GroupPlan& G);
void group_remap_resample(const GroupPlan& G);   // into each solve's tmp
void group_copy_tmp_to_fini(const GroupPlan& G);
void group_remap_gate(const GroupPlan& G);        // E_map + decision of each solve (gated plans)
void group_spline(const GroupPlan& G);           // fini -> eta
size_t group_big_smem(const Grid& g);            // the large windows' shared memory for grid g
bool group_map_prepare();

// adaptive computing domain (api.cu launches, elements.cu kernels)
// node rectangle of |f_ini| > f_th into ds->fbox (reset first)
void launch_fth_box(vm_solver* s);
// f_ini <- 0 outside the node rectangle of ds->fbox
void launch_fth_cut(vm_solver* s);
// the map's site rectangle from the existing elements' positions into ds->rect
void launch_domain_rect(vm_solver* s);
// map.cu: owner slots outside ds->rect tagged SLOT_OUTSIDE
void launch_clear_outside(vm_solver* s);

// Does element (kk, ll) exist (inside the lattice and the part of it that
// covers the computing domain)?
__device__ __forceinline__ bool elem_exists(const Grid& g, int kk, int ll) {
  return kk >= g.klo && kk <= g.khi && ll >= g.llo && ll <= g.lhi;
}

// ---- exact-order FP64 arithmetic (never contracted into FMA) ----
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// Offset Q - Q_m of the second-order inverse map of one element at P
// (Sec. 2.1): y = T^-1 dP, s_l = dP^T G_l dP, dQ = y - T^-1 s / 2.
__device__ __forceinline__ void qofp_exact(const double* t, double Px, double Pv, double& dqx,
                                           double& dqv) {
  double dPx = dsub(Px, t[TY_X]), dPv = dsub(Pv, t[TY_V]);
  double yx = dadd(dmul(t[TY_TI00], dPx), dmul(t[TY_TI01], dPv));
  double yv = dadd(dmul(t[TY_TI10], dPx), dmul(t[TY_TI11], dPv));
  double g0 = dadd(dmul(t[TY_GX00], dPx), dmul(t[TY_GX01], dPv));
  double g1 = dadd(dmul(t[TY_GX01], dPx), dmul(t[TY_GX11], dPv));
  double sx = dadd(dmul(dPx, g0), dmul(dPv, g1));
  g0 = dadd(dmul(t[TY_GV00], dPx), dmul(t[TY_GV01], dPv));
  g1 = dadd(dmul(t[TY_GV01], dPx), dmul(t[TY_GV11], dPv));
  double sv = dadd(dmul(dPx, g0), dmul(dPv, g1));
  double cx = dadd(dmul(t[TY_TI00], sx), dmul(t[TY_TI01], sv));
  double cv = dadd(dmul(t[TY_TI10], sx), dmul(t[TY_TI11], sv));
  dqx = dsub(yx, dmul(0.5, cx));
  dqv = dsub(yv, dmul(0.5, cv));
}

// Squared Lagrangian distance in element spacings (Sec. 2.3.1, d[dQ]).
__device__ __forceinline__ double dist2_exact(const double* t, const Grid& g, double Px, double Pv,
                                              double& xi, double& ze) {
  double dqx, dqv;
  qofp_exact(t, Px, Pv, dqx, dqv);
  xi = dmul(dqx, g.inv_dxm);
  ze = dmul(dqv, g.inv_dvm);
  return dadd(dmul(xi, xi), dmul(ze, ze));
}

__device__ __forceinline__ double site_x(const Grid& g, long long i) {
  return dadd(g.x_lo, dmul((double)i, g.dx));
}
__device__ __forceinline__ double site_v(const Grid& g, long long j) {
  return dadd(g.v_lo, dmul((double)j, g.dv));
}

__device__ __forceinline__ unsigned long long dkey(double d) {
  return (unsigned long long)__double_as_longlong(d);
}

}  // namespace vm

namespace vm {
// The last CUDA error a library call met in this host thread (reported by
// vm_last_cuda_error), and the clearing of errors left unread by other code.
void note_cuda(cudaError_t e);
void clear_foreign_error();
}  // namespace vm

#define VM_CUDA_TRY(expr)                       \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) {                    \
      vm::note_cuda(e_);                        \
      return VM_E_CUDA;                         \
    }                                           \
  } while (0)
