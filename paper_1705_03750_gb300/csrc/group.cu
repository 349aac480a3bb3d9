// Many independent solves advanced together (Sec. 2.4 for each solve; the
// solves are independent problems): the host side of the group launches.
//
// A group holds solves of one precision.  Its plan is a device table of the
// solves' constants and buffers plus, per phase, the offsets of every
// solve's units in the phase's work list; each phase of a step is then one
// launch for the whole group (group_* in the kernels' translation units).
// The launch shapes (persistent blocks per phase) do not change any result,
// so they can be tuned on the steps of the run itself.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "group.cuh"

namespace vm {

namespace {

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

SolveDesc desc_of(const vm_solver* s, bool gated) {
  SolveDesc d;
  memset(&d, 0, sizeof d);
  d.g = s->g;
  d.g.gate = gated ? &s->ds->gate : nullptr;
  const float fa = (float)s->g.alpha, fb = (float)s->g.beta;
  d.alo = ((double)fa <= s->g.alpha) ? fa : nextafterf(fa, -INFINITY);
  d.ahi = ((double)fa >= s->g.alpha) ? fa : nextafterf(fa, INFINITY);
  d.blo = ((double)fb <= s->g.beta) ? fb : nextafterf(fb, -INFINITY);
  d.bhi = ((double)fb >= s->g.beta) ? fb : nextafterf(fb, INFINITY);
  d.map_windows = s->cfg.map_windows;
  d.fini = s->fini;
  d.eta = s->eta;
  d.f = s->f;
  d.tmp = s->tmp;
  d.map = s->map;
  d.slot1 = s->slot1;
  d.rec_key = s->rec_key;
  d.rec_site = s->rec_site;
  d.rec_cap = s->rec_cap;
  d.holes_a = s->holes_a;
  d.holes_b = s->holes_b;
  d.ovf1 = s->overflow_list;
  d.ovf2 = s->overflow_list2;
  d.gwin = s->gwin;
  d.gwin_words = global_window_words(s->g.nx, s->g.nv, s->g.pad);
  d.t1seed = s->t1seed;
  d.t1seed_cap = s->t1seed_cap;
  d.el = s->el;
  d.tay = s->tay;
  d.tayf = s->tayf;
  d.M = s->M;
  d.a = s->a;
  d.da = s->da;
  d.d2a = s->d2a;
  d.thx = s->thomas_x;
  d.thv = s->thomas_v;
  d.thxf = s->thomas_xf;
  d.thvf = s->thomas_vf;
  d.Mpart = s->Mpart;
  d.ds = s->ds;
  d.n_s = s->cfg.n_s;
  d.emap_thr = s->cfg.emap_remap;
  return d;
}

// Per-phase unit counts of one solve, in the order of the offset arrays.
enum { U_ELEM64 = 0, U_PAIR, U_ROWS, U_DIFF, U_SITES, U_COPY, U_ROWS4, U_COLS, U_SOLVE, U_TILES, U_N };

void units_of(const vm_solver* s, int (&u)[U_N]) {
  const long long n = (long long)s->g.nx * s->g.nv;
  u[U_ELEM64] = cdiv(s->g.ne, 64);
  u[U_PAIR] = cdiv(s->g.ne, 8);
  u[U_ROWS] = s->g.nx;
  u[U_DIFF] = cdiv(s->g.nx, 128);
  u[U_SITES] = std::max(1, cdiv(n / 4, 256));
  u[U_COPY] = cdiv(n, 4096);
  u[U_ROWS4] = cdiv(s->g.nx, 4);
  u[U_COLS] = cdiv(s->g.nv, 32);
  u[U_SOLVE] = 1;
  u[U_TILES] = recon_tiles_of(s->g);
}

}  // namespace

size_t group_table_bytes(int ns) {
  return ((size_t)ns * sizeof(SolveDesc) + 255) / 256 * 256 + (size_t)(U_N + 1) * (ns + 1) * sizeof(int) + 256;
}

vm_status group_check(vm_solver* const* solvers, int n) {
  if (!solvers || n < 1) return VM_E_INVALID_ARG;
  for (int i = 0; i < n; i++) {
    const vm_solver* s = solvers[i];
    if (!s) return VM_E_INVALID_ARG;
    if (!s->have_f) return VM_E_STATE;
    if (s->fp32 != solvers[0]->fp32) return VM_E_INVALID_ARG;
    if (s->g.recon_tiles != solvers[0]->g.recon_tiles) return VM_E_INVALID_ARG;
    // host decisions per step or per remap: not part of a group step (the
    // E_map criterion is decided on the device, see device_cycle)
    if (s->cfg.c_dyn > 0.0 || s->cfg.f_th > 0.0) return VM_E_INVALID_ARG;
    for (int j = 0; j < i; j++)
      if (solvers[j] == s) return VM_E_INVALID_ARG;
  }
  return VM_OK;
}

// Fill the plan of solvers[0..n) into the device table at d_table (at least
// group_table_bytes(n) bytes, 256-byte aligned), staging through the host
// buffer `host` (the same size, kept alive until the copy completes: the
// copy is asynchronous on `stream`).  gated: the plan of the remaps each
// solve's device decision may skip (its Grids carry the solves' gates).
void group_plan(GroupPlan& P, vm_solver* const* solvers, int n, void* d_table, void* host, cudaStream_t stream,
                bool gated) {
  memset(&P, 0, sizeof P);
  char* hb = (char*)host;
  char* db = (char*)d_table;
  const size_t dbytes = ((size_t)n * sizeof(SolveDesc) + 255) / 256 * 256;
  SolveDesc* hd = (SolveDesc*)hb;
  int* hoff = (int*)(hb + dbytes);
  int tot[U_N] = {0};
  size_t big = 0;
  for (int i = 0; i < n; i++) {
    hd[i] = desc_of(solvers[i], gated);
    int u[U_N];
    units_of(solvers[i], u);
    for (int k = 0; k < U_N; k++) {
      hoff[k * (n + 1) + i] = tot[k];
      tot[k] += u[k];
    }
    big = std::max(big, group_big_smem(solvers[i]->g));
  }
  for (int k = 0; k < U_N; k++) hoff[k * (n + 1) + n] = tot[k];
  const int* doff = (const int*)(db + dbytes);
  P.D = (const SolveDesc*)db;
  P.ns = n;
  P.fp32 = solvers[0]->fp32;
  P.stream = stream;
  P.off_elem64 = doff + U_ELEM64 * (n + 1);
  P.tot_elem64 = tot[U_ELEM64];
  P.off_pair = doff + U_PAIR * (n + 1);
  P.tot_pair = tot[U_PAIR];
  P.off_rows = doff + U_ROWS * (n + 1);
  P.tot_rows = tot[U_ROWS];
  P.off_diff = doff + U_DIFF * (n + 1);
  P.tot_diff = tot[U_DIFF];
  P.off_sites = doff + U_SITES * (n + 1);
  P.tot_sites = tot[U_SITES];
  P.off_copy = doff + U_COPY * (n + 1);
  P.tot_copy = tot[U_COPY];
  P.off_rows4 = doff + U_ROWS4 * (n + 1);
  P.tot_rows4 = tot[U_ROWS4];
  P.off_cols = doff + U_COLS * (n + 1);
  P.tot_cols = tot[U_COLS];
  P.off_solve = doff + U_SOLVE * (n + 1);
  P.off_tiles = doff + U_TILES * (n + 1);
  P.tot_tiles = tot[U_TILES];
  P.recon_tiles = solvers[0]->g.recon_tiles;
  P.off_dyn = (int*)(db + dbytes) + U_N * (n + 1);
  P.big_smem = big;
  P.big_blocks_cap = 0;
  cudaMemcpyAsync(d_table, host, dbytes + (size_t)U_N * (n + 1) * sizeof(int), cudaMemcpyHostToDevice, stream);
}

// Record an event before a phase when the plan carries timing events.
static inline void mark(const GroupPlan& P, const GroupTiming* T, int phase) {
  if (T) cudaEventRecord(T->ev[phase], P.stream);
}

void group_step_transport(const GroupPlan& P, const GroupTiming* T) {
  mark(P, T, GT_DRIFT);
  group_drift(P, true);
  mark(P, T, GT_MAP);
  group_map(P);
  mark(P, T, GT_RECON);
  group_reconstruct(P);
  mark(P, T, GT_SCAN);
  group_scan_force(P);
  mark(P, T, GT_KICK);
  group_kick(P);
  mark(P, T, GT_END);
}

void group_step_remap(const GroupPlan& P) {
  group_taylor(P);
  group_map(P);
  group_remap_resample(P);
  group_copy_tmp_to_fini(P);
  group_spline(P);
  group_reset(P);
}

// The remaps of a gated plan after a transport step: E_map and each solve's
// decision, then the remap launches, which skip the solves left shut.
void group_step_gated(const GroupPlan& P) {
  group_remap_gate(P);
  group_step_remap(P);
}

// Host counters of a solve after a group step (as vm_step keeps them; the
// cycle of a device_cycle solve is counted on the device).
void group_count_step(vm_solver* s, bool remapped) {
  s->nstep++;
  s->time += s->g.dt;
  s->last_dt = s->g.dt;
  if (!device_cycle(s)) s->cyc = remapped ? 0 : s->cyc + 1;
}

}  // namespace vm
