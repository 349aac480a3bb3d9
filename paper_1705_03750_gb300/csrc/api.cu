// C ABI of the solver (declared in include/vlamet.h): configuration,
// workspace layout, and the host-side sequencing of the kernels.  The host
// never touches grid data; it only launches and copies on request.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t fini, eta, f, tmp, map, slot1, rec_key, rec_site, holes_a, holes_b, ovf, gwin, seed, el, tay, tayf, M, a, da, d2a,
      thx, thv, thxf, thvf, rect, mpart, dpart, ds, total;
};

bool valid(const vm_config* c) {
  if (!c) return false;
  if (c->nx < 4 || c->nv < 4 || c->elem_stride < 1 || c->n_s < 1) return false;
  if (!(c->x_hi > c->x_lo) || !(c->v_hi > c->v_lo) || !(c->dt > 0.0) || !isfinite(c->G)) return false;
  if (c->precision != VM_FP64 && c->precision != VM_FP32_MIXED) return false;
  if (c->pad < 0 || c->max_hole_rounds < 0) return false;
  if (c->map_windows != 0 && c->map_windows != 1) return false;
  if (!(c->emap_remap >= 0.0) || !isfinite(c->emap_remap)) return false;
  if (!(c->c_dyn >= 0.0) || !isfinite(c->c_dyn)) return false;
  if (!(c->alpha >= 0.0) || !(c->beta >= 0.0)) return false;
  if (!(c->f_th >= 0.0) || !isfinite(c->f_th)) return false;
  if (c->recon_mode != 0 && c->recon_mode != 1) return false;
  // 32-bit site indices; element indices fit the 24-bit field of the owner slots
  if ((long long)c->nx * (long long)c->nv >= (1ll << 31) / 2) return false;
  const long long s = c->elem_stride;
  const long long Lx = 2 * ((c->nx - 1 + 2 * s - 1) / (2 * s)) + 3, Lv = 2 * ((c->nv - 1 + 2 * s - 1) / (2 * s)) + 3;
  if (Lx * Lv >= (1ll << 24)) return false;
  return true;
}

void lattice(const vm_config* c, int32_t* Kx, int32_t* Kv, int32_t* Lx, int32_t* Lv) {
  const int s = c->elem_stride;
  *Kx = (c->nx - 1 + 2 * s - 1) / (2 * s);
  *Kv = (c->nv - 1 + 2 * s - 1) / (2 * s);
  *Lx = 2 * *Kx + 3;
  *Lv = 2 * *Kv + 3;
}

Layout layout(const vm_config* c) {
  Layout L{};
  int32_t Kx, Kv, Lx, Lv;
  lattice(c, &Kx, &Kv, &Lx, &Lv);
  const size_t n = (size_t)c->nx * c->nv, ne = (size_t)Lx * Lv;
  const size_t sr = (c->precision == VM_FP32_MIXED) ? 4 : 8;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.fini = take(n * sr);
  L.eta = take(n * sr);
  L.f = take(n * sr);
  L.tmp = take(n * sr);
  L.map = take(n * 4);
  L.slot1 = take(n * 4);
  L.rec_key = take(n * 16);  // one record per site
  L.rec_site = take(n * 4);
  L.holes_a = take(n * 4);
  L.holes_b = take(2 * n * 4);
  L.ovf = take(2 * ne * 8);
  const long long pad = c->pad ? c->pad : c->elem_stride;
  L.gwin = take(vm::kGlobalBlocks * vm::global_window_words(c->nx, c->nv, pad) * 8);
  L.seed = take(std::min<size_t>(ne, vm::kSeedRecords) * 96 * 8);
  L.el = take(12 * ne * 8);
  L.tay = take(16 * ne * 8);
  L.tayf = take(32 * ne * 4);
  L.M = take(c->nx * 8);
  L.a = take(c->nx * 8);
  L.da = take(c->nx * 8);
  L.d2a = take(c->nx * 8);
  L.thx = take(2 * c->nx * 8);
  L.thv = take(2 * c->nv * 8);
  L.thxf = take(2 * c->nx * 4);
  L.thvf = take(2 * c->nv * 4);
  L.rect = take(4 * vm::kRectBlocks * 8);
  L.mpart = take((size_t)c->nx * (size_t)((c->nv + 255) / 256) * 8);
  L.dpart = take(6 * vm::kRectBlocks * 8);
  L.ds = take(sizeof(vm::DevState));
  L.total = o;
  return L;
}

// LU factors of the constant spline system (rows (1,4,1), ends (4,2) and
// (2,4)): c'_i and 1/den_i of the Thomas sweeps.
void thomas(int n, std::vector<double>& out) {
  out.assign(2 * (size_t)n, 0.0);
  double cprev = 0.0;
  for (int i = 0; i < n; i++) {
    const double sub = (i == 0) ? 0.0 : ((i == n - 1) ? 2.0 : 1.0);
    const double sup = (i == n - 1) ? 0.0 : ((i == 0) ? 2.0 : 1.0);
    const double den = 4.0 - sub * cprev;
    const double cp = sup / den;
    out[i] = cp;
    out[n + i] = 1.0 / den;
    cprev = cp;
  }
}

size_t ne_total(const vm_solver* s) { return (size_t)s->g.ne; }
using vm::SLOT_MASK;

// Launch errors of this call (cleared, so that one failed launch does not
// make every later call report it).
vm_status check_launch(vm_solver* s) {
  (void)s;
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return VM_OK;
  vm::note_cuda(e);
  return VM_E_CUDA;
}

}  // namespace

namespace vm {

thread_local cudaError_t t_last_cuda = cudaSuccess;

void note_cuda(cudaError_t e) { t_last_cuda = e; }

// An error that earlier CUDA calls of other code in this thread left unread
// (a query that found work not yet done, a failed allocation the caller
// recovered from) is not this call's: drop it before launching, so that the
// check after the launches sees only ours.  An error that has corrupted the
// context persists and makes our own launches fail.
void clear_foreign_error() { (void)cudaGetLastError(); }

namespace {
long long floor_div(long long a, long long b) {  // b > 0
  const long long q = a / b;
  return (q * b > a) ? q - 1 : q;
}
}  // namespace

// Adaptive computing domain (Sec. 2.2.1, eq. constrf; Sec. 2.3), after f_ini
// changed (vm_set_f, remap): the node rectangle of |f_ini| > f_th, read back
// (synchronises), f_ini cut to it, and the lattice lines that exist: the
// last line at or before its first node and the first at or after its last
// node (integer arithmetic on the lines' index positions (n-1)/2 + (k-K-1)s),
// plus one extra layer on every side.
cudaError_t domain_update(vm_solver* s) {
  Grid& g = s->g;
  if (!g.fth_on) return cudaSuccess;
  int32_t box[4] = {g.nx, -1, g.nv, -1};
  cudaError_t e = cudaMemcpyAsync(s->ds->fbox, box, sizeof box, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return e;
  launch_fth_box(s);
  e = cudaMemcpyAsync(box, s->ds->fbox, sizeof box, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return e;
  if (box[1] < 0) {  // nothing above the threshold: no element exists
    g.klo = g.llo = 0;
    g.khi = g.lhi = -1;
  } else {
    const long long s2 = 2ll * g.s;
    const long long klo = g.Kx + 1 + floor_div(2ll * box[0] - (g.nx - 1), s2) - 1;
    const long long khi = g.Kx + 1 - floor_div(-(2ll * box[1] - (g.nx - 1)), s2) + 1;
    const long long llo = g.Kv + 1 + floor_div(2ll * box[2] - (g.nv - 1), s2) - 1;
    const long long lhi = g.Kv + 1 - floor_div(-(2ll * box[3] - (g.nv - 1)), s2) + 1;
    g.klo = (int32_t)std::max(0ll, klo);
    g.khi = (int32_t)std::min<long long>(g.Lx - 1, khi);
    g.llo = (int32_t)std::max(0ll, llo);
    g.lhi = (int32_t)std::min<long long>(g.Lv - 1, lhi);
  }
  launch_fth_cut(s);
  return cudaGetLastError();
}

// One transport step t -> t + dt (Sec. 2.4): predictor drift + Taylor terms
// at t + dt/2, map, f(t + dt/2) and M(i), force, kick + corrector.  Only
// enqueues work (safe inside a stream capture); host counters untouched.
void step_transport(vm_solver* s) {
  launch_drift(s, true);
  launch_map(s);
  launch_reconstruct(s);
  launch_scan_force(s);
  launch_kick_drift(s);
}

// Remap at the current elements (Secs. 2.2.2, 2.3.2); enqueue only.
cudaError_t step_remap(vm_solver* s) {
  launch_taylor(s);
  launch_map(s);
  launch_remap_resample(s, s->tmp);
  // the resampled f becomes f_ini (a copy, not a pointer swap, so that a
  // captured step keeps its buffers)
  cudaError_t e = cudaMemcpyAsync(s->fini, s->tmp, s->n * s->sreal, cudaMemcpyDeviceToDevice, s->stream);
  if (e != cudaSuccess) return e;
  e = domain_update(s);
  if (e != cudaSuccess) return e;
  launch_spline_solve(s, s->fini, s->eta);
  launch_reset_elements(s);
  return cudaSuccess;
}

// The remap after a step, behind the device's decision (Sec. 2.3.2): E_map
// and the decision kernel, then the remap's launches with the Grid's gate
// set, each of which returns at once unless the decision opened it.
// Enqueue only; host counters untouched.
void step_remap_gated(vm_solver* s) {
  launch_remap_gate(s);
  s->g.gate = &s->ds->gate;
  launch_taylor(s);
  launch_map(s);
  launch_remap_resample(s, s->tmp);
  launch_copy_gated(s);
  launch_spline_solve(s, s->fini, s->eta);
  launch_reset_elements(s);
  s->g.gate = nullptr;
}

// Device copies of the remap cycle, from the host's (cycle, forced remaps);
// the gate shut.  Not inside a stream capture (a pageable source).
cudaError_t cycle_to_device(vm_solver* s) {
  struct {
    long long emap_remaps;
    int32_t cyc, gate;
  } c{(long long)s->emap_remaps, s->cyc, 0};
  static_assert(offsetof(DevState, cyc) == offsetof(DevState, emap_remaps) + 8 &&
                    offsetof(DevState, gate) == offsetof(DevState, cyc) + 4 && sizeof c == 16,
                "cycle fields of DevState");
  return cudaMemcpyAsync(&s->ds->emap_remaps, &c, sizeof c, cudaMemcpyHostToDevice, s->stream);
}

// Host copies of a device-kept cycle (synchronises).
cudaError_t cycle_to_host(vm_solver* s) {
  if (!device_cycle(s)) return cudaSuccess;
  int32_t cyc = 0;
  long long er = 0;
  cudaError_t e = cudaMemcpyAsync(&cyc, &s->ds->cyc, sizeof cyc, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&er, &s->ds->emap_remaps, sizeof er, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) {
    s->cyc = cyc;
    s->emap_remaps = er;
  }
  return e;
}

}  // namespace vm

namespace {

// Largest projected density of s->f, computed and read back (synchronises).
vm_status rho_max_now(vm_solver* s, double* rho) {
  vm::DevState* d = s->ds;
  VM_CUDA_TRY(cudaMemsetAsync(&d->rho_max_bits, 0, sizeof d->rho_max_bits, s->stream));
  vm::launch_rho_max(s);
  unsigned long long bits = 0;
  VM_CUDA_TRY(cudaMemcpyAsync(&bits, &d->rho_max_bits, sizeof bits, cudaMemcpyDeviceToHost, s->stream));
  vm_status st = vm_sync(s);
  if (st != VM_OK) return st;
  memcpy(rho, &bits, 8);
  return VM_OK;
}

// E_map of the current influence map, computed and read back (synchronises).
vm_status emap_now(vm_solver* s, double* e) {
  vm::DevState* d = s->ds;
  VM_CUDA_TRY(cudaMemsetAsync(&d->emap2_bits, 0, sizeof d->emap2_bits, s->stream));
  vm::launch_emap(s);
  unsigned long long bits = 0;
  VM_CUDA_TRY(cudaMemcpyAsync(&bits, &d->emap2_bits, sizeof bits, cudaMemcpyDeviceToHost, s->stream));
  vm_status st = vm_sync(s);
  if (st != VM_OK) return st;
  double e2;
  memcpy(&e2, &bits, 8);
  *e = sqrt(e2);
  return VM_OK;
}

vm_status remap_internal(vm_solver* s) {
  if (vm::step_remap(s) != cudaSuccess) return VM_E_CUDA;
  s->cyc = 0;
  if (vm::device_cycle(s)) VM_CUDA_TRY(cudaMemsetAsync(&s->ds->cyc, 0, 2 * sizeof(int32_t), s->stream));
  return check_launch(s);
}

// 8 bytes per site of scratch for the copy calls: the second hole list,
// which only lives inside one influence map.
void* staging(vm_solver* s) { return s->holes_b; }

vm_status read_real(vm_solver* s, const void* src, void* out, int32_t dtype, int32_t on_device) {
  if (!out || (dtype != VM_DTYPE_F64 && dtype != VM_DTYPE_F32)) return VM_E_INVALID_ARG;
  const size_t esz = dtype == VM_DTYPE_F64 ? 8 : 4;
  const bool same = (esz == s->sreal);
  if (on_device) {
    if (same) {
      VM_CUDA_TRY(cudaMemcpyAsync(out, src, s->n * esz, cudaMemcpyDeviceToDevice, s->stream));
    } else {
      vm::launch_convert(s, src, out, dtype, s->n);
    }
    return check_launch(s);
  }
  if (same) {
    VM_CUDA_TRY(cudaMemcpyAsync(out, src, s->n * esz, cudaMemcpyDeviceToHost, s->stream));
  } else {
    vm::launch_convert(s, src, staging(s), dtype, s->n);
    VM_CUDA_TRY(cudaMemcpyAsync(out, staging(s), s->n * esz, cudaMemcpyDeviceToHost, s->stream));
  }
  return vm_sync(s);
}

const char* const kKernelNames[vm::KID_N] = {
    "drift_taylor", "taylor", "kick_drift", "reset_elements", "scan_force", "diagnostics",
    "map_begin", "claim_small", "claim_large", "find_holes", "holes", "resolve", "read_map",
    "reconstruct", "remap_resample", "convert", "spline_rows", "spline_cols", "claim_pair", "emap_gate"};

}  // namespace

namespace vm {

int prof_begin(vm_solver* s, int kid) {
  if (!s->prof) return -1;
  if (s->prof_n >= PROF_CAP) prof_flush(s);
  const int slot = s->prof_n++;
  if (slot >= s->prof_created) {
    cudaEventCreate(&s->prof_ev[2 * slot]);
    cudaEventCreate(&s->prof_ev[2 * slot + 1]);
    s->prof_created = slot + 1;
  }
  s->prof_kind[slot] = kid;
  cudaEventRecord(s->prof_ev[2 * slot], s->stream);
  return slot;
}

void prof_end(vm_solver* s, int slot) {
  if (slot < 0) return;
  cudaEventRecord(s->prof_ev[2 * slot + 1], s->stream);
}

// Wait for the recorded launches and fold their durations into the totals.
void prof_flush(vm_solver* s) {
  if (s->prof_n == 0) return;
  cudaEventSynchronize(s->prof_ev[2 * (s->prof_n - 1) + 1]);
  for (int i = 0; i < s->prof_n; i++) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->prof_ev[2 * i], s->prof_ev[2 * i + 1]) == cudaSuccess) {
      s->prof_ms[s->prof_kind[i]] += ms;
      s->prof_count[s->prof_kind[i]]++;
    }
  }
  s->prof_n = 0;
}

}  // namespace vm

extern "C" {

void vm_config_default(vm_config* c) {
  if (!c) return;
  memset(c, 0, sizeof *c);
  c->alpha = sqrt(3.0) / 4.0;
  c->beta = 0.5 * (1.0 - sqrt(3.0) / 2.0);
  c->precision = VM_FP64;
}

size_t vm_workspace_bytes(const vm_config* c) {
  if (!valid(c)) return 0;
  return layout(c).total;
}

const char* vm_status_string(vm_status st) {
  switch (st) {
    case VM_OK: return "ok";
    case VM_E_INVALID_ARG: return "invalid argument";
    case VM_E_OOM: return "workspace too small";
    case VM_E_CUDA: return "CUDA runtime error";
    case VM_E_INTERNAL: return "internal consistency check failed";
    case VM_E_NOT_CONVERGED: return "unexplored-site repair did not converge";
    case VM_E_PATCH_OVERFLOW: return "influence region larger than the largest flood-fill window";
    case VM_E_BUDGET: return "memory budget exceeded";
    case VM_E_STATE: return "call out of order";
    case VM_E_IO: return "checkpoint file could not be written or read";
  }
  return "unknown status";
}

vm_status vm_create(const vm_config* c, void* d_workspace, size_t bytes, void* stream, vm_solver** out) {
  return vm::solver_create(c, d_workspace, bytes, (cudaStream_t)stream, true, out);
}

}  // extern "C"

// Create a solver on the caller's workspace; with sync = false the
// initialisation (workspace clear, spline factors) is only queued on the
// stream (the serving loop creates solvers while earlier work still runs).
vm_status vm::solver_create(const vm_config* c, void* d_workspace, size_t bytes, cudaStream_t stream, bool sync,
                            vm_solver** out) {
  if (!out) return VM_E_INVALID_ARG;
  *out = nullptr;
  if (!valid(c) || !d_workspace || ((uintptr_t)d_workspace & 255)) return VM_E_INVALID_ARG;
  const Layout L = layout(c);
  if (bytes < L.total) return VM_E_OOM;
  vm_solver* s = (vm_solver*)calloc(1, sizeof(vm_solver));
  if (!s) return VM_E_OOM;
  s->cfg = *c;
  if (s->cfg.pad == 0) s->cfg.pad = c->elem_stride;
  if (s->cfg.max_hole_rounds == 0) s->cfg.max_hole_rounds = c->nx + c->nv;
  s->stream = stream;
  s->fp32 = (c->precision == VM_FP32_MIXED);
  s->sreal = s->fp32 ? 4 : 8;
  s->n = (size_t)c->nx * c->nv;
  vm::Grid& g = s->g;
  g.nx = c->nx;
  g.nv = c->nv;
  g.s = c->elem_stride;
  g.pad = s->cfg.pad;
  lattice(c, &g.Kx, &g.Kv, &g.Lx, &g.Lv);
  g.ne = g.Lx * g.Lv;
  // Derived constants, one operation at a time (no contraction).
  g.x_lo = c->x_lo;
  g.v_lo = c->v_lo;
  g.dx = (c->x_hi - c->x_lo) / (double)(c->nx - 1);
  g.dv = (c->v_hi - c->v_lo) / (double)(c->nv - 1);
  g.dxm = (double)c->elem_stride * g.dx;
  g.dvm = (double)c->elem_stride * g.dv;
  g.inv_dx = 1.0 / g.dx;
  g.inv_dv = 1.0 / g.dv;
  g.inv_dxm = 1.0 / g.dxm;
  g.inv_dvm = 1.0 / g.dvm;
  g.r_vx = g.dvm / g.dxm;
  g.r_xv = g.dxm / g.dvm;
  g.cx = 0.5 * (c->x_lo + c->x_hi);
  g.cv = 0.5 * (c->v_lo + c->v_hi);
  g.dxdv = g.dx * g.dv;
  g.alpha = c->alpha;
  g.beta = c->beta;
  g.dt = c->dt;
  g.half_dt = 0.5 * c->dt;
  g.A = 2.0 * kPi * c->G;
  g.literal_fd = c->literal_fd;
  g.max_hole_rounds = s->cfg.max_hole_rounds;
  g.fth_on = c->f_th > 0.0 ? 1 : 0;
  g.recon_tiles = (c->precision == VM_FP32_MIXED && c->recon_mode == 1) ? 1 : 0;
  g.klo = 0;
  g.khi = g.Lx - 1;
  g.llo = 0;
  g.lhi = g.Lv - 1;
  char* base = (char*)d_workspace;
  s->fini = base + L.fini;
  s->eta = base + L.eta;
  s->f = base + L.f;
  s->tmp = base + L.tmp;
  s->map = (uint32_t*)(base + L.map);
  s->slot1 = (uint32_t*)(base + L.slot1);
  s->rec_key = (unsigned long long*)(base + L.rec_key);
  s->rec_site = (int32_t*)(base + L.rec_site);
  // each site is listed at most once per map
  s->rec_cap = (int32_t)s->n;
  s->holes_a = (int32_t*)(base + L.holes_a);
  s->holes_b = (int32_t*)(base + L.holes_b);
  s->overflow_list = (int2*)(base + L.ovf);
  s->overflow_list2 = s->overflow_list + ne_total(s);
  s->gwin = (unsigned long long*)(base + L.gwin);
  s->t1seed = (unsigned long long*)(base + L.seed);
  s->t1seed_cap = (int32_t)std::min<size_t>(ne_total(s), vm::kSeedRecords);
  s->el = (double*)(base + L.el);
  s->tay = (double*)(base + L.tay);
  s->tayf = (float*)(base + L.tayf);
  s->M = (double*)(base + L.M);
  s->a = (double*)(base + L.a);
  s->da = (double*)(base + L.da);
  s->d2a = (double*)(base + L.d2a);
  s->thomas_x = (double*)(base + L.thx);
  s->thomas_v = (double*)(base + L.thv);
  s->thomas_xf = (float*)(base + L.thxf);
  s->thomas_vf = (float*)(base + L.thvf);
  s->rect_part = (double*)(base + L.rect);
  s->Mpart = (double*)(base + L.mpart);
  s->diag_part = (double*)(base + L.dpart);
  s->ds = (vm::DevState*)(base + L.ds);
  if (!vm::map_prepare(g) || !vm::recon_prepare()) {
    free(s);
    return VM_E_INVALID_ARG;
  }
  std::vector<double> tx, tv;
  thomas(c->nx, tx);
  thomas(c->nv, tv);
  std::vector<float> txf(tx.begin(), tx.end()), tvf(tv.begin(), tv.end());
  vm_status st = VM_OK;
  do {
    if (cudaMemsetAsync(base, 0, L.total, s->stream) != cudaSuccess) { st = VM_E_CUDA; break; }
    // owner slots start empty (all-ones: an epoch no map uses)
    if (cudaMemsetAsync(s->map, 0xFF, s->n * 4, s->stream) != cudaSuccess) { st = VM_E_CUDA; break; }
    if (cudaMemsetAsync(s->slot1, 0xFF, s->n * 4, s->stream) != cudaSuccess) { st = VM_E_CUDA; break; }
    // contested-site records start (and stay, between maps) empty
    if (cudaMemsetAsync(s->rec_key, 0xFF, s->n * 16, s->stream) != cudaSuccess) { st = VM_E_CUDA; break; }
    if (cudaMemcpyAsync(s->thomas_x, tx.data(), tx.size() * 8, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->thomas_v, tv.data(), tv.size() * 8, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->thomas_xf, txf.data(), txf.size() * 4, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->thomas_vf, tvf.data(), tvf.size() * 4, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
      st = VM_E_CUDA;
      break;
    }
    vm::DevState init{};
    init.det_min_key = ~0ull;
    init.det_max_key = 0ull;
    if (cudaMemcpyAsync(s->ds, &init, sizeof init, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) { st = VM_E_CUDA; break; }
    if (sync && cudaStreamSynchronize(s->stream) != cudaSuccess) { st = VM_E_CUDA; break; }
  } while (0);
  if (st != VM_OK) {
    free(s);
    return st;
  }
  *out = s;
  return VM_OK;
}

extern "C" {

void vm_destroy(vm_solver* s) {
  if (!s) return;
  // the caller frees the workspace after this returns: no work of this
  // solver may still be running on it
  cudaStreamSynchronize(s->stream);
  for (int i = 0; i < 2 * s->prof_created; i++) cudaEventDestroy(s->prof_ev[i]);
  free(s);
}

vm_status vm_profile(vm_solver* s, int32_t enable) {
  if (!s) return VM_E_INVALID_ARG;
  vm::prof_flush(s);
  for (int k = 0; k < vm::KID_N; k++) {
    s->prof_ms[k] = 0.0;
    s->prof_count[k] = 0;
  }
  s->prof = enable ? 1 : 0;
  return VM_OK;
}

int32_t vm_profile_read(vm_solver* s, vm_kernel_stat* out, int32_t max) {
  if (!s) return -1;
  vm::prof_flush(s);
  int32_t n = 0;
  for (int k = 0; k < vm::KID_N; k++) {
    if (s->prof_count[k] == 0) continue;
    if (out && n < max) {
      memset(&out[n], 0, sizeof out[n]);
      strncpy(out[n].name, kKernelNames[k], sizeof out[n].name - 1);
      out[n].launches = s->prof_count[k];
      out[n].total_ms = s->prof_ms[k];
    }
    n++;
  }
  return n;
}

vm_status vm_lattice(const vm_solver* s, int32_t* ne, int32_t* Lx, int32_t* Lv) {
  if (!s) return VM_E_INVALID_ARG;
  if (ne) *ne = s->g.ne;
  if (Lx) *Lx = s->g.Lx;
  if (Lv) *Lv = s->g.Lv;
  return VM_OK;
}

int64_t vm_launch_count(const vm_solver* s) { return s ? s->launches : 0; }

vm_status vm_set_f(vm_solver* s, const double* f0, int32_t on_device) {
  if (!s || !f0) return VM_E_INVALID_ARG;
  vm::clear_foreign_error();
  const size_t bytes = s->n * 8;
  if (!s->fp32) {
    VM_CUDA_TRY(cudaMemcpyAsync(s->fini, f0, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                s->stream));
  } else {
    const double* src = f0;
    if (!on_device) {
      VM_CUDA_TRY(cudaMemcpyAsync(staging(s), f0, bytes, cudaMemcpyHostToDevice, s->stream));
      src = (const double*)staging(s);
    }
    vm::launch_store_real(s, src, s->fini, s->n);
  }
  VM_CUDA_TRY(vm::domain_update(s));
  VM_CUDA_TRY(cudaMemcpyAsync(s->f, s->fini, s->n * s->sreal, cudaMemcpyDeviceToDevice, s->stream));
  vm::launch_spline_solve(s, s->fini, s->eta);
  vm::launch_reset_elements(s);
  s->have_f = 1;
  s->nstep = 0;
  s->emap_remaps = 0;
  s->time = 0.0;
  s->last_dt = 0.0;
  s->cyc = 0;
  VM_CUDA_TRY(vm::cycle_to_device(s));
  return check_launch(s);
}

vm_status vm_set_elements(vm_solver* s, const double* soa12, int32_t on_device) {
  if (!s || !soa12) return VM_E_INVALID_ARG;
  VM_CUDA_TRY(cudaMemcpyAsync(s->el, soa12, 12 * (size_t)s->g.ne * 8,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
  if (!on_device) VM_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return VM_OK;
}

vm_status vm_get_elements(vm_solver* s, double* soa12, int32_t on_device) {
  if (!s || !soa12) return VM_E_INVALID_ARG;
  VM_CUDA_TRY(cudaMemcpyAsync(soa12, s->el, 12 * (size_t)s->g.ne * 8,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
  return on_device ? VM_OK : vm_sync(s);
}

vm_status vm_compute_map(vm_solver* s) {
  if (!s) return VM_E_INVALID_ARG;
  vm::clear_foreign_error();
  vm::launch_taylor(s);
  vm::launch_map(s);
  return check_launch(s);
}

vm_status vm_reconstruct(vm_solver* s) {
  if (!s) return VM_E_INVALID_ARG;
  vm::clear_foreign_error();
  if (!s->have_f) return VM_E_STATE;
  vm::launch_taylor(s);
  vm::launch_map(s);
  vm::launch_reconstruct(s);
  vm::launch_scan_force(s);
  return check_launch(s);
}

vm_status vm_step(vm_solver* s, int32_t nsteps) {
  if (!s || nsteps < 0) return VM_E_INVALID_ARG;
  vm::clear_foreign_error();
  if (!s->have_f) return VM_E_STATE;
  for (int32_t it = 0; it < nsteps; it++) {
    if (s->cfg.c_dyn > 0.0) {
      // Sec. 2.4: this step's dt from the last reconstructed f
      double rho = 0.0;
      vm_status st = rho_max_now(s, &rho);
      if (st != VM_OK) return st;
      double dt = s->cfg.dt;
      if (rho > 0.0) {
        const double lim = s->cfg.c_dyn / sqrt(rho);
        if (lim < dt) dt = lim;
      }
      s->g.dt = dt;
      s->g.half_dt = 0.5 * dt;
    }
    vm::step_transport(s);
    s->nstep++;
    s->time += s->g.dt;
    s->last_dt = s->g.dt;
    if (vm::device_cycle(s)) {
      // E_map and the cycle decide on the device; no round trip
      vm::step_remap_gated(s);
      continue;
    }
    s->cyc++;
    bool remap = s->cyc >= s->cfg.n_s;
    if (!remap && s->cfg.emap_remap > 0.0) {
      // E_map of this step's map (Sec. 2.3.2), read back to decide
      double e = 0.0;
      vm_status st = emap_now(s, &e);
      if (st != VM_OK) return st;
      if (e > s->cfg.emap_remap) {
        remap = true;
        s->emap_remaps++;
      }
    }
    if (remap) {
      vm_status st = remap_internal(s);
      if (st != VM_OK) return st;
    }
  }
  return check_launch(s);
}

vm_status vm_remap(vm_solver* s) {
  if (!s) return VM_E_INVALID_ARG;
  vm::clear_foreign_error();
  if (!s->have_f) return VM_E_STATE;
  return remap_internal(s);
}

vm_status vm_density_force(vm_solver* s, double* M, double* a, double* da, double* d2a, int32_t on_device) {
  if (!s) return VM_E_INVALID_ARG;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t b = (size_t)s->g.nx * 8;
  if (M) VM_CUDA_TRY(cudaMemcpyAsync(M, s->M, b, kind, s->stream));
  if (a) VM_CUDA_TRY(cudaMemcpyAsync(a, s->a, b, kind, s->stream));
  if (da) VM_CUDA_TRY(cudaMemcpyAsync(da, s->da, b, kind, s->stream));
  if (d2a) VM_CUDA_TRY(cudaMemcpyAsync(d2a, s->d2a, b, kind, s->stream));
  return on_device ? VM_OK : vm_sync(s);
}

vm_status vm_read_f(vm_solver* s, void* out, int32_t dtype, int32_t on_device) {
  if (!s) return VM_E_INVALID_ARG;
  return read_real(s, s->f, out, dtype, on_device);
}

vm_status vm_read_fini(vm_solver* s, void* out, int32_t dtype, int32_t on_device) {
  if (!s) return VM_E_INVALID_ARG;
  return read_real(s, s->fini, out, dtype, on_device);
}

vm_status vm_read_eta(vm_solver* s, void* out, int32_t dtype, int32_t on_device) {
  if (!s) return VM_E_INVALID_ARG;
  return read_real(s, s->eta, out, dtype, on_device);
}

vm_status vm_read_map(vm_solver* s, int32_t* out, int32_t on_device) {
  if (!s || !out) return VM_E_INVALID_ARG;
  if (on_device) {
    vm::launch_read_map(s, out);
    return check_launch(s);
  }
  vm::launch_read_map(s, (int32_t*)staging(s));
  VM_CUDA_TRY(cudaMemcpyAsync(out, staging(s), s->n * 4, cudaMemcpyDeviceToHost, s->stream));
  return vm_sync(s);
}

vm_status vm_sync(vm_solver* s) {
  if (!s) return VM_E_INVALID_ARG;
  int32_t err = 0;
  VM_CUDA_TRY(cudaMemcpyAsync(&err, &s->ds->err, sizeof err, cudaMemcpyDeviceToHost, s->stream));
  VM_CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (err) {
    VM_CUDA_TRY(cudaMemsetAsync(&s->ds->err, 0, sizeof(int32_t), s->stream));
    VM_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (err & vm::ERR_INTERNAL) return VM_E_INTERNAL;
    if (err & vm::ERR_PATCH_OVERFLOW) return VM_E_PATCH_OVERFLOW;
    if (err & vm::ERR_NOT_CONVERGED) return VM_E_NOT_CONVERGED;
    return VM_E_CUDA;
  }
  return VM_OK;
}

vm_status vm_diagnostics(vm_solver* s, vm_diag* d) {
  if (!s || !d) return VM_E_INVALID_ARG;
  // zero the accumulators: sum_mass, sum_kin, sum_pot, and the det keys
  vm::DevState h{};
  const size_t off = offsetof(vm::DevState, sum_mass), end = offsetof(vm::DevState, rect);
  h.det_min_key = ~0ull;
  h.det_max_key = 0ull;
  VM_CUDA_TRY(cudaMemcpyAsync((char*)s->ds + off, (char*)&h + off, end - off, cudaMemcpyHostToDevice, s->stream));
  vm::launch_diagnostics(s);
  vm::launch_emap(s);
  VM_CUDA_TRY(cudaMemcpyAsync(&h, s->ds, sizeof h, cudaMemcpyDeviceToHost, s->stream));
  vm_status st = vm_sync(s);
  if (st != VM_OK) return st;
  auto decode = [](unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    double d;
    memcpy(&d, &b, 8);
    return d;
  };
  d->mass = h.sum_mass;
  d->energy = h.sum_kin + (s->cfg.G != 0.0 ? -h.sum_pot / (8.0 * kPi * s->cfg.G) : 0.0);
  d->detT_min = decode(h.det_min_key);
  d->detT_max = decode(h.det_max_key);
  d->step = s->nstep;
  d->cycle = vm::device_cycle(s) ? h.cyc : s->cyc;
  d->holes = h.holes_found;
  d->hole_rounds = h.hole_rounds;
  d->overflow_elements = h.overflow_stat;
  d->tier1_more = h.t1_more;
  d->last_tier_elements = s->cfg.map_windows == 0 ? h.overflow3_stat : h.overflow_stat;
  d->exact_tests = h.n_exact;
  d->bad_where = h.bad_where;
  d->entropy = h.sum_ent;
  d->l1 = h.sum_l1;
  d->l2 = h.sum_l2;
  double e2;
  memcpy(&e2, &h.emap2_bits, 8);
  d->emap = sqrt(e2);
  d->emap_remaps = vm::device_cycle(s) ? (int64_t)h.emap_remaps : s->emap_remaps;
  d->time = s->time;
  d->last_dt = s->last_dt;
  d->lattice_range[0] = s->g.klo;
  d->lattice_range[1] = s->g.khi;
  d->lattice_range[2] = s->g.llo;
  d->lattice_range[3] = s->g.lhi;
  for (int q = 0; q < 4; q++) d->site_rect[q] = s->g.fth_on ? h.rect[q] : (q == 1 ? s->g.nx - 1 : (q == 3 ? s->g.nv - 1 : 0));
  return VM_OK;
}

int32_t vm_last_cuda_error(void) { return (int32_t)vm::t_last_cuda; }

const char* vm_cuda_error_name(int32_t code) { return cudaGetErrorName((cudaError_t)code); }

}  // extern "C"

// ---------------------------------------------------------------------------
// checkpoints
// ---------------------------------------------------------------------------

namespace {

constexpr char kCkMagic[8] = {'V', 'L', 'M', 'T', 'C', 'K', 'P', 'T'};
constexpr uint32_t kCkVersion = 3;

struct CkHeader {
  char magic[8];
  uint32_t version;
  int32_t nx, nv, elem_stride, precision, ne, have_f, cyc;
  int64_t nstep;
  uint64_t sreal;
  double x_lo, x_hi, v_lo, v_hi, dt, G, alpha, beta;
  double time, last_dt;  // Sec. 2.4: elapsed time and the last step (variable time steps)
  int64_t emap_remaps;
  double f_th;            // adaptive computing domain: threshold and existing lattice range
  int32_t lattice[4];
};

CkHeader ck_header(const vm_solver* s) {
  CkHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kCkMagic, sizeof kCkMagic);
  h.version = kCkVersion;
  h.nx = s->cfg.nx;
  h.nv = s->cfg.nv;
  h.elem_stride = s->cfg.elem_stride;
  h.precision = s->cfg.precision;
  h.ne = s->g.ne;
  h.have_f = s->have_f;
  h.cyc = s->cyc;
  h.nstep = s->nstep;
  h.sreal = s->sreal;
  h.x_lo = s->cfg.x_lo;
  h.x_hi = s->cfg.x_hi;
  h.v_lo = s->cfg.v_lo;
  h.v_hi = s->cfg.v_hi;
  h.dt = s->cfg.dt;
  h.G = s->cfg.G;
  h.alpha = s->g.alpha;
  h.beta = s->g.beta;
  h.time = s->time;
  h.last_dt = s->last_dt;
  h.emap_remaps = s->emap_remaps;
  h.f_th = s->cfg.f_th;
  h.lattice[0] = s->g.klo;
  h.lattice[1] = s->g.khi;
  h.lattice[2] = s->g.llo;
  h.lattice[3] = s->g.lhi;
  return h;
}

// The arrays of a checkpoint, in file order.
struct CkArray {
  void* dev;
  size_t bytes;
};

void ck_arrays(const vm_solver* s, CkArray (&a)[4]) {
  a[0] = {s->el, 12 * (size_t)s->g.ne * 8};
  a[1] = {s->fini, s->n * s->sreal};
  a[2] = {s->eta, s->n * s->sreal};
  a[3] = {s->f, s->n * s->sreal};
}

bool same_run(const CkHeader& a, const CkHeader& b) {
  return a.nx == b.nx && a.nv == b.nv && a.elem_stride == b.elem_stride && a.precision == b.precision &&
         a.ne == b.ne && a.sreal == b.sreal && a.x_lo == b.x_lo && a.x_hi == b.x_hi && a.v_lo == b.v_lo &&
         a.v_hi == b.v_hi && a.dt == b.dt && a.G == b.G && a.alpha == b.alpha && a.beta == b.beta &&
         a.f_th == b.f_th;
}

}  // namespace

vm_status vm_save(vm_solver* s, const char* path) {
  if (!s || !path) return VM_E_INVALID_ARG;
  if (!s->have_f) return VM_E_STATE;
  vm_status st = vm_sync(s);
  if (st != VM_OK) return st;
  VM_CUDA_TRY(vm::cycle_to_host(s));
  FILE* fp = fopen(path, "wb");
  if (!fp) return VM_E_IO;
  const CkHeader h = ck_header(s);
  bool ok = fwrite(&h, sizeof h, 1, fp) == 1;
  CkArray arr[4];
  ck_arrays(s, arr);
  std::vector<char> buf;
  for (int k = 0; k < 4 && ok; k++) {
    buf.resize(arr[k].bytes);
    cudaError_t e = cudaMemcpyAsync(buf.data(), arr[k].dev, arr[k].bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
      vm::note_cuda(e);
      fclose(fp);
      return VM_E_CUDA;
    }
    ok = fwrite(buf.data(), 1, arr[k].bytes, fp) == arr[k].bytes;
  }
  ok = (fclose(fp) == 0) && ok;
  return ok ? VM_OK : VM_E_IO;
}

vm_status vm_load(vm_solver* s, const char* path) {
  if (!s || !path) return VM_E_INVALID_ARG;
  vm_status st = vm_sync(s);
  if (st != VM_OK) return st;
  FILE* fp = fopen(path, "rb");
  if (!fp) return VM_E_IO;
  CkHeader h;
  if (fread(&h, sizeof h, 1, fp) != 1 || memcmp(h.magic, kCkMagic, sizeof kCkMagic) != 0 ||
      h.version != kCkVersion || !h.have_f) {
    fclose(fp);
    return VM_E_IO;
  }
  if (!same_run(h, ck_header(s))) {
    fclose(fp);
    return VM_E_INVALID_ARG;
  }
  CkArray arr[4];
  ck_arrays(s, arr);
  std::vector<char> buf;
  for (int k = 0; k < 4; k++) {
    buf.resize(arr[k].bytes);
    if (fread(buf.data(), 1, arr[k].bytes, fp) != arr[k].bytes) {
      fclose(fp);
      return VM_E_IO;
    }
    // (the host buffer is reused for the next array: each copy completes first)
    cudaError_t e = cudaMemcpyAsync(arr[k].dev, buf.data(), arr[k].bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
      vm::note_cuda(e);
      fclose(fp);
      return VM_E_CUDA;
    }
  }
  fclose(fp);
  s->have_f = 1;
  s->nstep = h.nstep;
  s->cyc = h.cyc;
  s->time = h.time;
  s->last_dt = h.last_dt;
  s->emap_remaps = h.emap_remaps;
  s->g.klo = h.lattice[0];
  s->g.khi = h.lattice[1];
  s->g.llo = h.lattice[2];
  s->g.lhi = h.lattice[3];
  VM_CUDA_TRY(vm::cycle_to_device(s));
  return VM_OK;
}
