// Serving solves with continuous batching, in the library.
//
// Requests (a grid, an initial condition, a number of steps) are submitted at
// any time; the server admits them first come, first served, as soon as a
// slot and enough of its device pool are free (each solve's exact workspace,
// first-fit with coalescing), keeps every admitted solve's state resident,
// and advances ALL active solves together: every step of a tick is one group
// step (group.cu: one launch per phase for the whole active set, the remaps
// of the solves whose cycle ends in one more group, and the solves that remap
// on the E_map criterion behind their own device decisions in a third), so
// requests that arrive
// while others run join the next step's launches.  A solve that has taken
// all its steps has its pixel masses and force copied to pinned host memory
// behind an event; the poll that finds the event complete hands the result
// over and frees the solve's slot and memory for the next request.  The host
// never waits for the device except to keep at most two ticks in flight.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <vector>

#include "common.cuh"
#include "group.cuh"

namespace {

constexpr int kInFlight = 2;     // ticks queued ahead of the device
constexpr int kTableSlots = 16;  // plan tables in the pool
// of them, two (alternating) for the transport plan, two for the gated plan,
// and the rest a ring for the host-cycle remaps
constexpr int kPlanSlots = 4;

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// First-fit allocator over [0, size) of the caller's pool, 256-byte units,
// adjacent free blocks merged.
struct PoolAlloc {
  std::map<size_t, size_t> free_;  // offset -> length
  size_t size = 0, used = 0, peak = 0;
  void init(size_t base, size_t n) {
    size = n;
    free_.clear();
    if (n > base) free_[base] = n - base;
  }
  bool take(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used += bytes;
      if (used > peak) peak = used;
      return true;
    }
    return false;
  }
  void give(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    used -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct Req {
  int64_t id = 0;
  vm_config cfg;
  int32_t steps = 0, left = 0;
  double* pinned = nullptr;  // f0 at submission, the result at completion
  size_t pinned_cap = 0;
  vm_solver* s = nullptr;
  size_t ws_off = 0, ws_bytes = 0;
  cudaEvent_t done_ev = nullptr;
  int32_t status = VM_OK;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  std::vector<double> result;  // M, a, da, d2a
  bool finished = false, reported = false;
};

}  // namespace

struct vm_server {
  vm_server_config c;
  char* pool = nullptr;
  size_t pool_bytes = 0;
  cudaStream_t stream = nullptr;
  PoolAlloc alloc;
  // plan tables: device slots, each with its pinned staging copy and an event
  // after its last use; slots 0-1 hold the transport plan of the stepping
  // set and 2-3 the gated plan of its device-cycle solves (each pair
  // alternating, so that a rebuild never overwrites a table queued steps
  // still read), slots 4.. a ring for the host-cycle remap subsets
  size_t table_bytes = 0;
  char* h_tables = nullptr;
  cudaEvent_t table_ev[kTableSlots];
  int table_next = kPlanSlots;
  int plan_slot = 0, gated_slot = 0;
  cudaEvent_t tick_ev[kInFlight];
  int tick_next = 0, ticks_queued = 0;
  // the plans of the current stepping set (rebuilt when the set changes):
  // transport of all, gated remaps of the device-cycle solves (if any)
  vm::GroupPlan plan, plan_g;
  bool have_gated = false;
  std::vector<vm_solver*> plan_set;
  bool plan_valid = false;
  std::deque<Req*> waiting;
  std::vector<Req*> active;
  std::map<int64_t, Req*> all;
  std::vector<std::pair<size_t, double*>> pinned_free;  // reusable pinned buffers (capacity, pointer)
  int64_t next_id = 1;
  int64_t ticks = 0, group_steps = 0, remap_groups = 0;
  int32_t peak_active = 0;
  std::chrono::steady_clock::time_point t0;
};

namespace {

double* pinned_get(vm_server* S, size_t n, size_t* cap) {
  for (size_t k = 0; k < S->pinned_free.size(); k++)
    if (S->pinned_free[k].first >= n) {
      double* p = S->pinned_free[k].second;
      *cap = S->pinned_free[k].first;
      S->pinned_free.erase(S->pinned_free.begin() + (long)k);
      return p;
    }
  void* p = nullptr;
  if (cudaHostAlloc(&p, n * sizeof(double), cudaHostAllocDefault) != cudaSuccess) return nullptr;
  *cap = n;
  return (double*)p;
}

void pinned_put(vm_server* S, double* p, size_t cap) {
  if (p) S->pinned_free.emplace_back(cap, p);
}

enum PlanKind { PK_TRANSPORT, PK_GATED, PK_REMAP };

// A plan-table slot whose last use has completed: the other slot of the
// transport or gated pair, or the next slot of the remap ring.
int table_slot(vm_server* S, PlanKind kind) {
  int k;
  if (kind == PK_TRANSPORT) {
    k = S->plan_slot = (S->plan_slot + 1) % 2;
  } else if (kind == PK_GATED) {
    k = 2 + (S->gated_slot = (S->gated_slot + 1) % 2);
  } else {
    k = S->table_next;
    S->table_next = (k + 1 - kPlanSlots) % (kTableSlots - kPlanSlots) + kPlanSlots;
  }
  cudaEventSynchronize(S->table_ev[k]);
  return k;
}

void plan_into_slot(vm_server* S, vm::GroupPlan& P, const std::vector<vm_solver*>& set, PlanKind kind) {
  const int k = table_slot(S, kind);
  vm::group_plan(P, set.data(), (int)set.size(), S->pool + (size_t)k * S->table_bytes,
                 S->h_tables + (size_t)k * S->table_bytes, S->stream, kind == PK_GATED);
  cudaEventRecord(S->table_ev[k], S->stream);  // re-recorded after the plan's last use
  P.big_blocks_cap = 0;
}

void mark_slot_used(vm_server* S, const vm::GroupPlan& P) {
  const size_t k = (size_t)((const char*)P.D - S->pool) / S->table_bytes;
  if (k < (size_t)kTableSlots) cudaEventRecord(S->table_ev[k], S->stream);
}

// Results of solves whose completion event has passed; slots and memory back.
int retire(vm_server* S) {
  int n = 0;
  std::vector<Req*> keep;
  for (Req* r : S->active) {
    if (r->left == 0 && r->done_ev && cudaEventQuery(r->done_ev) == cudaSuccess) {
      const size_t nx = (size_t)r->cfg.nx;
      r->result.assign(r->pinned, r->pinned + 4 * nx);
      int32_t err = 0;
      memcpy(&err, r->pinned + 4 * nx, sizeof err);
      if (err & vm::ERR_INTERNAL)
        r->status = VM_E_INTERNAL;
      else if (err & vm::ERR_PATCH_OVERFLOW)
        r->status = VM_E_PATCH_OVERFLOW;
      else if (err & vm::ERR_NOT_CONVERGED)
        r->status = VM_E_NOT_CONVERGED;
      r->t_finish = now_s(S->t0);
      r->finished = true;
      pinned_put(S, r->pinned, r->pinned_cap);
      r->pinned = nullptr;
      free(r->s);  // host struct only: its work is complete (the event)
      r->s = nullptr;
      S->alloc.give(r->ws_off, r->ws_bytes);
      cudaEventDestroy(r->done_ev);
      r->done_ev = nullptr;
      n++;
    } else {
      keep.push_back(r);
    }
  }
  if (n) S->plan_valid = false;
  S->active.swap(keep);
  return n;
}

void admit(vm_server* S) {
  while (!S->waiting.empty() && (int32_t)S->active.size() < S->c.max_active) {
    Req* r = S->waiting.front();
    size_t off = 0;
    if (!S->alloc.take(r->ws_bytes, &off)) break;  // first come, first served: no overtaking
    S->waiting.pop_front();
    r->ws_off = off;
    r->t_admit = now_s(S->t0);
    vm_status st = vm::solver_create(&r->cfg, S->pool + off, r->ws_bytes, S->stream, false, &r->s);
    if (st == VM_OK) {
      // f0 from the request's pinned buffer through the solver's staging area
      void* stg = r->s->holes_b;
      const size_t bytes = (size_t)r->cfg.nx * r->cfg.nv * sizeof(double);
      if (cudaMemcpyAsync(stg, r->pinned, bytes, cudaMemcpyHostToDevice, S->stream) != cudaSuccess) st = VM_E_CUDA;
      if (st == VM_OK) st = vm_set_f(r->s, (const double*)stg, 1);
    }
    if (st == VM_OK && cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming) != cudaSuccess) st = VM_E_CUDA;
    if (st != VM_OK) {
      r->status = st;
      r->finished = true;
      r->t_finish = now_s(S->t0);
      if (r->s) {
        cudaStreamSynchronize(S->stream);
        free(r->s);
        r->s = nullptr;
      }
      S->alloc.give(off, r->ws_bytes);
      pinned_put(S, r->pinned, r->pinned_cap);
      r->pinned = nullptr;
      continue;
    }
    S->active.push_back(r);
    S->plan_valid = false;
  }
  if ((int32_t)S->active.size() > S->peak_active) S->peak_active = (int32_t)S->active.size();
}

// One tick: steps_per_tick group steps of the active solves with steps left.
vm_status tick(vm_server* S) {
  for (int k = 0; k < S->c.steps_per_tick; k++) {
    std::vector<vm_solver*> set;
    std::vector<Req*> reqs;
    for (Req* r : S->active)
      if (r->left > 0) {
        set.push_back(r->s);
        reqs.push_back(r);
      }
    if (set.empty()) break;
    if (!S->plan_valid || set != S->plan_set) {
      plan_into_slot(S, S->plan, set, PK_TRANSPORT);
      std::vector<vm_solver*> gated;
      for (vm_solver* s : set)
        if (vm::device_cycle(s)) gated.push_back(s);
      S->have_gated = !gated.empty();
      if (S->have_gated) plan_into_slot(S, S->plan_g, gated, PK_GATED);
      S->plan_set = set;
      S->plan_valid = true;
    }
    vm::group_step_transport(S->plan);
    mark_slot_used(S, S->plan);
    if (S->have_gated) {
      vm::group_step_gated(S->plan_g);
      mark_slot_used(S, S->plan_g);
    }
    S->group_steps++;
    std::vector<vm_solver*> remap;
    for (Req* r : reqs) {
      vm_solver* s = r->s;
      s->nstep++;
      s->time += s->g.dt;
      s->last_dt = s->g.dt;
      if (vm::device_cycle(s)) continue;  // its cycle and remaps are on the device
      s->cyc++;
      if (s->cyc >= s->cfg.n_s) remap.push_back(s);
    }
    if (!remap.empty()) {
      vm::GroupPlan R;
      plan_into_slot(S, R, remap, PK_REMAP);
      vm::group_step_remap(R);
      mark_slot_used(S, R);
      S->remap_groups++;
      for (vm_solver* s : remap) s->cyc = 0;
    }
    for (Req* r : reqs) {
      if (--r->left > 0) continue;
      // the last step: pixel masses and force to the pinned buffer, then the event
      const size_t b = (size_t)r->cfg.nx * sizeof(double);
      double* h = r->pinned;
      cudaMemcpyAsync(h, r->s->M, b, cudaMemcpyDeviceToHost, S->stream);
      cudaMemcpyAsync(h + r->cfg.nx, r->s->a, b, cudaMemcpyDeviceToHost, S->stream);
      cudaMemcpyAsync(h + 2 * r->cfg.nx, r->s->da, b, cudaMemcpyDeviceToHost, S->stream);
      cudaMemcpyAsync(h + 3 * r->cfg.nx, r->s->d2a, b, cudaMemcpyDeviceToHost, S->stream);
      // and the solve's device error word (a map that did not converge, a failed bounds check)
      cudaMemcpyAsync(h + 4 * r->cfg.nx, &r->s->ds->err, sizeof(int32_t), cudaMemcpyDeviceToHost, S->stream);
      cudaEventRecord(r->done_ev, S->stream);
    }
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    vm::note_cuda(e);
    return VM_E_CUDA;
  }
  return VM_OK;
}

}  // namespace

extern "C" {

size_t vm_server_pool_bytes(const vm_server_config* c) {
  if (!c || c->max_active < 1) return 0;
  return (size_t)kTableSlots * ((vm::group_table_bytes(c->max_active) + 255) & ~size_t(255));
}

vm_status vm_server_create(const vm_server_config* c, void* d_pool, size_t pool_bytes, void* cuda_stream,
                           vm_server** out) {
  if (!out || !c || !d_pool || ((uintptr_t)d_pool & 255) || c->max_active < 1 || c->steps_per_tick < 1)
    return VM_E_INVALID_ARG;
  if (c->precision != VM_FP64 && c->precision != VM_FP32_MIXED) return VM_E_INVALID_ARG;
  *out = nullptr;
  const size_t reserve = vm_server_pool_bytes(c);
  if (pool_bytes <= reserve) return VM_E_OOM;
  if (!vm::group_map_prepare()) return VM_E_CUDA;
  vm_server* S = new vm_server();
  S->c = *c;
  S->pool = (char*)d_pool;
  S->pool_bytes = pool_bytes;
  S->stream = (cudaStream_t)cuda_stream;
  S->table_bytes = reserve / kTableSlots;
  S->alloc.init(reserve, std::min(pool_bytes, reserve + c->budget_bytes));
  S->t0 = std::chrono::steady_clock::now();
  void* h = nullptr;
  bool ok = cudaHostAlloc(&h, reserve, cudaHostAllocDefault) == cudaSuccess;
  S->h_tables = (char*)h;
  for (int k = 0; ok && k < kTableSlots; k++) {
    ok = cudaEventCreateWithFlags(&S->table_ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (ok) cudaEventRecord(S->table_ev[k], S->stream);
  }
  for (int k = 0; ok && k < kInFlight; k++) {
    ok = cudaEventCreateWithFlags(&S->tick_ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (ok) cudaEventRecord(S->tick_ev[k], S->stream);
  }
  if (!ok) {
    vm_server_destroy(S);
    return VM_E_CUDA;
  }
  *out = S;
  return VM_OK;
}

vm_status vm_server_submit(vm_server* S, const vm_config* cfg, const double* f0, int32_t nsteps, int64_t* id) {
  if (!S || !cfg || !f0 || !id || nsteps < 1) return VM_E_INVALID_ARG;
  if (cfg->precision != S->c.precision) return VM_E_INVALID_ARG;
  if (cfg->c_dyn > 0.0 || cfg->f_th > 0.0) return VM_E_INVALID_ARG;
  const size_t need = vm_workspace_bytes(cfg);
  if (need == 0) return VM_E_INVALID_ARG;
  if (((need + 255) & ~size_t(255)) > S->alloc.size - vm_server_pool_bytes(&S->c)) return VM_E_BUDGET;
  Req* r = new Req();
  r->id = S->next_id++;
  r->cfg = *cfg;
  r->steps = r->left = nsteps;
  r->ws_bytes = need;
  const size_t n = (size_t)cfg->nx * cfg->nv;
  // f0 at submission; at completion M, a, a', a'' and the error word
  r->pinned = pinned_get(S, std::max(n, 4 * (size_t)cfg->nx + 1), &r->pinned_cap);
  if (!r->pinned) {
    delete r;
    return VM_E_OOM;
  }
  memcpy(r->pinned, f0, n * sizeof(double));
  r->t_submit = now_s(S->t0);
  S->waiting.push_back(r);
  S->all[r->id] = r;
  *id = r->id;
  return VM_OK;
}

vm_status vm_server_poll(vm_server* S, vm_server_done* done, int32_t max_done, int32_t* n_done) {
  if (!S || (max_done > 0 && !done)) return VM_E_INVALID_ARG;
  vm::clear_foreign_error();
  retire(S);
  admit(S);
  // keep at most kInFlight ticks queued: wait (without blocking) for the oldest
  const int slot = S->tick_next;
  vm_status st = VM_OK;
  if (cudaEventQuery(S->tick_ev[slot]) == cudaSuccess) {
    st = tick(S);
    cudaEventRecord(S->tick_ev[slot], S->stream);
    S->tick_next = (slot + 1) % kInFlight;
    S->ticks++;
  }
  int32_t k = 0;
  for (auto& kv : S->all) {
    Req* r = kv.second;
    if (!r->finished || r->reported || k >= max_done) continue;
    done[k].id = r->id;
    done[k].status = r->status;
    done[k].submit_s = r->t_submit;
    done[k].admit_s = r->t_admit;
    done[k].finish_s = r->t_finish;
    r->reported = true;
    k++;
  }
  if (n_done) *n_done = k;
  return st;
}

vm_status vm_server_result(vm_server* S, int64_t id, double* M, double* a, double* da, double* d2a) {
  if (!S) return VM_E_INVALID_ARG;
  auto it = S->all.find(id);
  if (it == S->all.end()) return VM_E_INVALID_ARG;
  Req* r = it->second;
  if (!r->finished) return VM_E_STATE;
  if (r->status != VM_OK) return (vm_status)r->status;
  const size_t nx = (size_t)r->cfg.nx;
  double* outs[4] = {M, a, da, d2a};
  for (int q = 0; q < 4; q++)
    if (outs[q]) memcpy(outs[q], r->result.data() + q * nx, nx * sizeof(double));
  return VM_OK;
}

vm_status vm_server_stats(const vm_server* S, vm_server_stat* st) {
  if (!S || !st) return VM_E_INVALID_ARG;
  memset(st, 0, sizeof *st);
  st->waiting = (int32_t)S->waiting.size();
  st->active = (int32_t)S->active.size();
  int32_t fin = 0;
  for (auto& kv : S->all) fin += kv.second->finished ? 1 : 0;
  st->finished = fin;
  st->peak_active = S->peak_active;
  st->used_bytes = (int64_t)S->alloc.used;
  st->peak_bytes = (int64_t)S->alloc.peak;
  st->ticks = S->ticks;
  st->group_steps = S->group_steps;
  st->remap_groups = S->remap_groups;
  return VM_OK;
}

void vm_server_destroy(vm_server* S) {
  if (!S) return;
  cudaStreamSynchronize(S->stream);
  for (auto& kv : S->all) {
    Req* r = kv.second;
    if (r->s) free(r->s);
    if (r->done_ev) cudaEventDestroy(r->done_ev);
    if (r->pinned) cudaFreeHost(r->pinned);
    delete r;
  }
  for (auto& pf : S->pinned_free) cudaFreeHost(pf.second);
  for (int k = 0; k < kTableSlots; k++)
    if (S->table_ev[k]) cudaEventDestroy(S->table_ev[k]);
  for (int k = 0; k < kInFlight; k++)
    if (S->tick_ev[k]) cudaEventDestroy(S->tick_ev[k]);
  if (S->h_tables) cudaFreeHost(S->h_tables);
  delete S;
}

}  // extern "C"
