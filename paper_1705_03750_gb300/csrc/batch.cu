// Batched stepping of many independent solves.
//
// A batch is a group of solves (group.cu): each phase of a step is one
// launch whose blocks walk the work list of every solve's units (rows,
// element chunks, escaped elements...), so a step of the whole batch is
// about twenty launches whatever the number of solves.  Those launches are
// recorded once into a CUDA graph (a transport step, and a transport step
// followed by a remap; every solve whose cycle the host keeps shares one
// remap phase), and a batch step is one graph launch.  Solves that remap on
// the E_map criterion keep their cycle on the device: every step of the
// graph ends with their E_map, each one's decision and their remap
// launches, which skip the solves that do not remap this step.  The number of persistent blocks of
// each phase can be tuned on the run's own steps (vm_batch_autotune): it
// changes no result, only the time.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "group.cuh"

struct vm_batch {
  std::vector<vm_solver*> solvers;
  std::vector<vm_solver*> hosts;   // cycle kept on the host (one shared remap phase)
  std::vector<vm_solver*> gated;   // cycle kept on the device (device_cycle)
  cudaStream_t capture = nullptr;  // capture stream (owned)
  cudaStream_t user = nullptr;     // stream the graphs are launched on
  cudaEvent_t sync = nullptr;
  void* d_table = nullptr;         // plan tables (device, owned): all, hosts, gated
  std::vector<char> h_table;       // their host staging copy
  vm::GroupPlan plan;              // every solve (transport); carries the launch shapes
  vm::GroupPlan plan_h, plan_g;    // remaps of the host-cycle / device-cycle solves
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // [0] transport step, [1] transport + remap
  int64_t launches_per[2] = {0, 0};
  int32_t n_s = 0;
  // launch-shape tuning: chosen blocks per SM and the time measured with it,
  // per timed phase (drift, map, reconstruction, scan, kick)
  int32_t tuned = 0;
  int32_t bps[5] = {0, 0, 0, 0, 0};
  double tuned_ms[5] = {0, 0, 0, 0, 0};
};

namespace {

void destroy_batch(vm_batch* b) {
  if (!b) return;
  for (int k = 0; k < 2; k++)
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
  if (b->sync) cudaEventDestroy(b->sync);
  if (b->capture) cudaStreamSynchronize(b->capture);
  if (b->d_table) cudaFree(b->d_table);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

// The three plans on `stream`, with the launch shapes of b->plan.
void plans_on(const vm_batch* b, cudaStream_t stream, vm::GroupPlan& P, vm::GroupPlan& Ph, vm::GroupPlan& Pg) {
  P = b->plan;
  Ph = b->plan_h;
  Pg = b->plan_g;
  P.stream = Ph.stream = Pg.stream = stream;
  memcpy(Ph.shape, P.shape, sizeof P.shape);
  memcpy(Pg.shape, P.shape, sizeof P.shape);
}

// Enqueue one step: transport of every solve, the gated remaps, and (remap)
// the host-cycle solves' remap.
void enqueue_step(const vm_batch* b, const vm::GroupPlan& P, const vm::GroupPlan& Ph, const vm::GroupPlan& Pg,
                  bool remap, const vm::GroupTiming* T = nullptr) {
  vm::group_step_transport(P, T);
  if (!b->gated.empty()) vm::group_step_gated(Pg);
  if (remap && !b->hosts.empty()) vm::group_step_remap(Ph);
}

// Whether the next step ends the host-cycle solves' remap cycle.
bool host_remap_next(const vm_batch* b) { return !b->hosts.empty() && b->hosts[0]->cyc + 1 >= b->n_s; }

// Record one step of the whole batch into a graph.
vm_status capture(vm_batch* b, bool remap, cudaGraphExec_t* out, int64_t* launches) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return VM_E_CUDA;
  vm::GroupPlan P, Ph, Pg;
  plans_on(b, b->capture, P, Ph, Pg);
  enqueue_step(b, P, Ph, Pg, remap);
  const cudaError_t e = cudaStreamEndCapture(b->capture, &graph);
  if (e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return VM_E_CUDA;
  }
  size_t nodes = 0;
  cudaGraphGetNodes(graph, nullptr, &nodes);
  const cudaError_t ie = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return VM_E_CUDA;
  *launches = (int64_t)nodes;
  return VM_OK;
}

// Phases of the plan that follow each timed phase's launch shape.
void set_shape(vm::GroupPlan& P, int timed, int blocks) {
  using namespace vm;
  static const int kCount[5] = {2, 8, 3, 4, 2};
  static const int kPhases[5][8] = {
      {GP_DRIFT, GP_TAYLOR},
      {GP_PAIR, GP_SMALL, GP_BIG1, GP_BIG2, GP_BIG3, GP_RESOLVE, GP_FIND_HOLES, GP_HOLES},
      {GP_RECON, GP_REMAP, GP_COPY},
      {GP_SCAN, GP_DIFF, GP_ROWS, GP_COLS},
      {GP_KICK, GP_RESET}};
  for (int q = 0; q < kCount[timed]; q++) P.shape[kPhases[timed][q]].blocks = blocks;
}

// Order the batch's stream after work queued on the solvers' own streams.
vm_status enter(vm_batch* b) {
  for (vm_solver* s : b->solvers)
    if (cudaEventRecord(b->sync, s->stream) != cudaSuccess || cudaStreamWaitEvent(b->user, b->sync, 0) != cudaSuccess)
      return VM_E_CUDA;
  return VM_OK;
}

// Later calls on a solver's own stream see the batch's results.
vm_status leave(vm_batch* b) {
  if (cudaEventRecord(b->sync, b->user) != cudaSuccess) return VM_E_CUDA;
  for (vm_solver* s : b->solvers)
    if (cudaStreamWaitEvent(s->stream, b->sync, 0) != cudaSuccess) return VM_E_CUDA;
  return VM_OK;
}

void count(vm_batch* b, int kind) {
  for (vm_solver* s : b->solvers) {
    vm::group_count_step(s, kind == 1);
    s->launches += b->launches_per[kind] / (int64_t)b->solvers.size();
  }
}

}  // namespace

extern "C" vm_status vm_batch_create(vm_solver* const* solvers, int32_t n, int32_t nstreams, void* cuda_stream,
                                     vm_batch** out) {
  if (!out || !solvers || n < 1 || nstreams < 0) return VM_E_INVALID_ARG;
  *out = nullptr;
  vm::clear_foreign_error();
  vm_status st = vm::group_check(solvers, n);
  if (st != VM_OK) return st;
  std::vector<vm_solver*> hosts, gated;
  for (int32_t i = 0; i < n; i++) {
    if (solvers[i]->prof) return VM_E_STATE;
    (vm::device_cycle(solvers[i]) ? gated : hosts).push_back(solvers[i]);
  }
  const int32_t n_s = hosts.empty() ? 0 : hosts[0]->cfg.n_s, cyc = hosts.empty() ? 0 : hosts[0]->cyc;
  for (vm_solver* s : hosts)
    if (s->cfg.n_s != n_s || s->cyc != cyc) return VM_E_STATE;  // one remap phase for the host-cycle solves
  if (!vm::group_map_prepare()) return VM_E_CUDA;
  vm_batch* b = new vm_batch();
  b->solvers.assign(solvers, solvers + n);
  b->hosts = hosts;
  b->gated = gated;
  b->user = (cudaStream_t)cuda_stream;
  b->n_s = n_s;
  auto seg = [](int k) { return (vm::group_table_bytes(k) + 255) / 256 * 256; };
  const size_t t0 = seg(n), t1 = seg((int)hosts.size()), t2 = seg((int)gated.size());
  b->h_table.assign(t0 + t1 + t2, 0);
  if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->sync, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(&b->d_table, t0 + t1 + t2) != cudaSuccess)
    st = VM_E_CUDA;
  if (st == VM_OK) {
    char* d = (char*)b->d_table;
    char* h = b->h_table.data();
    vm::group_plan(b->plan, solvers, n, d, h, b->capture);
    if (!hosts.empty())
      vm::group_plan(b->plan_h, hosts.data(), (int)hosts.size(), d + t0, h + t0, b->capture);
    if (!gated.empty())
      vm::group_plan(b->plan_g, gated.data(), (int)gated.size(), d + t0 + t1, h + t0 + t1, b->capture, true);
    if (cudaStreamSynchronize(b->capture) != cudaSuccess) st = VM_E_CUDA;
  }
  // pending work of the solvers is done before the first replay
  for (int32_t i = 0; st == VM_OK && i < n; i++)
    if (cudaStreamSynchronize(solvers[i]->stream) != cudaSuccess) st = VM_E_CUDA;
  if (st == VM_OK) st = capture(b, false, &b->exec[0], &b->launches_per[0]);
  if (st == VM_OK) st = capture(b, true, &b->exec[1], &b->launches_per[1]);
  if (st != VM_OK) {
    destroy_batch(b);
    return st;
  }
  *out = b;
  return VM_OK;
}

extern "C" vm_status vm_batch_step(vm_batch* b, int32_t nsteps) {
  if (!b || nsteps < 0) return VM_E_INVALID_ARG;
  vm::clear_foreign_error();
  vm_status st = enter(b);
  if (st != VM_OK) return st;
  for (int32_t it = 0; it < nsteps; it++) {
    const int kind = host_remap_next(b) ? 1 : 0;
    if (cudaGraphLaunch(b->exec[kind], b->user) != cudaSuccess) return VM_E_CUDA;
    count(b, kind);
  }
  return leave(b);
}

extern "C" vm_status vm_batch_autotune(vm_batch* b, int32_t trials) {
  if (!b || trials < 1) return VM_E_INVALID_ARG;
  vm::clear_foreign_error();
  vm_status st = enter(b);
  if (st != VM_OK) return st;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  static const int kCand[4] = {1, 2, 4, 8};
  double best[5];
  int pick[5];
  for (int t = 0; t < 5; t++) {
    best[t] = 1e30;
    pick[t] = 4;
  }
  vm::GroupTiming T;
  for (int e = 0; e < vm::GT_N; e++)
    if (cudaEventCreate(&T.ev[e]) != cudaSuccess) return VM_E_CUDA;
  vm::GroupPlan P, Ph, Pg;
  plans_on(b, b->user, P, Ph, Pg);
  for (int c = 0; c < 4 && st == VM_OK; c++) {
    for (int t = 0; t < 5; t++) set_shape(P, t, kCand[c] * sms);
    memcpy(Pg.shape, P.shape, sizeof P.shape);
    double acc[5] = {0, 0, 0, 0, 0};
    int timed = 0;
    while (timed < trials && st == VM_OK) {
      // the step before a host-cycle remap runs with the remap (untimed)
      if (host_remap_next(b)) {
        if (cudaGraphLaunch(b->exec[1], b->user) != cudaSuccess) st = VM_E_CUDA;
        count(b, 1);
        continue;
      }
      // the transport phases timed; the gated remaps follow untimed
      enqueue_step(b, P, Ph, Pg, false, &T);
      if (cudaEventSynchronize(T.ev[vm::GT_END]) != cudaSuccess) st = VM_E_CUDA;
      for (int t = 0; t < 5 && st == VM_OK; t++) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, T.ev[t], T.ev[t + 1]);
        acc[t] += ms;
      }
      count(b, 0);
      timed++;
    }
    for (int t = 0; t < 5; t++)
      if (acc[t] < best[t]) {
        best[t] = acc[t];
        pick[t] = kCand[c];
      }
  }
  for (int e = 0; e < vm::GT_N; e++) cudaEventDestroy(T.ev[e]);
  if (st != VM_OK) return st;
  for (int t = 0; t < 5; t++) {
    set_shape(b->plan, t, pick[t] * sms);
    b->bps[t] = pick[t];
    b->tuned_ms[t] = best[t] / trials;
  }
  b->tuned = 1;
  if (cudaStreamSynchronize(b->user) != cudaSuccess) return VM_E_CUDA;
  st = capture(b, false, &b->exec[0], &b->launches_per[0]);
  if (st == VM_OK) st = capture(b, true, &b->exec[1], &b->launches_per[1]);
  if (st != VM_OK) return st;
  return leave(b);
}

extern "C" int32_t vm_batch_tuning(const vm_batch* b, int32_t* blocks_per_sm, double* ms) {
  if (!b) return -1;
  for (int t = 0; t < 5; t++) {
    if (blocks_per_sm) blocks_per_sm[t] = b->bps[t];
    if (ms) ms[t] = b->tuned_ms[t];
  }
  return b->tuned;
}

extern "C" int64_t vm_batch_launches_per_step(const vm_batch* b, int32_t with_remap) {
  return b ? b->launches_per[with_remap ? 1 : 0] : 0;
}

extern "C" void vm_batch_destroy(vm_batch* b) { destroy_batch(b); }
