// Batched stepping of many independent solves.
//
// One time step of every solve in the batch is recorded once into a CUDA
// graph (stream capture): the solves are spread over K streams forked from
// and joined back to one capture stream, so kernels of different solves run
// concurrently, and a step of the whole batch is then a single graph launch.
// Two graphs are kept: a transport step, and a transport step followed by a
// remap; every solve of a batch shares its remap phase.  Replays are exact
// repetitions of the same launches: all per-step state (element state, the
// map epoch, the remap copy) lives on the device.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "common.cuh"

struct vm_batch {
  std::vector<vm_solver*> solvers;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork;
  cudaStream_t capture;     // capture stream (owned)
  cudaStream_t user;        // stream the graphs are launched on
  cudaGraphExec_t exec[2];  // [0] transport step, [1] transport + remap
  int64_t launches_per[2];
  int32_t n_s;
};

namespace {

void destroy_batch(vm_batch* b) {
  if (!b) return;
  for (int k = 0; k < 2; k++)
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
  for (auto e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto st : b->streams) cudaStreamDestroy(st);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

// Record one step of every solve into a graph.
vm_status capture(vm_batch* b, bool remap, cudaGraphExec_t* out, int64_t* launches) {
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return VM_E_CUDA;
  bool ok = cudaEventRecord(b->fork, b->capture) == cudaSuccess;
  for (auto st : b->streams) ok = ok && cudaStreamWaitEvent(st, b->fork, 0) == cudaSuccess;
  int64_t count = 0;
  for (size_t i = 0; ok && i < b->solvers.size(); i++) {
    vm_solver* s = b->solvers[i];
    const cudaStream_t saved = s->stream;
    const int32_t saved_prof = s->prof;
    const int64_t l0 = s->launches;
    s->stream = b->streams[i % b->streams.size()];
    s->prof = 0;
    vm::step_transport(s);
    if (remap) ok = vm::step_remap(s) == cudaSuccess;
    count += s->launches - l0;
    s->launches = l0;
    s->stream = saved;
    s->prof = saved_prof;
  }
  for (size_t k = 0; ok && k < b->streams.size(); k++) {
    ok = cudaEventRecord(b->joins[k], b->streams[k]) == cudaSuccess &&
         cudaStreamWaitEvent(b->capture, b->joins[k], 0) == cudaSuccess;
  }
  const cudaError_t e = cudaStreamEndCapture(b->capture, &graph);
  if (!ok || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return VM_E_CUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return VM_E_CUDA;
  *launches = count;
  return VM_OK;
}

}  // namespace

extern "C" vm_status vm_batch_create(vm_solver* const* solvers, int32_t n, int32_t nstreams, void* cuda_stream,
                                     vm_batch** out) {
  if (!out || !solvers || n < 1 || nstreams < 1) return VM_E_INVALID_ARG;
  *out = nullptr;
  const int32_t n_s = solvers[0] ? solvers[0]->cfg.n_s : 0;
  const int32_t cyc = solvers[0] ? solvers[0]->cyc : 0;
  for (int32_t i = 0; i < n; i++) {
    const vm_solver* s = solvers[i];
    if (!s) return VM_E_INVALID_ARG;
    if (!s->have_f || s->prof) return VM_E_STATE;
    if (s->cfg.n_s != n_s || s->cyc != cyc) return VM_E_STATE;  // one remap phase per batch
    // host decisions per step or per remap: not capturable
    if (s->cfg.emap_remap > 0.0 || s->cfg.c_dyn > 0.0 || s->cfg.f_th > 0.0) return VM_E_INVALID_ARG;
    for (int32_t j = 0; j < i; j++)
      if (solvers[j] == s) return VM_E_INVALID_ARG;
  }
  vm_batch* b = new vm_batch();
  memset(b->exec, 0, sizeof b->exec);
  b->fork = nullptr;
  b->capture = nullptr;
  b->solvers.assign(solvers, solvers + n);
  b->user = (cudaStream_t)cuda_stream;
  b->n_s = n_s;
  if (nstreams > n) nstreams = n;
  vm_status st = VM_OK;
  if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    st = VM_E_CUDA;
  for (int32_t k = 0; st == VM_OK && k < nstreams; k++) {
    cudaStream_t sk;
    cudaEvent_t ek;
    if (cudaStreamCreateWithFlags(&sk, cudaStreamNonBlocking) != cudaSuccess) {
      st = VM_E_CUDA;
      break;
    }
    b->streams.push_back(sk);
    if (cudaEventCreateWithFlags(&ek, cudaEventDisableTiming) != cudaSuccess) {
      st = VM_E_CUDA;
      break;
    }
    b->joins.push_back(ek);
  }
  // pending work of the solvers is done before the capture's first replay
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
  // order after any work the caller queued on the solvers' own streams
  for (vm_solver* s : b->solvers) {
    if (cudaEventRecord(b->fork, s->stream) != cudaSuccess || cudaStreamWaitEvent(b->user, b->fork, 0) != cudaSuccess)
      return VM_E_CUDA;
  }
  for (int32_t it = 0; it < nsteps; it++) {
    const vm_solver* s0 = b->solvers[0];
    const int kind = (s0->cyc + 1 >= b->n_s) ? 1 : 0;
    if (cudaGraphLaunch(b->exec[kind], b->user) != cudaSuccess) return VM_E_CUDA;
    for (vm_solver* s : b->solvers) {
      s->nstep++;
      s->cyc = kind ? 0 : s->cyc + 1;
      s->launches += b->launches_per[kind] / (int64_t)b->solvers.size();
    }
  }
  // later calls on a solver's own stream see the batch's results
  if (cudaEventRecord(b->fork, b->user) != cudaSuccess) return VM_E_CUDA;
  for (vm_solver* s : b->solvers)
    if (cudaStreamWaitEvent(s->stream, b->fork, 0) != cudaSuccess) return VM_E_CUDA;
  return VM_OK;
}

extern "C" int64_t vm_batch_launches_per_step(const vm_batch* b, int32_t with_remap) {
  return b ? b->launches_per[with_remap ? 1 : 0] : 0;
}

extern "C" void vm_batch_destroy(vm_batch* b) { destroy_batch(b); }
