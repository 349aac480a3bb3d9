// Host side of the group launches (group.cu), shared by the batch and the
// serving loop.
#pragma once

#include "common.cuh"

namespace vm {

// Phases timed by the launch-shape tuner (events before each, and at the end).
enum { GT_DRIFT = 0, GT_MAP, GT_RECON, GT_SCAN, GT_KICK, GT_END, GT_N };
struct GroupTiming {
  cudaEvent_t ev[GT_N];
};

// Device bytes of the plan table of ns solves (also the host staging size).
size_t group_table_bytes(int ns);
// Solvers that may form a group: same precision, no per-step host decisions.
vm_status group_check(vm_solver* const* solvers, int n);
// Plan of solvers[0..n) in the device table (asynchronous upload on stream);
// gated: a plan of remaps decided on the device (device_cycle solves).
void group_plan(GroupPlan& P, vm_solver* const* solvers, int n, void* d_table, void* host, cudaStream_t stream,
                bool gated = false);
// One transport step / one remap of every solve of the plan (enqueue only);
// a gated plan's remaps after a transport step, each behind its solve's own
// decision (E_map criterion and cycle, Sec. 2.3.2).
void group_step_transport(const GroupPlan& P, const GroupTiming* T = nullptr);
void group_step_remap(const GroupPlan& P);
void group_step_gated(const GroupPlan& P);
void group_count_step(vm_solver* s, bool remapped);

}  // namespace vm
