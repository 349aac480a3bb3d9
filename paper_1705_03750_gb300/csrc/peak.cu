// Measured FP64 arithmetic peak of the current device (the denominator of
// the FP64 path's arithmetic roofline).  Every thread runs eight independent
// chains of fused multiply-adds for `iters` rounds; the grid fills every SM
// several times over.  The result is the FLOP count (2 per FMA) over the
// CUDA-event time of the launch.
#include "common.cuh"

namespace {

__global__ void __launch_bounds__(256) k_fma64(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; k++) s += x[k];
  if (s == 12345.678) out[0] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" vm_status vm_measure_fp64_peak(int32_t iters, void* cuda_stream, double* flops_per_s) {
  if (!flops_per_s || iters < 1) return VM_E_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  VM_CUDA_TRY(cudaGetDevice(&dev));
  VM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  VM_CUDA_TRY(cudaEventCreate(&e0));
  VM_CUDA_TRY(cudaEventCreate(&e1));
  k_fma64<<<blocks, threads, 0, st>>>(nullptr, iters / 8 + 1, 0.999999, 1e-9);  // warm-up
  cudaEventRecord(e0, st);
  k_fma64<<<blocks, threads, 0, st>>>(nullptr, iters, 0.999999, 1e-9);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    vm::note_cuda(e);
    return VM_E_CUDA;
  }
  *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return VM_OK;
}
