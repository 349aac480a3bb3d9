// Pixel masses and force from a caller's f, without any device allocation.
//
// Some callers cannot allocate device memory: a plugin whose host
// application owns the whole device heap and forbids direct cudaMalloc, or a
// loop that must never pay the device-wide synchronisation that cudaMalloc
// and cudaFree can trigger.  For them this file provides one entry point
// whose only scratch (the pixel masses between the row sums and the mass
// scan, plus a small control block) lives in a file-scope device array that
// every GPU loading the library keeps until the process exits.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kMaxNx = 16384;  // VM_STATIC_FORCE_MAX_NX in include/vlamet.h

struct ForceScratch {
  double M[kMaxNx];
  vm::DevState ds;
};

// The shared scratch.  Host code must not pass this name to a kernel: on the
// host it is only a stand-in symbol, not a device address.
static __device__ __align__(256) ForceScratch g_force_scratch;

constexpr int kMaxDevices = 64;
ForceScratch* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch on the current device, looked up once per
// device (with that device current) by cudaGetSymbolAddress.
vm_status scratch_address(ForceScratch** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return VM_E_CUDA;
  if (dev >= kMaxDevices) return VM_E_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_force_scratch) != cudaSuccess || !p) return VM_E_CUDA;
    g_scratch_addr[dev] = static_cast<ForceScratch*>(p);
  }
  *out = g_scratch_addr[dev];
  return VM_OK;
}

// M(i) = (sum_j f(i,j)) dx dv, one block per x row (Sec. 2.5).
template <typename R>
__global__ void __launch_bounds__(256) k_row_mass(const R* __restrict__ f, int nx, int nv, double dxdv,
                                                  double* __restrict__ M) {
  __shared__ double sh[8];
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) acc += (double)f[(size_t)i * nv + j];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
    M[i] = vm::dmul(t, dxdv);
  }
}

}  // namespace

extern "C" vm_status vm_force_from_f_static(const void* f, int32_t dtype, int32_t nx, int32_t nv, double x_lo,
                                            double x_hi, double v_lo, double v_hi, double G, int32_t literal_fd,
                                            double* M_out, double* a, double* da, double* d2a,
                                            void* cuda_stream) {
  if (!f || !a || !da || !d2a) return VM_E_INVALID_ARG;
  if (nx < 4 || nv < 4 || nx > kMaxNx) return VM_E_INVALID_ARG;
  if (!(x_hi > x_lo) || !(v_hi > v_lo)) return VM_E_INVALID_ARG;
  if (dtype != VM_DTYPE_F64 && dtype != VM_DTYPE_F32) return VM_E_INVALID_ARG;
  ForceScratch* scratch = nullptr;
  vm_status st = scratch_address(&scratch);
  if (st != VM_OK) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  vm::Grid g{};
  g.nx = nx;
  g.nv = nv;
  g.dx = (x_hi - x_lo) / (double)(nx - 1);
  g.dv = (v_hi - v_lo) / (double)(nv - 1);
  g.dxdv = g.dx * g.dv;
  g.A = 2.0 * 3.14159265358979323846 * G;
  g.literal_fd = literal_fd;
  // Every entry of M is overwritten by the row sums; nothing in the scratch
  // needs clearing beforehand.
  if (dtype == VM_DTYPE_F64)
    k_row_mass<double><<<nx, 256, 0, stream>>>((const double*)f, nx, nv, g.dxdv, scratch->M);
  else
    k_row_mass<float><<<nx, 256, 0, stream>>>((const float*)f, nx, nv, g.dxdv, scratch->M);
  vm::launch_scan_force_raw(g, scratch->M, a, da, d2a, &scratch->ds, stream);
  if (M_out) {
    if (cudaMemcpyAsync(M_out, scratch->M, (size_t)nx * sizeof(double), cudaMemcpyDeviceToDevice, stream) !=
        cudaSuccess)
      return VM_E_CUDA;
  }
  return cudaPeekAtLastError() == cudaSuccess ? VM_OK : VM_E_CUDA;
}
