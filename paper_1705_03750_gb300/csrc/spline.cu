// Cubic B-spline coefficients of f_ini (Sec. 2.2.2): for every x row a
// tridiagonal system along v, then for every v column one along x.  The
// systems share one constant matrix (rows (1, 4, 1)/6 with the zero-slope
// ghosts eta_{-1} = eta_1, eta_n = eta_{n-2}), so its LU factors c'_i and
// 1/den_i are computed once on the host and each system is one forward and
// one backward sweep.
//
// Row systems are contiguous in memory: a warp owns 32 rows and walks them
// in 32 x 32 tiles staged in shared memory, so global loads and stores stay
// coalesced while each lane runs the sequential sweep of its own row.  Column
// systems are strided by nv: one thread per column, so a warp's loads at a
// given step are 32 consecutive values.
#include "common.cuh"

namespace vm {
namespace {

constexpr int RW = 4;  // warps per block for the row sweeps

template <typename R, typename C>
__global__ void __launch_bounds__(32 * RW) k_rows(Grid g, const R* __restrict__ src, R* __restrict__ dst,
                                                  const C* __restrict__ th) {
  __shared__ R tile[RW][32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row0 = (blockIdx.x * RW + w) * 32;
  if (row0 >= g.nx) return;
  const int nv = g.nv;
  const C* cp = th;
  const C* inv = th + nv;
  const int myrow = row0 + lane;
  R (*T)[33] = tile[w];
  // forward sweep: d'_j = (6 f_j - sub_j d'_{j-1}) / den_j
  R dprev = R(0);
  for (int c0 = 0; c0 < nv; c0 += 32) {
    for (int rr = 0; rr < 32; rr++) {
      const int r = row0 + rr, c = c0 + lane;
      T[rr][lane] = (r < g.nx && c < nv) ? src[(size_t)r * nv + c] : R(0);
    }
    __syncwarp();
    const int cend = min(32, nv - c0);
    for (int cc = 0; cc < cend; cc++) {
      const int j = c0 + cc;
      const R sub = (j == 0) ? R(0) : ((j == nv - 1) ? R(2) : R(1));
      const R d = (R(6) * T[lane][cc] - sub * dprev) * (R)inv[j];
      T[lane][cc] = d;
      dprev = d;
    }
    __syncwarp();
    for (int rr = 0; rr < 32; rr++) {
      const int r = row0 + rr, c = c0 + lane;
      if (r < g.nx && c < nv) dst[(size_t)r * nv + c] = T[rr][lane];
    }
    __syncwarp();
  }
  // backward sweep: eta_j = d'_j - c'_j eta_{j+1}
  R enext = R(0);
  const int last0 = ((nv - 1) / 32) * 32;
  for (int c0 = last0; c0 >= 0; c0 -= 32) {
    for (int rr = 0; rr < 32; rr++) {
      const int r = row0 + rr, c = c0 + lane;
      T[rr][lane] = (r < g.nx && c < nv) ? dst[(size_t)r * nv + c] : R(0);
    }
    __syncwarp();
    const int cend = min(32, nv - c0);
    for (int cc = cend - 1; cc >= 0; cc--) {
      const int j = c0 + cc;
      const R e = (j == nv - 1) ? T[lane][cc] : (T[lane][cc] - (R)cp[j] * enext);
      T[lane][cc] = e;
      enext = e;
    }
    __syncwarp();
    for (int rr = 0; rr < 32; rr++) {
      const int r = row0 + rr, c = c0 + lane;
      if (r < g.nx && c < nv) dst[(size_t)r * nv + c] = T[rr][lane];
    }
    __syncwarp();
  }
  (void)myrow;
}

// One thread per column.  The sweeps are sequential in the row, but the
// loads are not: they are issued a chunk of CK rows at a time, so that one
// memory latency covers CK steps of the recurrence.
template <typename R, typename C>
__global__ void __launch_bounds__(128) k_cols(Grid g, R* __restrict__ x, const C* __restrict__ th) {
  constexpr int CK = 16;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.nv) return;
  const int nx = g.nx, nv = g.nv;
  const C* cp = th;
  const C* inv = th + nx;
  R dprev = R(0);
  for (int i0 = 0; i0 < nx; i0 += CK) {
    R v[CK];
#pragma unroll
    for (int u = 0; u < CK; u++) v[u] = (i0 + u < nx) ? x[(size_t)(i0 + u) * nv + j] : R(0);
#pragma unroll
    for (int u = 0; u < CK; u++) {
      const int i = i0 + u;
      if (i < nx) {
        const R sub = (i == 0) ? R(0) : ((i == nx - 1) ? R(2) : R(1));
        const R d = (R(6) * v[u] - sub * dprev) * (R)inv[i];
        x[(size_t)i * nv + j] = d;
        dprev = d;
      }
    }
  }
  R enext = dprev;  // d'_{nx-1} = eta_{nx-1}
  for (int i1 = nx - 2; i1 >= 0; i1 -= CK) {
    R v[CK];
#pragma unroll
    for (int u = 0; u < CK; u++) v[u] = (i1 - u >= 0) ? x[(size_t)(i1 - u) * nv + j] : R(0);
#pragma unroll
    for (int u = 0; u < CK; u++) {
      const int i = i1 - u;
      if (i >= 0) {
        const R e = v[u] - (R)cp[i] * enext;
        x[(size_t)i * nv + j] = e;
        enext = e;
      }
    }
  }
}

}  // namespace

void launch_spline_solve(vm_solver* s, const void* src, void* dst) {
  const unsigned rb = (unsigned)((s->g.nx + 32 * RW - 1) / (32 * RW));
  const unsigned cb = (unsigned)((s->g.nv + 127) / 128);
  int ps = prof_begin(s, KID_SPLINE_ROWS);
  if (s->fp32)
    k_rows<float, float><<<rb, 32 * RW, 0, s->stream>>>(s->g, (const float*)src, (float*)dst, s->thomas_vf);
  else
    k_rows<double, double><<<rb, 32 * RW, 0, s->stream>>>(s->g, (const double*)src, (double*)dst, s->thomas_v);
  prof_end(s, ps);
  ps = prof_begin(s, KID_SPLINE_COLS);
  if (s->fp32)
    k_cols<float, float><<<cb, 128, 0, s->stream>>>(s->g, (float*)dst, s->thomas_xf);
  else
    k_cols<double, double><<<cb, 128, 0, s->stream>>>(s->g, (double*)dst, s->thomas_x);
  prof_end(s, ps);
  s->launches += 2;
}

}  // namespace vm
