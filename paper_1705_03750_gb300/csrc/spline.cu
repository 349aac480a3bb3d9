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

// Row systems, one warp per row: both sweeps are linear recurrences,
// d_j = a_j d_{j-1} + b_j (forward: a_j = -sub_j / den_j, b_j = 6 f_j / den_j)
// and eta_j = -c'_j eta_{j+1} + d_j (backward).  A recurrence over a group of
// 32 consecutive entries is an inclusive scan of affine maps (a, b), composed
// as (a2, b2) o (a1, b1) = (a2 a1, a2 b1 + b2), in five shuffle steps; the
// group then continues from the previous group's last value.  Loads and
// stores are coalesced (32 consecutive entries per warp instruction).
template <typename R, typename C>
__device__ __forceinline__ void rows_scan_body(const Grid& g, const R* __restrict__ src, R* __restrict__ dst,
                                               const C* __restrict__ th, int vb) {
  const int lane = threadIdx.x & 31;
  const int row = vb * 4 + (threadIdx.x >> 5);
  if (row >= g.nx) return;
  const int nv = g.nv;
  const C* cp = th;
  const C* inv = th + nv;
  const R* f = src + (size_t)row * nv;
  R* d = dst + (size_t)row * nv;
  // forward
  R carry = R(0);
  for (int j0 = 0; j0 < nv; j0 += 32) {
    const int j = j0 + lane;
    R a = R(1), b = R(0);  // identity for lanes past the end
    if (j < nv) {
      const R sub = (j == 0) ? R(0) : ((j == nv - 1) ? R(2) : R(1));
      const R iv = (R)inv[j];
      a = -sub * iv;
      b = R(6) * f[j] * iv;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const R ap = __shfl_up_sync(0xffffffffu, a, o), bp = __shfl_up_sync(0xffffffffu, b, o);
      if (lane >= o) {
        b = a * bp + b;
        a = a * ap;
      }
    }
    const R v = a * carry + b;
    if (j < nv) d[j] = v;
    carry = __shfl_sync(0xffffffffu, v, 31);
  }
  __syncwarp();
  // backward: eta_{nv-1} = d_{nv-1}; groups from the end, scanned towards lower j
  carry = R(0);
  const int last0 = ((nv - 1) / 32) * 32;
  for (int j0 = last0; j0 >= 0; j0 -= 32) {
    const int j = j0 + lane;
    R a = R(1), b = R(0);
    if (j < nv) {
      a = (j == nv - 1) ? R(0) : -(R)cp[j];
      b = d[j];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const R an = __shfl_down_sync(0xffffffffu, a, o), bn = __shfl_down_sync(0xffffffffu, b, o);
      if (lane + o < 32) {
        b = a * bn + b;
        a = a * an;
      }
    }
    const R v = a * carry + b;
    if (j < nv) d[j] = v;
    carry = __shfl_sync(0xffffffffu, v, 0);
  }
}

// Column systems, one thread per column (a warp: 32 consecutive columns, so
// every load and store is coalesced).  The sweeps are sequential in the row,
// the loads are not: the next CK rows are loaded while the current CK are
// swept (double buffering), so that memory latency overlaps the recurrence.
template <typename R, typename C>
__global__ void __launch_bounds__(128) k_rows_scan(Grid g, const R* __restrict__ src, R* __restrict__ dst,
                                                   const C* __restrict__ th) {
  if (gate_shut(g)) return;
  rows_scan_body(g, src, dst, th, blockIdx.x);
}

template <typename R, typename C>
__device__ __forceinline__ void cols_body(const Grid& g, R* __restrict__ x, const C* __restrict__ th, int vb) {
  constexpr int CK = 32;
  const int j = vb * blockDim.x + threadIdx.x;
  if (j >= g.nv) return;
  const int nx = g.nx, nv = g.nv;
  const C* cp = th;
  const C* inv = th + nx;
  R cur[CK], nxt[CK];
  // forward
#pragma unroll
  for (int u = 0; u < CK; u++) cur[u] = (u < nx) ? x[(size_t)u * nv + j] : R(0);
  R dprev = R(0);
  for (int i0 = 0; i0 < nx; i0 += CK) {
#pragma unroll
    for (int u = 0; u < CK; u++) {
      const int i = i0 + CK + u;
      nxt[u] = (i < nx) ? x[(size_t)i * nv + j] : R(0);
    }
#pragma unroll
    for (int u = 0; u < CK; u++) {
      const int i = i0 + u;
      if (i < nx) {
        const R sub = (i == 0) ? R(0) : ((i == nx - 1) ? R(2) : R(1));
        const R d = (R(6) * cur[u] - sub * dprev) * (R)inv[i];
        x[(size_t)i * nv + j] = d;
        dprev = d;
      }
    }
#pragma unroll
    for (int u = 0; u < CK; u++) cur[u] = nxt[u];
  }
  // backward: eta_{nx-1} = d'_{nx-1}, then eta_i = d'_i - c'_i eta_{i+1}
  R enext = dprev;
#pragma unroll
  for (int u = 0; u < CK; u++) cur[u] = (nx - 2 - u >= 0) ? x[(size_t)(nx - 2 - u) * nv + j] : R(0);
  for (int i1 = nx - 2; i1 >= 0; i1 -= CK) {
#pragma unroll
    for (int u = 0; u < CK; u++) {
      const int i = i1 - CK - u;
      nxt[u] = (i >= 0) ? x[(size_t)i * nv + j] : R(0);
    }
#pragma unroll
    for (int u = 0; u < CK; u++) {
      const int i = i1 - u;
      if (i >= 0) {
        const R e = cur[u] - (R)cp[i] * enext;
        x[(size_t)i * nv + j] = e;
        enext = e;
      }
    }
#pragma unroll
    for (int u = 0; u < CK; u++) cur[u] = nxt[u];
  }
}

template <typename R, typename C>
__global__ void __launch_bounds__(32) k_cols(Grid g, R* __restrict__ x, const C* __restrict__ th) {
  if (gate_shut(g)) return;
  cols_body(g, x, th, blockIdx.x);
}

// ---- group launches: f_ini -> eta of every solve ----
template <typename R>
__global__ void __launch_bounds__(128) k_rows_group(const SolveDesc* __restrict__ D, const int* __restrict__ off,
                                                  int ns, int total) {
  GROUP_LOOP(off, ns, total)
  if constexpr (sizeof(R) == 4)
    rows_scan_body<float, float>(gsh, (const float*)d.fini, (float*)d.eta, d.thvf, vb);
  else
    rows_scan_body<double, double>(gsh, (const double*)d.fini, (double*)d.eta, d.thv, vb);
  GROUP_END
}

template <typename R>
__global__ void __launch_bounds__(32) k_cols_group(const SolveDesc* __restrict__ D, const int* __restrict__ off,
                                                 int ns, int total) {
  GROUP_LOOP(off, ns, total)
  if constexpr (sizeof(R) == 4)
    cols_body<float, float>(gsh, (float*)d.eta, d.thxf, vb);
  else
    cols_body<double, double>(gsh, (double*)d.eta, d.thx, vb);
  GROUP_END
}

}  // namespace

void launch_spline_solve(vm_solver* s, const void* src, void* dst) {
  const unsigned rb = (unsigned)((s->g.nx + 32 * RW - 1) / (32 * RW));
  const unsigned cb = (unsigned)((s->g.nv + 31) / 32);
  int ps = prof_begin(s, KID_SPLINE_ROWS);
  const unsigned sb = (unsigned)((s->g.nx + 3) / 4);
  (void)rb;
  if (s->fp32)
    k_rows_scan<float, float><<<sb, 128, 0, s->stream>>>(s->g, (const float*)src, (float*)dst, s->thomas_vf);
  else
    k_rows_scan<double, double><<<sb, 128, 0, s->stream>>>(s->g, (const double*)src, (double*)dst, s->thomas_v);
  prof_end(s, ps);
  ps = prof_begin(s, KID_SPLINE_COLS);
  if (s->fp32)
    k_cols<float, float><<<cb, 32, 0, s->stream>>>(s->g, (float*)dst, s->thomas_xf);
  else
    k_cols<double, double><<<cb, 32, 0, s->stream>>>(s->g, (double*)dst, s->thomas_x);
  prof_end(s, ps);
  s->launches += 2;
}

void group_spline(const GroupPlan& G) {
  if (G.fp32) {
    k_rows_group<float><<<group_grid(G, GP_ROWS, G.tot_rows4), 128, 0, G.stream>>>(G.D, G.off_rows4, G.ns, G.tot_rows4);
    k_cols_group<float><<<group_grid(G, GP_COLS, G.tot_cols), 32, 0, G.stream>>>(G.D, G.off_cols, G.ns, G.tot_cols);
  } else {
    k_rows_group<double><<<group_grid(G, GP_ROWS, G.tot_rows4), 128, 0, G.stream>>>(G.D, G.off_rows4, G.ns,
                                                                                  G.tot_rows4);
    k_cols_group<double><<<group_grid(G, GP_COLS, G.tot_cols), 32, 0, G.stream>>>(G.D, G.off_cols, G.ns, G.tot_cols);
  }
}

}  // namespace vm
