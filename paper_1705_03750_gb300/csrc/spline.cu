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
// systems are strided by nv: a lane per column, so a warp's loads at a given
// step are 32 consecutive values, and warps split the rows into chunks
// joined by their carries.
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

template <typename R, typename C>
__global__ void __launch_bounds__(128) k_rows_scan(Grid g, const R* __restrict__ src, R* __restrict__ dst,
                                                   const C* __restrict__ th) {
  if (gate_shut(g)) return;
  rows_scan_body(g, src, dst, th, blockIdx.x);
}

// Column systems: a block per 32 consecutive columns (lane = column, so
// every load and store is coalesced) and CW warps, warp w owning a chunk of
// consecutive rows.  Both sweeps are affine recurrences in the row,
//   forward  d_i = (6 f_i - sub_i d_{i-1}) / den_i = a_i d_{i-1} + (6 f_i / den_i),  a_i = -sub_i / den_i,
//   backward e_i = d_i - c'_i e_{i+1},
// so each warp first runs its chunk from a zero carry, keeping the chunk's
// composition (the product of its factors A, and its last value B); warp 0
// then chains the chunks' carries in order (CW steps per column); and each
// warp adds to every row the product of the chunk's factors up to that row
// times the carry that enters the chunk.  The whole column takes about
// 3 nx / CW dependent steps instead of 2 nx.
constexpr int CW = 32;  // warps per column block

template <typename R, typename C>
__device__ __forceinline__ void cols_body(const Grid& g, R* __restrict__ x, const C* __restrict__ th, int vb) {
  __shared__ R cB[CW][32];  // per chunk and column: the chunk's last value from a zero carry
  __shared__ R cC[CW][32];  // ... then the carry entering the chunk
  __shared__ C cA[CW];      // per chunk: the product of its factors (the same for every column)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = g.nx, nv = g.nv;
  const int j = vb * 32 + lane;
  const bool col = j < nv;
  const C* cp = th;
  const C* inv = th + nx;
  const int L = (nx + CW - 1) / CW;
  const int i0 = min(w * L, nx), i1 = min(i0 + L, nx);  // this warp's rows [i0, i1)
  R* xc = x + (col ? j : 0);
  // forward, each chunk from a zero carry
  {
    R d = R(0);
    C A = C(1);
#pragma unroll 8
    for (int i = i0; i < i1; i++) {
      const C sub = (i == 0) ? C(0) : ((i == nx - 1) ? C(2) : C(1));
      const R f = col ? xc[(size_t)i * nv] : R(0);
      d = (R(6) * f - (R)sub * d) * (R)inv[i];
      A *= -sub * inv[i];
      if (col) xc[(size_t)i * nv] = d;
    }
    cB[w][lane] = d;
    if (lane == 0) cA[w] = A;
  }
  __syncthreads();
  if (w == 0) {
    R c = R(0);
    for (int q = 0; q < CW; q++) {
      cC[q][lane] = c;
      c = (R)cA[q] * c + cB[q][lane];
    }
  }
  __syncthreads();
  // forward completed (d_i += P_i carry), then the backward sweep of the
  // chunk from a zero carry: e_i = d_i - c'_i e_{i+1}, e at i1 taken as 0
  {
    const R cin = cC[w][lane];
    C P = C(1);
#pragma unroll 8
    for (int i = i0; i < i1; i++) {
      const C sub = (i == 0) ? C(0) : ((i == nx - 1) ? C(2) : C(1));
      P *= -sub * inv[i];
      if (col) xc[(size_t)i * nv] += (R)P * cin;
    }
    R e = R(0);
    C Q = C(1);
#pragma unroll 8
    for (int i = i1 - 1; i >= i0; i--) {
      const C c = (i == nx - 1) ? C(0) : cp[i];
      const R d = col ? xc[(size_t)i * nv] : R(0);
      e = d - (R)c * e;
      Q *= -c;
      if (col) xc[(size_t)i * nv] = e;
    }
    __syncthreads();  // every warp has read its cC entry
    cB[w][lane] = e;
    if (lane == 0) cA[w] = Q;
  }
  __syncthreads();
  if (w == 0) {
    R c = R(0);
    for (int q = CW - 1; q >= 0; q--) {
      cC[q][lane] = c;
      c = (R)cA[q] * c + cB[q][lane];
    }
  }
  __syncthreads();
  {
    const R cin = cC[w][lane];
    C Q = C(1);
#pragma unroll 8
    for (int i = i1 - 1; i >= i0; i--) {
      const C c = (i == nx - 1) ? C(0) : cp[i];
      Q *= -c;
      if (col) xc[(size_t)i * nv] += (R)Q * cin;
    }
  }
}

template <typename R, typename C>
__global__ void __launch_bounds__(32 * CW) k_cols(Grid g, R* __restrict__ x, const C* __restrict__ th) {
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
__global__ void __launch_bounds__(32 * CW) k_cols_group(const SolveDesc* __restrict__ D, const int* __restrict__ off,
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
    k_cols<float, float><<<cb, 32 * CW, 0, s->stream>>>(s->g, (float*)dst, s->thomas_xf);
  else
    k_cols<double, double><<<cb, 32 * CW, 0, s->stream>>>(s->g, (double*)dst, s->thomas_x);
  prof_end(s, ps);
  s->launches += 2;
}

void group_spline(const GroupPlan& G) {
  if (G.fp32) {
    k_rows_group<float><<<group_grid(G, GP_ROWS, G.tot_rows4), 128, 0, G.stream>>>(G.D, G.off_rows4, G.ns, G.tot_rows4);
    k_cols_group<float><<<group_grid(G, GP_COLS, G.tot_cols), 32 * CW, 0, G.stream>>>(G.D, G.off_cols, G.ns,
                                                                                    G.tot_cols);
  } else {
    k_rows_group<double><<<group_grid(G, GP_ROWS, G.tot_rows4), 128, 0, G.stream>>>(G.D, G.off_rows4, G.ns,
                                                                                  G.tot_rows4);
    k_cols_group<double><<<group_grid(G, GP_COLS, G.tot_cols), 32 * CW, 0, G.stream>>>(G.D, G.off_cols, G.ns,
                                                                                     G.tot_cols);
  }
}

}  // namespace vm
