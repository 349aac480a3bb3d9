// Influence map of the elements of metric (Sec. 2.3.1).
//
// Element-parallel percolation.  Each element is handled by one thread
// block that holds, in shared memory, bit masks of a window of the Eulerian
// grid centred on the element's start site: "evaluated" and "claimed"
// (the connected component grown so far).  The flood fill is lazy: each
// round dilates the component by one site in the four directions and runs
// the percolation test only on the newly reached sites, so the test runs
// once per site of the component and once per site of its rim, as in a
// breadth-first search, while the dilation itself is a few word operations
// per window row.
//
// Claims are resolved with one 128-bit atomic compare-and-swap minimum per
// claimed site on the key (bits of d^2, element index): the smallest
// distance wins, ties go to the smaller index.  A finalize pass turns keys
// into the int32 map, resets them and lists the sites nobody claimed; a
// single-block pass then repairs those in Jacobi rounds from their
// 4-neighbours.  Elements whose component reaches the edge of the small
// window are queued and redone with a 4x larger window.
//
// Every decision (ranges, the d comparisons, the claim order) is taken on
// FP64 values computed operation by operation in a fixed order.
#include "common.cuh"

namespace vm {
namespace {

__device__ __forceinline__ void alpha_range(double r, double alpha, int& lo, int& hi) {
  if (r < -alpha) {
    lo = -1;
    hi = 0;
  } else if (r < alpha) {
    lo = 0;
    hi = 0;
  } else {
    lo = 0;
    hi = 1;
  }
}

// Percolation test of site P for the centre element of a 3x3 block of
// Taylor records (index 4): it fails if an investigated, existing neighbour
// proposes a strictly smaller distance.
__device__ bool pass_test(const Grid& g, const double (*T9)[TY_N], const int* ex9, double Px,
                          double Pv, double& d2) {
  double xi, ze;
  d2 = dist2_exact(T9[4], g, Px, Pv, xi, ze);
  int a0, a1, b0, b1;
  alpha_range(xi, g.alpha, a0, a1);
  alpha_range(ze, g.alpha, b0, b1);
  for (int a = a0; a <= a1; a++)
    for (int b = b0; b <= b1; b++) {
      if (a == 0 && b == 0) continue;
      int q = (a + 1) * 3 + (b + 1);
      if (!ex9[q]) continue;
      double x2, z2;
      double dn = dist2_exact(T9[q], g, Px, Pv, x2, z2);
      if (dn < d2) return false;
    }
  return true;
}

// 128-bit compare-and-swap on global memory (sm_90 and later).
__device__ __forceinline__ ulonglong2 cas128(unsigned long long* addr, ulonglong2 cmp, ulonglong2 val) {
  ulonglong2 old;
  asm volatile(
      "{\n\t"
      ".reg .b128 c, v, r;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 v, {%4, %5};\n\t"
      "atom.global.cas.b128 r, [%6], c, v;\n\t"
      "mov.b128 {%0, %1}, r;\n\t"
      "}"
      : "=l"(old.x), "=l"(old.y)
      : "l"(cmp.x), "l"(cmp.y), "l"(val.x), "l"(val.y), "l"(addr)
      : "memory");
  return old;
}

// keys[2p] = element index, keys[2p+1] = bits of d^2 (a 128-bit integer
// whose order is the claim order).
__device__ __forceinline__ void claim_min(unsigned long long* key2, unsigned long long dbits,
                                          unsigned long long idx) {
  ulonglong2 cur = __ldcg(reinterpret_cast<const ulonglong2*>(key2));
  ulonglong2 val = make_ulonglong2(idx, dbits);
  while (dbits < cur.y || (dbits == cur.y && idx < cur.x)) {
    ulonglong2 prev = cas128(key2, cur, val);
    if (prev.x == cur.x && prev.y == cur.y) break;
    cur = prev;
  }
}

// Mask of window columns [lo, hi) within word w (64 columns per word).
__device__ __forceinline__ unsigned long long col_mask(int w, int lo, int hi) {
  int a = max(lo - 64 * w, 0), b = min(hi - 64 * w, 64);
  if (b <= a) return 0ull;
  unsigned long long up = (b >= 64) ? ~0ull : ((1ull << b) - 1ull);
  unsigned long long dn = (a <= 0) ? 0ull : ((1ull << a) - 1ull);
  return up & ~dn;
}

template <int ROWS, int WORDS, int T>
struct ClaimShared {
  double T9[9][TY_N];
  int ex9[9];
  unsigned long long comp[ROWS][WORDS];
  unsigned long long eval[ROWS][WORDS];
  int ok, any, ovf;
};

// One element per block.  ROWS window rows along x, WORDS*64 columns along v;
// T threads, each owning rows tid, tid+T, ...
template <int ROWS, int WORDS, int T>
__device__ void claim_element(const Grid& g, int m, const double* __restrict__ tay,
                              unsigned long long* __restrict__ keys, DevState* ds,
                              int32_t* __restrict__ ovf_list, bool last_resort,
                              ClaimShared<ROWS, WORDS, T>& S) {
  constexpr int COLS = 64 * WORDS;
  constexpr int RPT = ROWS / T;
  const int tid = threadIdx.x;
  const int k = m / g.Lv, l = m - k * g.Lv;
  for (int idx = tid; idx < 9 * TY_N; idx += T) {
    int q = idx / TY_N, c = idx - q * TY_N;
    int kk = k + q / 3 - 1, ll = l + q % 3 - 1;
    bool ex = kk >= 0 && kk < g.Lx && ll >= 0 && ll < g.Lv;
    S.T9[q][c] = ex ? tay[(size_t)(kk * g.Lv + ll) * TY_N + c] : 0.0;
    if (c == 0) S.ex9[q] = ex;
  }
  for (int r = tid; r < ROWS; r += T)
#pragma unroll
    for (int w = 0; w < WORDS; w++) {
      S.comp[r][w] = 0ull;
      S.eval[r][w] = 0ull;
    }
  if (tid == 0) {
    S.ok = 0;
    S.ovf = 0;
  }
  __syncthreads();
  // start: the grid site nearest to P_m
  const double us = dmul(dsub(S.T9[4][TY_X], g.x_lo), g.inv_dx);
  const double ws = dmul(dsub(S.T9[4][TY_V], g.v_lo), g.inv_dv);
  if (!(us > -1e9 && us < 1e9 && ws > -1e9 && ws < 1e9)) return;
  const long long i0 = (long long)floor(dadd(us, 0.5)), j0 = (long long)floor(dadd(ws, 0.5));
  const int pad = g.pad;
  if (i0 < -pad || i0 >= g.nx + pad || j0 < -pad || j0 >= g.nv + pad) return;
  const long long r0 = i0 - ROWS / 2, c0 = j0 - COLS / 2;
  // window columns / rows inside the padded lattice
  const int clo = (int)max(0ll, (long long)(-pad) - c0);
  const int chi = (int)min((long long)COLS, (long long)(g.nv + pad) - c0);
  const int rlo = (int)max(0ll, (long long)(-pad) - r0);
  const int rhi = (int)min((long long)ROWS, (long long)(g.nx + pad) - r0);
  if (tid == 0) {
    double d2;
    double Px = site_x(g, i0), Pv = site_v(g, j0);
    bool ok = pass_test(g, S.T9, S.ex9, Px, Pv, d2);
    const int rs = ROWS / 2, cs = COLS / 2;
    S.eval[rs][cs >> 6] |= 1ull << (cs & 63);
    if (ok) {
      S.comp[rs][cs >> 6] |= 1ull << (cs & 63);
      if (i0 >= 0 && i0 < g.nx && j0 >= 0 && j0 < g.nv)
        claim_min(keys + 2 * ((size_t)i0 * g.nv + j0), dkey(d2), (unsigned long long)m);
    }
    S.ok = ok;
  }
  __syncthreads();
  if (!S.ok) return;
  unsigned long long front[RPT][WORDS];
  for (int it = 0; it < ROWS * COLS; it++) {
    bool anyf = false;
#pragma unroll
    for (int q = 0; q < RPT; q++) {
      const int r = tid + q * T;
#pragma unroll
      for (int w = 0; w < WORDS; w++) {
        unsigned long long c = S.comp[r][w];
        unsigned long long d = c | (c << 1) | (c >> 1);
        if (w > 0) d |= S.comp[r][w - 1] >> 63;
        if (w < WORDS - 1) d |= S.comp[r][w + 1] << 63;
        if (r > 0) d |= S.comp[r - 1][w];
        if (r < ROWS - 1) d |= S.comp[r + 1][w];
        unsigned long long valid = (r >= rlo && r < rhi) ? col_mask(w, clo, chi) : 0ull;
        front[q][w] = d & ~S.eval[r][w] & valid;
        anyf |= front[q][w] != 0ull;
      }
    }
    if (!__syncthreads_or(anyf)) break;
#pragma unroll
    for (int q = 0; q < RPT; q++) {
      const int r = tid + q * T;
      const long long i = r0 + r;
#pragma unroll
      for (int w = 0; w < WORDS; w++) {
        unsigned long long fr = front[q][w];
        if (!fr) continue;
        S.eval[r][w] |= fr;
        unsigned long long add = 0ull;
        while (fr) {
          int b = __ffsll((long long)fr) - 1;
          fr &= fr - 1ull;
          const long long j = c0 + 64 * w + b;
          double d2;
          if (pass_test(g, S.T9, S.ex9, site_x(g, i), site_v(g, j), d2)) {
            add |= 1ull << b;
            if (i >= 0 && i < g.nx && j >= 0 && j < g.nv)
              claim_min(keys + 2 * ((size_t)i * g.nv + j), dkey(d2), (unsigned long long)m);
          }
        }
        S.comp[r][w] |= add;
      }
    }
    __syncthreads();
  }
  // Did the component reach a window edge beyond which the padded lattice
  // continues?  Then the window was too small for this element.
  bool ovf = false;
#pragma unroll
  for (int q = 0; q < RPT; q++) {
    const int r = tid + q * T;
    unsigned long long rowany = 0ull;
#pragma unroll
    for (int w = 0; w < WORDS; w++) rowany |= S.comp[r][w];
    if (!rowany) continue;
    if (r == 0 && rlo == 0 && r0 - 1 >= -pad) ovf = true;
    if (r == ROWS - 1 && rhi == ROWS && r0 + ROWS < g.nx + pad) ovf = true;
    if ((S.comp[r][0] & 1ull) && clo == 0 && c0 - 1 >= -pad) ovf = true;
    if ((S.comp[r][WORDS - 1] >> 63) && chi == COLS && c0 + COLS < g.nv + pad) ovf = true;
  }
  if (__syncthreads_or(ovf) && tid == 0) {
    if (last_resort) {
      atomicOr(&ds->err, ERR_PATCH_OVERFLOW);
    } else {
      int slot = atomicAdd(&ds->noverflow, 1);
      ovf_list[slot] = m;
    }
  }
}

constexpr int SR = 64, SW = 2, ST = 32;    // small window: 64 x 128 sites, one warp
constexpr int BR = 256, BW = 4, BT = 256;  // large window: 256 x 256 sites

__global__ void __launch_bounds__(ST) k_claim_small(Grid g, const double* __restrict__ tay,
                                                    unsigned long long* __restrict__ keys, DevState* ds,
                                                    int32_t* __restrict__ ovf_list) {
  __shared__ ClaimShared<SR, SW, ST> S;
  claim_element<SR, SW, ST>(g, blockIdx.x, tay, keys, ds, ovf_list, false, S);
}

__global__ void __launch_bounds__(BT) k_claim_large(Grid g, const double* __restrict__ tay,
                                                    unsigned long long* __restrict__ keys, DevState* ds,
                                                    int32_t* __restrict__ ovf_list) {
  __shared__ ClaimShared<BR, BW, BT> S;
  const int n = ds->noverflow;
  for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
    claim_element<BR, BW, BT>(g, ovf_list[idx], tay, keys, ds, ovf_list, true, S);
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ds->overflow_stat = n;
}

// Keys -> map; reset keys for the next map; list the unclaimed sites.
__global__ void k_finalize(Grid g, unsigned long long* __restrict__ keys, int32_t* __restrict__ map,
                           int32_t* __restrict__ holes, DevState* ds) {
  const size_t n = (size_t)g.nx * g.nv;
  const ulonglong2 empty = make_ulonglong2(KEY_EMPTY, KEY_EMPTY);
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    ulonglong2 kv = reinterpret_cast<ulonglong2*>(keys)[p];
    int32_t m = -1;
    if (kv.y == KEY_EMPTY && kv.x == KEY_EMPTY) {
      int slot = atomicAdd(&ds->nholes, 1);
      holes[slot] = (int32_t)p;
    } else {
      m = (int32_t)kv.x;
      reinterpret_cast<ulonglong2*>(keys)[p] = empty;
    }
    map[p] = m;
  }
}

constexpr int HT = 1024;

// Unexplored sites (Sec. 2.3.1, end): Jacobi rounds; in each round every
// hole takes, among the elements its in-grid 4-neighbours held at the end of
// the previous round, the one with the smallest d at the hole, then the
// smaller index.
__global__ void __launch_bounds__(HT) k_holes(Grid g, const double* __restrict__ tay,
                                              int32_t* __restrict__ map, int32_t* la, int32_t* lb,
                                              int32_t* cho, DevState* ds) {
  __shared__ int n_s, next_s;
  if (threadIdx.x == 0) {
    n_s = ds->nholes;
    ds->holes_found = n_s;
  }
  __syncthreads();
  int rounds = 0;
  while (n_s > 0) {
    if (rounds >= g.max_hole_rounds) {
      if (threadIdx.x == 0) atomicOr(&ds->err, ERR_NOT_CONVERGED);
      break;
    }
    const int n = n_s;
    for (int idx = threadIdx.x; idx < n; idx += HT) {
      const int p = la[idx];
      const int i = p / g.nv, j = p - i * g.nv;
      const double Px = site_x(g, i), Pv = site_v(g, j);
      int best = -1;
      unsigned long long bestk = 0;
      const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
      for (int q = 0; q < 4; q++) {
        const int ii = i + di[q], jj = j + dj[q];
        if (ii < 0 || ii >= g.nx || jj < 0 || jj >= g.nv) continue;
        const int cand = map[(size_t)ii * g.nv + jj];
        if (cand < 0) continue;
        double xi, ze;
        unsigned long long key = dkey(dist2_exact(tay + (size_t)cand * TY_N, g, Px, Pv, xi, ze));
        if (best < 0 || key < bestk || (key == bestk && cand < best)) {
          best = cand;
          bestk = key;
        }
      }
      cho[idx] = best;
    }
    if (threadIdx.x == 0) next_s = 0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < n; idx += HT) {
      const int c = cho[idx];
      if (c >= 0) {
        map[la[idx]] = c;
      } else {
        int slot = atomicAdd(&next_s, 1);
        lb[slot] = la[idx];
      }
    }
    __syncthreads();
    int32_t* t = la;
    la = lb;
    lb = t;
    rounds++;
    if (threadIdx.x == 0) n_s = next_s;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ds->hole_rounds = rounds;
    ds->nholes = 0;
  }
}

}  // namespace

void launch_map(vm_solver* s) {
  // counters: nholes, holes_found, hole_rounds, noverflow
  cudaMemsetAsync(&s->ds->nholes, 0, 4 * sizeof(int32_t), s->stream);
  k_claim_small<<<s->g.ne, ST, 0, s->stream>>>(s->g, s->tay, s->keys, s->ds, s->overflow_list);
  k_claim_large<<<152, BT, 0, s->stream>>>(s->g, s->tay, s->keys, s->ds, s->overflow_list);
  unsigned nb = (unsigned)((s->n + 255) / 256);
  if (nb > 152 * 16) nb = 152 * 16;
  k_finalize<<<nb, 256, 0, s->stream>>>(s->g, s->keys, s->map, s->holes_a, s->ds);
  k_holes<<<1, HT, 0, s->stream>>>(s->g, s->tay, s->map, s->holes_a, s->holes_b,
                                    s->holes_b + s->n, s->ds);
  s->launches += 4;
}

}  // namespace vm
