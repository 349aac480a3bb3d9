// Influence map of the elements of metric (Sec. 2.3.1).
//
// Element-parallel percolation: the claimed set of element m is the
// 4-connected component, containing the grid site nearest to P_m, of the
// sites that pass m's test (no investigated neighbour proposes a strictly
// smaller d).  Each element is flood-filled inside a window of bit masks
// held in shared memory (evaluated / passing / claimed), with the window
// sized in three tiers:
//
//   1. a 64 x 128 window, one warp per element, one percolation test per
//      newly reached site (lazy breadth-first growth: the test runs once per
//      site of the component and of its rim);
//   2. for the elements whose component reached the edge of tier 1, up to
//      three attempts with larger windows, in an order set by the sides it
//      escaped from: a band window 128 sites across and as long as shared
//      memory allows along v (the whole padded lattice at 4096^2), the same
//      along x, and a 256 x 256 window.  Elements of the outer layer whose
//      neighbours have moved away claim long thin bands; to cross them in
//      few rounds, any 64-site word the component reaches is evaluated
//      whole, and the component is then extended through runs of passing
//      sites inside the word with one carry-propagating addition.
//
// Claims are resolved by one 128-bit atomic compare-and-swap minimum per
// claimed site on the key (bits of d^2, element index): smallest distance
// wins, ties go to the smaller index.  A finalize pass turns keys into the
// int32 map, resets them and lists unclaimed sites; one block repairs those
// in Jacobi rounds from their 4-neighbours.
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
// Taylor records (index 4).
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
      const int q = (a + 1) * 3 + (b + 1);
      if (!ex9[q]) continue;
      double x2, z2;
      const double dn = dist2_exact(T9[q], g, Px, Pv, x2, z2);
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

// keys[2p] = element index, keys[2p+1] = bits of d^2: as a 128-bit integer
// its order is the claim order.
__device__ __forceinline__ void claim_min(unsigned long long* key2, unsigned long long dbits,
                                          unsigned long long idx) {
  ulonglong2 cur = __ldcg(reinterpret_cast<const ulonglong2*>(key2));
  const ulonglong2 val = make_ulonglong2(idx, dbits);
  while (dbits < cur.y || (dbits == cur.y && idx < cur.x)) {
    const ulonglong2 prev = cas128(key2, cur, val);
    if (prev.x == cur.x && prev.y == cur.y) break;
    cur = prev;
  }
}

__device__ __forceinline__ void claim_site(const Grid& g, unsigned long long* keys, long long i, long long j,
                                           double d2, int m) {
  if (i >= 0 && i < g.nx && j >= 0 && j < g.nv)
    claim_min(keys + 2 * ((size_t)i * g.nv + j), dkey(d2), (unsigned long long)m);
}

// Mask of window columns [lo, hi) within word w (64 columns per word).
__device__ __forceinline__ unsigned long long col_mask(int w, int lo, int hi) {
  const int a = max(lo - 64 * w, 0), b = min(hi - 64 * w, 64);
  if (b <= a) return 0ull;
  const unsigned long long up = (b >= 64) ? ~0ull : ((1ull << b) - 1ull);
  const unsigned long long dn = (a <= 0) ? 0ull : ((1ull << a) - 1ull);
  return up & ~dn;
}

// Bits of P reachable from the seeds S (S inside P) through runs of set
// bits of P, in both directions along the word.
__device__ __forceinline__ unsigned long long run_fill(unsigned long long S, unsigned long long P) {
  S &= P;
  const unsigned long long up = (((P + S) ^ P) & P) | S;
  const unsigned long long Pr = __brevll(P), Sr = __brevll(S);
  const unsigned long long dn = __brevll((((Pr + Sr) ^ Pr) & Pr) | Sr);
  return up | dn;
}

enum : int { MODE_BAND_V = 0, MODE_BAND_X = 1, MODE_FAT = 2 };

__device__ __forceinline__ void load_T9(const Grid& g, int m, const double* __restrict__ tay,
                                        double (*T9)[TY_N], int* ex9) {
  const int k = m / g.Lv, l = m - k * g.Lv;
  for (int idx = threadIdx.x; idx < 9 * TY_N; idx += blockDim.x) {
    const int q = idx / TY_N, c = idx - q * TY_N;
    const int kk = k + q / 3 - 1, ll = l + q % 3 - 1;
    const bool ex = kk >= 0 && kk < g.Lx && ll >= 0 && ll < g.Lv;
    T9[q][c] = ex ? tay[(size_t)(kk * g.Lv + ll) * TY_N + c] : 0.0;
    if (c == 0) ex9[q] = ex;
  }
}

// ---------------------------------------------------------------------------
// tier 1: 64 x 128 window, one warp per element, lazy per-site growth
// ---------------------------------------------------------------------------

constexpr int SR = 64, SW = 2, ST = 32;

struct SmallShared {
  double T9[9][TY_N];
  int ex9[9];
  unsigned long long comp[SR][SW];
  unsigned long long eval[SR][SW];
  int ok;
};

__global__ void __launch_bounds__(ST) k_claim_small(Grid g, const double* __restrict__ tay,
                                                    unsigned long long* __restrict__ keys, DevState* ds,
                                                    int2* __restrict__ ovf_list) {
  constexpr int COLS = 64 * SW, RPT = SR / ST;
  __shared__ SmallShared S;
  const int m = blockIdx.x, tid = threadIdx.x;
  load_T9(g, m, tay, S.T9, S.ex9);
  for (int r = tid; r < SR; r += ST)
#pragma unroll
    for (int w = 0; w < SW; w++) {
      S.comp[r][w] = 0ull;
      S.eval[r][w] = 0ull;
    }
  __syncthreads();
  const double us = dmul(dsub(S.T9[4][TY_X], g.x_lo), g.inv_dx);
  const double ws = dmul(dsub(S.T9[4][TY_V], g.v_lo), g.inv_dv);
  if (!(us > -1e9 && us < 1e9 && ws > -1e9 && ws < 1e9)) return;
  const long long i0 = (long long)floor(dadd(us, 0.5)), j0 = (long long)floor(dadd(ws, 0.5));
  const int pad = g.pad;
  if (i0 < -pad || i0 >= g.nx + pad || j0 < -pad || j0 >= g.nv + pad) return;
  const long long r0 = i0 - SR / 2, c0 = j0 - COLS / 2;
  const int clo = (int)max(0ll, (long long)(-pad) - c0);
  const int chi = (int)min((long long)COLS, (long long)(g.nv + pad) - c0);
  const int rlo = (int)max(0ll, (long long)(-pad) - r0);
  const int rhi = (int)min((long long)SR, (long long)(g.nx + pad) - r0);
  if (tid == 0) {
    double d2;
    const bool ok = pass_test(g, S.T9, S.ex9, site_x(g, i0), site_v(g, j0), d2);
    S.eval[SR / 2][(COLS / 2) >> 6] |= 1ull << ((COLS / 2) & 63);
    if (ok) {
      S.comp[SR / 2][(COLS / 2) >> 6] |= 1ull << ((COLS / 2) & 63);
      claim_site(g, keys, i0, j0, d2, m);
    }
    S.ok = ok;
  }
  __syncthreads();
  if (!S.ok) return;
  unsigned long long front[RPT][SW];
  for (int it = 0; it < SR * COLS; it++) {
    bool anyf = false;
#pragma unroll
    for (int q = 0; q < RPT; q++) {
      const int r = tid + q * ST;
#pragma unroll
      for (int w = 0; w < SW; w++) {
        const unsigned long long c = S.comp[r][w];
        unsigned long long d = c | (c << 1) | (c >> 1);
        if (w > 0) d |= S.comp[r][w - 1] >> 63;
        if (w < SW - 1) d |= S.comp[r][w + 1] << 63;
        if (r > 0) d |= S.comp[r - 1][w];
        if (r < SR - 1) d |= S.comp[r + 1][w];
        const unsigned long long valid = (r >= rlo && r < rhi) ? col_mask(w, clo, chi) : 0ull;
        front[q][w] = d & ~S.eval[r][w] & valid;
        anyf |= front[q][w] != 0ull;
      }
    }
    if (!__syncthreads_or(anyf)) break;
#pragma unroll
    for (int q = 0; q < RPT; q++) {
      const int r = tid + q * ST;
      const long long i = r0 + r;
#pragma unroll
      for (int w = 0; w < SW; w++) {
        unsigned long long fr = front[q][w];
        if (!fr) continue;
        S.eval[r][w] |= fr;
        unsigned long long add = 0ull;
        while (fr) {
          const int b = __ffsll((long long)fr) - 1;
          fr &= fr - 1ull;
          const long long j = c0 + 64 * w + b;
          double d2;
          if (pass_test(g, S.T9, S.ex9, site_x(g, i), site_v(g, j), d2)) {
            add |= 1ull << b;
            claim_site(g, keys, i, j, d2, m);
          }
        }
        S.comp[r][w] |= add;
      }
    }
    __syncthreads();
  }
  // Escaped the window?  Record on which sides, to pick the next window.
  bool esc_rows = false, esc_cols = false;
#pragma unroll
  for (int q = 0; q < RPT; q++) {
    const int r = tid + q * ST;
    unsigned long long rowany = 0ull;
#pragma unroll
    for (int w = 0; w < SW; w++) rowany |= S.comp[r][w];
    if (!rowany) continue;
    if (r == 0 && rlo == 0 && r0 - 1 >= -pad) esc_rows = true;
    if (r == SR - 1 && rhi == SR && r0 + SR < g.nx + pad) esc_rows = true;
    if ((S.comp[r][0] & 1ull) && clo == 0 && c0 - 1 >= -pad) esc_cols = true;
    if ((S.comp[r][SW - 1] >> 63) && chi == COLS && c0 + COLS < g.nv + pad) esc_cols = true;
  }
  const bool er = __syncthreads_or(esc_rows), ec = __syncthreads_or(esc_cols);
  if ((er || ec) && tid == 0) {
    const int sides = (er ? 1 : 0) | (ec ? 2 : 0);
    const int slot = atomicAdd(&ds->noverflow, 1);
    ovf_list[slot] = make_int2(m, sides << 4);   // attempt 0
  }
}

// ---------------------------------------------------------------------------
// tiers 2 and 3: cooperative block, word-granular evaluation
// ---------------------------------------------------------------------------

constexpr int BT = 256;       // threads
constexpr int BAND_R = 128;   // band window: rows across the band
constexpr int FAT_R = 256, FAT_W = 4;
constexpr int LIST_CAP = 1024;
constexpr size_t SMEM_MAX = 227 * 1024;

// Order of the window modes tried for an element, by the sides its
// component escaped tier 1 from (1: rows, 2: columns, 3: both).
__device__ __forceinline__ int mode_for(int sides, int attempt) {
  const int seq[4][3] = {{MODE_FAT, MODE_BAND_V, MODE_BAND_X},
                         {MODE_BAND_X, MODE_FAT, MODE_BAND_V},
                         {MODE_BAND_V, MODE_FAT, MODE_BAND_X},
                         {MODE_BAND_V, MODE_BAND_X, MODE_FAT}};
  return seq[sides & 3][attempt];
}

struct BigHeader {
  double T9[9][TY_N];
  int ex9[9];
  int ok, nlist, active, esc;
  int list[LIST_CAP];
};

// Window geometry: "rows" run across, "words" along the bit axis.  For
// MODE_BAND_X the bit axis is x (transposed window), otherwise v.
struct Win {
  bool trans;
  int R, W;              // rows, 64-bit words per row
  long long r0, c0;      // lattice coordinate of row 0 / bit 0
  int rlo, rhi, clo, chi;
  long long nrow_lat, ncol_lat;  // lattice extent along rows / bits (without pad)
};

__device__ __forceinline__ void site_of(const Win& W, int r, int c, long long& i, long long& j) {
  if (W.trans) {
    j = W.r0 + r;
    i = W.c0 + c;
  } else {
    i = W.r0 + r;
    j = W.c0 + c;
  }
}

// 64-bit words along a band window for a lattice side n: the whole padded
// side if it fits in shared memory, else as many as fit.
__host__ __device__ __forceinline__ int band_words(long long n, int pad) {
  const long long full = (n + 2 * pad + 63) / 64;
  const long long fit = (long long)((SMEM_MAX - sizeof(BigHeader)) / (3 * 8 * BAND_R));
  return (int)(full < fit ? full : fit);
}

__global__ void __launch_bounds__(BT) k_claim_big(Grid g, const double* __restrict__ tay,
                                                  unsigned long long* __restrict__ keys, DevState* ds,
                                                  const int2* __restrict__ list_in, const int* __restrict__ n_in,
                                                  int* __restrict__ stat, int2* __restrict__ list_out,
                                                  int* __restrict__ n_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BigHeader& H = *reinterpret_cast<BigHeader*>(smem_raw);
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(BigHeader));
  const int tid = threadIdx.x;
  const int pad = g.pad;
  const int n = *n_in;
  for (int item = blockIdx.x; item < n; item += gridDim.x) {
    const int m = list_in[item].x;
    const int sides = list_in[item].y >> 4, attempt = list_in[item].y & 15;
    const int mode = mode_for(sides, attempt);
    load_T9(g, m, tay, H.T9, H.ex9);
    __syncthreads();
    const double us = dmul(dsub(H.T9[4][TY_X], g.x_lo), g.inv_dx);
    const double ws = dmul(dsub(H.T9[4][TY_V], g.v_lo), g.inv_dv);
    const long long i0 = (long long)floor(dadd(us, 0.5)), j0 = (long long)floor(dadd(ws, 0.5));
    Win W;
    W.trans = (mode == MODE_BAND_X);
    const long long along0 = W.trans ? i0 : j0, across0 = W.trans ? j0 : i0;
    W.nrow_lat = W.trans ? g.nv : g.nx;
    W.ncol_lat = W.trans ? g.nx : g.nv;
    if (mode == MODE_FAT) {
      W.R = FAT_R;
      W.W = FAT_W;
      W.r0 = across0 - FAT_R / 2;
      W.c0 = along0 - 32 * FAT_W;
    } else {
      W.R = BAND_R;
      W.W = band_words(W.ncol_lat, pad);
      W.r0 = across0 - BAND_R / 2;
      // centred on the start, kept inside the padded lattice
      long long c0 = along0 - 32ll * W.W;
      const long long hi = W.ncol_lat + pad - 64ll * W.W;
      if (c0 > hi) c0 = hi;
      if (c0 < -pad) c0 = -pad;
      W.c0 = c0;
    }
    const int COLS = 64 * W.W;
    W.clo = (int)max(0ll, (long long)(-pad) - W.c0);
    W.chi = (int)min((long long)COLS, W.ncol_lat + pad - W.c0);
    W.rlo = (int)max(0ll, (long long)(-pad) - W.r0);
    W.rhi = (int)min((long long)W.R, W.nrow_lat + pad - W.r0);
    const int NW = W.R * W.W;
    unsigned long long* comp = bits;
    unsigned long long* eval = bits + NW;
    unsigned long long* pass = bits + 2 * NW;
    for (int q = tid; q < 3 * NW; q += BT) bits[q] = 0ull;
    if (tid == 0) {
      H.ok = 0;
      H.esc = 0;
    }
    __syncthreads();
    const int rs = (int)(across0 - W.r0), cs = (int)(along0 - W.c0);
    if (tid == 0) {
      double d2;
      const bool ok = pass_test(g, H.T9, H.ex9, site_x(g, i0), site_v(g, j0), d2);
      const int q = rs * W.W + (cs >> 6);
      eval[q] |= 1ull << (cs & 63);
      if (ok) {
        pass[q] |= 1ull << (cs & 63);
        comp[q] |= 1ull << (cs & 63);
        claim_site(g, keys, i0, j0, d2, m);
      }
      H.ok = ok;
    }
    __syncthreads();
    if (H.ok) {
      for (int it = 0; it < NW * 64; it++) {
        if (tid == 0) {
          H.nlist = 0;
          H.active = 0;
        }
        __syncthreads();
        // A: growth candidates of every word; words needing evaluation are listed
        bool act = false;
        for (int q = tid; q < NW; q += BT) {
          const int r = q / W.W, w = q - r * W.W;
          const unsigned long long c = comp[q];
          unsigned long long d = c | (c << 1) | (c >> 1);
          if (w > 0) d |= comp[q - 1] >> 63;
          if (w < W.W - 1) d |= comp[q + 1] << 63;
          if (r > 0) d |= comp[q - W.W];
          if (r < W.R - 1) d |= comp[q + W.W];
          const unsigned long long valid = (r >= W.rlo && r < W.rhi) ? col_mask(w, W.clo, W.chi) : 0ull;
          const unsigned long long gr = d & ~c & valid;
          if (gr & ~eval[q]) {
            act = true;
            const int slot = atomicAdd(&H.nlist, 1);
            if (slot < LIST_CAP) H.list[slot] = q;
          } else if (gr & pass[q]) {
            act = true;
          }
        }
        if (!__syncthreads_or(act)) break;
        // C: evaluate every still-unevaluated valid site of the listed words
        const int nl = min(H.nlist, LIST_CAP);
        for (int e = tid; e < nl * 64; e += BT) {
          const int q = H.list[e >> 6], b = e & 63;
          const int r = q / W.W, w = q - r * W.W;
          const unsigned long long valid = (r >= W.rlo && r < W.rhi) ? col_mask(w, W.clo, W.chi) : 0ull;
          if (!(((valid & ~eval[q]) >> b) & 1ull)) continue;
          long long i, j;
          site_of(W, r, 64 * w + b, i, j);
          double d2;
          if (pass_test(g, H.T9, H.ex9, site_x(g, i), site_v(g, j), d2))
            atomicOr(&pass[q], 1ull << b);
        }
        __syncthreads();
        for (int e = tid; e < nl; e += BT) {
          const int q = H.list[e];
          const int r = q / W.W, w = q - r * W.W;
          eval[q] |= (r >= W.rlo && r < W.rhi) ? col_mask(w, W.clo, W.chi) : 0ull;
        }
        __syncthreads();
        // D: extend the component through passing runs inside each word.  A
        // word may see its neighbours' growth of this same phase; that only
        // adds connected passing sites earlier, so the fixed point is the same.
        for (int q = tid; q < NW; q += BT) {
          const int r = q / W.W, w = q - r * W.W;
          const unsigned long long c = comp[q];
          unsigned long long d = c | (c << 1) | (c >> 1);
          if (w > 0) d |= comp[q - 1] >> 63;
          if (w < W.W - 1) d |= comp[q + 1] << 63;
          if (r > 0) d |= comp[q - W.W];
          if (r < W.R - 1) d |= comp[q + W.W];
          const unsigned long long seeds = d & ~c & pass[q];
          if (!seeds) continue;
          const unsigned long long nw = run_fill(seeds | c, pass[q]);
          unsigned long long add = nw & ~c;
          comp[q] = c | nw;
          while (add) {
            const int b = __ffsll((long long)add) - 1;
            add &= add - 1ull;
            long long i, j;
            site_of(W, r, 64 * w + b, i, j);
            if (i >= 0 && i < g.nx && j >= 0 && j < g.nv) {
              double xi, ze;
              const double d2 = dist2_exact(H.T9[4], g, site_x(g, i), site_v(g, j), xi, ze);
              claim_site(g, keys, i, j, d2, m);
            }
          }
        }
        __syncthreads();
      }
      // escaped this window as well?
      bool esc = false;
      for (int q = tid; q < NW; q += BT) {
        const unsigned long long c = comp[q];
        if (!c) continue;
        const int r = q / W.W, w = q - r * W.W;
        if (r == 0 && W.rlo == 0 && W.r0 - 1 >= -pad) esc = true;
        if (r == W.R - 1 && W.rhi == W.R && W.r0 + W.R < W.nrow_lat + pad) esc = true;
        if (w == 0 && (c & 1ull) && W.clo == 0 && W.c0 - 1 >= -pad) esc = true;
        if (w == W.W - 1 && (c >> 63) && W.chi == COLS && W.c0 + COLS < W.ncol_lat + pad) esc = true;
      }
      if (__syncthreads_or(esc) && tid == 0) {
        if (list_out != nullptr) {
          const int slot = atomicAdd(n_out, 1);
          list_out[slot] = make_int2(m, (sides << 4) | (attempt + 1));
        } else {
          atomicOr(&ds->err, ERR_PATCH_OVERFLOW);
        }
      }
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && tid == 0) *stat = n;
}

// Keys -> map; reset keys for the next map; list the unclaimed sites.
__global__ void k_finalize(Grid g, unsigned long long* __restrict__ keys, int32_t* __restrict__ map,
                           int32_t* __restrict__ holes, DevState* ds) {
  const size_t n = (size_t)g.nx * g.nv;
  const ulonglong2 empty = make_ulonglong2(KEY_EMPTY, KEY_EMPTY);
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const ulonglong2 kv = reinterpret_cast<ulonglong2*>(keys)[p];
    int32_t m = -1;
    if (kv.y == KEY_EMPTY && kv.x == KEY_EMPTY) {
      const int slot = atomicAdd(&ds->nholes, 1);
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
        const unsigned long long key = dkey(dist2_exact(tay + (size_t)cand * TY_N, g, Px, Pv, xi, ze));
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
        const int slot = atomicAdd(&next_s, 1);
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

size_t big_smem_bytes(const Grid& g) {
  long long nw = FAT_R * FAT_W;
  nw = max(nw, (long long)BAND_R * band_words(g.nv, g.pad));
  nw = max(nw, (long long)BAND_R * band_words(g.nx, g.pad));
  return sizeof(BigHeader) + 3 * (size_t)nw * sizeof(unsigned long long);
}

}  // namespace

// Opt the large-window kernel in to the shared memory its windows need.
bool map_prepare(const Grid& g) {
  const size_t need = big_smem_bytes(g);
  if (need > SMEM_MAX) return false;
  return cudaFuncSetAttribute(k_claim_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need) == cudaSuccess;
}

void launch_map(vm_solver* s) {
  // counters: nholes, holes_found, hole_rounds, noverflow, overflow_stat, noverflow2,
  // overflow2_stat, noverflow3, overflow3_stat
  int ps = prof_begin(s, KID_MAP_CLEAR);
  cudaMemsetAsync(&s->ds->nholes, 0, 9 * sizeof(int32_t), s->stream);
  prof_end(s, ps);
  ps = prof_begin(s, KID_CLAIM_SMALL);
  k_claim_small<<<s->g.ne, ST, 0, s->stream>>>(s->g, s->tay, s->keys, s->ds, s->overflow_list);
  prof_end(s, ps);
  const size_t smem = big_smem_bytes(s->g);
  ps = prof_begin(s, KID_CLAIM_LARGE);
  DevState* d = s->ds;
  k_claim_big<<<2 * 152, BT, smem, s->stream>>>(s->g, s->tay, s->keys, d, s->overflow_list, &d->noverflow,
                                                &d->overflow_stat, s->overflow_list2, &d->noverflow2);
  k_claim_big<<<152, BT, smem, s->stream>>>(s->g, s->tay, s->keys, d, s->overflow_list2, &d->noverflow2,
                                            &d->overflow2_stat, s->overflow_list, &d->noverflow3);
  k_claim_big<<<152, BT, smem, s->stream>>>(s->g, s->tay, s->keys, d, s->overflow_list, &d->noverflow3,
                                            &d->overflow3_stat, nullptr, nullptr);
  prof_end(s, ps);
  unsigned nb = (unsigned)((s->n + 255) / 256);
  if (nb > 152 * 16) nb = 152 * 16;
  ps = prof_begin(s, KID_FINALIZE);
  k_finalize<<<nb, 256, 0, s->stream>>>(s->g, s->keys, s->map, s->holes_a, s->ds);
  prof_end(s, ps);
  ps = prof_begin(s, KID_HOLES);
  k_holes<<<1, HT, 0, s->stream>>>(s->g, s->tay, s->map, s->holes_a, s->holes_b, s->holes_b + s->n, s->ds);
  prof_end(s, ps);
  s->launches += 6;
}

}  // namespace vm
