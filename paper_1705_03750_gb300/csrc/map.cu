// Influence map of the elements of metric (Sec. 2.3.1).
//
// Element-parallel percolation: the claimed set of element m is the
// 4-connected component, containing the grid site nearest to P_m, of the
// sites that pass m's test (no investigated neighbour proposes a strictly
// smaller d).  Each element is flood-filled inside a window of bit masks
// (tested / passing / component), sized in tiers:
//
//   0. a 16 x 32 window per half warp (one 32-bit row per half-lane), two
//      elements per warp; nearly every component fits.  Its escapes go to
//      tier 1, except outer elements (a neighbour missing), which claim
//      boundary bands and go straight to tier 2 with tier 0's masks;
//   1. a 32 x 64 window held in registers (one 64-bit row per lane), one
//      warp per element.  Both tiers run the same rounds: the first tests
//      the region predicted by the linear part of the element's map (its
//      inner part, where a bound on the second-order terms shows that every
//      site passes, needs no test);
//      the component is then closed through the passing sites by shuffle
//      scans, and further rounds test only sites next to it left untested
//      (the 32 lanes share a round's tests: lane e of a pass takes the
//      e-th untested site, found by a search of the rows' counts);
//   2. for the elements whose component reached the edge of tier 1, up to
//      two attempts with larger windows in shared memory, in an order set by
//      the sides it escaped from (a band window 128 sites across and up to
//      1280 along v or along x, or a 160 x 768 window), the first starting
//      from tier 1's masks of the element; then
//   3. the whole padded lattice, its masks in global memory.
//      Outer-layer elements whose neighbours moved away claim long thin
//      bands; to cross them in few rounds, any 64-site word near the
//      component is tested whole (three rows ahead, one word ahead) and the
//      component is extended through runs of passing sites inside a word
//      with one carry-propagating addition.
//
// A window whose component reaches its edge claims nothing: the next, larger
// window's component contains it.  Claims are made once the component is
// final, with several atomic exchanges in flight per thread.
//
// Decisions.  The percolation's outcome is fixed by FP64 values evaluated in
// one operation order (the exact test).  Each test is first run in FP32 in
// element units together with a rigorous bound on the distance between the
// FP32 value and the FP64 one (forward error of the evaluation, <= gamma_k
// times the same expression on absolute values, bounded per element by
// C1 |p| + C2 |p|^2); the FP32 result is used only when every range and
// distance comparison clears its bound, otherwise the exact FP64 test runs.
// The outcome is therefore identical to the all-FP64 evaluation.
//
// Claims.  A claimed site's owner slot takes (epoch << 24 | m) with one
// atomic exchange.  A claim that displaces a current-epoch owner folds into
// the site's record (a 128-bit key per site, empty between maps), by a
// 128-bit compare-and-swap minimum, the exact FP64 keys (bits of d^2,
// element index) of the displaced owner and of itself, and lists the site
// for resolution if it is the first to flag it (second slot = epoch): every
// claimant of a contested site reaches the record, so its minimum is the
// exact winner, and FP64 work is spent only on contested sites.
// Unclaimed sites are repaired in Jacobi rounds from their 4-neighbours.
#include <math.h>

#include <algorithm>
#include <climits>

#include "common.cuh"

namespace vm {
namespace {

// ---------------------------------------------------------------------------
// exact FP64 test
// ---------------------------------------------------------------------------

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

// Percolation test of site P for the centre element of a 3x3 block of FP64
// Taylor records (index 4).
__device__ __noinline__ bool pass_exact(const Grid& g, const double (*T9)[TY_N], const int* ex9, double Px, double Pv) {
  double xi, ze;
  const double d2 = dist2_exact(T9[4], g, Px, Pv, xi, ze);
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

// ---------------------------------------------------------------------------
// FP32 test with certified decisions
// ---------------------------------------------------------------------------

// Bound constants: a monomial of the FP32 q passes through at most ~22
// roundings (its coefficient, computed in FP32 from the FP64 terms, up to
// ten; the inputs p about four, twice in a square; three fused operations):
// gamma_22(2^-24) < 1.4e-6 against 2e-6.  d^2 then errs by at most about
// 2 gamma_22 + 2 ulp relative to the squared bounds: < 2.8e-6 against 4e-6.
// The absolute term covers the last-bit differences between the FP32 inputs'
// source values and the FP64 evaluation's own inputs.
constexpr float kRelQ = 2.0e-6f, kRelD = 4.0e-6f, kAbs = 1.0e-9f;

struct QF {
  float qx, qv, ax, av;  // offset in element units and bounds of |terms|
};

__device__ __forceinline__ QF qeval(const float* __restrict__ F, float px, float pv) {
  QF r;
  // (scalar loads from shared memory: in the tier-1 test loop 16-byte loads
  // cost more registers than they save issue slots)
  const float tx = fmaf(F[TF_AX], px, fmaf(F[TF_BX], pv, F[TF_T00])), ux = fmaf(F[TF_CX], pv, F[TF_T01]);
  const float tv = fmaf(F[TF_AV], px, fmaf(F[TF_BV], pv, F[TF_T10])), uv = fmaf(F[TF_CV], pv, F[TF_T11]);
  r.qx = fmaf(px, tx, pv * ux);
  r.qv = fmaf(px, tv, pv * uv);
  const float P = fmaxf(fabsf(px), fabsf(pv));
  r.ax = F[TF_C1X] * P + F[TF_C2X] * (P * P);
  r.av = F[TF_C1V] * P + F[TF_C2V] * (P * P);
  return r;
}

// Range of one axis from q with |q - r| <= e, r the FP64 value: 1 = {-1,0},
// 2 = {0}, 3 = {0,1}, 0 = cannot tell.
__device__ __forceinline__ int range_f(float q, float e, float alo, float ahi) {
  if (q + e < -ahi) return 1;
  if (q - e >= -alo && q + e < alo) return 2;
  if (q - e >= ahi) return 3;
  return 0;
}

// The map reads words 0-15 of the FP32 records (TF_MW, as four float4).
// Their shared-memory copies have a stride of 20 words, so that lanes
// evaluating different neighbours read the same word from different banks.
constexpr int TF_M = 20, TF_MW = 16;
static_assert(TF_C2V < TF_MW && TF_MW <= TF_M && TF_M % 4 == 0, "map's FP32 record words");

struct Ctx9 {
  const float (*F9)[TF_M];
  const int* ex9;
  const float* offu;  // (i0 - u_m') for the 9 elements, i0 the window's start site
  const float* offv;
  float inv_s, alo, ahi;
};

// 1: passes, 0: fails; negative: the bound does not settle it (run the exact
// test).  -1: the alpha ranges themselves are open, or (kOpen false) some
// comparison is; with kOpen, -2 - mask: the ranges are settled and only the
// comparisons with the neighbours in `mask` (bit q) are open, every other
// neighbour being certainly not closer (the windows' tiers, whose rare
// fallbacks are cheaper than carrying the mask, stop at the first open one).
template <bool kOpen = false>
__device__ __forceinline__ int pass_f32(const Ctx9& c, float di, float dj) {
  const QF m = qeval(c.F9[4], (di + c.offu[4]) * c.inv_s, (dj + c.offv[4]) * c.inv_s);
  const float ex = kRelQ * m.ax + kAbs * (1.f + m.ax), ev = kRelQ * m.av + kAbs * (1.f + m.av);
  const int ra = range_f(m.qx, ex, c.alo, c.ahi), rb = range_f(m.qv, ev, c.alo, c.ahi);
  if (!ra || !rb) return -1;
  if (ra == 2 && rb == 2) return 1;  // inside the alpha box on both axes: no neighbour to ask
  const float d2 = m.qx * m.qx + m.qv * m.qv;
  const float A2 = m.ax * m.ax + m.av * m.av;
  const float e2 = kRelD * A2 + kAbs * (1.f + A2);
  // The neighbours to compare with: (A, 0), (0, B) and (A, B) for the
  // nonzero ones of A, B (the side of the alpha box q leaves on each axis).
  // At most three evaluations, in one loop whose trip count is the only
  // thing that differs between lanes.
  const int A = ra - 2, B = rb - 2;
  const int qa = (A + 1) * 3 + 1, qb = 3 + (B + 1), qab = (A + 1) * 3 + (B + 1);
  const int cnt = (A != 0 && B != 0) ? 3 : 1;
  int open = 0;  // (kOpen) neighbours whose comparison the bound leaves open
  for (int t = 0; t < cnt; t++) {
    const int q = (t == 0) ? (A != 0 ? qa : qb) : (t == 1 ? qb : qab);
    if (!c.ex9[q]) continue;
    const QF n = qeval(c.F9[q], (di + c.offu[q]) * c.inv_s, (dj + c.offv[q]) * c.inv_s);
    const float d2n = n.qx * n.qx + n.qv * n.qv;
    const float An = n.ax * n.ax + n.av * n.av;
    const float en = kRelD * An + kAbs * (1.f + An);
    if (d2n + en < d2 - e2) return 0;
    if (!(d2n - en >= d2 + e2)) {
      if (!kOpen) return -1;
      open |= 1 << q;
    }
  }
  return open ? -2 - open : 1;
}

// ---------------------------------------------------------------------------
// claims
// ---------------------------------------------------------------------------

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

// key2[0] = element index, key2[1] = bits of d^2: as a 128-bit integer its
// order is the claim order (smaller d, then smaller index).
__device__ __forceinline__ void key_min(unsigned long long* key2, unsigned long long dbits, unsigned long long idx) {
  ulonglong2 cur = __ldcg(reinterpret_cast<const ulonglong2*>(key2));
  const ulonglong2 val = make_ulonglong2(idx, dbits);
  while (dbits < cur.y || (dbits == cur.y && idx < cur.x)) {
    const ulonglong2 prev = cas128(key2, cur, val);
    if (prev.x == cur.x && prev.y == cur.y) break;
    cur = prev;
  }
}

struct Slots {
  uint32_t* slot0;
  uint32_t* slot1;
  unsigned long long* rec_key;
  int32_t* rec_site;
  int rec_cap;
  const double* tay;
  DevState* ds;
  uint32_t epoch;  // filled in on the device from ds->epoch
  // tier 1's masks of escaped elements (32 rows x {component, tested,
  // passing}), handed to tier 2's first window; seed_cap records at most
  unsigned long long* seed;
  int seed_cap;
};

// The map's epoch lives on the device (so that a captured step replays
// correctly): every map kernel reads it once.
__device__ __forceinline__ Slots with_epoch(Slots S) {
  S.epoch = *(volatile uint32_t*)&S.ds->epoch;
  return S;
}

// Start of a map: next epoch, counters cleared.
__device__ __forceinline__ void map_begin_body(DevState* ds) {
  {
    ds->epoch = (ds->epoch + 1) % kEpochs;
    ds->nholes = ds->holes_found = ds->hole_rounds = 0;
    ds->noverflow = ds->overflow_stat = ds->noverflow2 = ds->overflow2_stat = 0;
    ds->noverflow3 = ds->overflow3_stat = 0;
    ds->nrec = 0;
    ds->t1_more = 0;
    ds->n_exact = 0;
    ds->take[0] = ds->take[1] = ds->take[2] = 0;
    ds->noverflow_back = 0;
    ds->nseed = 0;
    ds->n_pair_esc = 0;
    ds->emap2_bits = 0ull;  // E_map describes the current map only
    ds->emap_hit = 0;
  }
}

__global__ void k_map_begin(DevState* ds, const int32_t* gate) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && !(gate != nullptr && __ldcg(gate) == 0)) map_begin_body(ds);
}

__device__ __noinline__ void contest(const Slots& S, const Grid& g, long long i, long long j, size_t p, int m,
                                     uint32_t displaced) {
  const uint32_t E = S.epoch;
  // The site's record is its own 128-bit key slot, empty between maps.  The
  // claimant that first flags the site in this map's epoch lists it for the
  // resolution (each site at most once per map).
  const uint32_t rs = __ldcg(&S.slot1[p]);
  if ((rs >> 24) != E && atomicCAS(&S.slot1[p], rs, E << 24) == rs) {
    const int r = atomicAdd(&S.ds->nrec, 1);
    if (r < S.rec_cap)
      S.rec_site[r] = (int32_t)p;
    else
      atomicOr(&S.ds->err, ERR_PATCH_OVERFLOW);  // (cannot happen: rec_cap is the site count)
  }
  unsigned long long* key = S.rec_key + 2 * p;
  const double Px = site_x(g, i), Pv = site_v(g, j);
  double xi, ze;
  const int mo = (int)(displaced & SLOT_MASK);
  if (mo >= g.ne || p >= (size_t)g.nx * g.nv) {
    VM_BAD(S.ds, 1);
    return;
  }
  key_min(key, dkey(dist2_exact(S.tay + (size_t)mo * TY_N, g, Px, Pv, xi, ze)), (unsigned long long)mo);
  key_min(key, dkey(dist2_exact(S.tay + (size_t)m * TY_N, g, Px, Pv, xi, ze)), (unsigned long long)m);
}

// Claims of up to N sites (pos: row-major site index, or ~0 for none) with
// all N exchanges issued before any result is looked at.
template <int N>
__device__ __forceinline__ void claim_sites(const Slots& S, const Grid& g, const size_t (&pos)[N], int m) {
  const uint32_t tag = (S.epoch << 24) | (uint32_t)m;
  uint32_t old[N];
#pragma unroll
  for (int u = 0; u < N; u++) old[u] = (pos[u] != ~(size_t)0) ? atomicExch(&S.slot0[pos[u]], tag) : tag;
#pragma unroll
  for (int u = 0; u < N; u++) {
    // first claimant this map, or the same element again: nothing to resolve
    if ((old[u] >> 24) != S.epoch || old[u] == tag) continue;
    const long long i = (long long)(pos[u] / (size_t)g.nv), j = (long long)(pos[u] - (size_t)i * g.nv);
    contest(S, g, i, j, pos[u], m, old[u]);
  }
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

enum : int { MODE_BAND_V = 0, MODE_BAND_X = 1, MODE_FAT = 2, MODE_GLOBAL = 3 };

// Shared part of every window: the element's 3x3 neighbourhood in FP64 and
// FP32, and the FP32 offsets of their positions from the start site.
struct Elem9 {
  double T9[9][TY_N];
  float F9[9][TF_M];
  int ex9[9];
  float offu[9], offv[9];
};

__device__ __forceinline__ void load_elem9(const Grid& g, int m, const double* __restrict__ tay,
                                           const float* __restrict__ tayf, Elem9& E) {
  const int k = m / g.Lv, l = m - k * g.Lv;
  for (int idx = threadIdx.x; idx < 9 * TY_N; idx += blockDim.x) {
    const int q = idx / TY_N, c = idx - q * TY_N;
    const int kk = k + q / 3 - 1, ll = l + q % 3 - 1;
    const bool ex = elem_exists(g, kk, ll);
    E.T9[q][c] = ex ? tay[(size_t)(kk * g.Lv + ll) * TY_N + c] : 0.0;
    if (c == 0) E.ex9[q] = ex;
  }
  for (int idx = threadIdx.x; idx < 9 * TF_MW; idx += blockDim.x) {
    const int q = idx / TF_MW, c = idx - q * TF_MW;
    const int kk = k + q / 3 - 1, ll = l + q % 3 - 1;
    const bool ex = elem_exists(g, kk, ll);
    E.F9[q][c] = ex ? tayf[(size_t)(kk * g.Lv + ll) * TF_N + c] : 0.f;
  }
}

__device__ __forceinline__ bool start_site(const Grid& g, const Elem9& E, long long& i0, long long& j0) {
  const double us = E.T9[4][TY_U], ws = E.T9[4][TY_W];
  if (!(us > -1e9 && us < 1e9 && ws > -1e9 && ws < 1e9)) return false;
  i0 = (long long)floor(dadd(us, 0.5));
  j0 = (long long)floor(dadd(ws, 0.5));
  return !(i0 < -g.pad || i0 >= g.nx + g.pad || j0 < -g.pad || j0 >= g.nv + g.pad);
}

// Offsets i0 - u_m' of the neighbourhood (FP64 difference, then FP32).
__device__ __forceinline__ void set_offsets(Elem9& E, long long i0, long long j0) {
  const int q = threadIdx.x;
  if (q < 9) {
    E.offu[q] = E.ex9[q] ? (float)((double)i0 - E.T9[q][TY_U]) : 0.f;
    E.offv[q] = E.ex9[q] ? (float)((double)j0 - E.T9[q][TY_W]) : 0.f;
  }
}

__device__ __forceinline__ Ctx9 ctx_of(const Grid& g, const Elem9& E, float alo, float ahi) {
  Ctx9 c;
  c.F9 = E.F9;
  c.ex9 = E.ex9;
  c.offu = E.offu;
  c.offv = E.offv;
  c.inv_s = 1.0f / (float)g.s;
  c.alo = alo;
  c.ahi = ahi;
  return c;
}

// The exact test restricted to the neighbours whose comparison the FP32
// bound left open, the alpha ranges being settled: the other neighbours of
// the ranges are certainly not closer, so the outcome is the full test's.
__device__ __noinline__ bool pass_exact_open(const Grid& g, const double (*T9)[TY_N], int open, double Px,
                                             double Pv) {
  double xi, ze;
  const double d2 = dist2_exact(T9[4], g, Px, Pv, xi, ze);
  for (int q = 0; q < 9; q++) {
    if (!((open >> q) & 1)) continue;
    double x2, z2;
    if (dist2_exact(T9[q], g, Px, Pv, x2, z2) < d2) return false;
  }
  return true;
}

// Test of one site in the large windows: their band sites far from the
// element leave comparisons open far more often than the small windows'.
// The exact test of site (i, j) after the FP32 test left it open with
// result r (-1: every neighbour of the ranges; -2 - mask: those in mask).
__device__ __forceinline__ bool exact_open(const Grid& g, const Elem9& E, int r, long long i, long long j) {
  if (r == -1) return pass_exact(g, E.T9, E.ex9, site_x(g, i), site_v(g, j));
  return pass_exact_open(g, E.T9, -2 - r, site_x(g, i), site_v(g, j));
}

__device__ __forceinline__ bool test_site(const Grid& g, const Elem9& E, const Ctx9& c, long long i0, long long j0,
                                          long long i, long long j) {
  const int r = pass_f32<true>(c, (float)(int)(i - i0), (float)(int)(j - j0));
  if (r >= 0) return r == 1;
  return exact_open(g, E, r, i, j);
}

// ---------------------------------------------------------------------------
// tier 1: 32 x 64 window held in registers, one warp per element
// ---------------------------------------------------------------------------

constexpr int TR = 32, TCAP = 256, TE = 4;  // rows (one per lane), list capacity, elements per block
constexpr unsigned FULL = 0xffffffffu;

// The exact test of site (i, j) for element (k, l), FP64 records read from
// global memory (the rare fallback of the FP32 test).
__device__ __noinline__ bool pass_exact_g(const Grid& g, const double* __restrict__ tay, int k, int l, double Px,
                                          double Pv) {
  double xi, ze;
  const double d2 = dist2_exact(tay + (size_t)(k * g.Lv + l) * TY_N, g, Px, Pv, xi, ze);
  int a0, a1, b0, b1;
  alpha_range(xi, g.alpha, a0, a1);
  alpha_range(ze, g.alpha, b0, b1);
  for (int a = a0; a <= a1; a++)
    for (int b = b0; b <= b1; b++) {
      if (a == 0 && b == 0) continue;
      const int kk = k + a, ll = l + b;
      if (!elem_exists(g, kk, ll)) continue;
      double x2, z2;
      if (dist2_exact(tay + (size_t)(kk * g.Lv + ll) * TY_N, g, Px, Pv, x2, z2) < d2) return false;
    }
  return true;
}

struct __align__(16) WarpShared {
  float F9[9][TF_M];
  int ex9[9];
  float offu[9], offv[9];
  unsigned long long passed[TR];  // passing sites found by one round, per window row
  unsigned long long unsure[TR];  // sites of the round the FP32 bound could not settle
  unsigned short item[TCAP];      // compacted list of the claims (lane << 6 | bit)
};

// Inclusive sum of v over the lanes of the warp.
__device__ __forceinline__ int warp_incl(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Bits of `comp` carried along the columns of the window (down and up the
// lanes) through vertical runs of `pass` (comp inside pass): a segmented
// OR-scan, log2(32) shuffle steps each way.
__device__ __forceinline__ unsigned long long vfill(unsigned long long comp, unsigned long long pass, int lane) {
  unsigned long long gd = comp, ad = pass, gu = comp, au = pass;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long g1 = __shfl_up_sync(FULL, gd, d), a1 = __shfl_up_sync(FULL, ad, d);
    const unsigned long long g2 = __shfl_down_sync(FULL, gu, d), a2 = __shfl_down_sync(FULL, au, d);
    if (lane >= d) {
      gd |= g1 & ad;
      ad &= a1;
    }
    if (lane + d < 32) {
      gu |= g2 & au;
      au &= a2;
    }
  }
  return gd | gu;
}

// Position of the n-th set bit (from 0, counted from bit 0) of x; x has
// more than n set bits.
__device__ __forceinline__ int nth_bit(unsigned long long x, int n) {
  int pos = 0;
  unsigned w = (unsigned)x;
  int c = __popc(w);
  if (n >= c) { n -= c; pos = 32; w = (unsigned)(x >> 32); }
  c = __popc(w & 0xFFFFu); if (n >= c) { n -= c; pos += 16; w >>= 16; }
  c = __popc(w & 0xFFu); if (n >= c) { n -= c; pos += 8; w >>= 8; }
  c = __popc(w & 0xFu); if (n >= c) { n -= c; pos += 4; w >>= 4; }
  c = __popc(w & 0x3u); if (n >= c) { n -= c; pos += 2; w >>= 2; }
  if (n >= (int)(w & 1u)) pos += 1;
  return pos;
}

// Write the positions of the set bits of `bits` (one word per lane) with
// list index in [b0, b0 + TCAP) to the list; excl / incl: the lane's range.
__device__ __forceinline__ void list_chunk(unsigned short* item, unsigned long long bits, int excl, int incl, int b0,
                                           int lane) {
  if (excl >= b0 + TCAP || incl <= b0) return;
  int idx = excl;
  while (bits) {
    const int b = __ffsll((long long)bits) - 1;
    bits &= bits - 1ull;
    if (idx >= b0 + TCAP) break;
    if (idx >= b0) item[idx - b0] = (unsigned short)((lane << 6) | b);
    idx++;
  }
}

// Lane r owns window row r: its component / tested / passing bits are three
// 64-bit registers.  The first round tests the sites of the region the
// linear part of the map predicts (its parallelogram, widened by one site
// and by a bound on the second-order terms); every round then closes the
// component through all sites known to pass (vertical scan + horizontal
// runs, to a fixed point) and tests the sites next to it not yet tested.
// The 32 lanes share a round's tests (the e-th test of a pass goes to
// lane e, whatever row holds it).  The order of the
// tests does not change the result: the component is the connected set of
// passing sites reached from the start, and the loop ends only when every
// site next to it has been tested.  Claims are made once at the end.
__device__ __forceinline__ void claim_element(const Grid& g, const double* __restrict__ tay,
                                              const float* __restrict__ tayf, const Slots& S, float alo, float ahi,
                                              int2* __restrict__ ovf_list, WarpShared& sh, int lane, int m);

// One element per warp, the elements whose component escaped tier 0's
// window (list of n_in entries).  (A warp-strided loop that prefetched the
// next element's records cut the set-up latency but cost more in register
// spills than it saved.)
__device__ __forceinline__ void claim_small_body(const Grid& g, const double* __restrict__ tay,
                                                         const float* __restrict__ tayf, Slots Sin, float alo,
                                                         float ahi, int2* __restrict__ ovf_list,
                                                         const int32_t* __restrict__ list_in,
                                                         const int* __restrict__ n_in, int vb, int vg) {
  __shared__ WarpShared shw[TE];
  const Slots S = with_epoch(Sin);
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int n = *n_in;
  for (int idx = vb * TE + wq; idx < n; idx += vg * TE) {
    const int m = list_in[idx];
    if (m < 0 || m >= g.ne) {  // (never expected; keeps every index in bounds)
      if (lane == 0) VM_BAD(S.ds, 6);
      continue;
    }
    claim_element(g, tay, tayf, S, alo, ahi, ovf_list, shw[wq], lane, m);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32 * TE, 8) k_claim_small(Grid g, const double* __restrict__ tay,
                                                         const float* __restrict__ tayf, Slots Sin, float alo,
                                                         float ahi, int2* __restrict__ ovf_list,
                                                         const int32_t* __restrict__ list_in,
                                                         const int* __restrict__ n_in) {
  if (gate_shut(g)) return;
  claim_small_body(g, tay, tayf, Sin, alo, ahi, ovf_list, list_in, n_in, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void claim_element(const Grid& g, const double* __restrict__ tay,
                                              const float* __restrict__ tayf, const Slots& S, float alo, float ahi,
                                              int2* __restrict__ ovf_list, WarpShared& sh, int lane, int m) {
  const int k = m / g.Lv, l = m - k * g.Lv;
  // The 3x3 neighbourhood's FP64 index positions (lanes 0-8) and FP32
  // records (16 bytes per lane and load): every load issued before any is
  // used, so the set-up costs one memory round trip.
  double uq = 0.0, wpos = 0.0;
  bool exq = false;
  if (lane < 9) {
    const int kk = k + lane / 3 - 1, ll = l + lane % 3 - 1;
    exq = elem_exists(g, kk, ll);
    if (exq) {
      const double2 uw = __ldg(reinterpret_cast<const double2*>(tayf + (size_t)(kk * g.Lv + ll) * TF_N + TF_UD));
      uq = uw.x;
      wpos = uw.y;
    }
  }
  for (int idx = lane; idx < 9 * (TF_MW / 4); idx += 32) {
    const int q = idx / (TF_MW / 4), c4 = idx - q * (TF_MW / 4);
    const int kk = k + q / 3 - 1, ll = l + q % 3 - 1;
    const bool ex = elem_exists(g, kk, ll);
    const float4 v = ex ? __ldg(reinterpret_cast<const float4*>(tayf + (size_t)(kk * g.Lv + ll) * TF_N) + c4)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
    reinterpret_cast<float4*>(sh.F9[q])[c4] = v;
    if (c4 == 0) sh.ex9[q] = ex;
  }
  // start site (FP64 index position of P_m: lane 4 holds the centre)
  const double us = __shfl_sync(FULL, uq, 4), ws = __shfl_sync(FULL, wpos, 4);
  if (!(us > -1e9 && us < 1e9 && ws > -1e9 && ws < 1e9)) return;
  const long long i0 = (long long)floor(dadd(us, 0.5)), j0 = (long long)floor(dadd(ws, 0.5));
  const int pad = g.pad;
  if (i0 < -pad || i0 >= g.nx + pad || j0 < -pad || j0 >= g.nv + pad) return;
  if (lane < 9) {
    sh.offu[lane] = exq ? (float)((double)i0 - uq) : 0.f;
    sh.offv[lane] = exq ? (float)((double)j0 - wpos) : 0.f;
  }
  __syncwarp();
  Ctx9 c;
  c.F9 = sh.F9;
  c.ex9 = sh.ex9;
  c.offu = sh.offu;
  c.offv = sh.offv;
  c.inv_s = 1.0f / (float)g.s;
  c.alo = alo;
  c.ahi = ahi;
  const long long r0 = i0 - TR / 2, c0 = j0 - 32;
  const long long irow = r0 + lane;
  const int clo = (int)max(0ll, (long long)(-pad) - c0);
  const int chi = (int)min(64ll, (long long)(g.nv + pad) - c0);
  const unsigned long long valid = (irow >= -pad && irow < g.nx + pad) ? col_mask(0, clo, chi) : 0ull;
  // test of window site (row wr, column wb); offsets from the start in
  // 32-bit integers (a 64-bit conversion would take the FP64 pipe)
  // FP32 test of window site (row wr, column wb): 1 passes, 0 fails, -1 the
  // bound does not settle it (the exact test runs after the round, outside
  // the test loop, so that the loop makes no call).  Offsets from the start
  // in 32-bit integers (a 64-bit conversion would take the FP64 pipe).
  auto test = [&](int wr, int wb) -> int { return pass_f32(c, (float)(wr - TR / 2), (float)(wb - 32)); };
  // The start site decides whether there is a component at all; it is
  // tested with the first round (or certified with the inner sites).
  unsigned long long comp = 0ull, tested = 0ull, passing = 0ull;
  const unsigned long long seedbit = (lane == TR / 2) ? (1ull << 32) : 0ull;

  // predicted region, row by row: |T p|_x <= hx and |T p|_v <= hv for the
  // columns of this lane's row (p in element units).  Its inner part (the
  // sites expected well inside the alpha box, whose tests compare with no
  // neighbour) is listed first, so that the lanes of one pass of the tests
  // mostly take the same path.
  unsigned long long fa, fb;
  {
    const float* F = sh.F9[4];
    const float T00 = F[TF_T00], T01 = F[TF_T01], T10 = F[TF_T10], T11 = F[TF_T11];
    const float inv_s = c.inv_s, sf = (float)g.s;
    const float det = fabsf(T00 * T11 - T01 * T10);
    const float ext = (det > 1e-20f) ? fmaxf(fabsf(T11) + fabsf(T01), fabsf(T10) + fabsf(T00)) * __frcp_rn(det) : 0.f;
    const float P = 0.6f * ext + inv_s;
    const float sx = F[TF_C2X] * P * P, sv = F[TF_C2V] * P * P;
    const float hx = 0.52f + 1.1f * fmaxf(fabsf(T00), fabsf(T01)) * inv_s + sx;
    const float hv = 0.52f + 1.1f * fmaxf(fabsf(T10), fabsf(T11)) * inv_s + sv;
    const float ix = alo - 0.02f - sx, iv = alo - 0.02f - sv;
    const float px = ((float)(lane - TR / 2) + sh.offu[4]) * inv_s;
    const float r01 = (fabsf(T01) > 1e-20f) ? __frcp_rn(T01) : 0.f, r11 = (fabsf(T11) > 1e-20f) ? __frcp_rn(T11) : 0.f;
    // columns b with |a + cf * pv(b)| <= h for both rows of T, pv(b) = (b - 32 + offv) / s
    auto cols = [&](float h1, float h2) -> unsigned long long {
      float lo = -1e30f, hi = 1e30f;
      auto cut = [&](float a, float cf, float rcf, float h) {
        if (rcf != 0.f) {
          const float t1 = (-h - a) * rcf, t2 = (h - a) * rcf;
          lo = fmaxf(lo, fminf(t1, t2));
          hi = fminf(hi, fmaxf(t1, t2));
        } else if (!(fabsf(a) <= h)) {
          lo = 1e30f;
          hi = -1e30f;
        }
      };
      cut(T00 * px, T01, r01, h1);
      cut(T10 * px, T11, r11, h2);
      const float blo = fminf(fmaxf(lo * sf - sh.offv[4] + 32.f, -1.f), 65.f);
      const float bhi = fminf(fmaxf(hi * sf - sh.offv[4] + 32.f, -1.f), 65.f);
      const int ilo = max((int)ceilf(blo), 0), ihi = min((int)floorf(bhi), 63);
      return (ihi >= ilo) ? col_mask(0, ilo, ihi + 1) : 0ull;
    };
    const unsigned long long pred = (cols(hx, hv) | seedbit) & valid;
    unsigned long long inner = (ix > 0.f && iv > 0.f) ? cols(ix, iv) & pred : 0ull;
    // Inner sites need no test when it is certain that they pass: on them
    // |T p| <= alpha - 0.02 - sx (the interval above), and q differs from
    // T p by at most C2 P^2 (second-order terms, P = max |p| over the row's
    // inner run) plus roundings far below 1e-3 (of T, p, and the interval).
    // Then |q| < alpha on both axes: no neighbour is investigated, the site
    // passes (in the FP64 test as in the FP32 one).
    unsigned long long sure = 0ull;
    if (inner && fmaxf(fmaxf(fabsf(T00), fabsf(T01)), fmaxf(fabsf(T10), fabsf(T11))) < 50.f) {
      const int blo = __ffsll((long long)inner) - 1, bhi = 63 - __clzll((long long)inner);
      const float pvlo = ((float)(blo - 32) + sh.offv[4]) * inv_s, pvhi = ((float)(bhi - 32) + sh.offv[4]) * inv_s;
      const float Pr = fmaxf(fabsf(px), fmaxf(fabsf(pvlo), fabsf(pvhi)));
      if (F[TF_C2X] * Pr * Pr + 2e-3f <= 0.02f + sx && F[TF_C2V] * Pr * Pr + 2e-3f <= 0.02f + sv) sure = inner;
    }
    tested |= sure;
    passing |= sure;
    fa = pred & inner & ~sure;
    fb = pred & ~inner;
    // the owner slots the claims will exchange: towards L2 now (the first
    // and last in-grid site of this row's predicted run)
    const unsigned long long ing = pred & ((irow >= 0 && irow < g.nx) ? col_mask(0, (int)max(0ll, -c0),
                                                                               (int)min(64ll, (long long)g.nv - c0))
                                                                      : 0ull);
    if (ing) {
      const size_t rowp = (size_t)irow * g.nv + c0;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(S.slot0 + rowp + (__ffsll((long long)ing) - 1)));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(S.slot0 + rowp + (63 - __clzll((long long)ing))));
    }
  }
  int rounds = 0;
  for (int it = 0; it < TR * 64; it++) {
    // the sites to test: fa's listed before fb's
    const int ca = __popcll(fa), cb = __popcll(fb);
    const int inca = warp_incl(ca, lane), incb = warp_incl(cb, lane);
    const int ta = __shfl_sync(FULL, inca, 31);
    const int total = ta + __shfl_sync(FULL, incb, 31);
    // (the first pass always closes the component: certified sites may
    // already extend it with nothing left to test)
    if (total == 0 && it > 0) break;
    if (total > 0) rounds++;
    sh.passed[lane] = 0ull;
    sh.unsure[lane] = 0ull;
    __syncwarp();
    // Test e of the round (fa's sites, then fb's, row by row) is found by
    // a binary search of the lanes' inclusive counts (both lists' counts
    // packed in one word) and a select in the row's word.
    const unsigned incp = (unsigned)inca | ((unsigned)incb << 16);
    for (int e0 = 0; e0 < total; e0 += 32) {
      const int e = e0 + lane;
      const bool inA = e < ta;
      const int key = inA ? e : e - ta, sh16 = inA ? 0 : 16;
      int r = 0;
#pragma unroll
      for (int st = 16; st; st >>= 1) {
        const unsigned v = __shfl_sync(FULL, incp, r + st - 1);
        if ((int)((v >> sh16) & 0xFFFFu) <= key) r += st;
      }
      const unsigned vr = __shfl_sync(FULL, incp, r);
      const unsigned long long wa = __shfl_sync(FULL, fa, r), wb = __shfl_sync(FULL, fb, r);
      if (e < total) {
        const unsigned long long w = inA ? wa : wb;
        const int b = nth_bit(w, key - ((int)((vr >> sh16) & 0xFFFFu) - __popcll(w)));
        const int res = test(r, b);
        if (res == 1) atomicOr(&sh.passed[r], 1ull << b);
        if (res < 0) atomicOr(&sh.unsure[r], 1ull << b);
      }
    }
    __syncwarp();
    tested |= fa | fb;
    passing |= sh.passed[lane];
    // the exact FP64 test of this row's unsettled sites (rare)
    for (unsigned long long un = sh.unsure[lane]; un; un &= un - 1ull) {
      const int b = __ffsll((long long)un) - 1;
      atomicAdd(&S.ds->n_exact, 1);
      if (pass_exact_g(g, tay, k, l, site_x(g, irow), site_v(g, c0 + b))) passing |= 1ull << b;
    }
    if (it == 0) {
      if (!__shfl_sync(FULL, (unsigned)((passing >> 32) & 1ull), TR / 2)) return;  // the start fails
      comp = seedbit;
    }
    // close the component through every site known to pass
    for (int f = 0; f < TR * 64; f++) {
      const unsigned long long nc = run_fill(vfill(comp, passing, lane), passing);
      const bool grew = nc != comp;
      comp = nc;
      if (!__any_sync(FULL, grew)) break;
    }
    unsigned long long up = __shfl_up_sync(FULL, comp, 1), dn = __shfl_down_sync(FULL, comp, 1);
    if (lane == 0) up = 0ull;
    if (lane == TR - 1) dn = 0ull;
    fa = 0ull;
    fb = (comp | (comp << 1) | (comp >> 1) | up | dn) & ~comp & valid & ~tested;
  }
  if (rounds > 1 && lane == 0) atomicAdd(&S.ds->t1_more, 1);

  // Escaped the window?  Record on which sides, to pick the next window;
  // the larger window claims a superset of this component.
  const bool er = __any_sync(FULL, comp != 0ull && ((lane == 0 && r0 - 1 >= -pad) ||
                                                    (lane == TR - 1 && r0 + TR < g.nx + pad)));
  const bool ec = __any_sync(FULL, ((comp & 1ull) && clo == 0 && c0 - 1 >= -pad) ||
                                       ((comp >> 63) && chi == 64 && c0 + 64 < g.nv + pad));
  if (er || ec) {
    int seed = -1;
    if (lane == 0) {
      // Outer elements (a neighbour missing) that left along v claim the
      // long boundary bands, the longest jobs of the next tier: they are
      // listed from the front and taken first, the others from the end.
      const int sides = (er ? 1 : 0) | (ec ? 2 : 0);
      bool outer = false;
      for (int q = 0; q < 9; q++) outer |= !sh.ex9[q];
      const int slot = (outer && sides == 2) ? atomicAdd(&S.ds->noverflow, 1)
                                             : g.ne - 1 - atomicAdd(&S.ds->noverflow_back, 1);
      seed = atomicAdd(&S.ds->nseed, 1);
      if (seed >= S.seed_cap) seed = -1;
      // attempt 0; bits 8 and up: the masks' record + 1 (0: none)
      ovf_list[slot] = make_int2(m, ((seed + 1) << 8) | (sides << 4));
    }
    // the window's masks for the next tier (its first window starts from them)
    seed = __shfl_sync(FULL, seed, 0);
    if (seed >= 0) {
      unsigned long long* rec = S.seed + (size_t)seed * (3 * TR);
      rec[lane] = comp;
      rec[TR + lane] = tested;
      rec[2 * TR + lane] = passing;
    }
    return;
  }
  // claims: the component's sites compacted into the list, four exchanges
  // in flight per lane
  const int cnt = __popcll(comp);
  const int incl = warp_incl(cnt, lane);
  const int total = __shfl_sync(FULL, incl, 31);
  for (int b0 = 0; b0 < total; b0 += TCAP) {
    __syncwarp();
    list_chunk(sh.item, comp, incl - cnt, incl, b0, lane);
    __syncwarp();
    const int n = min(total - b0, TCAP);
    for (int e = lane; e < n; e += 4 * 32) {
      size_t pos[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int ee = e + 32 * u;
        pos[u] = ~(size_t)0;
        if (ee < n) {
          const int code = sh.item[ee];
          const long long i = r0 + (code >> 6), j = c0 + (code & 63);
          if (i >= 0 && i < g.nx && j >= 0 && j < g.nv) pos[u] = (size_t)i * g.nv + j;
        }
      }
      claim_sites(S, g, pos, m);
    }
  }
}

// ---------------------------------------------------------------------------
// tier 0: a 16 x 32 window per half warp, two elements per warp
// ---------------------------------------------------------------------------
//
// The same flood fill as tier 1 on a window a quarter of its size: nearly
// every component of an element of a few sites a side fits in 16 x 32, and
// the shuffle scans, the fill and the list work of one warp then serve two
// elements.  Half h = lane / 16 takes element 2w + h; half-lane r owns window
// row r as one 32-bit mask.  Every shuffle is a 16-wide one over the whole
// warp, so loops run until both halves are done, a finished half idling.
// A component that reaches the window's edge goes to tier 1.

constexpr int PR = 16, PC = 32, TP = 4;  // window rows, columns; warps per block

struct __align__(16) HalfShared {
  float F9[9][TF_M];
  int ex9[9];
  float offu[9], offv[9];
  unsigned passed[PR];
  unsigned unsure[PR];
  unsigned short item[PR * PC];  // the component's sites for the claims (row << 5 | column)
};

// Inclusive sum of v over the 16 lanes of the half.
__device__ __forceinline__ int half_incl(int v, int hl) {
#pragma unroll
  for (int o = 1; o < 16; o <<= 1) {
    const int t = __shfl_up_sync(FULL, v, o, 16);
    if (hl >= o) v += t;
  }
  return v;
}

// vfill on 16 rows of 32-bit masks.
__device__ __forceinline__ unsigned vfill16(unsigned comp, unsigned pass, int hl) {
  unsigned gd = comp, ad = pass, gu = comp, au = pass;
#pragma unroll
  for (int d = 1; d < 16; d <<= 1) {
    const unsigned g1 = __shfl_up_sync(FULL, gd, d, 16), a1 = __shfl_up_sync(FULL, ad, d, 16);
    const unsigned g2 = __shfl_down_sync(FULL, gu, d, 16), a2 = __shfl_down_sync(FULL, au, d, 16);
    if (hl >= d) {
      gd |= g1 & ad;
      ad &= a1;
    }
    if (hl + d < 16) {
      gu |= g2 & au;
      au &= a2;
    }
  }
  return gd | gu;
}

// run_fill on 32-bit words.
__device__ __forceinline__ unsigned run_fill32(unsigned S, unsigned P) {
  S &= P;
  const unsigned up = (((P + S) ^ P) & P) | S;
  const unsigned Pr = __brev(P), Sr = __brev(S);
  const unsigned dn = __brev((((Pr + Sr) ^ Pr) & Pr) | Sr);
  return up | dn;
}

__device__ __forceinline__ unsigned col_mask32(int lo, int hi) {
  const int a = max(lo, 0), b = min(hi, 32);
  if (b <= a) return 0u;
  const unsigned up = (b >= 32) ? ~0u : ((1u << b) - 1u);
  const unsigned dn = (a <= 0) ? 0u : ((1u << a) - 1u);
  return up & ~dn;
}

// Position of the n-th set bit (from 0) of a 32-bit x with more than n set bits.
__device__ __forceinline__ int nth_bit32(unsigned w, int n) {
  int pos = 0, c = __popc(w & 0xFFFFu);
  if (n >= c) { n -= c; pos = 16; w >>= 16; }
  c = __popc(w & 0xFFu); if (n >= c) { n -= c; pos += 8; w >>= 8; }
  c = __popc(w & 0xFu); if (n >= c) { n -= c; pos += 4; w >>= 4; }
  c = __popc(w & 0x3u); if (n >= c) { n -= c; pos += 2; w >>= 2; }
  if (n >= (int)(w & 1u)) pos += 1;
  return pos;
}

__device__ __forceinline__ void claim_pair_body(const Grid& g, const double* __restrict__ tay,
                                                         const float* __restrict__ tayf, Slots Sin, float alo,
                                                         float ahi, int32_t* __restrict__ esc_list,
                                                         int2* __restrict__ ovf_list, int vb) {
  __shared__ HalfShared shp[2 * TP];
  const Slots S = with_epoch(Sin);
  const int lane = threadIdx.x & 31, h = lane >> 4, hl = lane & 15;
  const int wq = threadIdx.x >> 5;
  HalfShared& sh = shp[2 * wq + h];
  const int m = (vb * TP + wq) * 2 + h;
  if (__all_sync(FULL, m >= g.ne)) return;
  bool live = m < g.ne;
  const int k = live ? m / g.Lv : 0, l = live ? m - k * g.Lv : 0;
  live = live && elem_exists(g, k, l);  // elements off the computing domain claim nothing
  // set-up: the 3x3 neighbourhood's index positions as integer part and
  // FP32 fraction (half-lanes 0-8; integer INT_MIN/2 where not finite) and
  // FP32 records, every load issued before any is used
  int uiq = 0, wiq = 0;
  float ufq = 0.f, wfq = 0.f;
  bool exq = false;
  if (live && hl < 9) {
    const int kk = k + hl / 3 - 1, ll = l + hl % 3 - 1;
    exq = elem_exists(g, kk, ll);
    if (exq) {
      const float* R = tayf + (size_t)(kk * g.Lv + ll) * TF_N;
      const int2 iw = __ldg(reinterpret_cast<const int2*>(R + TF_UI));
      const float2 fw = __ldg(reinterpret_cast<const float2*>(R + TF_UF));
      uiq = iw.x;
      wiq = iw.y;
      ufq = fw.x;
      wfq = fw.y;
    }
  }
  {
    // the 36 float4 of the nine records over the 16 half-lanes: all loads
    // issued, then all stores
    constexpr int NV = (9 * (TF_MW / 4) + 15) / 16;
    float4 v[NV];
#pragma unroll
    for (int u = 0; u < NV; u++) {
      const int idx = hl + 16 * u;
      const int q = idx / (TF_MW / 4), c4 = idx - q * (TF_MW / 4);
      const int kk = k + q / 3 - 1, ll = l + q % 3 - 1;
      const bool ex = live && idx < 9 * (TF_MW / 4) && elem_exists(g, kk, ll);
      v[u] = ex ? __ldg(reinterpret_cast<const float4*>(tayf + (size_t)(kk * g.Lv + ll) * TF_N) + c4)
                : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < NV; u++) {
      const int idx = hl + 16 * u;
      const int q = idx / (TF_MW / 4), c4 = idx - q * (TF_MW / 4);
      const int kk = k + q / 3 - 1, ll = l + q % 3 - 1;
      if (live && idx < 9 * (TF_MW / 4)) {
        reinterpret_cast<float4*>(sh.F9[q])[c4] = v[u];
        if (c4 == 0) sh.ex9[q] = elem_exists(g, kk, ll);
      }
    }
  }
  // the start site floor(u + 1/2) (u = ui + uf exactly in FP64): ui + 1
  // when the fraction is at least 1/2, settled by its FP32 rounding unless
  // that is 1/2 itself (then the FP64 index position decides); the offsets
  // i0 - u of the nine positions in FP32 from the integer difference and
  // the fraction (the same rounding as the FP64 difference rounded to FP32,
  // within the FP32 tests' bound)
  const int uis = __shfl_sync(FULL, uiq, 4, 16), wis = __shfl_sync(FULL, wiq, 4, 16);
  const float ufs = __shfl_sync(FULL, ufq, 4, 16), wfs = __shfl_sync(FULL, wfq, 4, 16);
  live = live && uis != INT_MIN / 2 && wis != INT_MIN / 2;  // (index position not finite: no element)
  long long i0 = 0, j0 = 0;
  if (live) {
    i0 = (long long)uis + (ufs > 0.5f ? 1 : 0);
    j0 = (long long)wis + (wfs > 0.5f ? 1 : 0);
    if (ufs == 0.5f || wfs == 0.5f) {
      const double2 uw = __ldg(reinterpret_cast<const double2*>(tayf + (size_t)m * TF_N + TF_UD));
      if (ufs == 0.5f) i0 = (long long)floor(dadd(uw.x, 0.5));
      if (wfs == 0.5f) j0 = (long long)floor(dadd(uw.y, 0.5));
    }
  }
  const int pad = g.pad;
  live = live && !(i0 < -pad || i0 >= g.nx + pad || j0 < -pad || j0 >= g.nv + pad);
  if (live && hl < 9) {
    sh.offu[hl] = exq ? (float)((int)i0 - uiq) - ufq : 0.f;
    sh.offv[hl] = exq ? (float)((int)j0 - wiq) - wfq : 0.f;
  }
  __syncwarp();
  Ctx9 c;
  c.F9 = sh.F9;
  c.ex9 = sh.ex9;
  c.offu = sh.offu;
  c.offv = sh.offv;
  c.inv_s = 1.0f / (float)g.s;
  c.alo = alo;
  c.ahi = ahi;
  const long long r0 = i0 - PR / 2, c0 = j0 - PC / 2;
  const long long irow = r0 + hl;
  const int clo = (int)max(0ll, (long long)(-pad) - c0);
  const int chi = (int)min((long long)PC, (long long)(g.nv + pad) - c0);
  const unsigned valid = (live && irow >= -pad && irow < g.nx + pad) ? col_mask32(clo, chi) : 0u;
  const unsigned seedbit = (hl == PR / 2) ? (1u << (PC / 2)) : 0u;
  unsigned comp = 0u, tested = 0u, passing = 0u, fa = 0u, fb = 0u;
  // predicted region (as in tier 1): the inner part certified or listed
  // first, the rest after it
  if (live) {
    const float* F = sh.F9[4];
    const float T00 = F[TF_T00], T01 = F[TF_T01], T10 = F[TF_T10], T11 = F[TF_T11];
    const float inv_s = c.inv_s, sf = (float)g.s;
    const float det = fabsf(T00 * T11 - T01 * T10);
    const float ext = (det > 1e-20f) ? fmaxf(fabsf(T11) + fabsf(T01), fabsf(T10) + fabsf(T00)) * __frcp_rn(det) : 0.f;
    const float P = 0.6f * ext + inv_s;
    const float sx = F[TF_C2X] * P * P, sv = F[TF_C2V] * P * P;
    const float hx = 0.52f + 1.1f * fmaxf(fabsf(T00), fabsf(T01)) * inv_s + sx;
    const float hv = 0.52f + 1.1f * fmaxf(fabsf(T10), fabsf(T11)) * inv_s + sv;
    const float ix = alo - 0.02f - sx, iv = alo - 0.02f - sv;
    const float px = ((float)(hl - PR / 2) + sh.offu[4]) * inv_s;
    const float r01 = (fabsf(T01) > 1e-20f) ? __frcp_rn(T01) : 0.f, r11 = (fabsf(T11) > 1e-20f) ? __frcp_rn(T11) : 0.f;
    auto cols = [&](float h1, float h2) -> unsigned {
      float lo = -1e30f, hi = 1e30f;
      auto cut = [&](float a, float cf, float rcf, float hh) {
        if (rcf != 0.f) {
          const float t1 = (-hh - a) * rcf, t2 = (hh - a) * rcf;
          lo = fmaxf(lo, fminf(t1, t2));
          hi = fminf(hi, fmaxf(t1, t2));
        } else if (!(fabsf(a) <= hh)) {
          lo = 1e30f;
          hi = -1e30f;
        }
      };
      cut(T00 * px, T01, r01, h1);
      cut(T10 * px, T11, r11, h2);
      const float blo = fminf(fmaxf(lo * sf - sh.offv[4] + (float)(PC / 2), -1.f), (float)(PC + 1));
      const float bhi = fminf(fmaxf(hi * sf - sh.offv[4] + (float)(PC / 2), -1.f), (float)(PC + 1));
      const int ilo = max((int)ceilf(blo), 0), ihi = min((int)floorf(bhi), PC - 1);
      return (ihi >= ilo) ? col_mask32(ilo, ihi + 1) : 0u;
    };
    const unsigned pred = (cols(hx, hv) | seedbit) & valid;
    const unsigned inner = (ix > 0.f && iv > 0.f) ? cols(ix, iv) & pred : 0u;
    // inner sites certified to pass (the bound argument of tier 1)
    unsigned sure = 0u;
    if (inner && fmaxf(fmaxf(fabsf(T00), fabsf(T01)), fmaxf(fabsf(T10), fabsf(T11))) < 50.f) {
      const int blo = __ffs(inner) - 1, bhi = 31 - __clz(inner);
      const float pvlo = ((float)(blo - PC / 2) + sh.offv[4]) * inv_s;
      const float pvhi = ((float)(bhi - PC / 2) + sh.offv[4]) * inv_s;
      const float Pr = fmaxf(fabsf(px), fmaxf(fabsf(pvlo), fabsf(pvhi)));
      if (F[TF_C2X] * Pr * Pr + 2e-3f <= 0.02f + sx && F[TF_C2V] * Pr * Pr + 2e-3f <= 0.02f + sv) sure = inner;
    }
    tested = sure;
    passing = sure;
    fa = pred & inner & ~sure;
    fb = pred & ~inner;
    const unsigned ing = pred & ((irow >= 0 && irow < g.nx)
                                     ? col_mask32((int)max(0ll, -c0), (int)min((long long)PC, (long long)g.nv - c0))
                                     : 0u);
    if (ing) {
      const size_t rowp = (size_t)irow * g.nv + c0;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(S.slot0 + rowp + (__ffs(ing) - 1)));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(S.slot0 + rowp + (31 - __clz(ing))));
    }
  }
  auto test = [&](int wr, int wb) -> int { return pass_f32(c, (float)(wr - PR / 2), (float)(wb - PC / 2)); };
  int rounds = 0;
  for (int it = 0; it < PR * PC; it++) {
    const int ca = __popc(fa), cb = __popc(fb);
    const int inca = half_incl(ca, hl), incb = half_incl(cb, hl);
    const int ta = __shfl_sync(FULL, inca, 15, 16);
    const int total = ta + __shfl_sync(FULL, incb, 15, 16);
    const bool fin = !live || (total == 0 && it > 0);
    if (__all_sync(FULL, fin)) break;
    if (!fin && total > 0) rounds++;
    sh.passed[hl] = 0u;
    sh.unsure[hl] = 0u;
    __syncwarp();
    const unsigned incp = (unsigned)inca | ((unsigned)incb << 16);
    const int tmax = max(total, __shfl_xor_sync(FULL, total, 16));
    for (int e0 = 0; e0 < tmax; e0 += 16) {
      const int e = e0 + hl;
      const bool inA = e < ta;
      const int key = inA ? e : e - ta, sh16 = inA ? 0 : 16;
      int r = 0;
#pragma unroll
      for (int st = 8; st; st >>= 1) {
        const unsigned v = __shfl_sync(FULL, incp, r + st - 1, 16);
        if ((int)((v >> sh16) & 0xFFFFu) <= key) r += st;
      }
      const unsigned vr = __shfl_sync(FULL, incp, r, 16);
      const unsigned wa = __shfl_sync(FULL, fa, r, 16), wb = __shfl_sync(FULL, fb, r, 16);
      if (e < total) {
        const unsigned w = inA ? wa : wb;
        const int b = nth_bit32(w, key - ((int)((vr >> sh16) & 0xFFFFu) - __popc(w)));
        const int res = test(r, b);
        if (res == 1) atomicOr(&sh.passed[r], 1u << b);
        if (res < 0) atomicOr(&sh.unsure[r], 1u << b);
      }
    }
    __syncwarp();
    tested |= fa | fb;
    passing |= sh.passed[hl];
    // the exact FP64 test of this row's unsettled sites (rare)
    for (unsigned un = sh.unsure[hl]; un; un &= un - 1u) {
      const int b = __ffs(un) - 1;
      atomicAdd(&S.ds->n_exact, 1);
      if (pass_exact_g(g, tay, k, l, site_x(g, irow), site_v(g, c0 + b))) passing |= 1u << b;
    }
    if (it == 0) {
      // the start decides whether there is a component at all
      const bool start = __shfl_sync(FULL, (passing >> (PC / 2)) & 1u, PR / 2, 16) != 0u;
      live = live && start;
      comp = live ? seedbit : 0u;
    }
    // close the component through every site known to pass
    for (int f = 0; f < PR * PC; f++) {
      const unsigned nc = run_fill32(vfill16(comp, passing, hl), passing);
      const bool grew = nc != comp;
      comp = nc;
      if (!__any_sync(FULL, grew)) break;
    }
    unsigned up = __shfl_up_sync(FULL, comp, 1, 16), dn = __shfl_down_sync(FULL, comp, 1, 16);
    if (hl == 0) up = 0u;
    if (hl == PR - 1) dn = 0u;
    fa = 0u;
    fb = live ? ((comp | (comp << 1) | (comp >> 1) | up | dn) & ~comp & valid & ~tested) : 0u;
  }
  if (live && rounds > 1 && hl == 0) atomicAdd(&S.ds->t1_more, 1);
  // Escaped the window?  Then tier 1 takes the element from the start.
  const unsigned hm = 0xFFFFu << (16 * h);
  const bool er = (__ballot_sync(FULL, comp != 0u && ((hl == 0 && r0 - 1 >= -pad) ||
                                                      (hl == PR - 1 && r0 + PR < g.nx + pad))) & hm) != 0u;
  const bool ec = (__ballot_sync(FULL, ((comp & 1u) && clo == 0 && c0 - 1 >= -pad) ||
                                           ((comp >> (PC - 1)) && chi == PC && c0 + PC < g.nv + pad)) & hm) != 0u;
  const bool esc = live && (er || ec);
  // An outer element (a neighbour missing) that escapes claims a boundary
  // band, which tier 1's window cannot hold either: it goes straight to
  // tier 2 (the v bands listed from the front), with this window's masks as the seed of
  // tier 2's first window (placed in a 32 x 64 record as tier 1's would
  // be).  The others start again in tier 1.
  bool outer = false;
  for (int q = 0; q < 9; q++) outer |= !sh.ex9[q];
  int seed = -1;
  if (esc && outer && hl == 0) {
    seed = atomicAdd(&S.ds->nseed, 1);
    if (seed >= S.seed_cap) seed = -1;
    const int sides = (er ? 1 : 0) | (ec ? 2 : 0);
    // the v bands (the longest jobs) from the front, taken first; the others
    // from the end
    const int slot = (sides == 2) ? atomicAdd(&S.ds->noverflow, 1) : g.ne - 1 - atomicAdd(&S.ds->noverflow_back, 1);
    ovf_list[slot] = make_int2(m, ((seed + 1) << 8) | (sides << 4));
  }
  seed = __shfl_sync(FULL, seed, 0, 16);
  if (esc && outer) {
    if (seed >= 0) {
      unsigned long long* rec = S.seed + (size_t)seed * (3 * TR);
      const int r = TR / 2 - PR / 2 + hl, sh0 = 32 - PC / 2;
      rec[r] = (unsigned long long)comp << sh0;
      rec[TR + r] = (unsigned long long)tested << sh0;
      rec[2 * TR + r] = (unsigned long long)passing << sh0;
      // the record's other rows
      rec[hl < 8 ? hl : TR - 16 + hl] = 0ull;
      rec[TR + (hl < 8 ? hl : TR - 16 + hl)] = 0ull;
      rec[2 * TR + (hl < 8 ? hl : TR - 16 + hl)] = 0ull;
    }
  } else if (esc && hl == 0) {
    esc_list[atomicAdd(&S.ds->n_pair_esc, 1)] = m;
  }
  const bool claim = live && !esc;
  // claims: the component's sites listed in row order, four exchanges in
  // flight per lane
  const int cnt = claim ? __popc(comp) : 0;
  const int incl = half_incl(cnt, hl);
  const int total = __shfl_sync(FULL, incl, 15, 16);
  if (claim) {
    int idx = incl - cnt;
    for (unsigned bits = comp; bits; bits &= bits - 1u) sh.item[idx++] = (unsigned short)((hl << 5) | (__ffs(bits) - 1));
  }
  __syncwarp();
  const int tmax = max(total, __shfl_xor_sync(FULL, total, 16));
  for (int e = hl; e < tmax; e += 4 * 16) {
    size_t pos[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int ee = e + 16 * u;
      pos[u] = ~(size_t)0;
      if (ee < total) {
        const int code = sh.item[ee];
        const long long i = r0 + (code >> 5), j = c0 + (code & 31);
        if (i >= 0 && i < g.nx && j >= 0 && j < g.nv) pos[u] = (size_t)i * g.nv + j;
      }
    }
    claim_sites(S, g, pos, m);
  }
}

__global__ void __launch_bounds__(32 * TP, 8) k_claim_pair(Grid g, const double* __restrict__ tay,
                                                         const float* __restrict__ tayf, Slots Sin, float alo,
                                                         float ahi, int32_t* __restrict__ esc_list,
                                                         int2* __restrict__ ovf_list) {
  if (gate_shut(g)) return;
  claim_pair_body(g, tay, tayf, Sin, alo, ahi, esc_list, ovf_list, blockIdx.x);
}

// ---------------------------------------------------------------------------
// tier 2: larger windows, cooperative block, word-granular tests
// ---------------------------------------------------------------------------

constexpr int BT = 256;       // threads
constexpr int BLOCKS_PER_SM = 3;
constexpr int BAND_R = 128, BAND_W = 20;  // band window: 128 rows across, up to 1280 sites along
constexpr int FAT_R = 160, FAT_W = 12;    // 160 x 768 sites
constexpr int LIST_CAP = 512;
constexpr int UNS_CAP = 512;  // sites per round whose FP32 test is left open, tested exactly together
constexpr int AHEAD = 3;      // rows tested ahead of the component per round
constexpr size_t SMEM_MAX = 227 * 1024;   // opt-in limit per block
constexpr size_t SMEM_SM = 228 * 1024;    // shared memory per SM

struct BigHeader {
  Elem9 E;
  int item, nlist, ok, bulk;
  int rmin, rmax, wmin, wmax;  // rows / words holding component bits
  int list[LIST_CAP];          // words to test this round
  unsigned long long lmask[LIST_CAP];  // their untested valid sites
  int lcnt[LIST_CAP];          // inclusive counts of the listed sites
  int wtot[BT / 32];           // per-warp totals of a block scan
  short plo[FAT_R > BAND_R ? FAT_R : BAND_R];  // per window row: columns of the predicted band
  short phi[FAT_R > BAND_R ? FAT_R : BAND_R];
  int nuns;                    // this round's sites left open by the FP32 test
  int uns_site[UNS_CAP];       // their window bit (word * 64 + bit)
  int uns_res[UNS_CAP];        // and the FP32 test's open result (-1, or -2 - neighbour mask)
};

// Block-wide inclusive sums out[e] = cnt(0) + ... + cnt(e) for e < n (each
// thread sums a contiguous run of entries); returns the total.  Called by
// every thread of the block.
template <class Cnt>
__device__ __forceinline__ int block_incl(int n, Cnt cnt, int* out, int* wtot) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int per = (n + BT - 1) / BT;
  const int a = min(tid * per, n), b = min(a + per, n);
  int sum = 0;
  for (int e = a; e < b; e++) {
    sum += cnt(e);
    out[e] = sum;
  }
  const int incl = warp_incl(sum, lane);
  if (lane == 31) wtot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int v = warp_incl(lane < BT / 32 ? wtot[lane] : 0, lane);
    __syncwarp();
    if (lane < BT / 32) wtot[lane] = v;
  }
  __syncthreads();
  const int off = incl - sum + (wid ? wtot[wid - 1] : 0);
  for (int e = a; e < b; e++) out[e] += off;
  const int total = wtot[BT / 32 - 1];
  __syncthreads();
  return total;
}

// Entry holding item e, at or after entry s0 (which holds an earlier item):
// a few steps forward, doubling, then a binary search of the last stretch.
__device__ __forceinline__ int find_entry_from(const int* incl, int s0, int n, int e) {
  int lo = s0, step = 1;
  while (lo + step < n && incl[lo + step - 1] <= e) {
    lo += step;
    step <<= 1;
  }
  int hi = min(lo + step, n) - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (incl[mid] > e)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

// Entry holding item e of a compacted list (first s with incl[s] > e; e is
// below incl[n - 1]).
__device__ __forceinline__ int find_entry(const int* incl, int n, int e) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (incl[mid] > e)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

// Window modes of the attempts after tier 1, by the sides its component
// escaped from (1: rows, 2: columns, 3: both); the last attempt covers the
// whole padded lattice, its bit masks in global memory.
__device__ __forceinline__ int mode_for(int sides, int attempt) {
  const int seq[4][2] = {{MODE_FAT, MODE_BAND_V}, {MODE_BAND_X, MODE_FAT}, {MODE_BAND_V, MODE_FAT},
                         {MODE_FAT, MODE_BAND_V}};
  return attempt >= 2 ? MODE_GLOBAL : seq[sides & 3][attempt < 0 ? 0 : attempt];
}

// 64-bit words along a band window for a lattice side n: the whole padded
// side, at most BAND_W.
__host__ __device__ __forceinline__ int band_words(long long n, int pad) {
  const long long full = (n + 2 * pad + 63) / 64;
  return (int)(full < BAND_W ? full : BAND_W);
}

// Rows and words of a window mode on a lattice (nrow x ncol sites before
// the pad, rows across and words along the bit axis): never more than the
// padded lattice holds.
__host__ __device__ __forceinline__ void window_dims(int mode, long long nrow, long long ncol, int pad, int& R,
                                                     int& W) {
  const long long rows_pad = nrow + 2 * pad, words_pad = (ncol + 2 * pad + 63) / 64;
  long long r, w;
  if (mode == MODE_GLOBAL) {
    r = rows_pad;
    w = words_pad;
  } else if (mode == MODE_FAT) {
    r = FAT_R < rows_pad ? FAT_R : rows_pad;
    w = FAT_W < words_pad ? FAT_W : words_pad;
  } else {
    r = BAND_R < rows_pad ? BAND_R : rows_pad;
    w = band_words(ncol, pad);
  }
  R = (int)r;
  W = (int)w;
}

// Window geometry: "rows" run across, "words" along the bit axis.  For
// MODE_BAND_X the bit axis is x (transposed window), otherwise v.
struct Win {
  bool trans;
  int R, W;              // rows, 64-bit words per row
  long long r0, c0;      // lattice coordinate of row 0 / bit 0
  int rlo, rhi, clo, chi;
  long long nrow_lat, ncol_lat;  // lattice extent along rows / bits (without pad)
};

// Centred on the start site, moved inside the padded lattice.
__device__ __forceinline__ Win make_window(int mode, const Grid& g, long long i0, long long j0) {
  Win W;
  const int pad = g.pad;
  W.trans = (mode == MODE_BAND_X);
  W.nrow_lat = W.trans ? g.nv : g.nx;
  W.ncol_lat = W.trans ? g.nx : g.nv;
  window_dims(mode, W.nrow_lat, W.ncol_lat, pad, W.R, W.W);
  const long long across0 = W.trans ? j0 : i0, along0 = W.trans ? i0 : j0;
  long long r0 = across0 - W.R / 2, c0 = along0 - 32ll * W.W;
  r0 = min(r0, W.nrow_lat + pad - W.R);
  c0 = min(c0, W.ncol_lat + pad - 64ll * W.W);
  W.r0 = max(r0, (long long)(-pad));
  W.c0 = max(c0, (long long)(-pad));
  const long long COLS = 64ll * W.W;
  W.clo = (int)max(0ll, (long long)(-pad) - W.c0);
  W.chi = (int)min(COLS, W.ncol_lat + pad - W.c0);
  W.rlo = (int)max(0ll, (long long)(-pad) - W.r0);
  W.rhi = (int)min((long long)W.R, W.nrow_lat + pad - W.r0);
  return W;
}

__device__ __forceinline__ void site_of(const Win& W, int r, int c, long long& i, long long& j) {
  if (W.trans) {
    j = W.r0 + r;
    i = W.c0 + c;
  } else {
    i = W.r0 + r;
    j = W.c0 + c;
  }
}

__device__ __forceinline__ unsigned long long valid_mask(const Win& W, int r, int w) {
  return (r >= W.rlo && r < W.rhi) ? col_mask(w, W.clo, W.chi) : 0ull;
}

__device__ __forceinline__ unsigned long long dilate(const unsigned long long* comp, const Win& W, int q) {
  const int r = q / W.W, w = q - r * W.W;
  const unsigned long long c = comp[q];
  unsigned long long d = c | (c << 1) | (c >> 1);
  if (w > 0) d |= comp[q - 1] >> 63;
  if (w < W.W - 1) d |= comp[q + 1] << 63;
  if (r > 0) d |= comp[q - W.W];
  if (r < W.R - 1) d |= comp[q + W.W];
  return d;
}

// Sites worth testing ahead of the component in word q: the word's column
// within AHEAD rows of it, the whole word if the word or a neighbouring word
// of its row holds some.  (Deeper speculation, 4 to 12 rows and two words,
// tested more sites than it saved rounds; growing inside a word one site per
// round, as the column rule alone does, made a component that starts from one
// site and runs along the bits take one round per site.)
__device__ __forceinline__ unsigned long long ahead(const unsigned long long* comp, const Win& W, int q) {
  const int r = q / W.W, w = q - r * W.W;
  unsigned long long d = dilate(comp, W, q);
  for (int k = 2; k <= AHEAD; k++) {
    if (r - k >= 0) d |= comp[q - k * W.W];
    if (r + k < W.R) d |= comp[q + k * W.W];
  }
  if (comp[q] || (w > 0 && comp[q - 1]) || (w < W.W - 1 && comp[q + 1])) d = ~0ull;
  return d;
}

// Flood fill of the elements queued by the previous tier, one element per
// block at a time.  Each round lists the words near the component that hold
// untested sites (AHEAD rows ahead, so that a component growing across the
// rows needs few rounds), tests them whole, and closes the component through
// the passing sites to a fixed point.  The loop ends when no site next to
// the component is untested or passing outside it.  kGlobal: the window is
// the whole padded lattice, its masks in a zeroed global scratch of the
// block, cleared again (over the touched box) before the next element.
template <bool kGlobal>
__device__ __forceinline__ void claim_big_body(const Grid& g, const double* __restrict__ tay,
                                                  const float* __restrict__ tayf, Slots Sin, float alo, float ahi,
                                                  const int2* __restrict__ list_in, const int* __restrict__ n_in,
                                                  const int* __restrict__ n_back,
                                                  int* __restrict__ stat, int2* __restrict__ list_out,
                                                  int* __restrict__ n_out, int* __restrict__ take,
                                                  unsigned long long* __restrict__ gwin, size_t gwin_words, int vb) {
  const Slots S = with_epoch(Sin);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BigHeader& H = *reinterpret_cast<BigHeader*>(smem_raw);
  unsigned long long* bits = kGlobal ? gwin + (size_t)vb * gwin_words
                                     : reinterpret_cast<unsigned long long*>(smem_raw + sizeof(BigHeader));
  const int tid = threadIdx.x;
  const int pad = g.pad;
  // n_in items from the front of the list, n_back (if given) from its end
  const int nf = *n_in, n = nf + (n_back ? *n_back : 0);
  // items are taken one at a time from a shared counter, so that blocks that
  // drew short components take more of them
  for (;;) {
    if (tid == 0) H.item = atomicAdd(take, 1);
    __syncthreads();
    const int item = H.item;
    if (item >= n) break;
    const int2 it2 = list_in[item < nf ? item : g.ne - 1 - (item - nf)];
    const int m = it2.x;
    if (m < 0 || m >= g.ne) {  // (never expected; keeps every index in bounds)
      if (tid == 0) VM_BAD(S.ds, 4);
      __syncthreads();  // every thread has read H.item before it is taken again
      continue;
    }
    const int sides = (it2.y >> 4) & 15, attempt = it2.y & 15, seed = (it2.y >> 8) - 1;
    const int mode = kGlobal ? MODE_GLOBAL : mode_for(sides, attempt);
    load_elem9(g, m, tay, tayf, H.E);
    __syncthreads();
    long long i0 = 0, j0 = 0;
    start_site(g, H.E, i0, j0);  // inside the padded lattice: tier 1 checked it
    set_offsets(H.E, i0, j0);
    const Win W = make_window(mode, g, i0, j0);
    const int NW = W.R * W.W;
    unsigned long long* comp = bits;
    unsigned long long* eval = bits + NW;
    unsigned long long* pass = bits + 2 * NW;
    if (!kGlobal) {
      for (int q = tid; q < 3 * NW; q += BT) bits[q] = 0ull;
    }
    __syncthreads();
    const Ctx9 c = ctx_of(g, H.E, alo, ahi);
    const long long across0 = W.trans ? j0 : i0, along0 = W.trans ? i0 : j0;
    const int rs = (int)(across0 - W.r0), cs = (int)(along0 - W.c0);
    if (tid == 0) {
      const bool ok = test_site(g, H.E, c, i0, j0, i0, j0);
      const int q = rs * W.W + (cs >> 6);
      H.rmin = H.rmax = rs;
      H.wmin = H.wmax = cs >> 6;
      eval[q] |= 1ull << (cs & 63);
      if (ok) {
        pass[q] |= 1ull << (cs & 63);
        comp[q] |= 1ull << (cs & 63);
      }
      H.ok = ok;
    }
    __syncthreads();
    // Tier 1's component, tested and passing masks, when this is the first
    // window of an element that escaped it (not transposed, in shared memory):
    // its component is a connected part of this window's, and its tests are
    // the same tests, so the fill continues from there.
    if (!kGlobal && seed >= 0 && seed < S.seed_cap && !W.trans && H.ok) {
      if (tid < TR) {
        const unsigned long long* rec = S.seed + (size_t)seed * (3 * TR);
        const unsigned long long mc = rec[tid], mt = rec[TR + tid], mp = rec[2 * TR + tid];
        const long long r = (i0 - TR / 2 + tid) - W.r0;
        const long long off = (j0 - 32) - W.c0;  // window bit of tier 1's column 0
        const long long w0 = (off >= 0) ? off / 64 : -((-off + 63) / 64);
        const int sh = (int)(off - 64 * w0);
        if (r >= 0 && r < W.R && (mc | mt | mp)) {
          for (int k = 0; k < 2; k++) {
            const long long w = w0 + k;
            if (w < 0 || w >= W.W) continue;
            auto part = [&](unsigned long long x) -> unsigned long long {
              return k == 0 ? (x << sh) : (sh ? (x >> (64 - sh)) : 0ull);
            };
            const int q = (int)(r * W.W + w);
            const unsigned long long vmask = valid_mask(W, (int)r, (int)w);
            comp[q] |= part(mc) & vmask;
            eval[q] |= part(mt) & vmask;
            pass[q] |= part(mp) & vmask;
            if (part(mc) & vmask) {
              atomicMin(&H.rmin, (int)r);
              atomicMax(&H.rmax, (int)r);
              atomicMin(&H.wmin, (int)w);
              atomicMax(&H.wmax, (int)w);
            }
          }
        }
      }
      __syncthreads();
    }
    // An outer element (a neighbour missing) claims a band that runs to the
    // padded lattice's edge on its open side.  Its first round also tests,
    // per window row, the columns where the linear part of its map keeps q
    // within a margin of the box on every side that has a neighbour (no
    // bound on a side without one): most of the band in one round instead
    // of a few rows per round.  Speculative only: the rounds still end only
    // when every site next to the component has been tested.
    if (!kGlobal) {
      bool outer = false;
      for (int q = 0; q < 9; q++) outer |= !H.E.ex9[q];
      const float* F = H.E.F9[4];
      const float T00 = F[TF_T00], T01 = F[TF_T01], T10 = F[TF_T10], T11 = F[TF_T11];
      const float Tm = fmaxf(fmaxf(fabsf(T00), fabsf(T01)), fmaxf(fabsf(T10), fabsf(T11)));
      const bool bulk = outer && H.ok && Tm < 1e6f;
      if (bulk) {
        const float inv_s = 1.0f / (float)g.s, sf = (float)g.s;
        const float h = 0.62f + 1.1f * Tm * inv_s;
        const float xlo = H.E.ex9[1] ? -h : -1e30f, xhi = H.E.ex9[7] ? h : 1e30f;
        const float vlo = H.E.ex9[3] ? -h : -1e30f, vhi = H.E.ex9[5] ? h : 1e30f;
        const long long acr0 = W.trans ? j0 : i0, alg0 = W.trans ? i0 : j0;
        const float offa = W.trans ? H.E.offv[4] : H.E.offu[4];
        const float C0 = (float)(W.c0 - alg0) + (W.trans ? H.E.offu[4] : H.E.offv[4]);
        const float cmax = (float)(64 * W.W);
        for (int r = tid; r < W.R; r += BT) {
          const float pf = ((float)(W.r0 + r - acr0) + offa) * inv_s;
          // q_x = ax + bx g, q_v = av + bv g along the row, g = (column + C0) / s
          const float ax = W.trans ? T01 * pf : T00 * pf, bx = W.trans ? T00 : T01;
          const float av = W.trans ? T11 * pf : T10 * pf, bv = W.trans ? T10 : T11;
          float glo = -1e30f, ghi = 1e30f;
          auto cut = [&](float a, float b, float lo, float hi) {
            if (fabsf(b) > 1e-20f) {
              const float t1 = (lo - a) / b, t2 = (hi - a) / b;
              glo = fmaxf(glo, fminf(t1, t2));
              ghi = fminf(ghi, fmaxf(t1, t2));
            } else if (!(a >= lo && a <= hi)) {
              glo = 1e30f;
              ghi = -1e30f;
            }
          };
          cut(ax, bx, xlo, xhi);
          cut(av, bv, vlo, vhi);
          const float clo = fminf(fmaxf(glo * sf - C0, -1.f), cmax), chi = fmaxf(fminf(ghi * sf - C0, cmax), -1.f);
          const int lo = max((int)ceilf(clo), 0), hi = min((int)floorf(chi), 64 * W.W - 1);
          H.plo[r] = (short)(lo <= hi ? lo : 1);
          H.phi[r] = (short)(lo <= hi ? hi : 0);
        }
      }
      if (tid == 0) H.bulk = bulk;
    }
    bool escaped = false;
    if (H.ok) {
      for (int it = 0; it < NW * 64; it++) {
        if (tid == 0) {
          H.nlist = 0;
          H.nuns = 0;
        }
        const int ra0 = max(H.rmin - AHEAD, 0), rb0 = min(H.rmax + AHEAD, W.R - 1);
        const int wa0 = max(H.wmin - 1, 0), wb0 = min(H.wmax + 1, W.W - 1);
        __syncthreads();
        const bool bulk = !kGlobal && it == 0 && H.bulk;
        const int ra = bulk ? 0 : ra0, rb = bulk ? W.R - 1 : rb0;
        const int wa = bulk ? 0 : wa0, wb = bulk ? W.W - 1 : wb0;
        const int bw = wb - wa + 1, nbox = (rb - ra + 1) * bw;
        // A: is the component open (an untested or passing site next to
        // it)?  List the words with untested sites near it, marking them
        // evaluated now (the list keeps which sites to test).
        bool open = false;
        for (int e = tid; e < nbox; e += BT) {
          const int r = ra + e / bw, w = wa + e % bw, q = r * W.W + w;
          const unsigned long long valid = valid_mask(W, r, w);
          const unsigned long long ev = eval[q];
          const unsigned long long near = dilate(comp, W, q) & ~comp[q] & valid;
          if (near & (~ev | pass[q])) open = true;
          unsigned long long todo = ahead(comp, W, q) & valid & ~ev;
          if (bulk) todo |= col_mask(w, H.plo[r], H.phi[r] + 1) & valid & ~ev;
          if (todo) {
            const int slot = atomicAdd(&H.nlist, 1);
            if (slot < LIST_CAP) {
              H.list[slot] = q;
              H.lmask[slot] = todo;
              eval[q] = ev | todo;
            }
          }
        }
        if (!__syncthreads_or(open)) break;
        // B: the listed sites' tests, compacted: test e goes to thread
        // e mod BT whatever word holds it
        const int nl = min(H.nlist, LIST_CAP);
        const int ntest = block_incl(nl, [&](int s) { return __popcll(H.lmask[s]); }, H.lcnt, H.wtot);
        int s = 0;  // a thread's entries only move forward: search on from the last one
        for (int e = tid; e < ntest; e += BT) {
          s = find_entry_from(H.lcnt, s, nl, e);
          const unsigned long long lm = H.lmask[s];
          const int b = nth_bit(lm, e - (H.lcnt[s] - __popcll(lm)));
          const int q = H.list[s];
          const int r = q / W.W, w = q - r * W.W;
          long long i, j;
          site_of(W, r, 64 * w + b, i, j);
          const int res = pass_f32<true>(c, (float)(int)(i - i0), (float)(int)(j - j0));
          if (res == 1) {
            atomicOr(&pass[q], 1ull << b);
          } else if (res < 0) {
            // left open: tested exactly below with the others, every lane busy
            // (an FP64 instruction takes the SM's FP64 unit for a whole warp)
            const int u = atomicAdd(&H.nuns, 1);
            if (u < UNS_CAP) {
              H.uns_site[u] = q * 64 + b;
              H.uns_res[u] = res;
            } else if (exact_open(g, H.E, res, i, j)) {
              atomicOr(&pass[q], 1ull << b);
            }
          }
        }
        __syncthreads();
        for (int u = tid; u < min(H.nuns, UNS_CAP); u += BT) {
          const int q = H.uns_site[u] >> 6, b = H.uns_site[u] & 63;
          const int r = q / W.W, w = q - r * W.W;
          long long i, j;
          site_of(W, r, 64 * w + b, i, j);
          if (exact_open(g, H.E, H.uns_res[u], i, j)) atomicOr(&pass[q], 1ull << b);
        }
        __syncthreads();
        // C: close the component through the passing sites (runs inside a
        // word at once, one row or word boundary per pass).  A word may see
        // its neighbours' growth of the same pass; that only adds connected
        // passing sites earlier, so the fixed point is the same.
        for (int p = 0; p < NW * 64; p++) {
          const int ca = max(H.rmin - 1, 0), cb = min(H.rmax + 1, W.R - 1);
          const int da = max(H.wmin - 1, 0), db = min(H.wmax + 1, W.W - 1);
          const int cw_ = db - da + 1, cbox = (cb - ca + 1) * cw_;
          __syncthreads();
          bool grew = false;
          for (int e = tid; e < cbox; e += BT) {
            const int r = ca + e / cw_, w = da + e % cw_, q = r * W.W + w;
            const unsigned long long cw = comp[q];
            const unsigned long long seeds = dilate(comp, W, q) & ~cw & pass[q];
            if (!seeds) continue;
            comp[q] = cw | run_fill(seeds | cw, pass[q]);
            grew = true;
            atomicMin(&H.rmin, r);
            atomicMax(&H.rmax, r);
            atomicMin(&H.wmin, w);
            atomicMax(&H.wmax, w);
          }
          if (!__syncthreads_or(grew)) break;
        }
      }
      // escaped this window?  (component bits on an edge that is not the
      // padded lattice's)
      bool esc = false;
      if (!kGlobal) {
        if (tid == 0) {
          esc = (H.rmin == 0 && W.rlo == 0 && W.r0 - 1 >= -pad) ||
                (H.rmax == W.R - 1 && W.rhi == W.R && W.r0 + W.R < W.nrow_lat + pad);
        }
        const bool left = H.wmin == 0 && W.clo == 0 && W.c0 - 1 >= -pad;
        const bool right = H.wmax == W.W - 1 && W.chi == 64 * W.W && W.c0 + 64ll * W.W < W.ncol_lat + pad;
        for (int r = H.rmin + tid; r <= H.rmax; r += BT) {
          if (left && (comp[r * W.W] & 1ull)) esc = true;
          if (right && (comp[r * W.W + W.W - 1] >> 63)) esc = true;
        }
      }
      escaped = __syncthreads_or(esc);
      if (escaped) {
        // the next, larger window claims a superset of this component
        if (tid == 0) {
          if (list_out != nullptr)
            list_out[atomicAdd(n_out, 1)] = make_int2(m, (sides << 4) | (attempt + 1));
          else
            atomicOr(&S.ds->err, ERR_PATCH_OVERFLOW);
        }
      } else {
        // claims: the component's sites compacted over the box's words
        // (their inclusive counts in the eval masks, no longer needed), up
        // to 8 exchanges in flight per thread
        const int bw = H.wmax - H.wmin + 1, nbox = (H.rmax - H.rmin + 1) * bw;
        int* ccnt = reinterpret_cast<int*>(eval);  // nbox <= NW ints fit in NW words
        auto word_of = [&](int e) { return (H.rmin + e / bw) * W.W + H.wmin + e % bw; };
        const int nsite = block_incl(nbox, [&](int e) { return __popcll(comp[word_of(e)]); }, ccnt, H.wtot);
        int xs = 0;  // (entries only move forward, as for the tests)
        for (int e0 = 0; e0 < nsite; e0 += 8 * BT) {
          size_t pos[8];
#pragma unroll
          for (int u = 0; u < 8; u++) {
            const int e = e0 + u * BT + tid;
            pos[u] = ~(size_t)0;
            if (e < nsite) {
              const int x = xs = find_entry_from(ccnt, xs, nbox, e), q = word_of(x);
              const unsigned long long cw = comp[q];
              const int b = nth_bit(cw, e - (ccnt[x] - __popcll(cw)));
              long long i, j;
              site_of(W, q / W.W, 64 * (q % W.W) + b, i, j);
              if (i >= 0 && i < g.nx && j >= 0 && j < g.nv) pos[u] = (size_t)i * g.nv + j;
            }
          }
          claim_sites(S, g, pos, m);
        }
      }
    }
    if (kGlobal) {
      // every word written lies within AHEAD rows and one word of the box
      __syncthreads();
      const int ra = max(H.rmin - AHEAD, 0), rb = min(H.rmax + AHEAD, W.R - 1);
      const int wa = max(H.wmin - 1, 0), wb = min(H.wmax + 1, W.W - 1);
      const int bw = wb - wa + 1, nbox = (rb - ra + 1) * bw;
      for (int e = tid; e < nbox; e += BT) {
        const int q = (ra + e / bw) * W.W + wa + e % bw;
        comp[q] = 0ull;
        eval[q] = 0ull;
        pass[q] = 0ull;
      }
      // and the claims' counts at the start of the eval masks
      const int ncl = escaped ? 0 : (H.rmax - H.rmin + 1) * (H.wmax - H.wmin + 1);
      for (int q = tid; q < (ncl + 1) / 2; q += BT) eval[q] = 0ull;
    }
    __syncthreads();
  }
  if (vb == 0 && tid == 0) *stat = n;
}

template <bool kGlobal>
__global__ void __launch_bounds__(BT, BLOCKS_PER_SM) k_claim_big(Grid g, const double* __restrict__ tay,
                                                  const float* __restrict__ tayf, Slots Sin, float alo, float ahi,
                                                  const int2* __restrict__ list_in, const int* __restrict__ n_in,
                                                  const int* __restrict__ n_back,
                                                  int* __restrict__ stat, int2* __restrict__ list_out,
                                                  int* __restrict__ n_out, int* __restrict__ take,
                                                  unsigned long long* __restrict__ gwin, size_t gwin_words) {
  if (gate_shut(g)) return;
  claim_big_body<kGlobal>(g, tay, tayf, Sin, alo, ahi, list_in, n_in, n_back, stat, list_out, n_out, take, gwin,
                          gwin_words, blockIdx.x);
}

// ---------------------------------------------------------------------------
// conflicts, extra claimants, holes
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long exact_key(const Grid& g, const double* __restrict__ tay, int m,
                                                        double Px, double Pv) {
  double xi, ze;
  return dkey(dist2_exact(tay + (size_t)m * TY_N, g, Px, Pv, xi, ze));
}

// Contested sites: the record's minimum is the owner; the record and the
// flag are emptied for the next map.
__device__ __forceinline__ void resolve_body(const Grid& g, const Slots& Sin, int vb, int vg) {
  const Slots S = with_epoch(Sin);
  const int n = min(S.ds->nrec, S.rec_cap);
  const size_t nsites = (size_t)g.nx * g.nv;
  for (int r = vb * blockDim.x + threadIdx.x; r < n; r += vg * blockDim.x) {
    const size_t p = (size_t)(uint32_t)S.rec_site[r];
    if (p >= nsites) {
      VM_BAD(S.ds, 2);
      continue;
    }
    const unsigned long long win = S.rec_key[2 * p];
    S.slot0[p] = (S.epoch << 24) | (uint32_t)win;
    S.rec_key[2 * p] = KEY_EMPTY;
    S.rec_key[2 * p + 1] = KEY_EMPTY;
    S.slot1[p] = SLOT_EMPTY;
  }
}

__global__ void k_resolve(Grid g, Slots Sin) {
  if (gate_shut(g)) return;
  resolve_body(g, Sin, blockIdx.x, gridDim.x);
}

// Sites no element claimed, four owner slots per 16-byte load (the slot
// array is 256-byte aligned); the list's order does not matter (the hole
// rounds are Jacobi rounds).
__device__ __forceinline__ void find_holes_body(const Grid& g, const uint32_t* __restrict__ slot0,
                                                int32_t* __restrict__ holes, DevState* ds, int vb, int vg) {
  const uint32_t epoch = *(volatile uint32_t*)&ds->epoch;
  const size_t n = (size_t)g.nx * g.nv, n4 = n / 4;
  const size_t t0 = vb * (size_t)blockDim.x + threadIdx.x, stride = (size_t)vg * blockDim.x;
  const uint4* s4 = reinterpret_cast<const uint4*>(slot0);
#pragma unroll 4
  for (size_t q = t0; q < n4; q += stride) {
    const uint4 t = __ldcs(s4 + q);  // read once: streamed past the caches
    const uint32_t e[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int u = 0; u < 4; u++)
      if ((e[u] >> 24) != epoch) holes[atomicAdd(&ds->nholes, 1)] = (int32_t)(4 * q + u);
  }
  for (size_t p = 4 * n4 + t0; p < n; p += stride)
    if ((slot0[p] >> 24) != epoch) holes[atomicAdd(&ds->nholes, 1)] = (int32_t)p;
}

__global__ void k_find_holes(Grid g, const uint32_t* __restrict__ slot0, int32_t* __restrict__ holes, DevState* ds) {
  if (gate_shut(g)) return;
  find_holes_body(g, slot0, holes, ds, blockIdx.x, gridDim.x);
}

constexpr int HT = 1024;

// Unexplored sites (Sec. 2.3.1, end): Jacobi rounds; in each round every
// hole takes, among the elements its in-grid 4-neighbours held at the end of
// the previous round, the one with the smallest d at the hole, then the
// smaller index.
__device__ __forceinline__ void holes_body(const Grid& g, const double* __restrict__ tay, uint32_t* __restrict__ slot0,
                                           int32_t* la, int32_t* lb, int32_t* cho, DevState* ds) {
  const uint32_t epoch = *(volatile uint32_t*)&ds->epoch;
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
      if (p < 0 || (size_t)p >= (size_t)g.nx * g.nv) {
        VM_BAD(ds, 3);
        cho[idx] = -2;  // dropped
        continue;
      }
      const int i = p / g.nv, j = p - i * g.nv;
      const double Px = site_x(g, i), Pv = site_v(g, j);
      int best = -1;
      unsigned long long bestk = 0;
      const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
      for (int q = 0; q < 4; q++) {
        const int ii = i + di[q], jj = j + dj[q];
        if (ii < 0 || ii >= g.nx || jj < 0 || jj >= g.nv) continue;
        const uint32_t t = slot0[(size_t)ii * g.nv + jj];
        if ((t >> 24) != epoch || (int)(t & SLOT_MASK) >= g.ne) continue;
        const int cand = (int)(t & SLOT_MASK);
        const unsigned long long key = exact_key(g, tay, cand, Px, Pv);
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
      const int ch = cho[idx];
      if (ch >= 0)
        slot0[la[idx]] = (epoch << 24) | (uint32_t)ch;
      else if (ch == -1)
        lb[atomicAdd(&next_s, 1)] = la[idx];
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

__global__ void __launch_bounds__(HT) k_holes(Grid g, const double* __restrict__ tay, uint32_t* __restrict__ slot0,
                                              int32_t* la, int32_t* lb, int32_t* cho, DevState* ds) {
  if (gate_shut(g)) return;
  holes_body(g, tay, slot0, la, lb, cho, ds);
}

// E_map (Sec. 2.3.2) of the current influence map: for every grid site with
// an owner m, and every existing neighbour n = m + (a, b) in the alpha
// ranges of the percolation test, the squared mismatch of the Lagrangian
// positions they propose in element spacings, ((a + xi_n) - xi_m)^2 +
// ((b + ze_n) - ze_m)^2 (Q_n - Q_m = (a dx_m, b dv_m) on the lattice), FP64
// in the oracle's order; the largest into ds->emap2_bits (bits of a
// non-negative double order as the values do).
__device__ __forceinline__ void emap_body(const Grid& g, const uint32_t* __restrict__ slot0,
                                          const double* __restrict__ tay, DevState* ds, int vb, int vg) {
  const uint32_t epoch = *(volatile uint32_t*)&ds->epoch;
  const size_t n = (size_t)g.nx * g.nv;
  double worst = 0.0;
  for (size_t p = (size_t)vb * blockDim.x + threadIdx.x; p < n; p += (size_t)vg * blockDim.x) {
    const uint32_t t = slot0[p];
    if ((t >> 24) != epoch) continue;
    const int m = (int)(t & SLOT_MASK);
    if (m >= g.ne) continue;
    const int i = (int)(p / (size_t)g.nv), j = (int)(p - (size_t)i * g.nv);
    const double Px = site_x(g, i), Pv = site_v(g, j);
    double xi, ze;
    dist2_exact(tay + (size_t)m * TY_N, g, Px, Pv, xi, ze);
    int a0, a1, b0, b1;
    alpha_range(xi, g.alpha, a0, a1);
    alpha_range(ze, g.alpha, b0, b1);
    const int k = m / g.Lv, l = m - k * g.Lv;
    for (int a = a0; a <= a1; a++)
      for (int b = b0; b <= b1; b++) {
        if (a == 0 && b == 0) continue;
        const int kk = k + a, ll = l + b;
        if (!elem_exists(g, kk, ll)) continue;
        double xn, zn;
        dist2_exact(tay + (size_t)(kk * g.Lv + ll) * TY_N, g, Px, Pv, xn, zn);
        const double mx = dsub(dadd((double)a, xn), xi), mv = dsub(dadd((double)b, zn), ze);
        const double e2 = dadd(dmul(mx, mx), dmul(mv, mv));
        if (e2 > worst) worst = e2;
      }
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_down_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0 && worst > 0.0)
    atomicMax(&ds->emap2_bits, (unsigned long long)__double_as_longlong(worst));
}

__global__ void k_emap(Grid g, const uint32_t* __restrict__ slot0, const double* __restrict__ tay, DevState* ds) {
  emap_body(g, slot0, tay, ds, blockIdx.x, gridDim.x);
}

// Whether the current map's E_map exceeds thr, without computing it: the
// same terms as emap_body, each settled from the FP32 records where their
// error bounds leave a margin (the bounds of the percolation's FP32 test on
// q, plus the roundings of the two FP32 differences), and from the exact
// FP64 terms at the sites where they do not (an alpha range that the bound
// leaves open, or a term within the margin of thr).  The outcome equals
// sqrt(max exact term) > thr.  Sets ds->emap_hit; blocks stop once it is set.
// Nothing to do when the step completes the remap cycle (the cycle decides).
constexpr float kRelE = 4.0e-6f;     // margin on thr^2 (FP32 squares and sums; thr^2 to FP32)
constexpr float kRndE = 2.4e-7f;     // two FP32 roundings of a difference of O(1) terms, doubled

// q of the FP32 record F at grid site (i, j) and its bounds (|q - xi| <= e);
// p from the record's integer and fraction split of the index position
// (FP32 and integer arithmetic only, as the reconstruction forms it).
__device__ __forceinline__ QF q_at_site(const float* __restrict__ F, int i, int j, float inv_s, float& ex,
                                        float& ev) {
  float f[TF_MW];  // words 0-15: the map's part of the record, 128-byte aligned
#pragma unroll
  for (int c = 0; c < TF_MW / 4; c++) {
    const float4 w = __ldg(reinterpret_cast<const float4*>(F) + c);
    f[4 * c] = w.x;
    f[4 * c + 1] = w.y;
    f[4 * c + 2] = w.z;
    f[4 * c + 3] = w.w;
  }
  static_assert(TF_UF < TF_MW && TF_WF < TF_MW && TF_UI % 2 == 0 && TF_WI == TF_UI + 1, "index split words");
  const int2 ui = __ldg(reinterpret_cast<const int2*>(F + TF_UI));  // UI, WI (8-byte aligned)
  const float px = ((float)(i - ui.x) - f[TF_UF]) * inv_s;
  const float pv = ((float)(j - ui.y) - f[TF_WF]) * inv_s;
  const QF r = qeval(f, px, pv);
  ex = kRelQ * r.ax + kAbs * (1.f + r.ax);
  ev = kRelQ * r.av + kAbs * (1.f + r.av);
  return r;
}

// The exact terms of one site (as emap_body): true when one of them exceeds thr.
__device__ __noinline__ bool emap_site_exceeds(const Grid& g, const double* __restrict__ tay, int m, long long i,
                                               long long j, double thr) {
  const double Px = site_x(g, i), Pv = site_v(g, j);
  double xi, ze;
  dist2_exact(tay + (size_t)m * TY_N, g, Px, Pv, xi, ze);
  int a0, a1, b0, b1;
  alpha_range(xi, g.alpha, a0, a1);
  alpha_range(ze, g.alpha, b0, b1);
  const int k = m / g.Lv, l = m - k * g.Lv;
  for (int a = a0; a <= a1; a++)
    for (int b = b0; b <= b1; b++) {
      if (a == 0 && b == 0) continue;
      const int kk = k + a, ll = l + b;
      if (!elem_exists(g, kk, ll)) continue;
      double xn, zn;
      dist2_exact(tay + (size_t)(kk * g.Lv + ll) * TY_N, g, Px, Pv, xn, zn);
      const double mx = dsub(dadd((double)a, xn), xi), mv = dsub(dadd((double)b, zn), ze);
      if (sqrt(dadd(dmul(mx, mx), dmul(mv, mv))) > thr) return true;
    }
  return false;
}

__device__ __forceinline__ void emap_test_body(const Grid& g, const uint32_t* __restrict__ slot0,
                                               const double* __restrict__ tay, const float* __restrict__ tayf,
                                               DevState* ds, double thr, int n_s, float alo, float ahi, int vb,
                                               int vg) {
  if (__ldcg(&ds->cyc) + 1 >= n_s) return;
  const uint32_t epoch = *(volatile uint32_t*)&ds->epoch;
  const float T2 = (float)(thr * thr);
  const float t_hi = T2 * (1.f + kRelE), t_lo = T2 * (1.f - kRelE);
  const float inv_s = 1.0f / (float)g.s;
  // rows by virtual block, sites of a row by thread (coalesced owner reads)
  for (int i = vb; i < g.nx; i += vg) {
    if (*(volatile int32_t*)&ds->emap_hit) return;
    const uint32_t* row = slot0 + (size_t)i * g.nv;
    for (int j = threadIdx.x; j < g.nv; j += blockDim.x) {
      const uint32_t t = row[j];
      if ((t >> 24) != epoch) continue;
      const int m = (int)(t & SLOT_MASK);
      if (m >= g.ne) continue;
      float exm, evm;
      const QF qm = q_at_site(tayf + (size_t)m * TF_N, i, j, inv_s, exm, evm);
      const int ra = range_f(qm.qx, exm, alo, ahi), rb = range_f(qm.qv, evm, alo, ahi);
      bool hit = false, open = (ra == 0 || rb == 0);
      if (!open && !(ra == 2 && rb == 2)) {
        // the terms of the settled alpha ranges: (A, 0), (0, B), (A, B) for
        // the nonzero ones of A, B
        const int A = ra - 2, B = rb - 2;
        const int k = m / g.Lv, l = m - k * g.Lv;
        for (int q = 0; q < 3 && !hit; q++) {
          const int a = (q == 1) ? 0 : A, b = (q == 0) ? 0 : B;
          if (a == 0 && b == 0) continue;
          if (q == 2 && (A == 0 || B == 0)) continue;
          const int kk = k + a, ll = l + b;
          if (!elem_exists(g, kk, ll)) continue;
          float exn, evn;
          const QF qn = q_at_site(tayf + (size_t)(kk * g.Lv + ll) * TF_N, i, j, inv_s, exn, evn);
          const float mx = ((float)a + qn.qx) - qm.qx, mv = ((float)b + qn.qv) - qm.qv;
          const float amx = fabsf(mx), amv = fabsf(mv);
          const float ux = exn + exm + kRndE * (1.f + fabsf(qn.qx) + amx);
          const float uv = evn + evm + kRndE * (1.f + fabsf(qn.qv) + amv);
          const float lx = fmaxf(amx - ux, 0.f), lv = fmaxf(amv - uv, 0.f);
          const float hx = amx + ux, hv = amv + uv;
          if (lx * lx + lv * lv > t_hi)
            hit = true;
          else if (!(hx * hx + hv * hv < t_lo))
            open = true;
        }
      }
      if (!hit && open) hit = emap_site_exceeds(g, tay, m, i, j, thr);
      if (hit) {
        atomicOr(&ds->emap_hit, 1);
        return;
      }
    }
  }
}

__global__ void k_emap_test(Grid g, const uint32_t* __restrict__ slot0, const double* __restrict__ tay,
                            const float* __restrict__ tayf, DevState* ds, double thr, int n_s, float alo, float ahi) {
  emap_test_body(g, slot0, tay, tayf, ds, thr, n_s, alo, ahi, blockIdx.x, gridDim.x);
}

// The remap decision of one solve after a step (Sec. 2.3.2), on the device:
// the cycle advances, and the remap runs at once when n_s steps are complete
// or, for thr > 0, when the step's E_map exceeds thr (emap_hit, counted).
// The same rule, in the same order, as the host's decision.
__device__ __forceinline__ void remap_decide(DevState* ds, int n_s, double thr) {
  const int cyc = ds->cyc + 1;
  bool remap = cyc >= n_s;
  if (!remap && thr > 0.0 && ds->emap_hit) {
    remap = true;
    ds->emap_remaps++;
  }
  ds->cyc = remap ? 0 : cyc;
  ds->gate = remap ? 1 : 0;
}

__global__ void k_remap_gate(DevState* ds, int n_s, double thr) {
  if (threadIdx.x == 0 && blockIdx.x == 0) remap_decide(ds, n_s, thr);
}

__global__ void k_read_map(const uint32_t* __restrict__ slot0, const DevState* ds, int32_t* __restrict__ out,
                           size_t n, int ne) {
  const uint32_t epoch = *(const volatile uint32_t*)&ds->epoch;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const uint32_t t = slot0[p];
    out[p] = ((t >> 24) == epoch && (int)(t & SLOT_MASK) < ne) ? (int32_t)(t & SLOT_MASK) : -1;
  }
}

// Adaptive computing domain: sites outside the map's rectangle ds->rect get
// the current epoch with no element (SLOT_OUTSIDE), so that they are
// neither holes to repair nor candidates of a repair, and read as unowned.
__global__ void k_clear_outside(Grid g, uint32_t* __restrict__ slot0, const DevState* ds) {
  const uint32_t epoch = *(const volatile uint32_t*)&ds->epoch;
  const int i0 = ds->rect[0], i1 = ds->rect[1], j0 = ds->rect[2], j1 = ds->rect[3];
  const uint32_t tag = (epoch << 24) | SLOT_OUTSIDE;
  for (int i = blockIdx.x; i < g.nx; i += gridDim.x) {
    uint32_t* row = slot0 + (size_t)i * g.nv;
    if (i < i0 || i > i1 || j0 > j1) {
      for (int j = threadIdx.x; j < g.nv; j += blockDim.x) row[j] = tag;
    } else {
      for (int j = threadIdx.x; j < j0; j += blockDim.x) row[j] = tag;
      for (int j = j1 + 1 + threadIdx.x; j < g.nv; j += blockDim.x) row[j] = tag;
    }
  }
}

// ---- group launches: the influence maps of every solve of a group ----

__device__ __forceinline__ Slots slots_of(const SolveDesc& d) {
  Slots S;
  S.slot0 = d.map;
  S.slot1 = d.slot1;
  S.rec_key = d.rec_key;
  S.rec_site = d.rec_site;
  S.rec_cap = d.rec_cap;
  S.tay = d.tay;
  S.ds = d.ds;
  S.epoch = 0u;
  S.seed = d.t1seed;
  S.seed_cap = d.t1seed_cap;
  return S;
}

__global__ void k_map_begin_group(const SolveDesc* __restrict__ D, int ns) {
  for (int sv = blockIdx.x * blockDim.x + threadIdx.x; sv < ns; sv += gridDim.x * blockDim.x)
    if (!gate_shut(D[sv].g)) map_begin_body(D[sv].ds);
}

// Units of a dynamic phase, per solve, from the solve's counters (read after
// the previous phase): an exclusive prefix into off[0..ns], one block.
__global__ void __launch_bounds__(1024) k_units(const SolveDesc* __restrict__ D, int ns, int kind, int cap,
                                              int* __restrict__ off) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < ns; base += blockDim.x) {
    const int sv = base + threadIdx.x;
    int u = 0;
    if (sv < ns) {
      const DevState* ds = D[sv].ds;
      const bool lastonly = D[sv].map_windows != 0;
      int n = 0;
      switch (kind) {
        case GC_PAIR_ESC: n = (ds->n_pair_esc + TE - 1) / TE; break;
        case GC_OVF1: n = lastonly ? 0 : ds->noverflow + ds->noverflow_back; break;
        case GC_OVF2: n = lastonly ? 0 : ds->noverflow2; break;
        case GC_OVF3: n = lastonly ? ds->noverflow + ds->noverflow_back : ds->noverflow3; break;
        case GC_REC: n = (min(ds->nrec, D[sv].rec_cap) + 255) / 256; break;
        default: n = ds->nholes > 0 ? 1 : 0; break;
      }
      u = gate_shut(D[sv].g) ? 0 : min(max(n, 0), cap);
    }
    int inc = u;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      const int w = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
      int wi = w;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      wsum[lane] = wi - w;
    }
    __syncthreads();
    if (sv < ns) off[sv] = carry + wsum[wid] + inc - u;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += wsum[wid] + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[ns] = carry;
}

// The loop of a dynamic phase: units [off[sv], off[sv + 1]) of solve sv,
// the unit count of the solve being the virtual grid.
#define GROUP_DYN_LOOP(off, ns)                                      \
  __shared__ Grid gsh;                                               \
  __shared__ int svsh;                                               \
  const int total_ = __ldcg((off) + (ns));                           \
  for (int u = blockIdx.x; u < total_; u += gridDim.x) {             \
    if (threadIdx.x == 0) {                                          \
      int lo = 0, hi = (ns) - 1;                                     \
      while (lo < hi) {                                              \
        const int mid = (lo + hi + 1) >> 1;                          \
        if (__ldcg((off) + mid) <= u) lo = mid; else hi = mid - 1;   \
      }                                                              \
      svsh = lo;                                                     \
      gsh = D[lo].g;                                                 \
    }                                                                \
    __syncthreads();                                                 \
    const int sv = svsh;                                             \
    const SolveDesc& d = D[sv];                                      \
    const int o0 = __ldcg((off) + sv);                               \
    const int vb = u - o0, vg = __ldcg((off) + sv + 1) - o0;         \
    (void)vg;

__global__ void __launch_bounds__(32 * TP, 8) k_claim_pair_group(const SolveDesc* __restrict__ D,
                                                               const int* __restrict__ off, int ns, int total) {
  GROUP_LOOP(off, ns, total)
  claim_pair_body(gsh, d.tay, d.tayf, slots_of(d), d.alo, d.ahi, d.holes_a, d.ovf1, vb);
  GROUP_END
}

__global__ void __launch_bounds__(32 * TE, 8) k_claim_small_group(const SolveDesc* __restrict__ D,
                                                                const int* __restrict__ off, int ns) {
  GROUP_DYN_LOOP(off, ns)
  claim_small_body(gsh, d.tay, d.tayf, slots_of(d), d.alo, d.ahi, d.ovf1, d.holes_a, &d.ds->n_pair_esc, vb, vg);
  GROUP_END
}

// attempt 0: the first large windows; 1: the second; 2: the whole lattice
template <int kAttempt>
__global__ void __launch_bounds__(BT, BLOCKS_PER_SM) k_claim_big_group(const SolveDesc* __restrict__ D,
                                                                      const int* __restrict__ off, int ns) {
  GROUP_DYN_LOOP(off, ns)
  DevState* ds = d.ds;
  const Slots S = slots_of(d);
  if (kAttempt == 0)
    claim_big_body<false>(gsh, d.tay, d.tayf, S, d.alo, d.ahi, d.ovf1, &ds->noverflow, &ds->noverflow_back,
                          &ds->overflow_stat, d.ovf2, &ds->noverflow2, &ds->take[0], nullptr, 0, vb);
  else if (kAttempt == 1)
    claim_big_body<false>(gsh, d.tay, d.tayf, S, d.alo, d.ahi, d.ovf2, &ds->noverflow2, nullptr,
                          &ds->overflow2_stat, d.ovf1, &ds->noverflow3, &ds->take[1], nullptr, 0, vb);
  else if (d.map_windows == 0)
    claim_big_body<true>(gsh, d.tay, d.tayf, S, d.alo, d.ahi, d.ovf1, &ds->noverflow3, nullptr, &ds->overflow3_stat,
                         nullptr, nullptr, &ds->take[2], d.gwin, d.gwin_words, vb);
  else
    claim_big_body<true>(gsh, d.tay, d.tayf, S, d.alo, d.ahi, d.ovf1, &ds->noverflow, &ds->noverflow_back,
                         &ds->overflow_stat, nullptr, nullptr, &ds->take[2], d.gwin, d.gwin_words, vb);
  GROUP_END
}

__global__ void k_resolve_group(const SolveDesc* __restrict__ D, const int* __restrict__ off, int ns) {
  GROUP_DYN_LOOP(off, ns)
  resolve_body(gsh, slots_of(d), vb, vg);
  GROUP_END
}

__global__ void k_find_holes_group(const SolveDesc* __restrict__ D, const int* __restrict__ off, int ns, int total) {
  GROUP_LOOP(off, ns, total)
  const int vg = __ldg(off + sv + 1) - __ldg(off + sv);
  find_holes_body(gsh, d.map, d.holes_a, d.ds, vb, vg);
  GROUP_END
}

__global__ void k_emap_test_group(const SolveDesc* __restrict__ D, const int* __restrict__ off, int ns,
                                  int total) {
  GROUP_LOOP_ALL(off, ns, total)
  const int vg = __ldg(off + sv + 1) - __ldg(off + sv);
  emap_test_body(gsh, d.map, d.tay, d.tayf, d.ds, d.emap_thr, d.n_s, d.alo, d.ahi, vb, vg);
  GROUP_END
}

__global__ void k_remap_gate_group(const SolveDesc* __restrict__ D, int ns) {
  for (int sv = blockIdx.x * blockDim.x + threadIdx.x; sv < ns; sv += gridDim.x * blockDim.x)
    remap_decide(D[sv].ds, D[sv].n_s, D[sv].emap_thr);
}

__global__ void __launch_bounds__(HT) k_holes_group(const SolveDesc* __restrict__ D, const int* __restrict__ off,
                                                  int ns) {
  GROUP_DYN_LOOP(off, ns)
  (void)vb;
  holes_body(gsh, d.tay, d.map, d.holes_a, d.holes_b, d.holes_b + (size_t)gsh.nx * gsh.nv, d.ds);
  GROUP_END
}

}  // namespace

void launch_clear_outside(vm_solver* s) {
  const unsigned nb = (unsigned)std::min(s->g.nx, 152 * 8);
  k_clear_outside<<<nb, 256, 0, s->stream>>>(s->g, s->map, s->ds);
  s->launches++;
}

void launch_emap(vm_solver* s) {
  unsigned nb = (unsigned)((s->n + 255) / 256);
  if (nb > 152 * 16) nb = 152 * 16;
  k_emap<<<nb, 256, 0, s->stream>>>(s->g, s->map, s->tay, s->ds);
  s->launches++;
}

namespace {
void alpha_bounds(double alpha, float& lo, float& hi);
}  // namespace

void launch_remap_gate(vm_solver* s) {
  const int ps = prof_begin(s, KID_EMAP);
  float alo, ahi;
  alpha_bounds(s->g.alpha, alo, ahi);
  unsigned nb = (unsigned)((s->n + 255) / 256);
  if (nb > 152 * 8) nb = 152 * 8;
  k_emap_test<<<nb, 256, 0, s->stream>>>(s->g, s->map, s->tay, s->tayf, s->ds, s->cfg.emap_remap, s->cfg.n_s, alo,
                                         ahi);
  k_remap_gate<<<1, 32, 0, s->stream>>>(s->ds, s->cfg.n_s, s->cfg.emap_remap);
  prof_end(s, ps);
  s->launches++;
}

void group_remap_gate(const GroupPlan& G) {
  if (G.tot_sites > 0)
    k_emap_test_group<<<group_grid(G, GP_EMAP, G.tot_sites), 256, 0, G.stream>>>(G.D, G.off_sites, G.ns,
                                                                                  G.tot_sites);
  k_remap_gate_group<<<(unsigned)((G.ns + 255) / 256), 256, 0, G.stream>>>(G.D, G.ns);
}

namespace {

size_t big_smem_bytes(const Grid& g) {
  long long nw = 0;
  int R, W;
  window_dims(MODE_FAT, g.nx, g.nv, g.pad, R, W);
  nw = max(nw, (long long)R * W);
  window_dims(MODE_BAND_V, g.nx, g.nv, g.pad, R, W);
  nw = max(nw, (long long)R * W);
  window_dims(MODE_BAND_X, g.nv, g.nx, g.pad, R, W);
  nw = max(nw, (long long)R * W);
  return sizeof(BigHeader) + 3 * (size_t)nw * sizeof(unsigned long long);
}

// alpha rounded down and up to FP32
void alpha_bounds(double alpha, float& lo, float& hi) {
  const float f = (float)alpha;
  lo = ((double)f <= alpha) ? f : nextafterf(f, -INFINITY);
  hi = ((double)f >= alpha) ? f : nextafterf(f, INFINITY);
}

}  // namespace

// Opt the large-window kernel in to shared memory.  The limit is a property
// of the kernel, shared by every solver of the process, so it is set to the
// largest size any grid can ask for rather than to this grid's need.
bool map_prepare(const Grid& g) {
  if (big_smem_bytes(g) > SMEM_MAX || BLOCKS_PER_SM * (big_smem_bytes(g) + 1024) > SMEM_SM) return false;
  return cudaFuncSetAttribute(k_claim_big<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_MAX) ==
         cudaSuccess;
}

void launch_map(vm_solver* s) {
  Slots S{s->map, s->slot1, s->rec_key, s->rec_site, s->rec_cap, s->tay, s->ds, 0u, s->t1seed, s->t1seed_cap};
  float alo, ahi;
  alpha_bounds(s->g.alpha, alo, ahi);
  int ps = prof_begin(s, KID_MAP_CLEAR);
  if (s->g.fth_on) launch_domain_rect(s);
  k_map_begin<<<1, 32, 0, s->stream>>>(s->ds, s->g.gate);
  prof_end(s, ps);
  // tier 0 (two elements per warp), its escapes to tier 1 through the first
  // hole list (free until the holes are looked for)
  ps = prof_begin(s, KID_CLAIM_PAIR);
  k_claim_pair<<<(unsigned)((s->g.ne + 2 * TP - 1) / (2 * TP)), 32 * TP, 0, s->stream>>>(s->g, s->tay, s->tayf, S,
                                                                                        alo, ahi, s->holes_a,
                                                                                        s->overflow_list);
  prof_end(s, ps);
  ps = prof_begin(s, KID_CLAIM_SMALL);
  const unsigned t1 = (unsigned)std::min<long long>(152 * 8, (s->g.ne + TE - 1) / TE);
  k_claim_small<<<t1, 32 * TE, 0, s->stream>>>(s->g, s->tay, s->tayf, S, alo, ahi, s->overflow_list, s->holes_a,
                                              &s->ds->n_pair_esc);
  prof_end(s, ps);
  const size_t smem = big_smem_bytes(s->g);
  DevState* d = s->ds;
  // Blocks of the large windows: the elements that can escape tier 1 are
  // few on a small lattice, and an idle block still takes a whole SM.
  const unsigned big1 = (unsigned)std::min<long long>(BLOCKS_PER_SM * 152, std::max<long long>(16, s->g.ne / 16));
  const unsigned big2 = big1;
  const unsigned bigG = (unsigned)std::min<long long>(kGlobalBlocks, big1);
  ps = prof_begin(s, KID_CLAIM_LARGE);
  if (s->cfg.map_windows == 0) {
    k_claim_big<false><<<big1, BT, smem, s->stream>>>(s->g, s->tay, s->tayf, S, alo, ahi, s->overflow_list,
                                                         &d->noverflow, &d->noverflow_back, &d->overflow_stat,
                                                         s->overflow_list2,
                                                         &d->noverflow2, &d->take[0], nullptr, 0);
    k_claim_big<false><<<big2, BT, smem, s->stream>>>(s->g, s->tay, s->tayf, S, alo, ahi, s->overflow_list2,
                                                     &d->noverflow2, nullptr, &d->overflow2_stat, s->overflow_list,
                                                     &d->noverflow3, &d->take[1], nullptr, 0);
  }
  // tier-1 escapes go straight here when the shared-memory windows are off
  int* n_last = s->cfg.map_windows == 0 ? &d->noverflow3 : &d->noverflow;
  int* stat_last = s->cfg.map_windows == 0 ? &d->overflow3_stat : &d->overflow_stat;
  k_claim_big<true><<<bigG, BT, sizeof(BigHeader), s->stream>>>(
      s->g, s->tay, s->tayf, S, alo, ahi, s->overflow_list, n_last,
      s->cfg.map_windows == 0 ? nullptr : &d->noverflow_back, stat_last, nullptr, nullptr, &d->take[2],
      s->gwin, global_window_words(s->g.nx, s->g.nv, s->g.pad));
  prof_end(s, ps);
  ps = prof_begin(s, KID_RESOLVE);
  k_resolve<<<(unsigned)std::min<size_t>(152, (s->n + 1023) / 1024), 256, 0, s->stream>>>(s->g, S);
  if (s->g.fth_on) launch_clear_outside(s);
  prof_end(s, ps);
  unsigned nb = (unsigned)((s->n / 4 + 255) / 256);
  if (nb > 152 * 16) nb = 152 * 16;
  if (nb == 0) nb = 1;
  ps = prof_begin(s, KID_FINALIZE);
  k_find_holes<<<nb, 256, 0, s->stream>>>(s->g, s->map, s->holes_a, s->ds);
  prof_end(s, ps);
  ps = prof_begin(s, KID_HOLES);
  k_holes<<<1, HT, 0, s->stream>>>(s->g, s->tay, s->map, s->holes_a, s->holes_b, s->holes_b + s->n, s->ds);
  prof_end(s, ps);
  s->launches += s->cfg.map_windows == 0 ? 10 : 8;
}

void launch_read_map(vm_solver* s, int32_t* dst) {
  unsigned nb = (unsigned)((s->n + 255) / 256);
  if (nb > 152 * 16) nb = 152 * 16;
  const int ps = prof_begin(s, KID_READ_MAP);
  k_read_map<<<nb, 256, 0, s->stream>>>(s->map, s->ds, dst, s->n, s->g.ne);
  prof_end(s, ps);
  s->launches++;
}

// The maps of every solve of a group: the single-solve sequence of launches,
// each over the group's work list (dynamic phases from each solve's counters).
size_t group_big_smem(const Grid& g) { return big_smem_bytes(g); }

void group_map(const GroupPlan& G) {
  cudaStream_t st = G.stream;
  const int ns = G.ns;
  const int persist = 152 * 8;
  k_map_begin_group<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(G.D, ns);
  if (G.tot_pair > 0)
    k_claim_pair_group<<<group_grid(G, GP_PAIR, G.tot_pair), 32 * TP, 0, st>>>(G.D, G.off_pair, ns, G.tot_pair);
  k_units<<<1, 1024, 0, st>>>(G.D, ns, GC_PAIR_ESC, persist, G.off_dyn);
  k_claim_small_group<<<group_grid(G, GP_SMALL, persist), 32 * TE, 0, st>>>(G.D, G.off_dyn, ns);
  const int capb = G.big_blocks_cap > 0 ? G.big_blocks_cap : BLOCKS_PER_SM * 152;
  k_units<<<1, 1024, 0, st>>>(G.D, ns, GC_OVF1, capb, G.off_dyn);
  k_claim_big_group<0><<<group_grid(G, GP_BIG1, BLOCKS_PER_SM * 152), BT, G.big_smem, st>>>(G.D, G.off_dyn, ns);
  k_units<<<1, 1024, 0, st>>>(G.D, ns, GC_OVF2, capb, G.off_dyn);
  k_claim_big_group<1><<<group_grid(G, GP_BIG2, BLOCKS_PER_SM * 152), BT, G.big_smem, st>>>(G.D, G.off_dyn, ns);
  k_units<<<1, 1024, 0, st>>>(G.D, ns, GC_OVF3, kGlobalBlocks, G.off_dyn);
  k_claim_big_group<2><<<group_grid(G, GP_BIG3, BLOCKS_PER_SM * 152), BT, sizeof(BigHeader), st>>>(G.D, G.off_dyn, ns);
  k_units<<<1, 1024, 0, st>>>(G.D, ns, GC_REC, 152, G.off_dyn);
  k_resolve_group<<<group_grid(G, GP_RESOLVE, 152 * 4), 256, 0, st>>>(G.D, G.off_dyn, ns);
  if (G.tot_sites > 0)
    k_find_holes_group<<<group_grid(G, GP_FIND_HOLES, G.tot_sites), 256, 0, st>>>(G.D, G.off_sites, ns, G.tot_sites);
  k_units<<<1, 1024, 0, st>>>(G.D, ns, GC_HOLES, 1, G.off_dyn);
  k_holes_group<<<group_grid(G, GP_HOLES, 152), HT, 0, st>>>(G.D, G.off_dyn, ns);
}

// Opt the group's large-window kernels in to shared memory (as map_prepare
// does), up to the per-block limit less their static shared memory.
template <typename K>
static cudaError_t opt_in(K kernel) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(SMEM_MAX - fa.sharedSizeBytes));
}

bool group_map_prepare() {
  cudaError_t e = opt_in(k_claim_big_group<0>);
  if (e == cudaSuccess) e = opt_in(k_claim_big_group<1>);
  if (e != cudaSuccess) note_cuda(e);
  return e == cudaSuccess;
}

}  // namespace vm
