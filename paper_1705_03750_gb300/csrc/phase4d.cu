// 4D phase-space (x, y, vx, vy) form of the metric semi-Lagrangian step, FP64.
//
// The paper implements 2D phase space and gives the 4D generalisation piece by
// piece: 60-number elements and the inverse map of eq. QofP (Sec. 2.1), the
// 15-point quadratic hypersurface (Sec. 2.2.1), percolation with per-axis
// ranges (Sec. 2.3), and Poisson's equation in the space dimensions on a fixed
// grid (Sec. 2.5).  Kernels of one step, on the caller's stream:
//
//   k4_drift        half drift of every element (one thread per element)
//   k4_taylor       T^-1 = adj(T)/det T and G_l = [T^-1]^T H_l T^-1
//   k4_percolate    one block per element: breadth-first flood fill of its
//                   component in a shared-memory bit window around its start
//                   site, frontier waves in shared memory, claims by a 128-bit
//                   compare-and-swap minimum of (d^2 bits, element index);
//                   k4_percolate_big fills the elements that left their window
//                   again over the whole padded lattice (global-memory bits)
//   k4_map_finish   owner of every site from its slot or record; hole list
//   k4_holes        Jacobi rounds of the unexplored-site repair (one block)
//   k4_recon        one block per (x, y) pixel: f at its vx-vy plane by the
//                   15-point interpolation of f_ini at Q(P); pixel mass by a
//                   block reduction (the v-integration fused in)
//   k4_accel        direct sum of the 2D Green function over the pixel masses
//                   for the nodes of the grid and a halo, sources split over
//                   blocks; k4_accel_sum adds the partial sums in order
//   k4_kick_drift   2D TSC of the field, its gradient and Hessian (centred
//                   differences) at the element; kick; second half drift
//   remap           k4_resample (Q_r blend of the beta set, 4^4-term cubic
//                   B-spline of eta), k4_spline_axis x 4 (batched tridiagonal
//                   solves along vy, vx, y, x), k4_reset
//
// Every integer decision (start sites, alpha and beta ranges, the d^2
// comparisons of the percolation, the nearest node of the interpolation) is
// taken on FP64 values computed in one fixed order without fused
// multiply-add (the __d*_rn intrinsics), the order of the FP64 restatement of
// the method, or on FP32 values whose rigorous error bound shows the same
// outcome; the map is therefore exactly the one that restatement gives for
// the same elements.  Values that feed no such decision (the interpolated f,
// the Q_r blend, the spline sums) use fused arithmetic and agree with it to
// rounding; the spline solve divides by the same pivots in the same order;
// the pixel masses are block sums and the field is summed over blocks, so
// element trajectories agree to rounding.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/vlamet4d.h"

namespace {

constexpr int NE4 = 60;  // doubles per element
constexpr int NT4 = 64;  // doubles per Taylor record
constexpr int FCAP = 512;  // frontier capacity of the flood fill (sites per wave)
constexpr int PERC_THREADS = 64;  // one block of two warps per element
static_assert(PERC_THREADS >= NT4, "a block loads its element's Taylor record one value per thread");
constexpr int ERR_NC = 1, ERR_OVF = 2, ERR_INT = 4;
constexpr unsigned long long KEY_EMPTY = ~0ull;

struct G4 {
  int32_t n[4];
  long long nsite;
  long long st[4];  // strides of f
  double lo[4], d[4], inv_d[4], dm[4], inv_dm[4], ctr[4];
  int32_t s, pad, K[4], L[4], ne;
  double alpha, beta, half_dt, dt, twoG, dV;
  int32_t E, We0, We1;  // field cache: nodes [-E, n0-1+E] x [-E, n1-1+E]
  int32_t R, W;         // flood window: side W = 2R+1 sites around the start site
  int32_t max_rounds;
};

struct Dev4 {
  int32_t err;
  int32_t nholes;
  int32_t bad_where;
  int32_t novf;  // elements whose component left the shared-memory window (this map)
  int32_t rounds;  // hole-repair rounds of the last map
  unsigned long long d2_evals;  // distance evaluations of the percolation kernels (cumulative)
};

// whole-lattice flood fill of the elements that left their window: per slot,
// a bit per site of the padded lattice and two frontier buffers
constexpr int BIG_SLOTS = 8;
constexpr int BIG_FCAP = 1 << 18;

__device__ __forceinline__ double M_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double A_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double S_(double a, double b) { return __dsub_rn(a, b); }

__device__ __forceinline__ void bad(Dev4* ds, int where) {
  atomicOr(&ds->err, ERR_INT);
  atomicCAS(&ds->bad_where, 0, where);
}

// symmetric index of (b, c) in the order 00,01,02,03,11,12,13,22,23,33
__host__ __device__ __forceinline__ int sym4(int b, int c) {
  if (b > c) {
    int t = b;
    b = c;
    c = t;
  }
  return 4 * b - (b * (b - 1)) / 2 + (c - b);
}

__device__ __forceinline__ long long nearest_i(double u) { return (long long)floor(A_(u, 0.5)); }

// ---------------------------------------------------------------------------
// Sec. 2.1: inverse map
// ---------------------------------------------------------------------------

// dQ = y - T^-1 s / 2, y = T^-1 dP, s_l = dP^T G_l dP
__device__ __forceinline__ void qofp4(const double* __restrict__ t, const double* P, double* dQ) {
  double dP[4], s[4];
  for (int a = 0; a < 4; a++) dP[a] = S_(P[a], t[a]);
  const double* Ti = t + 4;
#pragma unroll
  for (int l = 0; l < 4; l++) {
    const double* G = t + 20 + 10 * l;
    double g[4];
#pragma unroll
    for (int b = 0; b < 4; b++)
      g[b] = A_(A_(A_(M_(G[sym4(b, 0)], dP[0]), M_(G[sym4(b, 1)], dP[1])), M_(G[sym4(b, 2)], dP[2])),
                M_(G[sym4(b, 3)], dP[3]));
    s[l] = A_(A_(A_(M_(dP[0], g[0]), M_(dP[1], g[1])), M_(dP[2], g[2])), M_(dP[3], g[3]));
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    double y = A_(A_(A_(M_(Ti[4 * a], dP[0]), M_(Ti[4 * a + 1], dP[1])), M_(Ti[4 * a + 2], dP[2])),
                  M_(Ti[4 * a + 3], dP[3]));
    double c = A_(A_(A_(M_(Ti[4 * a], s[0]), M_(Ti[4 * a + 1], s[1])), M_(Ti[4 * a + 2], s[2])),
                  M_(Ti[4 * a + 3], s[3]));
    dQ[a] = S_(y, M_(0.5, c));
  }
}

// The same inverse map with fused multiply-adds, for values that feed no
// integer decision (or whose decision is re-taken in the exact order near
// its threshold): about half the FP64 instructions of qofp4.
__device__ __forceinline__ void qofp4_f(const double* __restrict__ t, const double* P, double* dQ) {
  double dP[4], s[4];
  for (int a = 0; a < 4; a++) dP[a] = P[a] - t[a];
  const double* Ti = t + 4;
#pragma unroll
  for (int l = 0; l < 4; l++) {
    const double* G = t + 20 + 10 * l;
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      double gb = G[sym4(b, 0)] * dP[0];
      gb = fma(G[sym4(b, 1)], dP[1], gb);
      gb = fma(G[sym4(b, 2)], dP[2], gb);
      gb = fma(G[sym4(b, 3)], dP[3], gb);
      acc = fma(dP[b], gb, acc);
    }
    s[l] = acc;
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    double y = Ti[4 * a] * dP[0], c = Ti[4 * a] * s[0];
    for (int b = 1; b < 4; b++) {
      y = fma(Ti[4 * a + b], dP[b], y);
      c = fma(Ti[4 * a + b], s[b], c);
    }
    dQ[a] = fma(-0.5, c, y);
  }
}

// squared Lagrangian distance in element spacings (Sec. 2.3.1, eq. distdef)
__device__ __forceinline__ double dist2_4(const G4& g, const double* __restrict__ t, const double* P,
                                          double* x) {
  double dQ[4], xl[4];
  qofp4(t, P, dQ);
  for (int a = 0; a < 4; a++) xl[a] = M_(dQ[a], g.inv_dm[a]);
  if (x)
    for (int a = 0; a < 4; a++) x[a] = xl[a];
  return A_(A_(A_(M_(xl[0], xl[0]), M_(xl[1], xl[1])), M_(xl[2], xl[2])), M_(xl[3], xl[3]));
}

__device__ __forceinline__ void elem_coords(const G4& g, int m, int* k) {
  for (int a = 3; a >= 0; a--) {
    k[a] = m % g.L[a];
    m /= g.L[a];
  }
}

__device__ __forceinline__ double site_coord(const G4& g, int a, long long i) {
  return A_(g.lo[a], M_((double)i, g.d[a]));
}

// ---------------------------------------------------------------------------
// elements
// ---------------------------------------------------------------------------

__global__ void k4_reset(G4 g, double* __restrict__ el) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.ne) return;
  int k[4];
  elem_coords(g, m, k);
  double* e = el + (size_t)NE4 * m;
  for (int q = 0; q < NE4; q++) e[q] = 0.0;
  for (int a = 0; a < 4; a++) {
    e[a] = A_(g.ctr[a], M_((double)(k[a] - g.K[a] - 1), g.dm[a]));
    e[4 + 5 * a] = 1.0;
  }
}

// half drift: x_a += v_a h, rows a = 0, 1 of T and H take rows a + 2 times h
__device__ __forceinline__ void drift_one(double* e, double h) {
  for (int a = 0; a < 2; a++) {
    e[a] = A_(e[a], M_(e[a + 2], h));
    for (int b = 0; b < 4; b++) e[4 + 4 * a + b] = A_(e[4 + 4 * a + b], M_(e[4 + 4 * (a + 2) + b], h));
    for (int q = 0; q < 10; q++) e[20 + 10 * a + q] = A_(e[20 + 10 * a + q], M_(e[20 + 10 * (a + 2) + q], h));
  }
}

__global__ void k4_drift(G4 g, double* __restrict__ el) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.ne) return;
  drift_one(el + (size_t)NE4 * m, g.half_dt);
}

// T^-1 by the adjugate from the 2x2 minors of rows 0-1 (s) and rows 2-3 (c)
__device__ void inverse4(const double* A, double* B) {
  const double a00 = A[0], a01 = A[1], a02 = A[2], a03 = A[3];
  const double a10 = A[4], a11 = A[5], a12 = A[6], a13 = A[7];
  const double a20 = A[8], a21 = A[9], a22 = A[10], a23 = A[11];
  const double a30 = A[12], a31 = A[13], a32 = A[14], a33 = A[15];
  const double s0 = S_(M_(a00, a11), M_(a10, a01)), s1 = S_(M_(a00, a12), M_(a10, a02));
  const double s2 = S_(M_(a00, a13), M_(a10, a03)), s3 = S_(M_(a01, a12), M_(a11, a02));
  const double s4 = S_(M_(a01, a13), M_(a11, a03)), s5 = S_(M_(a02, a13), M_(a12, a03));
  const double c5 = S_(M_(a22, a33), M_(a32, a23)), c4 = S_(M_(a21, a33), M_(a31, a23));
  const double c3 = S_(M_(a21, a32), M_(a31, a22)), c2 = S_(M_(a20, a33), M_(a30, a23));
  const double c1 = S_(M_(a20, a32), M_(a30, a22)), c0 = S_(M_(a20, a31), M_(a30, a21));
  const double det =
      A_(S_(A_(A_(S_(M_(s0, c5), M_(s1, c4)), M_(s2, c3)), M_(s3, c2)), M_(s4, c1)), M_(s5, c0));
  const double id = __ddiv_rn(1.0, det);
  B[0] = M_(A_(S_(M_(a11, c5), M_(a12, c4)), M_(a13, c3)), id);
  B[1] = M_(S_(S_(M_(a02, c4), M_(a01, c5)), M_(a03, c3)), id);
  B[2] = M_(A_(S_(M_(a31, s5), M_(a32, s4)), M_(a33, s3)), id);
  B[3] = M_(S_(S_(M_(a22, s4), M_(a21, s5)), M_(a23, s3)), id);
  B[4] = M_(S_(S_(M_(a12, c2), M_(a10, c5)), M_(a13, c1)), id);
  B[5] = M_(A_(S_(M_(a00, c5), M_(a02, c2)), M_(a03, c1)), id);
  B[6] = M_(S_(S_(M_(a32, s2), M_(a30, s5)), M_(a33, s1)), id);
  B[7] = M_(A_(S_(M_(a20, s5), M_(a22, s2)), M_(a23, s1)), id);
  B[8] = M_(A_(S_(M_(a10, c4), M_(a11, c2)), M_(a13, c0)), id);
  B[9] = M_(S_(S_(M_(a01, c2), M_(a00, c4)), M_(a03, c0)), id);
  B[10] = M_(A_(S_(M_(a30, s4), M_(a31, s2)), M_(a33, s0)), id);
  B[11] = M_(S_(S_(M_(a21, s2), M_(a20, s4)), M_(a23, s0)), id);
  B[12] = M_(S_(S_(M_(a11, c1), M_(a10, c3)), M_(a12, c0)), id);
  B[13] = M_(A_(S_(M_(a00, c3), M_(a01, c1)), M_(a02, c0)), id);
  B[14] = M_(S_(S_(M_(a31, s1), M_(a30, s3)), M_(a32, s0)), id);
  B[15] = M_(A_(S_(M_(a20, s3), M_(a21, s1)), M_(a22, s0)), id);
}

// FP32 record of an element's inverse map in element units, for the certified
// percolation tests: with p_b = (P_b - P_m,b)/dm_b,
//   xi_a = (Q_a - Q_m,a)/dm_a = sum_b A_ab p_b + sum_{b<=c} B_a,bc p_b p_c,
// A_ab = T^-1_ab dm_b/dm_a, B_a,bc = -(1/2)(2 - [b=c]) sum_l T^-1_al G_l,bc dm_b dm_c/dm_a
// (the same polynomial the FP64 evaluation computes in another order), and
// K_a = (1/2) sum_l |T^-1_al| max_bc |G_l,bc| dm_b dm_c / dm_a (bounds the
// absolute terms of that FP64 evaluation), nA_a = sum_b |A_ab|,
// nB_a = sum_bc |B_a,bc|.  Layout: A[16], B[40], K[4], nA[4], nB[4], pad.
constexpr int NF4 = 72;

__global__ void __launch_bounds__(128) k4_taylor(G4 g, const double* __restrict__ el, double* __restrict__ tay,
                                                 float* __restrict__ tay32) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.ne) return;
  const double* e = el + (size_t)NE4 * m;
  double* t = tay + (size_t)NT4 * m;
  double Ti[16];
  inverse4(e + 4, Ti);
  for (int a = 0; a < 4; a++) t[a] = e[a];
  for (int q = 0; q < 16; q++) t[4 + q] = Ti[q];
  for (int l = 0; l < 4; l++) {
    const double* h = e + 20 + 10 * l;
    double Am[4][4];
    for (int b = 0; b < 4; b++)
      for (int c = 0; c < 4; c++)
        Am[b][c] = A_(A_(A_(M_(h[sym4(b, 0)], Ti[c]), M_(h[sym4(b, 1)], Ti[4 + c])), M_(h[sym4(b, 2)], Ti[8 + c])),
                      M_(h[sym4(b, 3)], Ti[12 + c]));
    for (int b = 0; b < 4; b++)
      for (int c = b; c < 4; c++)
        t[20 + 10 * l + sym4(b, c)] =
            A_(A_(A_(M_(Ti[b], Am[0][c]), M_(Ti[4 + b], Am[1][c])), M_(Ti[8 + b], Am[2][c])), M_(Ti[12 + b], Am[3][c]));
  }
  int k[4];
  elem_coords(g, m, k);
  for (int a = 0; a < 4; a++) t[60 + a] = A_(g.ctr[a], M_((double)(k[a] - g.K[a] - 1), g.dm[a]));
  float* r = tay32 + (size_t)NF4 * m;
  for (int a = 0; a < 4; a++) {
    for (int b = 0; b < 4; b++) r[4 * a + b] = (float)(Ti[4 * a + b] * g.dm[b] * g.inv_dm[a]);
    double kmax = 0.0;
    for (int l = 0; l < 4; l++) {
      double gm = 0.0;
      for (int b = 0; b < 4; b++)
        for (int c = b; c < 4; c++) gm = fmax(gm, fabs(t[20 + 10 * l + sym4(b, c)]) * g.dm[b] * g.dm[c]);
      kmax += fabs(Ti[4 * a + l]) * gm;
    }
    r[56 + a] = (float)(0.5 * kmax * g.inv_dm[a] * 1.0000001);
    for (int b = 0; b < 4; b++)
      for (int c = b; c < 4; c++) {
        double v = 0.0;
        for (int l = 0; l < 4; l++) v += Ti[4 * a + l] * t[20 + 10 * l + sym4(b, c)];
        r[16 + 10 * a + sym4(b, c)] = (float)(-0.5 * (b == c ? 1.0 : 2.0) * v * g.dm[b] * g.dm[c] * g.inv_dm[a]);
      }
  }
  for (int a = 0; a < 4; a++) {
    float na = 0.f, nb = 0.f;
    for (int b = 0; b < 4; b++) na += fabsf(r[4 * a + b]);
    for (int q = 0; q < 10; q++) nb += fabsf(r[16 + 10 * a + q]);
    r[60 + a] = na * 1.000001f;
    r[64 + a] = nb * 1.000001f;
  }
  for (int q = 68; q < NF4; q++) r[q] = 0.f;
}

// FP32 offsets xi of an element at a site with rigorous bounds e_a >=
// |xi_a - x_a|, x_a the FP64 evaluation's (dQ_a / dm_a in the exact order).
// Roundings: products p_b p_c (1), coefficients (1), the FMA chain of 14
// terms (14): below 17 u = 1.0e-6 of the sum of absolute terms; the bound
// dp of the inputs p is carried through the linear and quadratic terms; the
// FP64 evaluation's own error (under 1e-14 of its absolute terms, bounded by
// K (sum |p|)^2 and the linear part) adds the last term.
constexpr float kRel4 = 2.0e-6f, kAbs4 = 1.0e-9f;

__device__ __forceinline__ void eval32_4(const float* __restrict__ R, const float* p, const float* dp, float* xi,
                                         float* e) {
  // the absolute terms bounded by the row norms: |sum A p| <= nA max|p|,
  // |sum B p p| <= nB max|p|^2, and the input bound likewise
  const float pm = fmaxf(fmaxf(fabsf(p[0]), fabsf(p[1])), fmaxf(fabsf(p[2]), fabsf(p[3])));
  const float dm = fmaxf(fmaxf(dp[0], dp[1]), fmaxf(dp[2], dp[3]));
  const float dpp = fmaf(2.f * pm, dm, dm * dm);
  const float S = 4.f * pm;
  float pp[10];
  for (int b = 0; b < 4; b++)
    for (int c = b; c < 4; c++) pp[sym4(b, c)] = p[b] * p[c];
  for (int a = 0; a < 4; a++) {
    float v = 0.f;
    for (int b = 0; b < 4; b++) v = fmaf(R[4 * a + b], p[b], v);
    for (int q = 0; q < 10; q++) v = fmaf(R[16 + 10 * a + q], pp[q], v);
    xi[a] = v;
    const float nA = R[60 + a], nB = R[64 + a];
    const float E = fmaf(nB, pm * pm, nA * pm);
    const float Ep = fmaf(nB, dpp, nA * dm);
    e[a] = kRel4 * E + kAbs4 * (1.f + E) + 1.00001f * Ep + 1e-13f * R[56 + a] * (S * S) * 16.f;
  }
}

// p_b = j_b h_b + r_b (element units) from the offset j of the site from a
// reference site, jh_b = (float)j_b * h_b looked up in a per-block table,
// and the element's FP32 offset r of that reference site; dp bounds its
// distance to the FP64 evaluation's dP_b / dm_b
__device__ __forceinline__ void p_of(const float* jh, const float* r, float* p, float* dp) {
  for (int b = 0; b < 4; b++) {
    p[b] = jh[b] + r[b];
    dp[b] = 6.0e-8f * (fabsf(r[b]) + 2.f * fabsf(jh[b]) + fabsf(p[b])) + 1e-12f;
  }
}

// d^2 in FP32 and a bound on its distance to the FP64 value
__device__ __forceinline__ float d2_32(const float* xi, const float* e, float* bd) {
  float d2 = 0.f, b = 0.f;
  for (int a = 0; a < 4; a++) {
    d2 = fmaf(xi[a], xi[a], d2);
    b = fmaf(e[a], 2.f * fabsf(xi[a]) + e[a], b);
  }
  *bd = b + 6e-7f * d2 + 1e-30f;
  return d2;
}

// ---------------------------------------------------------------------------
// Sec. 2.3.1: percolation
// ---------------------------------------------------------------------------

// 128-bit compare-and-swap on global memory (sm_90 and later)
__device__ __forceinline__ ulonglong2 cas128_4(ulonglong2* addr, ulonglong2 cmp, ulonglong2 val) {
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

// key.y = bits of d^2 (non-negative doubles order as integers), key.x = element:
// the smaller (d^2, index) wins the site
__device__ __forceinline__ void claim4(ulonglong2* key, unsigned long long dbits, unsigned long long idx) {
  ulonglong2 cur = __ldcg(key);
  const ulonglong2 val = make_ulonglong2(idx, dbits);
  while (dbits < cur.y || (dbits == cur.y && idx < cur.x)) {
    const ulonglong2 prev = cas128_4(key, cur, val);
    if (prev.x == cur.x && prev.y == cur.y) break;
    cur = prev;
  }
}

// Claim of in-grid site p by element m (Sec. 2.3.1: smaller d, then smaller
// index).  The site's slot takes m + 1 by an exchange; a first claimant needs
// nothing more.  A claim that displaces an owner folds the exact FP64 keys of
// both into the site's 128-bit record: every claimant after the first reaches
// the record with its own key and its predecessor's, so the record's minimum
// is the exact winner of a contested site, and FP64 distances are spent on
// contested sites only.
__device__ __forceinline__ void claim_site(const G4& g, uint32_t* __restrict__ slot, ulonglong2* __restrict__ key,
                                           long long p, int m, const double* tm, const double* __restrict__ tay,
                                           const long long* gs, bool have_d2, double d2, unsigned& nev, Dev4* ds) {
  const uint32_t old = atomicExch(slot + p, (uint32_t)m + 1u);
  if (old == 0u) return;
  double P[4];
  for (int a = 0; a < 4; a++) P[a] = site_coord(g, a, gs[a]);
  if (!have_d2) {
    d2 = dist2_4(g, tm, P, nullptr);
    nev++;
  }
  claim4(key + p, (unsigned long long)__double_as_longlong(d2), (unsigned long long)m);
  const int o = (int)old - 1;
  if (o == m) return;
  if (o < 0 || o >= g.ne) {
    bad(ds, 45);
    return;
  }
  nev++;
  const double d2o = dist2_4(g, tay + (size_t)NT4 * o, P, nullptr);
  claim4(key + p, (unsigned long long)__double_as_longlong(d2o), (unsigned long long)o);
}

// The percolation test (Sec. 2.3.1): the site passes for m unless an element
// of the alpha ranges (per axis: below -alpha {-1,0}, below alpha {0}, else
// {0,1}) proposes a strictly smaller distance.
__device__ bool passes4(const G4& g, const int* k, const double* tself, const double* __restrict__ tay,
                        const double* P, double* d2o, unsigned& nev) {
  double x[4];
  const double d2 = dist2_4(g, tself, P, x);
  *d2o = d2;
  nev++;
  int lo[4], hi[4];
  for (int a = 0; a < 4; a++) {
    if (x[a] < -g.alpha) {
      lo[a] = -1;
      hi[a] = 0;
    } else if (x[a] < g.alpha) {
      lo[a] = 0;
      hi[a] = 0;
    } else {
      lo[a] = 0;
      hi[a] = 1;
    }
  }
  for (int o0 = lo[0]; o0 <= hi[0]; o0++)
    for (int o1 = lo[1]; o1 <= hi[1]; o1++)
      for (int o2 = lo[2]; o2 <= hi[2]; o2++)
        for (int o3 = lo[3]; o3 <= hi[3]; o3++) {
          if ((o0 | o1 | o2 | o3) == 0) continue;
          const int k0 = k[0] + o0, k1 = k[1] + o1, k2 = k[2] + o2, k3 = k[3] + o3;
          if (k0 < 0 || k0 >= g.L[0] || k1 < 0 || k1 >= g.L[1] || k2 < 0 || k2 >= g.L[2] || k3 < 0 ||
              k3 >= g.L[3])
            continue;
          const int mm = ((k0 * g.L[1] + k1) * g.L[2] + k2) * g.L[3] + k3;
          nev++;
          if (dist2_4(g, tay + (size_t)NT4 * mm, P, nullptr) < d2) return false;
        }
  return true;
}

// One block per element: its 4-connected component of passing sites from the
// site nearest to its position, within the padded lattice [-pad, n-1+pad]^4,
// explored wave by wave inside a window of side W around the start site.
// Each wave runs in packed phases, so that the FP64 unit (a few operations
// per clock per SM on this part) sees as little work as possible and that on
// full warps:
//   1. expansion: the 8 neighbours of every frontier site are stamped in the
//      window's visited bits; newly reached sites form the test list;
//   2. own offsets: one lane per listed site evaluates the element's inverse
//      map in FP32 with a bound on its distance to the FP64 value
//      (eval32_4); the alpha ranges are decided where the bound settles them
//      (else the site is left to the exact test), and the (site, neighbour)
//      pairs they name are listed;
//   3. pair distances: one lane per pair, FP32 with bounds: a neighbour
//      certainly closer fails the site, one whose comparison the bound
//      leaves open sends the site to the exact test;
//   4. exact work: the sites left open run the FP64 test in the oracle's
//      order; every passing site's claim key takes its FP64 d^2.
// The outcome is the all-FP64 percolation's.  Passing sites are claimed and
// form the next frontier.  An element whose component would leave the window,
// or whose lists outgrow their buffers, is listed for k4_percolate_big.
constexpr int TCAP = 512;  // sites tested per wave
constexpr int PCAP = 1024;  // (site, neighbour) pairs per wave
enum : int { ST_PASS = 0, ST_OPEN = 1, ST_FAIL = 2 };

// list entries hold a site's four window coordinates, one byte each (W <= 25)
__device__ __forceinline__ void decode_w(int lw, int /*W*/, int* l) {
  l[0] = lw & 255;
  l[1] = (lw >> 8) & 255;
  l[2] = (lw >> 16) & 255;
  l[3] = (lw >> 24) & 255;
}
__device__ __forceinline__ int pack_w(const int* l) { return l[0] | (l[1] << 8) | (l[2] << 16) | (l[3] << 24); }

__global__ void __launch_bounds__(PERC_THREADS, 8) k4_percolate(G4 g, const double* __restrict__ el,
                                                    const double* __restrict__ tay,
                                                    const float* __restrict__ tay32, ulonglong2* __restrict__ key,
                                                    uint32_t* __restrict__ slot, int32_t* __restrict__ ovf_list,
                                                    Dev4* ds) {
  extern __shared__ uint32_t sm4[];
  const int W = g.W;
  const int nwin = W * W * W * W;
  const int nwords = (nwin + 31) >> 5;
  uint32_t* stamp = sm4;
  int32_t* front = (int32_t*)(sm4 + ((nwords + 3) & ~3));  // FCAP
  int32_t* tlist = front + FCAP;                             // TCAP
  int32_t* pairs = tlist + TCAP;                             // PCAP
  int32_t* status = pairs + PCAP;                            // TCAP
  float* d2f = (float*)(status + TCAP);                      // TCAP
  float* bdf = d2f + TCAP;                                   // TCAP
  __shared__ double tself[NT4];
  __shared__ float rself[NF4];
  __shared__ float roff[81][4];  // per offset code: the element's FP32 offset of the start site
  __shared__ float jht[4][32];   // (float)(l - R) * h_a for window coordinate l
  __shared__ double pst[4];      // the start site's coordinates
  __shared__ int org[4], kk[4];
  __shared__ int go, ncur, ntest, npairs, ovf;
  const int m = blockIdx.x;
  const int tid = threadIdx.x;
  unsigned nev = 0;
  if (tid < NT4) tself[tid] = tay[(size_t)NT4 * m + tid];
  for (int q = tid; q < NF4; q += blockDim.x) rself[q] = tay32[(size_t)NF4 * m + q];
  for (int w = tid; w < nwords; w += blockDim.x) stamp[w] = 0u;
  const float af = (float)g.alpha, aerr = 1e-7f * (1.f + af);
  if (tid == 0) {
    const double* e = el + (size_t)NE4 * m;
    int ok = 1;
    for (int a = 0; a < 4; a++) {
      const double u = M_(S_(e[a], g.lo[a]), g.inv_d[a]);
      if (!(u > -1e9 && u < 1e9)) {
        ok = 0;
        break;
      }
      const long long g0 = nearest_i(u);
      if (g0 < -g.pad || g0 >= g.n[a] + g.pad) ok = 0;
      org[a] = (int)g0 - g.R;
    }
    int kc[4];
    elem_coords(g, m, kc);
    for (int a = 0; a < 4; a++) kk[a] = kc[a];
    go = ok;
    ovf = 0;
    // the start site is the first wave's only site to test
    const int c = g.R;
    const int lc[4] = {c, c, c, c};
    tlist[0] = pack_w(lc);
    ntest = 1;
    ncur = 0;
  }
  __syncthreads();
  if (!go) return;
  if (tid == 0) {
    const int c = g.R;
    const int lw = ((c * W + c) * W + c) * W + c;
    stamp[lw >> 5] |= 1u << (lw & 31);
  }
  int kl[4];
  for (int a = 0; a < 4; a++) kl[a] = kk[a];
  if (tid < 4) pst[tid] = site_coord(g, tid, (long long)org[tid] + g.R);
  for (int q = tid; q < 4 * 32; q += blockDim.x) {
    const int a = q >> 5, l = q & 31;
    jht[a][l] = (float)(l - g.R) * (float)(g.d[a] * g.inv_dm[a]);
  }
  __syncthreads();
  // offsets (start site - P_m') / dm of the element and its 80 neighbours,
  // in FP64, rounded once to FP32
  for (int code = tid; code < 81; code += blockDim.x) {
    int o[4], c = code, ok = 1;
    for (int a = 3; a >= 0; a--) {
      o[a] = c % 3 - 1;
      c /= 3;
    }
    int mm = 0;
    for (int a = 0; a < 4; a++) {
      const int ka = kl[a] + o[a];
      ok &= (ka >= 0 && ka < g.L[a]);
      mm = mm * g.L[a] + ka;
    }
    for (int a = 0; a < 4; a++)
      roff[code][a] = ok ? (float)((pst[a] - __ldg(tay + (size_t)NT4 * mm + a)) * g.inv_dm[a]) : 0.f;
  }
  __syncthreads();
  bool first = true;
  while (true) {
    // 1. expansion of the frontier (the first wave tests the start site only)
    if (!first) {
      if (tid == 0) ntest = 0;
      __syncthreads();
      const int ntask = ncur * 8;
      for (int t = tid; t < ntask; t += blockDim.x) {
        const int e = t >> 3, dir = t & 7, ax = dir >> 1, sg = (dir & 1) ? 1 : -1;
        int l[4];
        decode_w(front[e], W, l);
        l[ax] += sg;
        const long long ga = (long long)org[ax] + l[ax];
        if (ga < -g.pad || ga >= g.n[ax] + g.pad) continue;
        if (l[ax] < 0 || l[ax] >= W) {
          ovf = 1;
          continue;
        }
        const int nw = ((l[0] * W + l[1]) * W + l[2]) * W + l[3];
        const uint32_t bit = 1u << (nw & 31);
        if (atomicOr(&stamp[nw >> 5], bit) & bit) continue;
        const int idx = atomicAdd(&ntest, 1);
        if (idx < TCAP)
          tlist[idx] = pack_w(l);
        else
          ovf = 1;
      }
    }
    first = false;
    if (tid == 0) npairs = 0;
    __syncthreads();
    const int nt = ovf ? 0 : min(ntest, TCAP);
    if (nt == 0) break;
    // 2. own offsets in FP32, certified alpha ranges, the pair list
    for (int i = tid; i < nt; i += blockDim.x) {
      int l[4];
      decode_w(tlist[i], W, l);
      float jh[4];
      for (int a = 0; a < 4; a++) jh[a] = jht[a][l[a]];
      float pv[4], dp[4], x[4], e[4];
      p_of(jh, roff[40], pv, dp);
      eval32_4(rself, pv, dp, x, e);
      float bd;
      d2f[i] = d2_32(x, e, &bd);
      bdf[i] = bd;
      int lo[4], hi[4], open = 0;
      for (int a = 0; a < 4; a++) {
        const float E = e[a] + aerr;
        // below -alpha: {-1,0}; below alpha: {0}; else {0,1}, each comparison certified
        const bool below_lo = x[a] + E < -af, above_lo = x[a] - E > -af;
        const bool below_hi = x[a] + E < af, above_hi = x[a] - E > af;
        if (below_lo) {
          lo[a] = -1;
          hi[a] = 0;
        } else if (above_lo && below_hi) {
          lo[a] = 0;
          hi[a] = 0;
        } else if (above_hi) {
          lo[a] = 0;
          hi[a] = 1;
        } else {
          open = 1;
          lo[a] = hi[a] = 0;
        }
      }
      status[i] = open ? ST_OPEN : ST_PASS;
      if (open) continue;
      int cnt = 0, codes[15];
      for (int o0 = lo[0]; o0 <= hi[0]; o0++)
        for (int o1 = lo[1]; o1 <= hi[1]; o1++)
          for (int o2 = lo[2]; o2 <= hi[2]; o2++)
            for (int o3 = lo[3]; o3 <= hi[3]; o3++) {
              if ((o0 | o1 | o2 | o3) == 0) continue;
              const int k0 = kl[0] + o0, k1 = kl[1] + o1, k2 = kl[2] + o2, k3 = kl[3] + o3;
              if (k0 < 0 || k0 >= g.L[0] || k1 < 0 || k1 >= g.L[1] || k2 < 0 || k2 >= g.L[2] || k3 < 0 ||
                  k3 >= g.L[3])
                continue;
              codes[cnt++] = (((o0 + 1) * 3 + (o1 + 1)) * 3 + (o2 + 1)) * 3 + (o3 + 1);
            }
      if (cnt) {
        const int at = atomicAdd(&npairs, cnt);
        if (at + cnt <= PCAP) {
          for (int q = 0; q < cnt; q++) pairs[at + q] = (i << 7) | codes[q];
        } else {
          ovf = 1;
        }
      }
    }
    __syncthreads();
    if (ovf) break;
    // 3. the neighbours' distances at the listed sites, FP32 with bounds
    const int np = npairs;
    for (int j = tid; j < np; j += blockDim.x) {
      const int pr = pairs[j];
      const int i = pr >> 7;
      int code = pr & 127, o[4];
      for (int a = 3; a >= 0; a--) {
        o[a] = code % 3 - 1;
        code /= 3;
      }
      const int mm = (((kl[0] + o[0]) * g.L[1] + (kl[1] + o[1])) * g.L[2] + (kl[2] + o[2])) * g.L[3] + (kl[3] + o[3]);
      int l[4];
      decode_w(tlist[i], W, l);
      float jh[4];
      for (int a = 0; a < 4; a++) jh[a] = jht[a][l[a]];
      float pv[4], dp[4], x[4], e[4], bn;
      p_of(jh, roff[pr & 127], pv, dp);
      eval32_4(tay32 + (size_t)NF4 * mm, pv, dp, x, e);
      const float dn = d2_32(x, e, &bn);
      const float dm = d2f[i], bm = bdf[i];
      if (dn + bn < dm - bm)
        status[i] = ST_FAIL;
      else if (!(dn - bn > dm + bm))
        atomicMax(&status[i], ST_OPEN);
    }
    if (tid == 0) ncur = 0;
    __syncthreads();
    // 4. exact tests where the bounds left them open; claims
    for (int i = tid; i < nt; i += blockDim.x) {
      const int st = status[i];
      if (st == ST_FAIL) continue;
      int l[4];
      decode_w(tlist[i], W, l);
      long long gs[4];
      for (int a = 0; a < 4; a++) gs[a] = (long long)org[a] + l[a];
      double d2 = 0.0;
      if (st == ST_OPEN) {
        double P[4];
        for (int a = 0; a < 4; a++) P[a] = site_coord(g, a, gs[a]);
        if (!passes4(g, kl, tself, tay, P, &d2, nev)) continue;
      }
      bool in = true;
      long long p = 0;
      for (int a = 0; a < 4; a++) {
        in = in && gs[a] >= 0 && gs[a] < g.n[a];
        p += gs[a] * g.st[a];
      }
      if (in) claim_site(g, slot, key, p, m, tself, tay, gs, st == ST_OPEN, d2, nev, ds);
      const int idx = atomicAdd(&ncur, 1);
      if (idx < FCAP)
        front[idx] = tlist[i];
      else
        ovf = 1;
    }
    __syncthreads();
    if (ovf || ncur == 0) break;
  }
  // the component reached the window's edge (or a list its buffer): the
  // element is filled again over the whole padded lattice (its claims so far
  // are a subset of the full component's, with the same keys)
  if (tid == 0 && ovf) ovf_list[atomicAdd(&ds->novf, 1)] = m;
  for (int o = 16; o > 0; o >>= 1) nev += __shfl_down_sync(0xffffffffu, nev, o);
  if ((tid & 31) == 0 && nev) atomicAdd(&ds->d2_evals, (unsigned long long)nev);
}

// Whole-lattice flood fill of the listed elements: the same breadth-first
// search over the padded lattice [-pad, n-1+pad]^4, with its visited bits and
// frontiers in global memory (one slot per block).
__global__ void __launch_bounds__(256) k4_percolate_big(G4 g, const double* __restrict__ el,
                                                        const double* __restrict__ tay, ulonglong2* __restrict__ key,
                                                        uint32_t* __restrict__ slot,
                                                        const int32_t* __restrict__ ovf_list, uint32_t* __restrict__ big,
                                                        Dev4* ds) {
  __shared__ double tself[NT4];
  __shared__ int kk[4];
  __shared__ int go, ncur, nnext, bad_wave;
  const int nlist = ds->novf;
  long long pw[4], npad = 1;
  for (int a = 0; a < 4; a++) {
    pw[a] = g.n[a] + 2 * g.pad;
    npad *= pw[a];
  }
  const long long nwords = (npad + 31) >> 5;
  const size_t slot_words = (size_t)((nwords + 63) & ~63ll) + 2 * (size_t)BIG_FCAP;
  uint32_t* stamp = big + (size_t)blockIdx.x * slot_words;
  int32_t* front0 = (int32_t*)(stamp + ((nwords + 63) & ~63ll));
  int32_t* front1 = front0 + BIG_FCAP;
  const int tid = threadIdx.x;
  unsigned nev = 0;
  for (int it = blockIdx.x; it < nlist; it += gridDim.x) {
    const int m = ovf_list[it];
    __syncthreads();
    if (tid < NT4) tself[tid] = tay[(size_t)NT4 * m + tid];
    for (long long w = tid; w < nwords; w += blockDim.x) stamp[w] = 0u;
    if (tid == 0) {
      const double* e = el + (size_t)NE4 * m;
      long long p0 = 0;
      bool ok = true;
      for (int a = 0; a < 4; a++) {
        const double u = M_(S_(e[a], g.lo[a]), g.inv_d[a]);
        const long long g0 = nearest_i(u);
        ok = ok && (g0 >= -g.pad && g0 < g.n[a] + g.pad);
        p0 = p0 * pw[a] + (g0 + g.pad);
      }
      int kc[4];
      elem_coords(g, m, kc);
      for (int a = 0; a < 4; a++) kk[a] = kc[a];
      go = ok;
      ncur = 0;
      bad_wave = 0;
      if (ok) front0[0] = (int32_t)p0;
    }
    __syncthreads();
    __threadfence_block();
    if (!go) continue;
    if (tid == 0) {
      // the start site passed in the window pass (the element overflowed from it)
      const long long p0 = front0[0];
      atomicOr(&stamp[p0 >> 5], 1u << (p0 & 31));
      ncur = 1;
    }
    __syncthreads();
    int kl[4];
    for (int a = 0; a < 4; a++) kl[a] = kk[a];
    int cur = 0;
    while (ncur > 0) {
      if (tid == 0) nnext = 0;
      __syncthreads();
      const int32_t* fc = cur ? front1 : front0;
      int32_t* fn = cur ? front0 : front1;
      const long long ntask = (long long)ncur * 8;
      for (long long t = tid; t < ntask; t += blockDim.x) {
        const long long e = t >> 3;
        const int dir = (int)(t & 7), ax = dir >> 1, sg = (dir & 1) ? 1 : -1;
        long long r = fc[e], gl[4];
        for (int a = 3; a >= 0; a--) {
          gl[a] = r % pw[a];
          r /= pw[a];
        }
        gl[ax] += sg;
        if (gl[ax] < 0 || gl[ax] >= pw[ax]) continue;
        const long long np = ((gl[0] * pw[1] + gl[1]) * pw[2] + gl[2]) * pw[3] + gl[3];
        const uint32_t bit = 1u << (np & 31);
        if (atomicOr(&stamp[np >> 5], bit) & bit) continue;
        double P[4], d2;
        long long gs[4];
        for (int a = 0; a < 4; a++) {
          gs[a] = gl[a] - g.pad;
          P[a] = site_coord(g, a, gs[a]);
        }
        if (!passes4(g, kl, tself, tay, P, &d2, nev)) continue;
        bool in = true;
        long long p = 0;
        for (int a = 0; a < 4; a++) {
          in = in && gs[a] >= 0 && gs[a] < g.n[a];
          p += gs[a] * g.st[a];
        }
        if (in) claim_site(g, slot, key, p, m, tself, tay, gs, true, d2, nev, ds);
        const int idx = atomicAdd(&nnext, 1);
        if (idx < BIG_FCAP)
          fn[idx] = (int32_t)np;
        else
          bad_wave = 1;
      }
      __syncthreads();
      if (tid == 0) {
        if (bad_wave) atomicOr(&ds->err, ERR_OVF);
        ncur = bad_wave ? 0 : min(nnext, BIG_FCAP);
      }
      cur ^= 1;
      __syncthreads();
    }
  }
  for (int o = 16; o > 0; o >>= 1) nev += __shfl_down_sync(0xffffffffu, nev, o);
  if ((tid & 31) == 0 && nev) atomicAdd(&ds->d2_evals, (unsigned long long)nev);
}

// owner of every site from its key (the key is emptied for the next map);
// sites nobody claimed go to the hole list
__global__ void k4_map_finish(G4 g, ulonglong2* __restrict__ key, uint32_t* __restrict__ slot,
                              int32_t* __restrict__ map, int32_t* __restrict__ holes, Dev4* ds) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.nsite) return;
  const ulonglong2 k = key[p];
  const uint32_t sl = slot[p];
  int owner = -1;
  if (k.y != KEY_EMPTY) {  // contested: the record's minimum
    if (k.x < (unsigned long long)g.ne)
      owner = (int)k.x;
    else
      bad(ds, 41);
    key[p] = make_ulonglong2(KEY_EMPTY, KEY_EMPTY);
  } else if (sl != 0u) {  // one claimant
    if (sl <= (uint32_t)g.ne)
      owner = (int)sl - 1;
    else
      bad(ds, 46);
  }
  if (sl != 0u) slot[p] = 0u;
  map[p] = owner;
  if (owner < 0) {
    const int i = atomicAdd(&ds->nholes, 1);
    holes[i] = (int32_t)p;
  }
}

// Unexplored sites (Sec. 2.3.1): in each round every hole takes, among the
// owners of its in-grid face neighbours at the end of the previous round, the
// one with the smallest (d^2 at the hole, index).  One block; rounds are
// separated by block barriers.
__global__ void __launch_bounds__(1024) k4_holes(G4 g, const double* __restrict__ tay, int32_t* __restrict__ map,
                                                 const int32_t* __restrict__ holes, int32_t* __restrict__ cand,
                                                 Dev4* ds) {
  __shared__ int remaining;
  const int nh = ds->nholes;
  if (threadIdx.x == 0) ds->rounds = 0;
  if (nh == 0) return;
  int rounds = 0;
  while (true) {
    if (threadIdx.x == 0) remaining = 0;
    for (int i = threadIdx.x; i < nh; i += blockDim.x) {
      const long long p = holes[i];
      const int cur = map[p];
      if (cur >= 0) {
        cand[i] = cur;
        continue;
      }
      long long gc[4], r = p;
      for (int a = 3; a >= 0; a--) {
        gc[a] = r % g.n[a];
        r /= g.n[a];
      }
      double P[4];
      for (int a = 0; a < 4; a++) P[a] = site_coord(g, a, gc[a]);
      int best = -1;
      unsigned long long bestk = 0;
      for (int a = 0; a < 4; a++)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          const long long ga = gc[a] + sgn;
          if (ga < 0 || ga >= g.n[a]) continue;
          const int c = map[p + sgn * g.st[a]];
          if (c < 0) continue;
          if (c >= g.ne) {
            bad(ds, 42);
            continue;
          }
          const unsigned long long kd =
              (unsigned long long)__double_as_longlong(dist2_4(g, tay + (size_t)NT4 * c, P, nullptr));
          if (best < 0 || kd < bestk || (kd == bestk && c < best)) {
            best = c;
            bestk = kd;
          }
        }
      cand[i] = best;
    }
    __syncthreads();
    int left = 0;
    for (int i = threadIdx.x; i < nh; i += blockDim.x) {
      map[holes[i]] = cand[i];
      left += cand[i] < 0;
    }
    if (left) atomicAdd(&remaining, left);
    __syncthreads();
    rounds++;
    const int rem = remaining;
    if (threadIdx.x == 0) ds->rounds = rounds;
    __syncthreads();
    if (rem == 0) break;
    if (rounds >= g.max_rounds) {
      if (threadIdx.x == 0) atomicOr(&ds->err, ERR_NC);
      break;
    }
  }
}

// ---------------------------------------------------------------------------
// Sec. 2.2.1: 15-point quadratic interpolation; transport reconstruction
// ---------------------------------------------------------------------------

__device__ __forceinline__ double F4at(const G4& g, const double* __restrict__ F, const long long* c) {
  for (int a = 0; a < 4; a++)
    if (c[a] < 0 || c[a] >= g.n[a]) return 0.0;
  return __ldg(F + c[0] * g.st[0] + c[1] * g.st[1] + c[2] * g.st[2] + c[3]);
}

// 15-point quadratic interpolation (Sec. 2.2.1) at index coordinates u: the
// nearest node, its 9-point cross (Lagrange weights on {-1,0,1} per axis),
// and per pair of axes the corner of the square of that pair's plane through
// the nearest node that holds the projection of u (from the integer parts);
// nodes outside the grid read 0.  Values in fused arithmetic; the stencil is
// chosen from u.
__device__ double qinterp4_f(const G4& g, const double* __restrict__ F, const double* u) {
  for (int a = 0; a < 4; a++)
    if (!(u[a] > -2.0 && u[a] < (double)g.n[a] + 1.0)) return 0.0;
  long long gn[4], gc[4];
  double dq[4];
  for (int a = 0; a < 4; a++) {
    gn[a] = (long long)floor(u[a] + 0.5);
    gc[a] = (long long)floor(u[a]);
    dq[a] = u[a] - (double)gn[a];
  }
  const double F0 = F4at(g, F, gn);
  double f = F0 * (1.0 - ((dq[0] * dq[0] + dq[1] * dq[1]) + (dq[2] * dq[2] + dq[3] * dq[3])));
  for (int a = 0; a < 4; a++) {
    long long c[4] = {gn[0], gn[1], gn[2], gn[3]};
    c[a] = gn[a] + 1;
    const double Fp = F4at(g, F, c);
    c[a] = gn[a] - 1;
    const double Fm = F4at(g, F, c);
    // (Fp dq (1 + dq) + Fm dq (dq - 1)) / 2
    f = fma(0.5 * dq[a], fma(Fp + Fm, dq[a], Fp - Fm), f);
  }
  for (int a = 0; a < 4; a++)
    for (int b = a + 1; b < 4; b++) {
      long long c00[4] = {gn[0], gn[1], gn[2], gn[3]};
      c00[a] = gc[a];
      c00[b] = gc[b];
      long long c11[4] = {c00[0], c00[1], c00[2], c00[3]}, c10[4] = {c00[0], c00[1], c00[2], c00[3]},
                c01[4] = {c00[0], c00[1], c00[2], c00[3]};
      c11[a] += 1;
      c11[b] += 1;
      c10[a] += 1;
      c01[b] += 1;
      const double cross = (F4at(g, F, c11) + F4at(g, F, c00)) - (F4at(g, F, c10) + F4at(g, F, c01));
      f = fma(cross * dq[a], dq[b], f);
    }
  return f;
}

// One block per (x, y) pixel: f(P) = f_ini(Q(P)) at every (vx, vy) site of
// the pixel through the owner's inverse map, and the pixel mass
// M = (sum f) dx dy dvx dvy.
__global__ void __launch_bounds__(256) k4_recon(G4 g, const double* __restrict__ tay, const int32_t* __restrict__ map,
                                                const double* __restrict__ fini, double* __restrict__ f,
                                                double* __restrict__ Mpix, Dev4* ds) {
  __shared__ double red[32];
  const int pix = blockIdx.x;
  const long long i0 = pix / g.n[1], i1 = pix % g.n[1];
  const int nvel = g.n[2] * g.n[3];
  const long long base = (long long)pix * nvel;
  double sum = 0.0;
  for (int q = threadIdx.x; q < nvel; q += blockDim.x) {
    const long long p = base + q;
    const int m = map[p];
    double fv = 0.0;
    if (m >= 0 && m < g.ne) {
      const double* t = tay + (size_t)NT4 * m;
      double P[4], dQ[4], u[4];
      P[0] = site_coord(g, 0, i0);
      P[1] = site_coord(g, 1, i1);
      P[2] = site_coord(g, 2, q / g.n[3]);
      P[3] = site_coord(g, 3, q % g.n[3]);
      // fused evaluation; the nearest node (the one decision the
      // interpolant is not continuous across) is re-taken in the exact order
      // when a coordinate lies within 1e-9 of a half-integer
      qofp4_f(t, P, dQ);
      bool tie = false;
      for (int a = 0; a < 4; a++) {
        u[a] = ((__ldg(t + 60 + a) + dQ[a]) - g.lo[a]) * g.inv_d[a];
        tie |= fabs((u[a] - floor(u[a])) - 0.5) < 1e-9;
      }
      if (tie) {
        qofp4(t, P, dQ);
        for (int a = 0; a < 4; a++) u[a] = M_(S_(A_(__ldg(t + 60 + a), dQ[a]), g.lo[a]), g.inv_d[a]);
      }
      fv = qinterp4_f(g, fini, u);
    } else if (m >= g.ne) {
      bad(ds, 43);
    }
    f[p] = fv;
    sum += fv;
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) Mpix[pix] = v * g.dV;
  }
}

// ---------------------------------------------------------------------------
// Sec. 2.5: Poisson in 2D space
// ---------------------------------------------------------------------------

// partial direct sums g_part[chunk][node] = sum over the chunk's pixels p !=
// node of M_p (r - r_p)/|r - r_p|^2, for the nodes of the cache block
constexpr int ACC_CHUNK = 1024;

__global__ void __launch_bounds__(256) k4_accel(G4 g, const double* __restrict__ Mpix, double2* __restrict__ part) {
  __shared__ double ms[ACC_CHUNK];
  const int nsrc = g.n[0] * g.n[1];
  const int c0 = blockIdx.y * ACC_CHUNK;
  const int cn = min(ACC_CHUNK, nsrc - c0);
  for (int q = threadIdx.x; q < cn; q += blockDim.x) ms[q] = Mpix[c0 + q];
  __syncthreads();
  const int nodes = g.We0 * g.We1;
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nodes) return;
  const long long i = node / g.We1 - g.E, j = node % g.We1 - g.E;
  double gx = 0.0, gy = 0.0;
  for (int q = 0; q < cn; q++) {
    const int src = c0 + q;
    const long long p0 = src / g.n[1], p1 = src % g.n[1];
    if (p0 == i && p1 == j) continue;
    const double rx = (double)(i - p0) * g.d[0];
    const double ry = (double)(j - p1) * g.d[1];
    const double c = ms[q] / (rx * rx + ry * ry);
    gx += c * rx;
    gy += c * ry;
  }
  part[(size_t)blockIdx.y * nodes + node] = make_double2(gx, gy);
}

__global__ void k4_accel_sum(G4 g, const double2* __restrict__ part, int nchunk, double2* __restrict__ gext) {
  const int nodes = g.We0 * g.We1;
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nodes) return;
  double gx = 0.0, gy = 0.0;
  for (int c = 0; c < nchunk; c++) {
    const double2 v = part[(size_t)c * nodes + node];
    gx += v.x;
    gy += v.y;
  }
  gext[node] = make_double2(-g.twoG * gx, -g.twoG * gy);
}

// acceleration at any node: the cache block, else the direct sum
__device__ double2 accel_node(const G4& g, const double* __restrict__ Mpix, const double2* __restrict__ gext,
                              long long i, long long j) {
  if (i >= -g.E && i < g.n[0] + g.E && j >= -g.E && j < g.n[1] + g.E)
    return gext[(i + g.E) * g.We1 + (j + g.E)];
  double gx = 0.0, gy = 0.0;
  for (long long p0 = 0; p0 < g.n[0]; p0++)
    for (long long p1 = 0; p1 < g.n[1]; p1++) {
      const double rx = (double)(i - p0) * g.d[0];
      const double ry = (double)(j - p1) * g.d[1];
      const double c = Mpix[p0 * g.n[1] + p1] / (rx * rx + ry * ry);
      gx += c * rx;
      gy += c * ry;
    }
  return make_double2(-g.twoG * gx, -g.twoG * gy);
}

// field record (g, J, K) at a node from the accelerations of its 3x3 block
__device__ __forceinline__ void field_block(const G4& g, const double2 b[3][3], double* o) {
  o[0] = b[1][1].x;
  o[1] = b[1][1].y;
  const double dx = g.d[0], dy = g.d[1];
  for (int a = 0; a < 2; a++) {
    const double v21 = a ? b[2][1].y : b[2][1].x, v01 = a ? b[0][1].y : b[0][1].x;
    const double v12 = a ? b[1][2].y : b[1][2].x, v10 = a ? b[1][0].y : b[1][0].x;
    const double v11 = a ? b[1][1].y : b[1][1].x;
    const double v22 = a ? b[2][2].y : b[2][2].x, v20 = a ? b[2][0].y : b[2][0].x;
    const double v02 = a ? b[0][2].y : b[0][2].x, v00 = a ? b[0][0].y : b[0][0].x;
    o[2 + 2 * a] = (v21 - v01) / (2.0 * dx);
    o[3 + 2 * a] = (v12 - v10) / (2.0 * dy);
    o[6 + 3 * a] = ((v21 + v01) - 2.0 * v11) / (dx * dx);
    o[7 + 3 * a] = (((v22 - v20) - v02) + v00) / ((4.0 * dx) * dy);
    o[8 + 3 * a] = ((v12 + v10) - 2.0 * v11) / (dy * dy);
  }
}

__global__ void k4_node_fields(G4 g, const double* __restrict__ Mpix, const double2* __restrict__ gext,
                               double* __restrict__ out) {
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.n[0] * g.n[1]) return;
  const long long i = node / g.n[1], j = node % g.n[1];
  double2 b[3][3];
  for (int p = 0; p < 3; p++)
    for (int q = 0; q < 3; q++) b[p][q] = accel_node(g, Mpix, gext, i + p - 1, j + q - 1);
  field_block(g, b, out + 12 * (size_t)node);
}

// Kick (Sec. 2.4) with the field interpolated at the drifted element by the
// 2D TSC weights: dv_a = g_a dt, dT_{2+a,.} = J_a. T_{0:2,.} dt,
// dH_{2+a,bc} = (J_a. H_{0:2,bc} + K_a,.. T_.b T_.c) dt; then the second half
// drift.
__global__ void __launch_bounds__(128) k4_kick_drift(G4 g, const double* __restrict__ Mpix,
                                                     const double2* __restrict__ gext, double* __restrict__ el) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.ne) return;
  double* e = el + (size_t)NE4 * m;
  const double ux = (e[0] - g.lo[0]) * g.inv_d[0];
  const double uy = (e[1] - g.lo[1]) * g.inv_d[1];
  if (ux > -1e9 && ux < 1e9 && uy > -1e9 && uy < 1e9) {
    const long long i = (long long)floor(ux + 0.5), j = (long long)floor(uy + 0.5);
    double wx[3], wy[3];
    {
      const double w = ux - (double)i;
      wx[0] = 0.5 * ((0.5 - w) * (0.5 - w));
      wx[1] = 0.75 - w * w;
      wx[2] = 0.5 * ((0.5 + w) * (0.5 + w));
      const double v = uy - (double)j;
      wy[0] = 0.5 * ((0.5 - v) * (0.5 - v));
      wy[1] = 0.75 - v * v;
      wy[2] = 0.5 * ((0.5 + v) * (0.5 + v));
    }
    double F[12];
    for (int c = 0; c < 12; c++) F[c] = 0.0;
    for (int p = 0; p < 3; p++) {
      double row[12];
      for (int c = 0; c < 12; c++) row[c] = 0.0;
      for (int q = 0; q < 3; q++) {
        double2 b[3][3];
        for (int pp = 0; pp < 3; pp++)
          for (int qq = 0; qq < 3; qq++) b[pp][qq] = accel_node(g, Mpix, gext, i + p + pp - 2, j + q + qq - 2);
        double nf[12];
        field_block(g, b, nf);
        for (int c = 0; c < 12; c++) row[c] += wy[q] * nf[c];
      }
      for (int c = 0; c < 12; c++) F[c] += wx[p] * row[c];
    }
    double Tx[2][4], Hx[2][10];
    for (int b = 0; b < 2; b++) {
      for (int q = 0; q < 4; q++) Tx[b][q] = e[4 + 4 * b + q];
      for (int q = 0; q < 10; q++) Hx[b][q] = e[20 + 10 * b + q];
    }
    const double dt = g.dt;
    for (int a = 0; a < 2; a++) {
      const double Ja0 = F[2 + 2 * a], Ja1 = F[3 + 2 * a];
      const double Kxx = F[6 + 3 * a], Kxy = F[7 + 3 * a], Kyy = F[8 + 3 * a];
      e[2 + a] += F[a] * dt;
      for (int q = 0; q < 4; q++) e[4 + 4 * (2 + a) + q] += (Ja0 * Tx[0][q] + Ja1 * Tx[1][q]) * dt;
      for (int b = 0; b < 4; b++)
        for (int c = b; c < 4; c++) {
          const int q = sym4(b, c);
          const double t1 = Ja0 * Hx[0][q] + Ja1 * Hx[1][q];
          const double t2 = (((Kxx * Tx[0][b]) * Tx[0][c] + (Kxy * Tx[0][b]) * Tx[1][c]) + (Kxy * Tx[1][b]) * Tx[0][c]) +
                            (Kyy * Tx[1][b]) * Tx[1][c];
          e[20 + 10 * (2 + a) + q] += (t1 + t2) * dt;
        }
    }
  }
  drift_one(e, g.half_dt);
}

// ---------------------------------------------------------------------------
// Secs. 2.2.2 and 2.3.2: remap
// ---------------------------------------------------------------------------

// Monaghan M4 kernel W(x), unnormalised (Sec. 2.3.2), fused arithmetic
__device__ __forceinline__ double W4f(double x) {
  if (x <= 1.0) return fma(0.75 * x, x * x, fma(-1.5 * x, x, 1.0));
  if (x <= 2.0) {
    const double r = 2.0 - x;
    return 0.25 * (r * r * r);
  }
  return 0.0;
}

// uniform cubic B-spline B(t), support [-2, 2], fused arithmetic
__device__ __forceinline__ double bspline3_f(double t) {
  t = fabs(t);
  if (t < 1.0) return fma(0.5 * t, t * t, fma(-t, t, 2.0 / 3.0));
  if (t < 2.0) {
    const double r = 2.0 - t;
    return (r * r * r) * (1.0 / 6.0);
  }
  return 0.0;
}

__device__ __forceinline__ long long ghost4(long long k, int n) {
  if (k >= 0 && k < n) return k;
  if (k == -1) return 1;
  if (k == n) return n - 2;
  return -1;
}

// Cubic B-spline of the coefficients eta at index coordinates u (Sec. 2.2.2):
// the sum over the 4^4 coefficients around u of eta_k prod_a B(u_a - k_a),
// with the zero-slope mirror ghosts, zero beyond its support.  Fused
// arithmetic; the sum is C2 in u, so the choice of the cell (floor(u)) where
// u lies on a knot does not change its value.
__device__ double spline_eval4_f(const G4& g, const double* __restrict__ eta, const double* u) {
  for (int a = 0; a < 4; a++)
    if (!(u[a] > -3.0 && u[a] < (double)(g.n[a] + 2))) return 0.0;
  double B[4][4];
  long long gk[4][4];
  for (int a = 0; a < 4; a++) {
    const long long k0 = (long long)floor(u[a]) - 1;
    for (int q = 0; q < 4; q++) {
      B[a][q] = bspline3_f(u[a] - (double)(k0 + q));
      gk[a][q] = ghost4(k0 + q, g.n[a]);
    }
  }
  double sum = 0.0;
  for (int q0 = 0; q0 < 4; q0++) {
    if (gk[0][q0] < 0) continue;
    for (int q1 = 0; q1 < 4; q1++) {
      if (gk[1][q1] < 0) continue;
      const double w01 = B[0][q0] * B[1][q1];
      for (int q2 = 0; q2 < 4; q2++) {
        if (gk[2][q2] < 0) continue;
        const double w012 = w01 * B[2][q2];
        const long long b012 = gk[0][q0] * g.st[0] + gk[1][q1] * g.st[1] + gk[2][q2] * g.st[2];
        double part = 0.0;
        for (int q3 = 0; q3 < 4; q3++) {
          if (gk[3][q3] < 0) continue;
          part = fma(__ldg(eta + b012 + gk[3][q3]), B[3][q3], part);
        }
        sum = fma(part, w012, sum);
      }
    }
  }
  return sum;
}

// f_new(P) = spline[f_ini](Q_r(P)), Q_r = sum W(2 d_m') Q(P, m') / sum W(2 d_m')
// over the beta set of the owner (per axis below -beta {-1,0}, below beta
// {-1,0,1}, else {0,1}; an offset with two or more non-zero components is
// dropped when one of them lies on a {-1,0,1} axis).  The beta ranges are
// decided on the owner's offsets in the exact order; the blend and the spline
// sum, continuous in their inputs, use fused arithmetic; an element whose
// FP32 distance is certainly at least one element spacing (weight 0) is
// skipped.
__global__ void __launch_bounds__(128) k4_resample(G4 g, const double* __restrict__ tay,
                                                  const float* __restrict__ tay32, const int32_t* __restrict__ map,
                                                  const double* __restrict__ eta, double* __restrict__ fnew, Dev4* ds) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.nsite) return;
  const int m = map[p];
  double val = 0.0;
  if (m >= 0 && m < g.ne) {
    long long gc[4], r = p;
    for (int a = 3; a >= 0; a--) {
      gc[a] = r % g.n[a];
      r /= g.n[a];
    }
    double P[4], x[4];
    for (int a = 0; a < 4; a++) P[a] = site_coord(g, a, gc[a]);
    const double* tm = tay + (size_t)NT4 * m;
    dist2_4(g, tm, P, x);
    int lo[4], hi[4], full[4];
    for (int a = 0; a < 4; a++) {
      lo[a] = (x[a] < -g.beta) ? -1 : ((x[a] < g.beta) ? -1 : 0);
      hi[a] = (x[a] < -g.beta) ? 0 : 1;
      full[a] = (lo[a] == -1 && hi[a] == 1);
    }
    int k[4];
    elem_coords(g, m, k);
    double num[4] = {0.0, 0.0, 0.0, 0.0}, den = 0.0;
    for (int o0 = lo[0]; o0 <= hi[0]; o0++)
      for (int o1 = lo[1]; o1 <= hi[1]; o1++)
        for (int o2 = lo[2]; o2 <= hi[2]; o2++)
          for (int o3 = lo[3]; o3 <= hi[3]; o3++) {
            const int o[4] = {o0, o1, o2, o3};
            int nz = 0, onfull = 0;
            for (int a = 0; a < 4; a++)
              if (o[a] != 0) {
                nz++;
                onfull |= full[a];
              }
            if (nz >= 2 && onfull) continue;
            int kk[4], ok = 1;
            for (int a = 0; a < 4; a++) {
              kk[a] = k[a] + o[a];
              ok &= (kk[a] >= 0 && kk[a] < g.L[a]);
            }
            if (!ok) continue;
            const int mm = ((kk[0] * g.L[1] + kk[1]) * g.L[2] + kk[2]) * g.L[3] + kk[3];
            const double* t = tay + (size_t)NT4 * mm;
            {
              // W(2d) = 0 for d >= 1: skip the FP64 evaluation where the FP32
              // distance and its bound show d^2 >= 1
              float pv[4], dp[4], xf[4], ef[4], bd;
              for (int a = 0; a < 4; a++) {
                pv[a] = (float)((P[a] - __ldg(t + a)) * g.inv_dm[a]);
                dp[a] = 1.8e-7f * fabsf(pv[a]) + 1e-12f;
              }
              eval32_4(tay32 + (size_t)NF4 * mm, pv, dp, xf, ef);
              const float d2f = d2_32(xf, ef, &bd);
              if (d2f - bd >= 1.f) continue;
            }
            double dQ[4], dd = 0.0;
            qofp4_f(t, P, dQ);
            for (int a = 0; a < 4; a++) {
              const double xa = dQ[a] * g.inv_dm[a];
              dd = fma(xa, xa, dd);
            }
            const double w = W4f(2.0 * sqrt(dd));
            for (int a = 0; a < 4; a++) num[a] = fma(w, __ldg(t + 60 + a) + dQ[a], num[a]);
            den += w;
          }
    double Qr[4];
    if (den > 0.0) {
      const double id = 1.0 / den;
      for (int a = 0; a < 4; a++) Qr[a] = num[a] * id;
    } else {
      double dQ[4];
      qofp4_f(tm, P, dQ);
      for (int a = 0; a < 4; a++) Qr[a] = __ldg(tm + 60 + a) + dQ[a];
    }
    double u[4];
    for (int a = 0; a < 4; a++) u[a] = (Qr[a] - g.lo[a]) * g.inv_d[a];
    val = spline_eval4_f(g, eta, u);
  } else if (m >= g.ne) {
    bad(ds, 44);
  }
  fnew[p] = val;
}

// Diagnostics: per (x, y) pixel, sum f and sum (vx^2 + vy^2) f of its
// velocity plane (one block per pixel, sums in a fixed order)
__global__ void __launch_bounds__(256) k4_diag_pix(G4 g, const double* __restrict__ f, double* __restrict__ out) {
  __shared__ double r0[8], r1[8];
  const int pix = blockIdx.x;
  const int nvel = g.n[2] * g.n[3];
  const long long base = (long long)pix * nvel;
  double s0 = 0.0, s1 = 0.0;
  for (int q = threadIdx.x; q < nvel; q += blockDim.x) {
    const double fv = f[base + q];
    const double vx = g.lo[2] + (double)(q / g.n[3]) * g.d[2];
    const double vy = g.lo[3] + (double)(q % g.n[3]) * g.d[3];
    s0 += fv;
    s1 += (vx * vx + vy * vy) * fv;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r0[threadIdx.x >> 5] = s0;
    r1[threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      a += r0[w];
      b += r1[w];
    }
    out[2 * pix] = a * g.dV;
    out[2 * pix + 1] = 0.5 * b * g.dV;
  }
}

// potential phi_p = 2 G sum_{q != p} M_q ln|r_p - r_q| at every pixel
__global__ void k4_diag_phi(G4 g, const double* __restrict__ pm, double* __restrict__ phi) {
  const int np = g.n[0] * g.n[1];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const long long i = p / g.n[1], j = p % g.n[1];
  double acc = 0.0;
  for (int q = 0; q < np; q++) {
    if (q == p) continue;
    const double rx = (double)(i - q / g.n[1]) * g.d[0], ry = (double)(j - q % g.n[1]) * g.d[1];
    acc += pm[2 * q] * (0.5 * log(rx * rx + ry * ry));
  }
  phi[p] = g.twoG * acc;
}

__device__ double det4_d(const double* A) {
  const double s0 = A[0] * A[5] - A[4] * A[1], s1 = A[0] * A[6] - A[4] * A[2];
  const double s2 = A[0] * A[7] - A[4] * A[3], s3 = A[1] * A[6] - A[5] * A[2];
  const double s4 = A[1] * A[7] - A[5] * A[3], s5 = A[2] * A[7] - A[6] * A[3];
  const double c5 = A[10] * A[15] - A[14] * A[11], c4 = A[9] * A[15] - A[13] * A[11];
  const double c3 = A[9] * A[14] - A[13] * A[10], c2 = A[8] * A[15] - A[12] * A[11];
  const double c1 = A[8] * A[14] - A[12] * A[10], c0 = A[8] * A[13] - A[12] * A[9];
  return ((((s0 * c5 - s1 * c4) + s2 * c3) + s3 * c2) - s4 * c1) + s5 * c0;
}

__global__ void k4_diag_det(G4 g, const double* __restrict__ el, double* __restrict__ det) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.ne) return;
  det[m] = det4_d(el + (size_t)NE4 * m + 4);
}

// Batched tridiagonal solves of the zero-slope cubic spline along one axis
// (Sec. 2.2.2), in place on eta, one thread per line.  tab holds, per node i
// of the axis, the sub-diagonal, the pivot and the eliminated super-diagonal
// of the Thomas algorithm (pivots computed once on the host).
__global__ void k4_spline_axis(G4 g, int ax, const double* __restrict__ tab, double* __restrict__ eta) {
  const long long nl = g.nsite / g.n[ax];
  const long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= nl) return;
  const long long st = g.st[ax];
  const long long base = (line / st) * (st * g.n[ax]) + (line % st);
  const int n = g.n[ax];
  const double* sub = tab;
  const double* den = tab + n;
  const double* cp = tab + 2 * n;
  double dp = 0.0;
  for (int i = 0; i < n; i++) {
    const double rhs = M_(6.0, eta[base + i * st]);
    dp = __ddiv_rn(S_(rhs, M_(__ldg(sub + i), dp)), __ldg(den + i));
    eta[base + i * st] = dp;
  }
  double nxt = eta[base + (long long)(n - 1) * st];
  for (int i = n - 2; i >= 0; i--) {
    nxt = S_(eta[base + i * st], M_(__ldg(cp + i), nxt));
    eta[base + i * st] = nxt;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {
enum K4Id { K_DRIFT, K_TAYLOR, K_PERC, K_PERC_BIG, K_FINISH, K_HOLES, K_RECON, K_ACCEL, K_ACCEL_SUM, K_KICK,
            K_RESAMPLE, K_SPLINE, K_RESET, K_FIELDS, K_DIAG, K_COUNT };
const char* const k4_names[K_COUNT] = {"drift", "taylor", "percolate", "percolate_big", "map_finish", "holes",
                                       "reconstruct", "accel", "accel_sum", "kick_drift", "resample", "spline_axis",
                                       "reset", "node_fields", "diagnostics"};
struct ProfRec {
  int id;
  cudaEvent_t a, b;
};
}  // namespace

struct vm_4d_solver {
  G4 g;
  bool profiling;
  std::vector<ProfRec> prof;
  cudaStream_t stream;
  char* ws;
  double *fini, *eta, *f, *el, *tay, *Mpix, *fld, *tab, *diag;
  float* tay32;
  ulonglong2* key;
  uint32_t* slot;
  int32_t *map, *holes, *cand, *ovf_list;
  uint32_t* big;
  double2 *gext, *part;
  Dev4* ds;
  int nchunk;
  size_t smem;
  int64_t launches;
  int have_f;
  int cyc;
  int n_s;
};

namespace {

constexpr size_t ALIGN = 256;
size_t up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

bool fill_grid(const vm_4d_config* c, G4* g) {
  if (!c) return false;
  memset(g, 0, sizeof *g);
  const int s = c->elem_stride;
  if (s < 1 || s > 8 || c->n_s < 1 || !(c->dt > 0.0) || c->pad < 0) return false;
  long long ns = 1;
  for (int a = 0; a < 4; a++) {
    if (c->n[a] < 4 || c->n[a] > 4096 || !(c->hi[a] > c->lo[a])) return false;
    ns *= c->n[a];
  }
  if (ns > (1ll << 31) - 1) return false;
  g->nsite = ns;
  g->s = s;
  g->pad = c->pad > 0 ? c->pad : s;
  long long ne = 1;
  for (int a = 0; a < 4; a++) {
    g->n[a] = c->n[a];
    g->lo[a] = c->lo[a];
    g->d[a] = (c->hi[a] - c->lo[a]) / (double)(c->n[a] - 1);
    g->dm[a] = (double)s * g->d[a];
    g->inv_d[a] = 1.0 / g->d[a];
    g->inv_dm[a] = 1.0 / g->dm[a];
    g->ctr[a] = 0.5 * (c->lo[a] + c->hi[a]);
    g->K[a] = (c->n[a] - 1 + 2 * s - 1) / (2 * s);
    g->L[a] = 2 * g->K[a] + 3;
    ne *= g->L[a];
  }
  if (ne > (1ll << 30)) return false;
  long long npad = 1;
  for (int a = 0; a < 4; a++) npad *= c->n[a] + 2 * g->pad;
  if (npad > (1ll << 31) - 1) return false;
  g->ne = (int32_t)ne;
  g->st[3] = 1;
  for (int a = 2; a >= 0; a--) g->st[a] = g->st[a + 1] * c->n[a + 1];
  g->alpha = c->alpha > 0.0 ? c->alpha : sqrt(3.0) / 4.0;
  g->beta = c->beta > 0.0 ? c->beta : 0.5 * (1.0 - sqrt(3.0) / 2.0);
  g->dt = c->dt;
  g->half_dt = 0.5 * c->dt;
  g->twoG = 2.0 * c->G;
  g->dV = ((g->d[0] * g->d[1]) * g->d[2]) * g->d[3];
  g->E = g->pad + 2 * s + 4;
  g->We0 = c->n[0] + 2 * g->E;
  g->We1 = c->n[1] + 2 * g->E;
  g->R = std::min(2 * s, 12);
  g->W = 2 * g->R + 1;
  g->max_rounds = c->max_hole_rounds > 0 ? c->max_hole_rounds : (c->n[0] + c->n[1] + c->n[2] + c->n[3]);
  return true;
}

int nchunks(const G4& g) {
  const int nsrc = g.n[0] * g.n[1];
  return (nsrc + ACC_CHUNK - 1) / ACC_CHUNK;
}

struct Layout {
  size_t diag, fini, eta, f, key, slot, map, holes, cand, el, tay, tay32, Mpix, fld, gext, part, tab, ovf, big, ds, total;
};

Layout layout(const G4& g) {
  Layout L;
  size_t o = 0;
  const size_t ns = (size_t)g.nsite;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = up(o + bytes);
    return at;
  };
  L.diag = take(8 * (3 * (size_t)g.n[0] * g.n[1] + (size_t)g.ne));
  L.fini = take(8 * ns);
  L.eta = take(8 * ns);
  L.f = take(8 * ns);
  L.key = take(16 * ns);
  L.slot = take(4 * ns);
  L.map = take(4 * ns);
  L.holes = take(4 * ns);
  L.cand = take(4 * ns);
  L.el = take(8 * (size_t)NE4 * g.ne);
  L.tay = take(8 * (size_t)NT4 * g.ne);
  L.tay32 = take(4 * (size_t)NF4 * g.ne);
  L.Mpix = take(8 * (size_t)g.n[0] * g.n[1]);
  L.fld = take(8 * 12 * (size_t)g.n[0] * g.n[1]);
  L.gext = take(16 * (size_t)g.We0 * g.We1);
  L.part = take(16 * (size_t)g.We0 * g.We1 * nchunks(g));
  int nmax = 0;
  for (int a = 0; a < 4; a++) nmax = std::max(nmax, g.n[a]);
  L.tab = take(8 * 3 * 4 * (size_t)nmax);
  L.ovf = take(4 * (size_t)g.ne);
  long long npad = 1;
  for (int a = 0; a < 4; a++) npad *= g.n[a] + 2 * g.pad;
  const size_t nwords = (size_t)((npad + 31) >> 5);
  L.big = take(4 * (size_t)BIG_SLOTS * (((nwords + 63) & ~(size_t)63) + 2 * (size_t)BIG_FCAP));
  L.ds = take(sizeof(Dev4));
  L.total = o;
  return L;
}

// pivots of the Thomas algorithm of the zero-slope spline along an axis of
// n nodes: rows (multiplied by 6) 4 e0 + 2 e1; e_{i-1} + 4 e_i + e_{i+1};
// 2 e_{n-2} + 4 e_{n-1}
void spline_table(int n, double* sub, double* den, double* cp) {
  for (int i = 0; i < n; i++) {
    const double sb = (i == 0) ? 0.0 : ((i == n - 1) ? 2.0 : 1.0);
    const double sp = (i == n - 1) ? 0.0 : ((i == 0) ? 2.0 : 1.0);
    const double dia = 4.0;
    sub[i] = sb;
    if (i == 0) {
      den[i] = dia;
      cp[i] = sp / dia;
    } else {
      const double d = dia - sb * cp[i - 1];
      den[i] = d;
      cp[i] = sp / d;
    }
  }
}

inline unsigned blocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

vm_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? VM_OK : VM_E_CUDA; }

vm_status launched(vm_4d_solver* s) {
  s->launches++;
  return cuda_ok(cudaGetLastError());
}

// per-launch events on the solver's stream while profiling is on
void prof_begin(vm_4d_solver* s, cudaEvent_t* a) {
  *a = nullptr;
  if (!s->profiling) return;
  if (cudaEventCreate(a) == cudaSuccess) cudaEventRecord(*a, s->stream);
}
void prof_end(vm_4d_solver* s, int id, cudaEvent_t a) {
  if (!s->profiling || !a) return;
  cudaEvent_t b;
  if (cudaEventCreate(&b) != cudaSuccess) return;
  cudaEventRecord(b, s->stream);
  s->prof.push_back({id, a, b});
}

#define K4_LAUNCH(s, id, ...)          \
  do {                                 \
    cudaEvent_t ev_;                   \
    prof_begin((s), &ev_);             \
    __VA_ARGS__;                       \
    prof_end((s), (id), ev_);          \
    if (launched(s)) return VM_E_CUDA; \
  } while (0)

vm_status run_map(vm_4d_solver* s) {
  const G4& g = s->g;
  K4_LAUNCH(s, K_TAYLOR, k4_taylor<<<blocks(g.ne, 128), 128, 0, s->stream>>>(g, s->el, s->tay, s->tay32));
  if (cudaMemsetAsync(&s->ds->nholes, 0, sizeof(int32_t), s->stream) != cudaSuccess ||
      cudaMemsetAsync(&s->ds->novf, 0, sizeof(int32_t), s->stream) != cudaSuccess)
    return VM_E_CUDA;
  K4_LAUNCH(s, K_PERC, k4_percolate<<<g.ne, PERC_THREADS, s->smem, s->stream>>>(g, s->el, s->tay, s->tay32, s->key, s->slot,
                                                                      s->ovf_list, s->ds));
  // returns at once when no element left its window
  K4_LAUNCH(s, K_PERC_BIG,
            k4_percolate_big<<<BIG_SLOTS, 256, 0, s->stream>>>(g, s->el, s->tay, s->key, s->slot, s->ovf_list, s->big, s->ds));
  K4_LAUNCH(s, K_FINISH, k4_map_finish<<<blocks(g.nsite, 256), 256, 0, s->stream>>>(g, s->key, s->slot, s->map, s->holes, s->ds));
  K4_LAUNCH(s, K_HOLES, k4_holes<<<1, 1024, 0, s->stream>>>(g, s->tay, s->map, s->holes, s->cand, s->ds));
  return VM_OK;
}

vm_status run_recon(vm_4d_solver* s) {
  const G4& g = s->g;
  K4_LAUNCH(s, K_RECON, k4_recon<<<g.n[0] * g.n[1], 256, 0, s->stream>>>(g, s->tay, s->map, s->fini, s->f, s->Mpix, s->ds));
  const int nodes = g.We0 * g.We1;
  K4_LAUNCH(s, K_ACCEL, k4_accel<<<dim3(blocks(nodes, 256), s->nchunk), 256, 0, s->stream>>>(g, s->Mpix, s->part));
  K4_LAUNCH(s, K_ACCEL_SUM, k4_accel_sum<<<blocks(nodes, 256), 256, 0, s->stream>>>(g, s->part, s->nchunk, s->gext));
  return VM_OK;
}

vm_status run_spline(vm_4d_solver* s) {
  const G4& g = s->g;
  int nmax = 0;
  for (int a = 0; a < 4; a++) nmax = std::max(nmax, g.n[a]);
  for (int a = 3; a >= 0; a--) {
    K4_LAUNCH(s, K_SPLINE,
              k4_spline_axis<<<blocks(g.nsite / g.n[a], 128), 128, 0, s->stream>>>(g, a, s->tab + 3 * (size_t)nmax * a, s->eta));
  }
  return VM_OK;
}

vm_status run_reset(vm_4d_solver* s) {
  s->cyc = 0;
  K4_LAUNCH(s, K_RESET, k4_reset<<<blocks(s->g.ne, 128), 128, 0, s->stream>>>(s->g, s->el));
  return VM_OK;
}

vm_status run_remap(vm_4d_solver* s) {
  const G4& g = s->g;
  vm_status st = run_map(s);
  if (st) return st;
  // f_ini <- spline(f_ini)(Q_r): the resample reads eta only
  K4_LAUNCH(s, K_RESAMPLE, k4_resample<<<blocks(g.nsite, 128), 128, 0, s->stream>>>(g, s->tay, s->tay32, s->map, s->eta, s->fini, s->ds));
  if (cudaMemcpyAsync(s->eta, s->fini, 8 * (size_t)g.nsite, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
    return VM_E_CUDA;
  st = run_spline(s);
  if (st) return st;
  return run_reset(s);
}

vm_status copy_out(vm_4d_solver* s, void* dst, const void* src, size_t bytes, int on_device) {
  if (!dst) return VM_E_INVALID_ARG;
  if (cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream) !=
      cudaSuccess)
    return VM_E_CUDA;
  return vm_4d_sync(s);
}

}  // namespace

extern "C" {

size_t vm_4d_workspace_bytes(const vm_4d_config* c) {
  G4 g;
  if (!fill_grid(c, &g)) return 0;
  return layout(g).total;
}

vm_status vm_4d_create(const vm_4d_config* c, void* d_ws, size_t bytes, void* stream, vm_4d_solver** out) {
  if (!out) return VM_E_INVALID_ARG;
  *out = nullptr;
  G4 g;
  if (!fill_grid(c, &g)) return VM_E_INVALID_ARG;
  if (!d_ws || ((uintptr_t)d_ws & (ALIGN - 1))) return VM_E_INVALID_ARG;
  const Layout L = layout(g);
  if (bytes < L.total) return VM_E_OOM;
  vm_4d_solver* s = new (std::nothrow) vm_4d_solver();
  if (!s) return VM_E_OOM;
  s->g = g;
  s->n_s = c->n_s;
  s->stream = (cudaStream_t)stream;
  s->ws = (char*)d_ws;
  s->diag = (double*)(s->ws + L.diag);
  s->fini = (double*)(s->ws + L.fini);
  s->eta = (double*)(s->ws + L.eta);
  s->f = (double*)(s->ws + L.f);
  s->key = (ulonglong2*)(s->ws + L.key);
  s->slot = (uint32_t*)(s->ws + L.slot);
  s->map = (int32_t*)(s->ws + L.map);
  s->holes = (int32_t*)(s->ws + L.holes);
  s->cand = (int32_t*)(s->ws + L.cand);
  s->el = (double*)(s->ws + L.el);
  s->tay = (double*)(s->ws + L.tay);
  s->tay32 = (float*)(s->ws + L.tay32);
  s->Mpix = (double*)(s->ws + L.Mpix);
  s->fld = (double*)(s->ws + L.fld);
  s->gext = (double2*)(s->ws + L.gext);
  s->part = (double2*)(s->ws + L.part);
  s->tab = (double*)(s->ws + L.tab);
  s->ovf_list = (int32_t*)(s->ws + L.ovf);
  s->big = (uint32_t*)(s->ws + L.big);
  s->ds = (Dev4*)(s->ws + L.ds);
  s->nchunk = nchunks(g);
  const int nwin = g.W * g.W * g.W * g.W;
  const int nwords = (nwin + 31) / 32;
  s->smem = 4 * (size_t)((nwords + 3) & ~3) + 4 * (size_t)(FCAP + TCAP + PCAP + TCAP) + 8 * (size_t)TCAP;
  if (cudaFuncSetAttribute(k4_percolate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem) != cudaSuccess) {
    delete s;
    return VM_E_CUDA;
  }
  int nmax = 0;
  for (int a = 0; a < 4; a++) nmax = std::max(nmax, g.n[a]);
  std::vector<double> tab(3 * 4 * (size_t)nmax, 0.0);
  for (int a = 0; a < 4; a++) {
    double* t = tab.data() + 3 * (size_t)nmax * a;
    spline_table(g.n[a], t, t + g.n[a], t + 2 * g.n[a]);
  }
  vm_status st = VM_OK;
  if (cudaMemcpyAsync(s->tab, tab.data(), 8 * tab.size(), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemsetAsync(s->key, 0xff, 16 * (size_t)g.nsite, s->stream) != cudaSuccess ||
      cudaMemsetAsync(s->slot, 0, 4 * (size_t)g.nsite, s->stream) != cudaSuccess ||
      cudaMemsetAsync(s->map, 0xff, 4 * (size_t)g.nsite, s->stream) != cudaSuccess ||
      cudaMemsetAsync(s->ds, 0, sizeof(Dev4), s->stream) != cudaSuccess ||
      cudaMemsetAsync(s->Mpix, 0, 8 * (size_t)g.n[0] * g.n[1], s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    st = VM_E_CUDA;
  if (st == VM_OK) st = run_reset(s);
  if (st != VM_OK) {
    delete s;
    return st;
  }
  *out = s;
  return VM_OK;
}

void vm_4d_destroy(vm_4d_solver* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  for (const ProfRec& r : s->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  delete s;
}

vm_status vm_4d_set_f(vm_4d_solver* s, const double* f, int on_device) {
  if (!s || !f) return VM_E_INVALID_ARG;
  const size_t b = 8 * (size_t)s->g.nsite;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(s->fini, f, b, k, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(s->f, s->fini, b, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(s->eta, s->fini, b, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
    return VM_E_CUDA;
  vm_status st = run_spline(s);
  if (st) return st;
  st = run_reset(s);
  if (st) return st;
  s->have_f = 1;
  if (!on_device) return cuda_ok(cudaStreamSynchronize(s->stream));  // the host buffer may be reused
  return VM_OK;
}

vm_status vm_4d_step(vm_4d_solver* s, int32_t nsteps) {
  if (!s || nsteps < 0) return VM_E_INVALID_ARG;
  if (!s->have_f) return VM_E_STATE;
  const G4& g = s->g;
  for (int32_t it = 0; it < nsteps; it++) {
    K4_LAUNCH(s, K_DRIFT, k4_drift<<<blocks(g.ne, 128), 128, 0, s->stream>>>(g, s->el));
    vm_status st = run_map(s);
    if (st) return st;
    st = run_recon(s);
    if (st) return st;
    K4_LAUNCH(s, K_KICK, k4_kick_drift<<<blocks(g.ne, 128), 128, 0, s->stream>>>(g, s->Mpix, s->gext, s->el));
    if (++s->cyc >= s->n_s) {
      st = run_remap(s);
      if (st) return st;
    }
  }
  return VM_OK;
}

vm_status vm_4d_reconstruct(vm_4d_solver* s) {
  if (!s) return VM_E_INVALID_ARG;
  if (!s->have_f) return VM_E_STATE;
  vm_status st = run_map(s);
  if (st) return st;
  return run_recon(s);
}

vm_status vm_4d_remap(vm_4d_solver* s) {
  if (!s) return VM_E_INVALID_ARG;
  if (!s->have_f) return VM_E_STATE;
  return run_remap(s);
}

vm_status vm_4d_read_f(vm_4d_solver* s, double* out, int on_device) {
  if (!s) return VM_E_INVALID_ARG;
  return copy_out(s, out, s->f, 8 * (size_t)s->g.nsite, on_device);
}

vm_status vm_4d_read_fini(vm_4d_solver* s, double* out, int on_device) {
  if (!s) return VM_E_INVALID_ARG;
  return copy_out(s, out, s->fini, 8 * (size_t)s->g.nsite, on_device);
}

vm_status vm_4d_read_eta(vm_4d_solver* s, double* out, int on_device) {
  if (!s) return VM_E_INVALID_ARG;
  return copy_out(s, out, s->eta, 8 * (size_t)s->g.nsite, on_device);
}

vm_status vm_4d_read_map(vm_4d_solver* s, int32_t* out, int on_device) {
  if (!s) return VM_E_INVALID_ARG;
  return copy_out(s, out, s->map, 4 * (size_t)s->g.nsite, on_device);
}

vm_status vm_4d_density_force(vm_4d_solver* s, double* M, double* field, int on_device) {
  if (!s) return VM_E_INVALID_ARG;
  const G4& g = s->g;
  const size_t npix = (size_t)g.n[0] * g.n[1];
  vm_status st = VM_OK;
  if (M) st = copy_out(s, M, s->Mpix, 8 * npix, on_device);
  if (st) return st;
  if (field) {
    K4_LAUNCH(s, K_FIELDS, k4_node_fields<<<blocks((long long)npix, 128), 128, 0, s->stream>>>(g, s->Mpix, s->gext, s->fld));
    st = copy_out(s, field, s->fld, 8 * 12 * npix, on_device);
  }
  return st;
}

vm_status vm_4d_get_elements(vm_4d_solver* s, double* out, int on_device) {
  if (!s) return VM_E_INVALID_ARG;
  return copy_out(s, out, s->el, 8 * (size_t)NE4 * s->g.ne, on_device);
}

vm_status vm_4d_set_elements(vm_4d_solver* s, const double* in, int on_device) {
  if (!s || !in) return VM_E_INVALID_ARG;
  if (cudaMemcpyAsync(s->el, in, 8 * (size_t)NE4 * s->g.ne,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
    return VM_E_CUDA;
  return cuda_ok(cudaStreamSynchronize(s->stream));
}

int32_t vm_4d_num_elements(const vm_4d_solver* s, int32_t* L4) {
  if (!s) return 0;
  if (L4)
    for (int a = 0; a < 4; a++) L4[a] = s->g.L[a];
  return s->g.ne;
}

int64_t vm_4d_launches(const vm_4d_solver* s) { return s ? s->launches : 0; }

vm_status vm_4d_map_stats(vm_4d_solver* s, int32_t* out3, int64_t* d2_evals) {
  if (!s || !out3) return VM_E_INVALID_ARG;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return VM_E_CUDA;
  Dev4 h;
  if (cudaMemcpy(&h, s->ds, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return VM_E_CUDA;
  out3[0] = h.novf;
  out3[1] = h.nholes;
  out3[2] = h.rounds;
  if (d2_evals) *d2_evals = (int64_t)h.d2_evals;
  return VM_OK;
}

vm_status vm_4d_diagnostics(vm_4d_solver* s, vm_4d_diag* out) {
  if (!s || !out) return VM_E_INVALID_ARG;
  const G4& g = s->g;
  const int np = g.n[0] * g.n[1];
  double* pm = s->diag;            // 2 per pixel: mass, kinetic energy
  double* phi = s->diag + 2 * (size_t)np;
  double* det = s->diag + 3 * (size_t)np;
  K4_LAUNCH(s, K_DIAG, k4_diag_pix<<<np, 256, 0, s->stream>>>(g, s->f, pm));
  K4_LAUNCH(s, K_DIAG, k4_diag_phi<<<blocks(np, 128), 128, 0, s->stream>>>(g, pm, phi));
  K4_LAUNCH(s, K_DIAG, k4_diag_det<<<blocks(g.ne, 128), 128, 0, s->stream>>>(g, s->el, det));
  std::vector<double> h(3 * (size_t)np + (size_t)g.ne);
  vm_status st = copy_out(s, h.data(), s->diag, 8 * h.size(), 0);
  if (st) return st;
  double mass = 0.0, ek = 0.0, ep = 0.0;
  for (int p = 0; p < np; p++) {
    mass += h[2 * (size_t)p];
    ek += h[2 * (size_t)p + 1];
    ep += 0.5 * h[2 * (size_t)p] * h[2 * (size_t)np + p];
  }
  double lo = INFINITY, hi = -INFINITY;
  for (int m = 0; m < g.ne; m++) {
    const double d = h[3 * (size_t)np + m];
    lo = std::min(lo, d);
    hi = std::max(hi, d);
  }
  out->mass = mass;
  out->ekin = ek;
  out->epot = ep;
  out->detT_min = lo;
  out->detT_max = hi;
  return VM_OK;
}

vm_status vm_4d_profile(vm_4d_solver* s, int on) {
  if (!s) return VM_E_INVALID_ARG;
  s->profiling = on != 0;
  return VM_OK;
}

int32_t vm_4d_profile_read(vm_4d_solver* s, int64_t* launches, double* ms, int32_t nmax) {
  if (!s) return 0;
  cudaStreamSynchronize(s->stream);
  const int n = std::min<int>(K_COUNT, nmax);
  for (int i = 0; i < n; i++) {
    if (launches) launches[i] = 0;
    if (ms) ms[i] = 0.0;
  }
  for (const ProfRec& r : s->prof) {
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    if (r.id < n) {
      if (launches) launches[r.id]++;
      if (ms) ms[r.id] += t;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  s->prof.clear();
  return K_COUNT;
}

const char* vm_4d_kernel_name(int32_t id) { return (id >= 0 && id < K_COUNT) ? k4_names[id] : nullptr; }

vm_status vm_4d_sync(vm_4d_solver* s) {
  if (!s) return VM_E_INVALID_ARG;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return VM_E_CUDA;
  Dev4 h;
  if (cudaMemcpy(&h, s->ds, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return VM_E_CUDA;
  if (h.err == 0) return VM_OK;
  const int32_t zero = 0;
  if (cudaMemcpy(&s->ds->err, &zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess) return VM_E_CUDA;
  if (h.err & ERR_INT) return VM_E_INTERNAL;
  if (h.err & ERR_OVF) return VM_E_PATCH_OVERFLOW;
  return VM_E_NOT_CONVERGED;
}

}  // extern "C"
