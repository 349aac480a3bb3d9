// Elements of metric (Sec. 2.1, 2.4) and the 1D force (Sec. 2.5).
//
// One thread per element for the drift, kick and Taylor kernels: the
// element arrays are ~1/s^2 of the grid, so these kernels are small next to
// the per-site work.  The element arithmetic is written operation by
// operation in a fixed order with non-contracting intrinsics, so that given
// the same force arrays the element trajectories are reproducible to the
// last bit by any FP64 restatement that uses the same order.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace vm {
namespace {

// FP32 record of element m (see TF_* in common.cuh) from its FP64 terms,
// in FP32 arithmetic (FP64 runs at 1/64 of the FP32 rate here): each
// coefficient carries up to ten roundings, within the budget of the
// certified decisions' bound constants; the bound coefficients are rounded
// upwards at every operation, with a slack of 1e-5 over the FP32 values
// that also covers their distance to the FP64 ones.
__device__ __forceinline__ void taylor_f32(const Grid& g, const double* t, float* __restrict__ F) {
  const float dxm = (float)g.dxm, dvm = (float)g.dvm;
  const float ti00 = (float)t[TY_TI00], ti01 = (float)t[TY_TI01], ti10 = (float)t[TY_TI10], ti11 = (float)t[TY_TI11];
  const float T00 = ti00, T01 = ti01 * (float)g.r_vx, T10 = ti10 * (float)g.r_xv, T11 = ti11;
  F[TF_T00] = T00;
  F[TF_T01] = T01;
  F[TF_T10] = T10;
  F[TF_T11] = T11;
  float gs[2], G00[2], G01[2], G11[2];
#pragma unroll
  for (int l = 0; l < 2; l++) {
    G00[l] = (float)t[TY_GX00 + 3 * l] * (dxm * dxm);
    G01[l] = (float)t[TY_GX01 + 3 * l] * (dxm * dvm);
    G11[l] = (float)t[TY_GX11 + 3 * l] * (dvm * dvm);
    gs[l] = __fadd_ru(__fadd_ru(fabsf(G00[l]), __fmul_ru(2.f, fabsf(G01[l]))), fabsf(G11[l]));
  }
  const float K00 = ti00 * (float)g.inv_dxm, K01 = ti01 * (float)g.inv_dxm;
  const float K10 = ti10 * (float)g.inv_dvm, K11 = ti11 * (float)g.inv_dvm;
  // -1/2 (K[a][0] s_x + K[a][1] s_v) = A_a p_x^2 + B_a p_x p_v + C_a p_v^2
  F[TF_AX] = -0.5f * (K00 * G00[0] + K01 * G00[1]);
  F[TF_BX] = -(K00 * G01[0] + K01 * G01[1]);
  F[TF_CX] = -0.5f * (K00 * G11[0] + K01 * G11[1]);
  F[TF_AV] = -0.5f * (K10 * G00[0] + K11 * G00[1]);
  F[TF_BV] = -(K10 * G01[0] + K11 * G01[1]);
  F[TF_CV] = -0.5f * (K10 * G11[0] + K11 * G11[1]);
  const float slack = 1.0f + 1e-5f;
  F[TF_C1X] = __fmul_ru(__fadd_ru(fabsf(T00), fabsf(T01)), slack);
  F[TF_C2X] = __fmul_ru(__fmul_ru(0.5f, __fadd_ru(__fmul_ru(fabsf(K00), gs[0]), __fmul_ru(fabsf(K01), gs[1]))), slack);
  F[TF_C1V] = __fmul_ru(__fadd_ru(fabsf(T10), fabsf(T11)), slack);
  F[TF_C2V] = __fmul_ru(__fmul_ru(0.5f, __fadd_ru(__fmul_ru(fabsf(K10), gs[0]), __fmul_ru(fabsf(K11), gs[1]))), slack);
  const double u = t[TY_U], w = t[TY_W];
  const double ui = floor(u), wi = floor(w);
  const bool ok = (u > -1e9 && u < 1e9 && w > -1e9 && w < 1e9);
  F[TF_UF] = ok ? (float)(u - ui) : 0.f;
  F[TF_WF] = ok ? (float)(w - wi) : 0.f;
  reinterpret_cast<int*>(F)[TF_UI] = ok ? (int)ui : INT_MIN / 2;
  reinterpret_cast<int*>(F)[TF_WI] = ok ? (int)wi : INT_MIN / 2;
  reinterpret_cast<double2*>(F + TF_UD)[0] = make_double2(u, w);
}

__device__ __forceinline__ void taylor_one(const Grid& g, const double* __restrict__ el, int m,
                                           double* __restrict__ tay, float* __restrict__ tayf) {
  const int ne = g.ne;
  double x = el[EL_X * ne + m], v = el[EL_V * ne + m];
  double Txx = el[EL_TXX * ne + m], Txv = el[EL_TXV * ne + m];
  double Tvx = el[EL_TVX * ne + m], Tvv = el[EL_TVV * ne + m];
  // T^-1 = adj(T) (1/det T): one division (FP64 division is slow here)
  const double det = dsub(dmul(Txx, Tvv), dmul(Txv, Tvx));
  const double id = 1.0 / det;
  const double Ti00 = dmul(Tvv, id), Ti01 = dmul(-Txv, id), Ti10 = dmul(-Tvx, id), Ti11 = dmul(Txx, id);
  double* t = tay + (size_t)m * TY_N;
  t[TY_X] = x;
  t[TY_V] = v;
  t[TY_TI00] = Ti00;
  t[TY_TI01] = Ti01;
  t[TY_TI10] = Ti10;
  t[TY_TI11] = Ti11;
#pragma unroll
  for (int l = 0; l < 2; l++) {
    double h0 = el[(EL_HXXX + 3 * l) * ne + m];
    double h1 = el[(EL_HXXV + 3 * l) * ne + m];
    double h2 = el[(EL_HXVV + 3 * l) * ne + m];
    // A = H_l T^-1, G_l = [T^-1]^T A
    double A00 = dadd(dmul(h0, Ti00), dmul(h1, Ti10));
    double A01 = dadd(dmul(h0, Ti01), dmul(h1, Ti11));
    double A10 = dadd(dmul(h1, Ti00), dmul(h2, Ti10));
    double A11 = dadd(dmul(h1, Ti01), dmul(h2, Ti11));
    t[TY_GX00 + 3 * l] = dadd(dmul(Ti00, A00), dmul(Ti10, A10));
    t[TY_GX01 + 3 * l] = dadd(dmul(Ti00, A01), dmul(Ti10, A11));
    t[TY_GX11 + 3 * l] = dadd(dmul(Ti01, A01), dmul(Ti11, A11));
  }
  int k = m / g.Lv, l = m - k * g.Lv;
  t[TY_QX] = dadd(g.cx, dmul((double)(k - g.Kx - 1), g.dxm));
  t[TY_QV] = dadd(g.cv, dmul((double)(l - g.Kv - 1), g.dvm));
  // index position of P_m, as the start site of the percolation uses it
  t[TY_U] = dmul(dsub(x, g.x_lo), g.inv_dx);
  t[TY_W] = dmul(dsub(v, g.v_lo), g.inv_dv);
  taylor_f32(g, t, tayf + (size_t)m * TF_N);
}

// Half drift (predictor or corrector of Sec. 2.4): x, T_x. and H_x.. move
// with v, T_v. and H_v..; optionally followed by the Taylor terms.
__device__ __forceinline__ void drift_body(const Grid& g, double* __restrict__ el, double* __restrict__ tay,
                                           float* __restrict__ tayf, int taylor, int vb) {
  int m = vb * blockDim.x + threadIdx.x;
  if (m >= g.ne) return;
  const int ne = g.ne;
  double h = g.half_dt;
  el[EL_X * ne + m] = dadd(el[EL_X * ne + m], dmul(el[EL_V * ne + m], h));
  el[EL_TXX * ne + m] = dadd(el[EL_TXX * ne + m], dmul(el[EL_TVX * ne + m], h));
  el[EL_TXV * ne + m] = dadd(el[EL_TXV * ne + m], dmul(el[EL_TVV * ne + m], h));
#pragma unroll
  for (int q = 0; q < 3; q++)
    el[(EL_HXXX + q) * ne + m] = dadd(el[(EL_HXXX + q) * ne + m], dmul(el[(EL_HVXX + q) * ne + m], h));
  if (taylor) taylor_one(g, el, m, tay, tayf);
}

__global__ void k_drift(Grid g, double* __restrict__ el, double* __restrict__ tay, float* __restrict__ tayf,
                        int taylor) {
  drift_body(g, el, tay, tayf, taylor, blockIdx.x);
}

__global__ void k_taylor(Grid g, const double* __restrict__ el, double* __restrict__ tay, float* __restrict__ tayf) {
  if (gate_shut(g)) return;
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < g.ne) taylor_one(g, el, m, tay, tayf);
}

// Dual TSC interpolation (Sec. 2.5) at index coordinate u; beyond the grid
// the values are lo (left) and hi (right).
__device__ __forceinline__ double tsc(const double* __restrict__ A, int nx, double lo, double hi,
                                      double u) {
  if (!(u > -1e9 && u < 1e9)) return (u < 0.0) ? lo : hi;
  long long i = (long long)floor(dadd(u, 0.5));
  double w = dsub(u, (double)i);
  double v0 = (i - 1 < 0) ? lo : ((i - 1 >= nx) ? hi : A[i - 1]);
  double v1 = (i < 0) ? lo : ((i >= nx) ? hi : A[i]);
  double v2 = (i + 1 < 0) ? lo : ((i + 1 >= nx) ? hi : A[i + 1]);
  double a = dsub(0.5, w), b = dadd(0.5, w);
  double wl = dmul(0.5, dmul(a, a));
  double wc = dsub(0.75, dmul(w, w));
  double wr = dmul(0.5, dmul(b, b));
  return dadd(dadd(dmul(wl, v0), dmul(wc, v1)), dmul(wr, v2));
}

// Kick with a, a', a'' at the drifted positions, then the corrector drift.
__device__ __forceinline__ void kick_body(const Grid& g, double* __restrict__ el, const double* __restrict__ a,
                                          const double* __restrict__ da, const double* __restrict__ d2a,
                                          const DevState* __restrict__ ds, int vb) {
  int m = vb * blockDim.x + threadIdx.x;
  if (m >= g.ne) return;
  const int ne = g.ne;
  double Mt = ds->Mtot;
  double alo = dmul(g.A, Mt), ahi = -dmul(g.A, Mt);
  double x = el[EL_X * ne + m];
  double u = dmul(dsub(x, g.x_lo), g.inv_dx);
  double am = tsc(a, g.nx, alo, ahi, u);
  double dam = tsc(da, g.nx, 0.0, 0.0, u);
  double d2am = tsc(d2a, g.nx, 0.0, 0.0, u);
  double dt = g.dt;
  double v = dadd(el[EL_V * ne + m], dmul(am, dt));
  double Txx = el[EL_TXX * ne + m], Txv = el[EL_TXV * ne + m];
  double Tvx = dadd(el[EL_TVX * ne + m], dmul(dmul(dam, Txx), dt));
  double Tvv = dadd(el[EL_TVV * ne + m], dmul(dmul(dam, Txv), dt));
  double Hx0 = el[EL_HXXX * ne + m], Hx1 = el[EL_HXXV * ne + m], Hx2 = el[EL_HXVV * ne + m];
  double Hv0 = dadd(el[EL_HVXX * ne + m], dmul(dadd(dmul(dam, Hx0), dmul(dmul(d2am, Txx), Txx)), dt));
  double Hv1 = dadd(el[EL_HVXV * ne + m], dmul(dadd(dmul(dam, Hx1), dmul(dmul(d2am, Txx), Txv)), dt));
  double Hv2 = dadd(el[EL_HVVV * ne + m], dmul(dadd(dmul(dam, Hx2), dmul(dmul(d2am, Txv), Txv)), dt));
  double h = g.half_dt;
  el[EL_X * ne + m] = dadd(x, dmul(v, h));
  el[EL_V * ne + m] = v;
  el[EL_TXX * ne + m] = dadd(Txx, dmul(Tvx, h));
  el[EL_TXV * ne + m] = dadd(Txv, dmul(Tvv, h));
  el[EL_TVX * ne + m] = Tvx;
  el[EL_TVV * ne + m] = Tvv;
  el[EL_HXXX * ne + m] = dadd(Hx0, dmul(Hv0, h));
  el[EL_HXXV * ne + m] = dadd(Hx1, dmul(Hv1, h));
  el[EL_HXVV * ne + m] = dadd(Hx2, dmul(Hv2, h));
  el[EL_HVXX * ne + m] = Hv0;
  el[EL_HVXV * ne + m] = Hv1;
  el[EL_HVVV * ne + m] = Hv2;
}

__global__ void k_kick_drift(Grid g, double* __restrict__ el, const double* __restrict__ a,
                             const double* __restrict__ da, const double* __restrict__ d2a,
                             const DevState* __restrict__ ds) {
  kick_body(g, el, a, da, d2a, ds, blockIdx.x);
}

// Isotropic elements on the lattice (remap, Sec. 1): P_m = Q_m, T = I, H = 0.
__device__ __forceinline__ void reset_body(const Grid& g, double* __restrict__ el, int vb) {
  int m = vb * blockDim.x + threadIdx.x;
  if (m >= g.ne) return;
  const int ne = g.ne;
  int k = m / g.Lv, l = m - k * g.Lv;
  el[EL_X * ne + m] = dadd(g.cx, dmul((double)(k - g.Kx - 1), g.dxm));
  el[EL_V * ne + m] = dadd(g.cv, dmul((double)(l - g.Kv - 1), g.dvm));
  el[EL_TXX * ne + m] = 1.0;
  el[EL_TXV * ne + m] = 0.0;
  el[EL_TVX * ne + m] = 0.0;
  el[EL_TVV * ne + m] = 1.0;
#pragma unroll
  for (int q = EL_HXXX; q < EL_N; q++) el[q * ne + m] = 0.0;
}

__global__ void k_reset(Grid g, double* __restrict__ el) {
  if (gate_shut(g)) return;
  reset_body(g, el, blockIdx.x);
}

constexpr int SCAN_T = 512;

// ---- error-free mass prefix (Sec. 2.5, eq. of a(i)) ----
//
// The pixel masses are summed in 128-bit fixed point: with E the binary
// exponent of max|M| (2^E <= max|M| < 2^(E+1)), every M(i) is scaled by
// 2^(111-E) (exact) and rounded to an integer.  A mass within 2^-59 of the
// largest is therefore converted without any error, a smaller one to
// 2^(E-111) absolute, and the sums of up to 2^15 such integers stay below
// 2^127.  Integer addition is exact and associative, so the prefix sums
// M_left(i), the total and each bracket M_tot - M_left(i) - M_left(i-1) are
// exact whatever the summation order, and the only rounding of a(i) is the
// final conversion to double (correctly rounded) and the product by 2 pi G.
// This is summation with its compensation carried exactly: it is at least
// as accurate as a TwoSum-compensated FP64 scan, deterministic, and runs on
// the integer pipes (FP64 runs at two lanes per SM per clock on this GPU).
typedef __int128 i128;
typedef unsigned __int128 u128;

// M * 2^up rounded to the nearest integer (ties to even), for |M| * 2^up <
// 2^112, as a signed 128-bit value: from the bits of M (integer operations
// only; FP64 runs at two lanes per SM per clock on this GPU).
__device__ __forceinline__ i128 fixed_of(double M, int up) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(M);
  const bool neg = (b >> 63) != 0;
  const int be = (int)((b >> 52) & 0x7ff);
  unsigned long long mant = b & 0x000fffffffffffffull;
  int e2;  // M = mant * 2^e2
  if (be == 0) {
    e2 = -1074;  // subnormal (or zero)
  } else {
    mant |= 0x0010000000000000ull;
    e2 = be - 1075;
  }
  const int sh = e2 + up;
  u128 U;
  if (sh >= 0) {
    U = (u128)mant << sh;  // sh <= 59 for |M| * 2^up < 2^112
  } else if (sh > -64) {
    const int k = -sh;
    const unsigned long long q = mant >> k, rem = mant & ((1ull << k) - 1ull), half = 1ull << (k - 1);
    U = (u128)(q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull));
  } else {
    U = 0;  // below half a unit
  }
  return neg ? -(i128)U : (i128)U;
}

// X * 2^e correctly rounded to double (ties to even), X != -2^127, for
// results in the normal range (tiny ones are scaled by scalbn).
__device__ __forceinline__ double double_of(i128 X, int e) {
  if (X == 0) return 0.0;
  const bool neg = X < 0;
  const u128 U = neg ? (u128)(-X) : (u128)X;
  const unsigned long long hi = (unsigned long long)(U >> 64), lo = (unsigned long long)U;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  const int top = 127 - lz;  // position of the leading bit
  // the 53 significant bits, the rounding bit and the sticky bits below it
  unsigned long long mant;
  bool up_;
  if (top <= 52) {
    mant = lo << (52 - top);
    up_ = false;
  } else {
    const int k = top - 52;  // bits dropped, 1..75
    const u128 q = U >> k;
    const u128 rem = U - (q << k);
    const u128 half = (u128)1 << (k - 1);
    mant = (unsigned long long)q;
    up_ = rem > half || (rem == half && (mant & 1ull));
  }
  if (up_) mant++;
  int ex = top + e;  // binary exponent of the result
  if (mant == (1ull << 53)) {  // rounding carried into a new bit
    mant >>= 1;
    ex++;
  }
  double r;
  if (ex >= -1022 && ex <= 1023) {
    r = __longlong_as_double((long long)(((unsigned long long)(ex + 1023) << 52) | (mant & 0x000fffffffffffffull)));
  } else {
    r = scalbn((double)mant, ex - 52);  // outside the normal range: not met by pixel masses
  }
  return neg ? -r : r;
}

__device__ __forceinline__ i128 shfl_up_i128(i128 v, int d) {
  const long long lo = __shfl_up_sync(0xffffffffu, (long long)(unsigned long long)(u128)v, d);
  const long long hi = __shfl_up_sync(0xffffffffu, (long long)((u128)v >> 64), d);
  return (i128)(((u128)(unsigned long long)hi << 64) | (u128)(unsigned long long)lo);
}

// Mass scan and force: one block.  Each thread takes a contiguous chunk of
// pixels: the largest |M| sets the common scale, the chunk sums are scanned
// across the block, and each thread walks its chunk once more, writing
// a(i) = 2 pi G (M_tot - M_left(i) - M_left(i-1)).
__device__ __forceinline__ void scan_body(const Grid& g, const double* __restrict__ M, double* __restrict__ a,
                                          DevState* ds) {
  __shared__ i128 sh[SCAN_T / 32];
  __shared__ double mx_s[SCAN_T / 32];
  __shared__ i128 tot_s;
  const int nx = g.nx, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int C = (nx + SCAN_T - 1) / SCAN_T;
  const int i0 = min(tid * C, nx), i1 = min(i0 + C, nx);
  double mx = 0.0;
  bool bad = false;
#pragma unroll 4
  for (int i = i0; i < i1; i++) {
    const double m = fabs(M[i]);
    mx = fmax(mx, m);  // NaN is dropped by fmax, and flagged
    bad |= !(m <= 1.0e300);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) mx_s[wid] = bad ? INFINITY : mx;
  __syncthreads();
  mx = 0.0;
#pragma unroll
  for (int w = 0; w < SCAN_T / 32; w++) mx = fmax(mx, mx_s[w]);
  if (!(mx <= 1.0e300) || mx == 0.0) {
    // no mass (a = 0), or a mass that is not a finite number (a = NaN)
    const double val = (mx == 0.0) ? 0.0 : __longlong_as_double(0x7ff8000000000000ll);
    for (int i = i0; i < i1; i++) a[i] = val;
    if (tid == 0) ds->Mtot = val;
    return;
  }
  const int E = ilogb(mx);
  const int up = 111 - E;  // M * 2^up < 2^112
  i128 loc = 0;
#pragma unroll 4
  for (int i = i0; i < i1; i++) loc += fixed_of(M[i], up);
  i128 inc = loc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const i128 o = shfl_up_i128(inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (tid == 0) {
    i128 run = 0;
#pragma unroll
    for (int w = 0; w < SCAN_T / 32; w++) {
      const i128 t = sh[w];
      sh[w] = run;  // exclusive prefix of the warp totals
      run += t;
    }
    tot_s = run;
  }
  __syncthreads();
  const i128 tot = tot_s;
  i128 left_prev = sh[wid] + (inc - loc);  // mass of the pixels before this chunk
#pragma unroll 4
  for (int i = i0; i < i1; i++) {
    const i128 left = left_prev + fixed_of(M[i], up);
    a[i] = dmul(g.A, double_of(tot - left - left_prev, -up));
    left_prev = left;
  }
  if (tid == 0) ds->Mtot = double_of(tot, -up);
}

__global__ void __launch_bounds__(SCAN_T) k_scan_force(Grid g, const double* __restrict__ M,
                                                       double* __restrict__ a, DevState* ds) {
  scan_body(g, M, a, ds);
}

// a' and a'' by centred differences (Sec. 2.5); beyond the grid a takes its
// limits +A M_tot (left) and -A M_tot (right).
__device__ __forceinline__ void diff_body(const Grid& g, const double* __restrict__ a, double* __restrict__ da,
                                          double* __restrict__ d2a, const DevState* __restrict__ ds, int vb) {
  const int i = vb * blockDim.x + threadIdx.x;
  const int nx = g.nx;
  if (i >= nx) return;
  const double Mt = ds->Mtot;
  const double twodx = g.literal_fd ? g.dx : dmul(2.0, g.dx);
  const double dx2 = dmul(g.dx, g.dx);
  const double am = (i > 0) ? a[i - 1] : dmul(g.A, Mt);
  const double ap = (i < nx - 1) ? a[i + 1] : -dmul(g.A, Mt);
  da[i] = dsub(ap, am) / twodx;
  d2a[i] = dsub(dadd(ap, am), dmul(2.0, a[i])) / dx2;
}

__global__ void k_force_diff(Grid g, const double* __restrict__ a, double* __restrict__ da,
                             double* __restrict__ d2a, const DevState* __restrict__ ds) {
  diff_body(g, a, da, d2a, ds, blockIdx.x);
}

// ---- group launches: every solve of a group in one launch per phase ----

__global__ void k_drift_group(const SolveDesc* __restrict__ D, const int* __restrict__ off, int ns, int total,
                              int taylor) {
  GROUP_LOOP(off, ns, total)
  drift_body(gsh, d.el, d.tay, d.tayf, taylor, vb);
  GROUP_END
}

__global__ void k_taylor_group(const SolveDesc* __restrict__ D, const int* __restrict__ off, int ns, int total) {
  GROUP_LOOP(off, ns, total)
  const int m = vb * blockDim.x + threadIdx.x;
  if (m < gsh.ne) taylor_one(gsh, d.el, m, d.tay, d.tayf);
  GROUP_END
}

__global__ void k_kick_group(const SolveDesc* __restrict__ D, const int* __restrict__ off, int ns, int total) {
  GROUP_LOOP(off, ns, total)
  kick_body(gsh, d.el, d.a, d.da, d.d2a, d.ds, vb);
  GROUP_END
}

__global__ void k_reset_group(const SolveDesc* __restrict__ D, const int* __restrict__ off, int ns, int total) {
  GROUP_LOOP(off, ns, total)
  reset_body(gsh, d.el, vb);
  GROUP_END
}

__global__ void __launch_bounds__(SCAN_T) k_scan_group(const SolveDesc* __restrict__ D,
                                                       const int* __restrict__ off, int ns, int total) {
  GROUP_LOOP(off, ns, total)
  (void)vb;
  scan_body(gsh, d.M, d.a, d.ds);
  GROUP_END
}

__global__ void k_diff_group(const SolveDesc* __restrict__ D, const int* __restrict__ off, int ns, int total) {
  GROUP_LOOP(off, ns, total)
  diff_body(gsh, d.a, d.da, d.d2a, d.ds, vb);
  GROUP_END
}

__device__ __forceinline__ unsigned long long order_key(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Diagnostics of the last f (Sec. 3.2): each block's sums into part[6 x
// blockIdx] (mass, kinetic energy, S, L1, L2, the potential term), added in
// block order by k_diag_sum, so that the totals do not depend on the order
// in which blocks finish; the det T range by atomic min/max (order-free).
template <typename R>
__global__ void k_diag(Grid g, const R* __restrict__ f, const double* __restrict__ a,
                       const double* __restrict__ el, DevState* ds, double* __restrict__ part) {
  __shared__ double red[5][32];
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // mass, kinetic energy, S, L1, L2 (Sec. 3.2)
  const size_t n = (size_t)g.nx * g.nv;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    int j = (int)(p % g.nv);
    double v = dadd(g.v_lo, dmul((double)j, g.dv));
    double fv = (double)f[p];
    acc[0] += fv * g.dxdv;
    acc[1] += 0.5 * (v * v) * fv * g.dxdv;
    if (fv != 0.0) acc[2] -= fv * log(fabs(fv)) * g.dxdv;
    acc[3] += fabs(fv) * g.dxdv;
    acc[4] += fv * fv * g.dxdv;
  }
#pragma unroll
  for (int c = 0; c < 5; c++)
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 5; c++) red[c][wid] = acc[c];
  }
  __syncthreads();
  // potential energy term, reduced like the others
  const double a8 = g.A * ds->Mtot;
  double ep = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.nx; i += gridDim.x * blockDim.x)
    ep += (a[i] * a[i] - a8 * a8) * g.dx;
  for (int o = 16; o > 0; o >>= 1) ep += __shfl_down_sync(0xffffffffu, ep, o);
  __shared__ double red_p[32];
  if (lane == 0) red_p[wid] = ep;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
#pragma unroll
      for (int c = 0; c < 5; c++) t[c] += red[c][w];
      t[5] += red_p[w];
    }
#pragma unroll
    for (int c = 0; c < 6; c++) part[6 * blockIdx.x + c] = t[c];
  }
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < g.ne; m += gridDim.x * blockDim.x) {
    const int ne = g.ne;
    const int km = m / g.Lv;
    if (!elem_exists(g, km, m - km * g.Lv)) continue;
    double d = el[EL_TXX * ne + m] * el[EL_TVV * ne + m] - el[EL_TXV * ne + m] * el[EL_TVX * ne + m];
    unsigned long long k = order_key(d);
    atomicMin(&ds->det_min_key, k);
    atomicMax(&ds->det_max_key, k);
  }
}

__global__ void k_diag_sum(const double* __restrict__ part, int nb, DevState* ds) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < nb; b++)
    for (int c = 0; c < 6; c++) t[c] += part[6 * b + c];
  ds->sum_mass = t[0];
  ds->sum_kin = t[1];
  ds->sum_ent = t[2];
  ds->sum_l1 = t[3];
  ds->sum_l2 = t[4];
  ds->sum_pot = t[5];
}

// Largest projected density rho(x_i) = (sum_j f(i, j)) dv of f (Sec. 2.4's
// time-step constraint): a block per x row, the positive maxima into
// ds->rho_max_bits (bits of a non-negative double order as the values do).
template <typename R>
__global__ void __launch_bounds__(256) k_rho_max(Grid g, const R* __restrict__ f, DevState* ds) {
  __shared__ double sh[8];
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int j = threadIdx.x; j < g.nv; j += blockDim.x) acc += (double)f[(size_t)i * g.nv + j];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
    const double rho = dmul(t, g.dv);
    if (rho > 0.0) atomicMax(&ds->rho_max_bits, (unsigned long long)__double_as_longlong(rho));
  }
}

// ---- adaptive computing domain (Sec. 2.2.1, eq. constrf; Sec. 2.3) ----

// Node rectangle of |f_ini| > f_th: a block per row, the row's smallest and
// largest such column, then atomics into ds->fbox (reset by the caller to
// nx, -1, nv, -1).
template <typename R>
__global__ void __launch_bounds__(256) k_fth_box(Grid g, const R* __restrict__ f, double f_th, DevState* ds) {
  __shared__ int lo_s, hi_s;
  const int i = blockIdx.x;
  if (threadIdx.x == 0) {
    lo_s = g.nv;
    hi_s = -1;
  }
  __syncthreads();
  int lo = g.nv, hi = -1;
  for (int j = threadIdx.x; j < g.nv; j += blockDim.x)
    if (fabs((double)f[(size_t)i * g.nv + j]) > f_th) {
      lo = min(lo, j);
      hi = max(hi, j);
    }
  if (hi >= 0) {
    atomicMin(&lo_s, lo);
    atomicMax(&hi_s, hi);
  }
  __syncthreads();
  if (threadIdx.x == 0 && hi_s >= 0) {
    atomicMin(&ds->fbox[0], i);
    atomicMax(&ds->fbox[1], i);
    atomicMin(&ds->fbox[2], lo_s);
    atomicMax(&ds->fbox[3], hi_s);
  }
}

// f_ini <- 0 outside the node rectangle ds->fbox.
template <typename R>
__global__ void k_fth_cut(Grid g, R* __restrict__ f, const DevState* ds) {
  const int i0 = ds->fbox[0], i1 = ds->fbox[1], j0 = ds->fbox[2], j1 = ds->fbox[3];
  for (int i = blockIdx.x; i < g.nx; i += gridDim.x) {
    R* row = f + (size_t)i * g.nv;
    const bool all = i < i0 || i > i1;
    for (int j = threadIdx.x; j < g.nv; j += blockDim.x)
      if (all || j < j0 || j > j1) row[j] = R(0);
  }
}

__device__ __forceinline__ unsigned long long okey(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double okey_inv(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}

// Site rectangle of a map: the extent of the existing elements' positions
// (Sec. 2.3), i from ceil((min x_m - x_lo)/dx) to floor((max x_m - x_lo)/dx)
// clamped to the grid, same along v, in the oracle's operation order.  Each
// block reduces its elements into rect_part; the last block to finish
// reduces the partials into ds->rect and re-arms the counter.
__global__ void __launch_bounds__(256) k_domain_rect(Grid g, const double* __restrict__ el,
                                                     unsigned long long* __restrict__ part, DevState* ds) {
  __shared__ unsigned long long red[4][8];
  __shared__ bool last;
  const int nk = g.khi - g.klo + 1, nl = g.lhi - g.llo + 1;
  const long long nact = (nk > 0 && nl > 0) ? (long long)nk * nl : 0;
  // keys ordered as the values; max of ~key = min of key
  unsigned long long kmin_x = 0, kmax_x = 0, kmin_v = 0, kmax_v = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nact; q += (long long)gridDim.x * blockDim.x) {
    const int k = g.klo + (int)(q / nl), l = g.llo + (int)(q % nl);
    const int m = k * g.Lv + l;
    const unsigned long long kx = okey(el[EL_X * g.ne + m]), kv = okey(el[EL_V * g.ne + m]);
    kmin_x = max(kmin_x, ~kx);
    kmax_x = max(kmax_x, kx);
    kmin_v = max(kmin_v, ~kv);
    kmax_v = max(kmax_v, kv);
  }
  unsigned long long v4[4] = {kmin_x, kmax_x, kmin_v, kmax_v};
#pragma unroll
  for (int c = 0; c < 4; c++)
    for (int o = 16; o > 0; o >>= 1) v4[c] = max(v4[c], __shfl_down_sync(0xffffffffu, v4[c], o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < 4; c++) red[c][wid] = v4[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 4; c++) {
      unsigned long long t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) t = max(t, red[c][w]);
      part[4 * blockIdx.x + c] = t;
    }
    __threadfence();
    last = (atomicAdd(&ds->rect_done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  unsigned long long t[4] = {0, 0, 0, 0};
  for (unsigned b = 0; b < gridDim.x; b++)
    for (int c = 0; c < 4; c++) t[c] = max(t[c], __ldcg(&part[4 * b + c]));
  ds->rect_done = 0;
  if (nact == 0 || t[1] == 0) {
    ds->rect[0] = ds->rect[2] = 0;
    ds->rect[1] = ds->rect[3] = -1;
    return;
  }
  const double xmin = okey_inv(~t[0]), xmax = okey_inv(t[1]), vmin = okey_inv(~t[2]), vmax = okey_inv(t[3]);
  if (!(xmin <= xmax) || !(vmin <= vmax)) {
    ds->rect[0] = ds->rect[2] = 0;
    ds->rect[1] = ds->rect[3] = -1;
    return;
  }
  const double a = ceil(dmul(dsub(xmin, g.x_lo), g.inv_dx)), b = floor(dmul(dsub(xmax, g.x_lo), g.inv_dx));
  const double c = ceil(dmul(dsub(vmin, g.v_lo), g.inv_dv)), d = floor(dmul(dsub(vmax, g.v_lo), g.inv_dv));
  ds->rect[0] = (int)(a < 0.0 ? 0.0 : (a > g.nx ? (double)g.nx : a));
  ds->rect[1] = (int)(b > g.nx - 1 ? (double)(g.nx - 1) : (b < -1.0 ? -1.0 : b));
  ds->rect[2] = (int)(c < 0.0 ? 0.0 : (c > g.nv ? (double)g.nv : c));
  ds->rect[3] = (int)(d > g.nv - 1 ? (double)(g.nv - 1) : (d < -1.0 ? -1.0 : d));
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Element kernels are FP64-bound (two FP64 lanes per SM per clock): small
// blocks spread a small lattice over many SMs.
constexpr int ET = 64;

}  // namespace

void launch_drift(vm_solver* s, bool taylor) {
  { const int ps_ = prof_begin(s, KID_DRIFT); k_drift<<<blocks_for(s->g.ne, ET), ET, 0, s->stream>>>(s->g, s->el, s->tay, s->tayf, taylor ? 1 : 0); prof_end(s, ps_); }
  s->launches++;
}

void launch_taylor(vm_solver* s) {
  { const int ps_ = prof_begin(s, KID_TAYLOR); k_taylor<<<blocks_for(s->g.ne, ET), ET, 0, s->stream>>>(s->g, s->el, s->tay, s->tayf); prof_end(s, ps_); }
  s->launches++;
}

void launch_kick_drift(vm_solver* s) {
  { const int ps_ = prof_begin(s, KID_KICK_DRIFT); k_kick_drift<<<blocks_for(s->g.ne, ET), ET, 0, s->stream>>>(s->g, s->el, s->a, s->da, s->d2a, s->ds); prof_end(s, ps_); }
  s->launches++;
}

void launch_reset_elements(vm_solver* s) {
  { const int ps_ = prof_begin(s, KID_RESET); k_reset<<<blocks_for(s->g.ne, ET), ET, 0, s->stream>>>(s->g, s->el); prof_end(s, ps_); }
  s->launches++;
}

unsigned group_grid(const GroupPlan& G, GroupPhase ph, int total) {
  const int b = G.shape[ph].blocks > 0 ? G.shape[ph].blocks : 152 * 4;
  return (unsigned)std::max(1, std::min(b, total));
}

void group_drift(const GroupPlan& G, bool taylor) {
  if (G.tot_elem64 == 0) return;
  k_drift_group<<<group_grid(G, GP_DRIFT, G.tot_elem64), ET, 0, G.stream>>>(G.D, G.off_elem64, G.ns, G.tot_elem64,
                                                                           taylor ? 1 : 0);
}

void group_taylor(const GroupPlan& G) {
  if (G.tot_elem64 == 0) return;
  k_taylor_group<<<group_grid(G, GP_TAYLOR, G.tot_elem64), ET, 0, G.stream>>>(G.D, G.off_elem64, G.ns, G.tot_elem64);
}

void group_kick(const GroupPlan& G) {
  if (G.tot_elem64 == 0) return;
  k_kick_group<<<group_grid(G, GP_KICK, G.tot_elem64), ET, 0, G.stream>>>(G.D, G.off_elem64, G.ns, G.tot_elem64);
}

void group_reset(const GroupPlan& G) {
  if (G.tot_elem64 == 0) return;
  k_reset_group<<<group_grid(G, GP_RESET, G.tot_elem64), ET, 0, G.stream>>>(G.D, G.off_elem64, G.ns, G.tot_elem64);
}

void group_scan_force(const GroupPlan& G) {
  k_scan_group<<<group_grid(G, GP_SCAN, G.ns), SCAN_T, 0, G.stream>>>(G.D, G.off_solve, G.ns, G.ns);
  k_diff_group<<<group_grid(G, GP_DIFF, G.tot_diff), 128, 0, G.stream>>>(G.D, G.off_diff, G.ns, G.tot_diff);
}

void launch_scan_force(vm_solver* s) {
  const int ps_ = prof_begin(s, KID_SCAN_FORCE);
  launch_scan_force_raw(s->g, s->M, s->a, s->da, s->d2a, s->ds, s->stream);
  prof_end(s, ps_);
  s->launches += 2;
}

// The same mass scan on caller-provided buffers (no solver), for the
// allocation-free entry point.
void launch_scan_force_raw(const Grid& g, const double* M, double* a, double* da, double* d2a, DevState* ds,
                           cudaStream_t stream) {
  k_scan_force<<<1, SCAN_T, 0, stream>>>(g, M, a, ds);
  k_force_diff<<<blocks_for(g.nx, 128), 128, 0, stream>>>(g, a, da, d2a, ds);
}

void launch_fth_box(vm_solver* s) {
  if (s->fp32)
    k_fth_box<float><<<s->g.nx, 256, 0, s->stream>>>(s->g, (const float*)s->fini, s->cfg.f_th, s->ds);
  else
    k_fth_box<double><<<s->g.nx, 256, 0, s->stream>>>(s->g, (const double*)s->fini, s->cfg.f_th, s->ds);
  s->launches++;
}

void launch_fth_cut(vm_solver* s) {
  const unsigned nb = (unsigned)std::min(s->g.nx, 152 * 8);
  if (s->fp32)
    k_fth_cut<float><<<nb, 256, 0, s->stream>>>(s->g, (float*)s->fini, s->ds);
  else
    k_fth_cut<double><<<nb, 256, 0, s->stream>>>(s->g, (double*)s->fini, s->ds);
  s->launches++;
}

void launch_domain_rect(vm_solver* s) {
  const long long nact = (long long)std::max(0, s->g.khi - s->g.klo + 1) * std::max(0, s->g.lhi - s->g.llo + 1);
  const unsigned nb = (unsigned)std::max(1ll, std::min<long long>(kRectBlocks, (nact + 255) / 256));
  k_domain_rect<<<nb, 256, 0, s->stream>>>(s->g, s->el, reinterpret_cast<unsigned long long*>(s->rect_part),
                                          s->ds);
  s->launches++;
}

void launch_rho_max(vm_solver* s) {
  if (s->fp32)
    k_rho_max<float><<<s->g.nx, 256, 0, s->stream>>>(s->g, (const float*)s->f, s->ds);
  else
    k_rho_max<double><<<s->g.nx, 256, 0, s->stream>>>(s->g, (const double*)s->f, s->ds);
  s->launches++;
}

void launch_diagnostics(vm_solver* s) {
  unsigned nb = blocks_for((long long)s->n, 256);
  if (nb > (unsigned)kRectBlocks) nb = kRectBlocks;  // 6 partial sums per block in diag_part
  double* part = s->diag_part;
  const int ps_ = prof_begin(s, KID_DIAG);
  if (s->fp32)
    k_diag<float><<<nb, 256, 0, s->stream>>>(s->g, (const float*)s->f, s->a, s->el, s->ds, part);
  else
    k_diag<double><<<nb, 256, 0, s->stream>>>(s->g, (const double*)s->f, s->a, s->el, s->ds, part);
  k_diag_sum<<<1, 32, 0, s->stream>>>(part, (int)nb, s->ds);
  prof_end(s, ps_);
  s->launches += 2;
}

}  // namespace vm
