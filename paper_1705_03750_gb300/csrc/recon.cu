// Per-site reconstruction of f (Sec. 2.2, Liouville: f(P) = f_ini(Q(P))).
//
// Transport (Sec. 2.2.1): Q from the element that owns the site, six-point
// quadratic interpolation of f_ini, and the v-reduction of the row fused in
// the same block (pixel mass M(i), Sec. 2.5).  Remap (Secs. 2.2.2, 2.3.2):
// Q_r blended over the beta set of elements with the Monaghan kernel, then
// the cubic B-spline of f_ini at Q_r.
//
// FP64 path: Q, the node choice and the interpolation in FP64, the decisions
// taken in a fixed operation order (the remap's blend, continuous in its
// inputs, in fused FP64 once the beta ranges are decided).  FP32-mixed path: Q from the element's FP32
// record in element units, anchored on the exact lattice position of Q_m, so
// that only the small offset carries FP32 rounding; the integer decisions
// (nearest node, containing square, beta ranges) are taken from the FP32
// value only when it clears a rigorous bound on its distance to the FP64
// value, and otherwise from the FP64 evaluation, so they are the FP64 path's.
#include <climits>
#include <math.h>

#include "common.cuh"

namespace vm {
namespace {

template <typename R>
__device__ __forceinline__ R F_at(const R* __restrict__ F, const Grid& g, long long i, long long j) {
  if (i < 0 || j < 0 || i >= g.nx || j >= g.nv) return R(0);
  return F[i * g.nv + j];
}

// Six-point quadratic interpolation (Sec. 2.2.1) at index coordinates (u, w).
__device__ __forceinline__ double qinterp(const double* __restrict__ F, const Grid& g, double u, double w) {
  if (!(u > -2.0 && u < (double)g.nx + 1.0 && w > -2.0 && w < (double)g.nv + 1.0)) return 0.0;
  const long long in = (long long)floor(dadd(u, 0.5)), jn = (long long)floor(dadd(w, 0.5));
  const long long ic = (long long)floor(u), jc = (long long)floor(w);
  const double dqx = dsub(u, (double)in), dqv = dsub(w, (double)jn);
  double f = dmul(F_at(F, g, in, jn), dsub(dsub(1.0, dmul(dqx, dqx)), dmul(dqv, dqv)));
  f = dadd(f, dmul(dmul(dmul(0.5, F_at(F, g, in + 1, jn)), dqx), dadd(1.0, dqx)));
  f = dadd(f, dmul(dmul(dmul(0.5, F_at(F, g, in - 1, jn)), dqx), dsub(dqx, 1.0)));
  f = dadd(f, dmul(dmul(dmul(0.5, F_at(F, g, in, jn + 1)), dqv), dadd(1.0, dqv)));
  f = dadd(f, dmul(dmul(dmul(0.5, F_at(F, g, in, jn - 1)), dqv), dsub(dqv, 1.0)));
  double cross = dsub(dsub(dadd(F_at(F, g, ic + 1, jc + 1), F_at(F, g, ic, jc)), F_at(F, g, ic + 1, jc)),
                      F_at(F, g, ic, jc + 1));
  return dadd(f, dmul(dmul(cross, dqx), dqv));
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
  __syncthreads();
  return t;
}

// Transport reconstruction of one x row per block, fused with M(i).
__device__ __forceinline__ uint32_t ds_epoch(const DevState* ds) { return *(const volatile uint32_t*)&ds->epoch; }

__device__ __forceinline__ int owner(const uint32_t* __restrict__ map, size_t p, uint32_t epoch, int ne) {
  const uint32_t t = map[p];
  const int m = (int)(t & SLOT_MASK);
  return ((t >> 24) == epoch && m < ne) ? m : -1;
}

// The columns [j0, j1] of row i inside the map's computing domain (the whole
// row unless the adaptive domain is on; empty when j0 > j1).
__device__ __forceinline__ void row_span(const Grid& g, const DevState* ds, int i, int& j0, int& j1) {
  j0 = 0;
  j1 = g.nv - 1;
  if (g.fth_on) {
    const int i0 = ds->rect[0], i1 = ds->rect[1];
    if (i < i0 || i > i1) {
      j0 = g.nv;
      j1 = -1;
    } else {
      j0 = max(ds->rect[2], 0);
      j1 = min(ds->rect[3], g.nv - 1);
    }
  }
}

// Zeros of row `row` outside [j0, j1].
template <typename R>
__device__ __forceinline__ void zero_outside(const Grid& g, R* __restrict__ row, int j0, int j1) {
  if (j0 > j1) {
    for (int j = threadIdx.x; j < g.nv; j += blockDim.x) row[j] = R(0);
    return;
  }
  for (int j = threadIdx.x; j < j0; j += blockDim.x) row[j] = R(0);
  for (int j = j1 + 1 + threadIdx.x; j < g.nv; j += blockDim.x) row[j] = R(0);
}

// FP64 path.  The integer decisions (nearest node, containing cell) come
// from the FP32 record's certified evaluation, which is the fixed-order FP64
// evaluation's whenever its bound clears every decision boundary (as on the
// FP32-mixed path); the offset Q - Q_m is then evaluated in FP64 with fused
// operations, anchored on the exact lattice position of Q_m, and the
// six-point value with fused operations (rounding changes only).  A site
// whose decision the bound leaves open (the step after a remap puts every
// Q on a node) is evaluated entirely in the fixed order.
__device__ __forceinline__ bool recon64_fast(const Grid& g, const double* __restrict__ t, const float* __restrict__ F,
                                             int m, int i, int j, double Px, double Pv,
                                             const double* __restrict__ fini, float inv_Lv, double& val);

__device__ __forceinline__ double qinterp64_fused(const double* __restrict__ F, const Grid& g, long long in,
                                                  long long jn, long long ic, long long jc, double x, double y) {
  const double hx = 0.5 * x, hy = 0.5 * y;
  double f = F_at(F, g, in, jn) * fma(-y, y, fma(-x, x, 1.0));
  f = fma(F_at(F, g, in + 1, jn), fma(hx, x, hx), f);
  f = fma(F_at(F, g, in - 1, jn), fma(hx, x, -hx), f);
  f = fma(F_at(F, g, in, jn + 1), fma(hy, y, hy), f);
  f = fma(F_at(F, g, in, jn - 1), fma(hy, y, -hy), f);
  const double cross = (F_at(F, g, ic + 1, jc + 1) + F_at(F, g, ic, jc)) - (F_at(F, g, ic + 1, jc) + F_at(F, g, ic, jc + 1));
  return fma(cross, x * y, f);
}

__device__ __forceinline__ void k_recon64_body(const Grid& g, const uint32_t* __restrict__ map, const DevState* ds,
                                                 const double* __restrict__ tay, const float* __restrict__ tayf,
                                                 const double* __restrict__ fini, double* __restrict__ f,
                                                 double* __restrict__ M, int vb) {
  using R = double;
  __shared__ double sh[32];
  const int i = vb;
  const double Px = site_x(g, i);
  int js, je;
  row_span(g, ds, i, js, je);
  zero_outside(g, f + (size_t)i * g.nv, js, je);
  const float inv_Lv = 1.0f / (float)g.Lv;
  double acc = 0.0;
  for (int j = js + threadIdx.x; j <= je; j += blockDim.x) {
    const size_t p = (size_t)i * g.nv + j;
    const int m = owner(map, p, ds_epoch(ds), g.ne);
    double val = 0.0;
    if (m >= 0) {
      const double* t = tay + (size_t)m * TY_N;
      const double Pv = site_v(g, j);
      if (!recon64_fast(g, t, tayf + (size_t)m * TF_N, m, i, j, Px, Pv, fini, inv_Lv, val)) {
        // a decision the FP32 bound cannot settle: the fixed order
        double dqx, dqv;
        qofp_exact(t, Px, Pv, dqx, dqv);
        const double u = dmul(dsub(dadd(t[TY_QX], dqx), g.x_lo), g.inv_dx);
        const double w = dmul(dsub(dadd(t[TY_QV], dqv), g.v_lo), g.inv_dv);
        val = qinterp(fini, g, u, w);
      }
    }
    const R out = (R)val;
    f[p] = out;
    acc += (double)out;
  }
  const double rowsum = block_sum(acc, sh);
  if (threadIdx.x == 0) M[i] = dmul(rowsum, g.dxdv);
}

__global__ void __launch_bounds__(256) k_recon64(Grid g, const uint32_t* __restrict__ map, const DevState* ds,
                                                 const double* __restrict__ tay, const float* __restrict__ tayf,
                                                 const double* __restrict__ fini, double* __restrict__ f,
                                                 double* __restrict__ M) {
  k_recon64_body(g, map, ds, tay, tayf, fini, f, M, blockIdx.x);
}

// Monaghan M4 kernel, unnormalised (Sec. 2.3.2).
__device__ __forceinline__ double W4(double x) {
  if (x <= 1.0) return dadd(dsub(1.0, dmul(1.5, dmul(x, x))), dmul(0.75, dmul(dmul(x, x), x)));
  if (x <= 2.0) {
    double r = dsub(2.0, x);
    return dmul(0.25, dmul(dmul(r, r), r));
  }
  return 0.0;
}

// Q_r of Sec. 2.3.2 for a site owned by element m.
__device__ __forceinline__ void blended_q(const Grid& g, const double* __restrict__ tay, int m, double Px,
                                          double Pv, double& Qx, double& Qv) {
  double xi, ze;
  dist2_exact(tay + (size_t)m * TY_N, g, Px, Pv, xi, ze);
  const double beta = g.beta;
  const int a0 = (xi < -beta) ? -1 : ((xi < beta) ? -1 : 0);
  const int a1 = (xi < -beta) ? 0 : 1;
  const int b0 = (ze < -beta) ? -1 : ((ze < beta) ? -1 : 0);
  const int b1 = (ze < -beta) ? 0 : 1;
  const bool full = (a0 == -1 && a1 == 1) || (b0 == -1 && b1 == 1);
  const int k = m / g.Lv, l = m - k * g.Lv;
  double nx_ = 0.0, nv_ = 0.0, den = 0.0;
  for (int a = a0; a <= a1; a++)
    for (int b = b0; b <= b1; b++) {
      if (full && a != 0 && b != 0) continue;
      const int kk = k + a, ll = l + b;
      if (!elem_exists(g, kk, ll)) continue;
      const double* t = tay + (size_t)(kk * g.Lv + ll) * TY_N;
      double dqx, dqv;
      qofp_exact(t, Px, Pv, dqx, dqv);
      const double x1 = dmul(dqx, g.inv_dxm), z1 = dmul(dqv, g.inv_dvm);
      const double d = sqrt(dadd(dmul(x1, x1), dmul(z1, z1)));
      const double wgt = W4(dmul(2.0, d));
      nx_ = dadd(nx_, dmul(wgt, dadd(t[TY_QX], dqx)));
      nv_ = dadd(nv_, dmul(wgt, dadd(t[TY_QV], dqv)));
      den = dadd(den, wgt);
    }
  if (den > 0.0) {
    Qx = nx_ / den;
    Qv = nv_ / den;
  } else {
    const double* t = tay + (size_t)m * TY_N;
    double dqx, dqv;
    qofp_exact(t, Px, Pv, dqx, dqv);
    Qx = dadd(t[TY_QX], dqx);
    Qv = dadd(t[TY_QV], dqv);
  }
}

// The same blend for the FP64 remap, the beta ranges decided on the owner's
// offsets in the fixed order (the one integer decision here) and the
// neighbours' inverse maps, weights and sums in fused FP64: Q_r is continuous
// in them (W(2d) vanishes at the support's edge), and so is the spline sum
// it feeds, so the fused values agree with the fixed order to rounding.
__device__ __forceinline__ void qofp_fused(const double* __restrict__ t, double Px, double Pv, double& dqx,
                                           double& dqv) {
  const double dPx = Px - t[TY_X], dPv = Pv - t[TY_V];
  const double yx = fma(t[TY_TI01], dPv, t[TY_TI00] * dPx), yv = fma(t[TY_TI11], dPv, t[TY_TI10] * dPx);
  const double sx = fma(dPx, fma(t[TY_GX01], dPv, t[TY_GX00] * dPx), dPv * fma(t[TY_GX11], dPv, t[TY_GX01] * dPx));
  const double sv = fma(dPx, fma(t[TY_GV01], dPv, t[TY_GV00] * dPx), dPv * fma(t[TY_GV11], dPv, t[TY_GV01] * dPx));
  dqx = fma(-0.5, fma(t[TY_TI01], sv, t[TY_TI00] * sx), yx);
  dqv = fma(-0.5, fma(t[TY_TI11], sv, t[TY_TI10] * sx), yv);
}

__device__ __forceinline__ void blended_q_fused(const Grid& g, const double* __restrict__ tay, int m, double Px,
                                                double Pv, double& Qx, double& Qv) {
  double xi, ze;
  dist2_exact(tay + (size_t)m * TY_N, g, Px, Pv, xi, ze);
  const double beta = g.beta;
  const int a0 = (xi < -beta) ? -1 : ((xi < beta) ? -1 : 0);
  const int a1 = (xi < -beta) ? 0 : 1;
  const int b0 = (ze < -beta) ? -1 : ((ze < beta) ? -1 : 0);
  const int b1 = (ze < -beta) ? 0 : 1;
  const bool full = (a0 == -1 && a1 == 1) || (b0 == -1 && b1 == 1);
  const int k = m / g.Lv, l = m - k * g.Lv;
  double nx_ = 0.0, nv_ = 0.0, den = 0.0;
  for (int a = a0; a <= a1; a++)
    for (int b = b0; b <= b1; b++) {
      if (full && a != 0 && b != 0) continue;
      const int kk = k + a, ll = l + b;
      if (!elem_exists(g, kk, ll)) continue;
      const double* t = tay + (size_t)(kk * g.Lv + ll) * TY_N;
      double dqx, dqv;
      qofp_fused(t, Px, Pv, dqx, dqv);
      const double x1 = dqx * g.inv_dxm, z1 = dqv * g.inv_dvm;
      const double x = 2.0 * sqrt(fma(x1, x1, z1 * z1));
      double wgt = 0.0;
      if (x <= 1.0) {
        wgt = fma(0.75 * x, x * x, fma(-1.5 * x, x, 1.0));
      } else if (x <= 2.0) {
        const double r = 2.0 - x;
        wgt = 0.25 * (r * r * r);
      }
      nx_ = fma(wgt, t[TY_QX] + dqx, nx_);
      nv_ = fma(wgt, t[TY_QV] + dqv, nv_);
      den += wgt;
    }
  if (den > 0.0) {
    const double id = 1.0 / den;
    Qx = nx_ * id;
    Qv = nv_ * id;
  } else {
    const double* t = tay + (size_t)m * TY_N;
    double dqx, dqv;
    qofp_fused(t, Px, Pv, dqx, dqv);
    Qx = t[TY_QX] + dqx;
    Qv = t[TY_QV] + dqv;
  }
}

__device__ __forceinline__ long long ghost(long long k, int n) {
  if (k >= 0 && k < n) return k;
  if (k == -1) return 1;
  if (k == n) return n - 2;
  return -1;
}

// Cubic B-spline f(u, w) = sum eta_kl B(u-k) B(w-l) over k, l in -1..n with
// the zero-slope mirror ghosts (Sec. 2.2.2); the finite sum is evaluated
// everywhere and vanishes three cells beyond the edge nodes.
template <typename R>
__device__ __forceinline__ double spline_eval(const R* __restrict__ eta, const Grid& g, double u, double w) {
  if (!(u > -3.0 && u < (double)(g.nx + 2) && w > -3.0 && w < (double)(g.nv + 2))) return 0.0;
  const long long ku = (long long)floor(u), kw = (long long)floor(w);
  const R tu = (R)(u - (double)ku), tw = (R)(w - (double)kw);
  const R one = R(1), six = R(6), two3 = R(2) / R(3), half = R(0.5);
  R bu[4], bw[4];
  {
    R s = one - tu;
    bu[0] = s * s * s / six;
    bu[1] = two3 - tu * tu + half * tu * tu * tu;
    bu[2] = two3 - s * s + half * s * s * s;
    bu[3] = tu * tu * tu / six;
    s = one - tw;
    bw[0] = s * s * s / six;
    bw[1] = two3 - tw * tw + half * tw * tw * tw;
    bw[2] = two3 - s * s + half * s * s * s;
    bw[3] = tw * tw * tw / six;
  }
  R sum = R(0);
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const long long gk = ghost(ku - 1 + a, g.nx);
    if (gk < 0) continue;
    R row = R(0);
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const long long gl = ghost(kw - 1 + b, g.nv);
      if (gl < 0) continue;
      row += eta[gk * g.nv + gl] * bw[b];
    }
    sum += row * bu[a];
  }
  return (double)sum;
}

__device__ __forceinline__ void k_remap64_body(const Grid& g, const uint32_t* __restrict__ map, const DevState* ds,
                                                 const double* __restrict__ tay, const double* __restrict__ eta,
                                                 double* __restrict__ out, int vb) {
  using R = double;
  const int i = vb;
  const double Px = site_x(g, i);
  int js, je;
  row_span(g, ds, i, js, je);
  zero_outside(g, out + (size_t)i * g.nv, js, je);
  for (int j = js + threadIdx.x; j <= je; j += blockDim.x) {
    const size_t p = (size_t)i * g.nv + j;
    const int m = owner(map, p, ds_epoch(ds), g.ne);
    double val = 0.0;
    if (m >= 0) {
      double Qx, Qv;
      blended_q_fused(g, tay, m, Px, site_v(g, j), Qx, Qv);
      const double u = (Qx - g.x_lo) * g.inv_dx;
      const double w = (Qv - g.v_lo) * g.inv_dv;
      val = spline_eval(eta, g, u, w);
    }
    out[p] = (R)val;
  }
}

__global__ void __launch_bounds__(256) k_remap64(Grid g, const uint32_t* __restrict__ map, const DevState* ds,
                                                 const double* __restrict__ tay, const double* __restrict__ eta,
                                                 double* __restrict__ out) {
  if (gate_shut(g)) return;
  k_remap64_body(g, map, ds, tay, eta, out, blockIdx.x);
}


// ---------------------------------------------------------------------------
// FP32-mixed path
// ---------------------------------------------------------------------------

constexpr float kRelQ = 2.0e-6f, kAbs = 1.0e-9f;

struct QF {
  float qx, qv, ex, ev;  // offset in element units and its bounds
};

__device__ __forceinline__ QF qeval(const float* __restrict__ F, float px, float pv) {
  QF r;
  // the record's first 16 words in four 16-byte loads (records are 128-byte
  // aligned): T, A, B, C of both axes, the bound coefficients
  const float4* F4 = reinterpret_cast<const float4*>(F);
  const float4 f0 = F4[0], f1 = F4[1], f2 = F4[2], f3 = F4[3];
  const float tx = fmaf(f1.x, px, fmaf(f1.y, pv, f0.x)), ux = fmaf(f1.z, pv, f0.y);
  const float tv = fmaf(f1.w, px, fmaf(f2.x, pv, f0.z)), uv = fmaf(f2.y, pv, f0.w);
  r.qx = fmaf(px, tx, pv * ux);
  r.qv = fmaf(px, tv, pv * uv);
  const float P = fmaxf(fabsf(px), fabsf(pv));
  const float ax = f2.z * P + f2.w * (P * P);
  const float av = f3.x * P + f3.y * (P * P);
  r.ex = kRelQ * ax + kAbs * (1.f + ax);
  r.ev = kRelQ * av + kAbs * (1.f + av);
  return r;
}

// p = (P - P_m)/Delta_m of site (i, j) for the element with record F.
__device__ __forceinline__ void p_of(const float* __restrict__ F, int i, int j, float inv_s, float& px, float& pv) {
  const int* Fi = reinterpret_cast<const int*>(F);
  px = ((float)(i - Fi[TF_UI]) - F[TF_UF]) * inv_s;
  pv = ((float)(j - Fi[TF_WI]) - F[TF_WF]) * inv_s;
}

// The lattice index position of Q_m (a multiple of 1/2): integer part and
// half flag, exactly (integer arithmetic: no load on the latency chain).
__device__ __forceinline__ void anchor(const Grid& g, int m, int& Bu, float& bu, int& Bw, float& bw) {
  const int k = m / g.Lv, l = m - k * g.Lv;
  const int u2 = (g.nx - 1) + 2 * (k - g.Kx - 1) * g.s;  // 2 * index of Q_m,x
  const int w2 = (g.nv - 1) + 2 * (l - g.Kv - 1) * g.s;
  Bu = u2 >> 1;  // floor
  bu = (u2 & 1) ? 0.5f : 0.f;
  Bw = w2 >> 1;
  bw = (w2 & 1) ? 0.5f : 0.f;
}

// The anchor with k = m / Lv from an FP32 reciprocal (m < 2^24 is exact in
// FP32, the quotient is off by at most one and corrected): a few
// instructions instead of an integer division per site.
__device__ __forceinline__ void anchor_r(const Grid& g, int m, float inv_Lv, int& Bu, float& bu, int& Bw, float& bw) {
  int k = (int)((float)m * inv_Lv);
  if (k * g.Lv > m) k--;
  if ((k + 1) * g.Lv <= m) k++;
  const int l = m - k * g.Lv;
  const int u2 = (g.nx - 1) + 2 * (k - g.Kx - 1) * g.s;
  const int w2 = (g.nv - 1) + 2 * (l - g.Kv - 1) * g.s;
  Bu = u2 >> 1;
  bu = (u2 & 1) ? 0.5f : 0.f;
  Bw = w2 >> 1;
  bw = (w2 & 1) ? 0.5f : 0.f;
}

// Is floor(x) certain for every value within e of x?
__device__ __forceinline__ bool floor_sure(float x, float e) {
  const float f = floorf(x);
  return (x - e > f) && (x + e < f + 1.f);
}

__device__ __forceinline__ float F_at32(const float* __restrict__ F, const Grid& g, int i, int j) {
  if (i < 0 || j < 0 || i >= g.nx || j >= g.nv) return 0.f;
  return __ldg(F + (size_t)i * g.nv + j);
}

// Six-point quadratic interpolation from the node choice and the offsets;
// the stencil entirely inside the grid (1 <= in <= nx-2, 1 <= jn <= nv-2;
// ic and jc are in-1 or in, jn-1 or jn).
__device__ __forceinline__ float qinterp32_in(const float* __restrict__ F, const Grid& g, int in, int jn, int ic,
                                              int jc, float x, float y) {
  const float* c = F + (size_t)in * g.nv + jn;
  const float* d = F + (size_t)ic * g.nv + jc;
  float f = __ldg(c) * (1.0f - x * x - y * y);
  f += 0.5f * x * (__ldg(c + g.nv) * (1.0f + x) + __ldg(c - g.nv) * (x - 1.0f));
  f += 0.5f * y * (__ldg(c + 1) * (1.0f + y) + __ldg(c - 1) * (y - 1.0f));
  f += (__ldg(d + g.nv + 1) + __ldg(d) - __ldg(d + g.nv) - __ldg(d + 1)) * x * y;
  return f;
}

// The same with every node checked (outside the grid f is 0).
__device__ __forceinline__ float qinterp32(const float* __restrict__ F, const Grid& g, int in, int jn, int ic, int jc,
                                           float x, float y) {
  float f = F_at32(F, g, in, jn) * (1.0f - x * x - y * y);
  f += 0.5f * x * (F_at32(F, g, in + 1, jn) * (1.0f + x) + F_at32(F, g, in - 1, jn) * (x - 1.0f));
  f += 0.5f * y * (F_at32(F, g, in, jn + 1) * (1.0f + y) + F_at32(F, g, in, jn - 1) * (y - 1.0f));
  f += (F_at32(F, g, ic + 1, jc + 1) + F_at32(F, g, ic, jc) - F_at32(F, g, ic + 1, jc) - F_at32(F, g, ic, jc + 1)) *
       x * y;
  return f;
}

// Per-thread row sum of FP32 values as an unevaluated float pair (hi + lo,
// Knuth's TwoSum), converted to double once per thread: ~2^-48 relative
// accuracy with FP32 arithmetic only.
struct FPair {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// The nearest nodes are certain but a containing square (cell) is not: the
// offset along that axis is within its bound of 0.  The cell enters f only
// through the cross term, weighted by x y, so the FP32 cell is taken when the
// largest change the other choice could make, 2 (|x| + e_u)(|y| + e_v) times
// the largest |cross difference| of the four cells around the node, is at
// most 1e-7 of the largest |F| of the node's 3x3 block: a proven bound on the
// effect on f, a tenth of the reconstruction's 1e-6 max|f| tolerance.  (Right
// after a remap every Q_v lies on a node, and without this rule every site
// took the FP64 evaluation.)  Returns false, with nothing set, otherwise.
__device__ __forceinline__ bool cell_free32(const Grid& g, const float* __restrict__ fini, int Bu, float ru,
                                            float eu, int Bw, float rw, float ew, int& in, int& jn, int& ic,
                                            int& jc, float& x, float& y) {
  if (!(floor_sure(ru + 0.5f, eu) && floor_sure(rw + 0.5f, ew))) return false;
  const float nu = floorf(ru + 0.5f), nw = floorf(rw + 0.5f);
  const int i0 = Bu + (int)nu, j0 = Bw + (int)nw;
  float Fb[3][3], fref = 0.f;
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      Fb[a][b] = F_at32(fini, g, i0 + a - 1, j0 + b - 1);
      fref = fmaxf(fref, fabsf(Fb[a][b]));
    }
  float cm = 0.f;
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++)
      cm = fmaxf(cm, fabsf(Fb[a + 1][b + 1] + Fb[a][b] - Fb[a + 1][b] - Fb[a][b + 1]));
  const float xx = ru - nu, yy = rw - nw;
  if (!(2.f * (fabsf(xx) + eu) * (fabsf(yy) + ew) * cm <= 1e-7f * fref)) return false;
  in = i0;
  jn = j0;
  ic = Bu + (int)floorf(ru);
  jc = Bw + (int)floorf(rw);
  x = xx;
  y = yy;
  return true;
}

// Value of f at site (i, j) owned by element m: every case (node choice by
// the FP64 evaluation when the FP32 bound cannot settle it, stencils that
// leave the grid).
__device__ __noinline__ float recon_site32(const Grid& g, const double* __restrict__ tay,
                                           const float* __restrict__ tayf, const float* __restrict__ fini, int i,
                                           int j, int m) {
  const float inv_s = 1.0f / (float)g.s, fs = (float)g.s;
  float val = 0.f;
  const float* F = tayf + (size_t)m * TF_N;
  float px, pv;
  p_of(F, i, j, inv_s, px, pv);
  const QF q = qeval(F, px, pv);
  int Bu, Bw;
  float bu, bw;
  anchor(g, m < 0 ? 0 : m, Bu, bu, Bw, bw);
  // index coordinates of Q relative to the anchor
  const float ru = bu + fs * q.qx, rw = bw + fs * q.qv;
  const float eu = fs * q.ex + 1e-6f * (1.f + fabsf(ru)), ew = fs * q.ev + 1e-6f * (1.f + fabsf(rw));
  int in, jn, ic, jc;
  float x, y;
  if (!(fabsf(ru) < 1e7f && fabsf(rw) < 1e7f)) {
    // far outside the grid (or not a number): no node of the stencil exists
    in = jn = ic = jc = -1000000;
    x = y = 0.f;
  } else if (floor_sure(ru + 0.5f, eu) && floor_sure(ru, eu) && floor_sure(rw + 0.5f, ew) && floor_sure(rw, ew)) {
    const float nu = floorf(ru + 0.5f), nw = floorf(rw + 0.5f);
    in = Bu + (int)nu;
    jn = Bw + (int)nw;
    ic = Bu + (int)floorf(ru);
    jc = Bw + (int)floorf(rw);
    x = ru - nu;
    y = rw - nw;
  } else if (cell_free32(g, fini, Bu, ru, eu, Bw, rw, ew, in, jn, ic, jc, x, y)) {
    // nodes certain; the cell taken from the FP32 value (see cell_free32)
  } else {
    // FP64 evaluation, as the FP64 path takes these decisions
    const double* t = tay + (size_t)m * TY_N;
    double dqx, dqv;
    qofp_exact(t, site_x(g, i), site_v(g, j), dqx, dqv);
    const double u = dmul(dsub(dadd(t[TY_QX], dqx), g.x_lo), g.inv_dx);
    const double w = dmul(dsub(dadd(t[TY_QV], dqv), g.v_lo), g.inv_dv);
    if (!(u > -2.0 && u < (double)g.nx + 1.0 && w > -2.0 && w < (double)g.nv + 1.0)) {
      in = jn = ic = jc = -1000000;
      x = y = 0.f;
    } else {
      in = (int)floor(dadd(u, 0.5));
      jn = (int)floor(dadd(w, 0.5));
      ic = (int)floor(u);
      jc = (int)floor(w);
      x = (float)dsub(u, (double)in);
      y = (float)dsub(w, (double)jn);
    }
  }
  if (in > -2 && in < g.nx + 2 && jn > -2 && jn < g.nv + 2) val = qinterp32(fini, g, in, jn, ic, jc, x, y);
  return val;
}

// The common case without branches: the FP32 node choice is certain and the
// whole stencil is inside the grid.  Otherwise *slow is set (the value is
// then recon_site32's); the loads stay in bounds either way, so that the
// loads of several sites can be in flight together.
__device__ __forceinline__ float recon_fast32(const Grid& g, const float* __restrict__ tayf,
                                              const float* __restrict__ fini, int i, int j, int m, float inv_Lv,
                                              bool* slow) {
  const float inv_s = 1.0f / (float)g.s, fs = (float)g.s;
  const float* F = tayf + (size_t)(m < 0 ? 0 : m) * TF_N;
  float px, pv;
  p_of(F, i, j, inv_s, px, pv);
  const QF q = qeval(F, px, pv);
  int Bu, Bw;
  float bu, bw;
  anchor_r(g, m < 0 ? 0 : m, inv_Lv, Bu, bu, Bw, bw);
  const float ru = bu + fs * q.qx, rw = bw + fs * q.qv;
  const float eu = fs * q.ex + 1e-6f * (1.f + fabsf(ru)), ew = fs * q.ev + 1e-6f * (1.f + fabsf(rw));
  const bool finite = fabsf(ru) < 1e6f && fabsf(rw) < 1e6f;
  const float ruc = finite ? ru : 0.f, rwc = finite ? rw : 0.f;
  // nearest node floor(r + 1/2) and cell floor(r) from one floor of 2r
  // (exact doubling): both are certain when [2r - 2e, 2r + 2e] holds no
  // integer (the rounded end points err towards failing the test)
  const float tu = 2.f * ruc, tw = 2.f * rwc;
  const float fu = floorf(tu), fw = floorf(tw);
  const int iu = (int)fu, iw = (int)fw;
  const float nu = (float)((iu + 1) >> 1), nw = (float)((iw + 1) >> 1);
  int in = Bu + ((iu + 1) >> 1), jn = Bw + ((iw + 1) >> 1);
  int ic = Bu + (iu >> 1), jc = Bw + (iw >> 1);
  const bool sure = finite && (tu - 2.f * eu > fu) && (tu + 2.f * eu < fu + 1.f) && (tw - 2.f * ew > fw) &&
                    (tw + 2.f * ew < fw + 1.f);
  const bool inside = in >= 1 && in <= g.nx - 2 && jn >= 1 && jn <= g.nv - 2;
  *slow = (m >= 0) && !(sure && inside);
  if (!(sure && inside)) {  // any in-grid stencil: its value is not used
    in = jn = 1;
    ic = jc = 0;
  }
  const float v = qinterp32_in(fini, g, in, jn, ic, jc, ruc - nu, rwc - nw);
  return (m >= 0) ? v : 0.f;
}

__device__ __forceinline__ void k_recon32_body(const Grid& g, const uint32_t* __restrict__ map, const DevState* ds,
                                                 const double* __restrict__ tay, const float* __restrict__ tayf,
                                                 const float* __restrict__ fini, float* __restrict__ f,
                                                 double* __restrict__ M, int vb) {
  __shared__ double sh[32];
  const int i = vb;
  const uint32_t epoch = ds_epoch(ds);
  FPair acc;
  const float inv_Lv = 1.0f / (float)g.Lv;
  const size_t row = (size_t)i * g.nv;
  int js, je;
  row_span(g, ds, i, js, je);
  zero_outside(g, f + row, js, je);
  // the owner of the thread's next site is loaded one iteration ahead
  int m = (js + (int)threadIdx.x <= je) ? owner(map, row + js + threadIdx.x, epoch, g.ne) : -1;
  for (int j = js + threadIdx.x; j <= je; j += blockDim.x) {
    const int jn = j + blockDim.x;
    const int mn = (jn <= je) ? owner(map, row + jn, epoch, g.ne) : -1;
    bool slow;
    float v = recon_fast32(g, tayf, fini, i, j, m, inv_Lv, &slow);
    if (slow) v = recon_site32(g, tay, tayf, fini, i, j, m);
    f[row + j] = v;
    acc.add(v);
    m = mn;
  }
  const double rowsum = block_sum(acc.value(), sh);
  if (threadIdx.x == 0) M[i] = dmul(rowsum, g.dxdv);
}

__device__ __forceinline__ bool recon64_fast(const Grid& g, const double* __restrict__ t, const float* __restrict__ F,
                                             int m, int i, int j, double Px, double Pv,
                                             const double* __restrict__ fini, float inv_Lv, double& val) {
  const float inv_s = 1.0f / (float)g.s, fs = (float)g.s;
  float px, pv;
  p_of(F, i, j, inv_s, px, pv);
  const QF q = qeval(F, px, pv);
  int Bu, Bw;
  float bu, bw;
  anchor_r(g, m, inv_Lv, Bu, bu, Bw, bw);
  const float ru = bu + fs * q.qx, rw = bw + fs * q.qv;
  const float eu = fs * q.ex + 1e-6f * (1.f + fabsf(ru)), ew = fs * q.ev + 1e-6f * (1.f + fabsf(rw));
  if (!(fabsf(ru) < 1e6f && fabsf(rw) < 1e6f)) return false;
  const float tu = 2.f * ru, tw = 2.f * rw;
  const float fu = floorf(tu), fw = floorf(tw);
  if (!((tu - 2.f * eu > fu) && (tu + 2.f * eu < fu + 1.f) && (tw - 2.f * ew > fw) && (tw + 2.f * ew < fw + 1.f)))
    return false;
  const int iu = (int)fu, iw = (int)fw;
  const long long in = Bu + ((iu + 1) >> 1), jn = Bw + ((iw + 1) >> 1);
  const long long ic = Bu + (iu >> 1), jc = Bw + (iw >> 1);
  // FP64 offset, fused, on the exact lattice index of Q_m
  const double dPx = Px - t[TY_X], dPv = Pv - t[TY_V];
  const double yx = fma(t[TY_TI00], dPx, t[TY_TI01] * dPv), yv = fma(t[TY_TI10], dPx, t[TY_TI11] * dPv);
  double g0 = fma(t[TY_GX00], dPx, t[TY_GX01] * dPv), g1 = fma(t[TY_GX01], dPx, t[TY_GX11] * dPv);
  const double sx = fma(dPx, g0, dPv * g1);
  g0 = fma(t[TY_GV00], dPx, t[TY_GV01] * dPv);
  g1 = fma(t[TY_GV01], dPx, t[TY_GV11] * dPv);
  const double sv = fma(dPx, g0, dPv * g1);
  const double dqx = fma(-0.5, fma(t[TY_TI00], sx, t[TY_TI01] * sv), yx);
  const double dqv = fma(-0.5, fma(t[TY_TI10], sx, t[TY_TI11] * sv), yv);
  const double u = fma(dqx, g.inv_dx, (double)Bu + (double)bu), w = fma(dqv, g.inv_dv, (double)Bw + (double)bw);
  val = qinterp64_fused(fini, g, in, jn, ic, jc, u - (double)in, w - (double)jn);
  return true;
}

__global__ void __launch_bounds__(256, 6) k_recon32(Grid g, const uint32_t* __restrict__ map, const DevState* ds,
                                                 const double* __restrict__ tay, const float* __restrict__ tayf,
                                                 const float* __restrict__ fini, float* __restrict__ f,
                                                 double* __restrict__ M) {
  k_recon32_body(g, map, ds, tay, tayf, fini, f, M, blockIdx.x);
}

// ---------------------------------------------------------------------------
// FP32-mixed reconstruction in tiles staged by bulk copies
// ---------------------------------------------------------------------------
//
// A block takes a tile of RT_R x rows by RT_C v columns (one column per
// thread).  Phase 1 takes every site's certified node and cell decisions
// (as recon_fast32, without touching f_ini) and the bounding rectangle of
// the six-point stencils of the tile; if that patch of f_ini fits the
// shared-memory budget (and rows are 16-byte aligned, nv % 4 == 0), one
// thread issues a bulk copy (cp.async.bulk, the TMA engine) of each of its
// rows inside the grid, completing on one mbarrier, while the others zero
// the parts outside the grid (F = 0 there).  Phase 2 interpolates from
// shared memory, writes f (a warp writes 128 contiguous bytes) and the
// tile's row sums.  Sites the bound leaves open take recon_site32 (global
// memory); a patch too large for the budget falls back to global gathers
// for the tile.  The pixel masses are the tiles' row sums added in order
// (k_row_mass).
constexpr int RT_R = 4, RT_C = 256, RT_PR = 32, RT_PC = 288;

struct __align__(16) TileShared {
  float patch[RT_PR * RT_PC];
  float2 xy[RT_R * RT_C];
  int2 node[RT_R * RT_C];  // (in, jn) of a certain site; (m, -) of a site for recon_site32
  unsigned char kind[RT_R * RT_C];  // 0: f = 0; 1: certain (bit 2: ic = in - 1, bit 3: jc = jn - 1); 2: slow
  double rsum[RT_R][RT_C / 32];
  unsigned long long bar;
  int bounds[4];
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// The certified decisions of site (i, j) owned by m (recon_fast32's test):
// 1 with the nodes and offsets when they are certain and finite, else 2.
__device__ __forceinline__ int decide32(const Grid& g, const float* __restrict__ tayf, int i, int j, int m,
                                        float inv_Lv, int& in, int& jn, int& dic, int& djc, float& x, float& y) {
  const float inv_s = 1.0f / (float)g.s, fs = (float)g.s;
  const float* F = tayf + (size_t)m * TF_N;
  float px, pv;
  p_of(F, i, j, inv_s, px, pv);
  const QF q = qeval(F, px, pv);
  int Bu, Bw;
  float bu, bw;
  anchor_r(g, m, inv_Lv, Bu, bu, Bw, bw);
  const float ru = bu + fs * q.qx, rw = bw + fs * q.qv;
  const float eu = fs * q.ex + 1e-6f * (1.f + fabsf(ru)), ew = fs * q.ev + 1e-6f * (1.f + fabsf(rw));
  if (!(fabsf(ru) < 1e6f && fabsf(rw) < 1e6f)) return 2;
  const float tu = 2.f * ru, tw = 2.f * rw;
  const float fu = floorf(tu), fw = floorf(tw);
  if (!((tu - 2.f * eu > fu) && (tu + 2.f * eu < fu + 1.f) && (tw - 2.f * ew > fw) && (tw + 2.f * ew < fw + 1.f)))
    return 2;
  const int iu = (int)fu, iw = (int)fw;
  const int nu = (iu + 1) >> 1, nw = (iw + 1) >> 1;
  in = Bu + nu;
  jn = Bw + nw;
  dic = (iu >> 1) - nu;  // 0 or -1
  djc = (iw >> 1) - nw;
  x = ru - (float)nu;
  y = rw - (float)nw;
  return 1;
}

// The six-point value (the arithmetic of qinterp32_in) from node values.
__device__ __forceinline__ float six_point(float c, float cxp, float cxm, float cyp, float cym, float d00, float d10,
                                           float d01, float d11, float x, float y) {
  float f = c * (1.0f - x * x - y * y);
  f += 0.5f * x * (cxp * (1.0f + x) + cxm * (x - 1.0f));
  f += 0.5f * y * (cyp * (1.0f + y) + cym * (y - 1.0f));
  f += (d11 + d00 - d10 - d01) * x * y;
  return f;
}

__device__ __forceinline__ void recon32_tile_body(const Grid& g, const uint32_t* __restrict__ map, const DevState* ds,
                                                  const double* __restrict__ tay, const float* __restrict__ tayf,
                                                  const float* __restrict__ fini, float* __restrict__ f,
                                                  double* __restrict__ Mpart, DevState* dse, int vb) {
  extern __shared__ __align__(16) unsigned char tile_raw[];
  TileShared& S = *reinterpret_cast<TileShared*>(tile_raw);
  const int ntj = (g.nv + RT_C - 1) / RT_C;
  const int ti = vb / ntj, tj = vb - ti * ntj;
  const int i0 = ti * RT_R, j = tj * RT_C + (int)threadIdx.x;
  const int tid = threadIdx.x;
  const uint32_t epoch = ds_epoch(ds);
  const float inv_Lv = 1.0f / (float)g.Lv;
  if (tid < 4) S.bounds[tid] = (tid & 1) ? INT_MIN : INT_MAX;
  __syncthreads();
  // phase 1: decisions
  int lo_i = INT_MAX, hi_i = INT_MIN, lo_j = INT_MAX, hi_j = INT_MIN;
#pragma unroll
  for (int r = 0; r < RT_R; r++) {
    const int i = i0 + r, q = r * RT_C + tid;
    unsigned char kd = 0;
    if (i < g.nx && j < g.nv) {
      int js, je;
      row_span(g, ds, i, js, je);
      const int m = (j >= js && j <= je) ? owner(map, (size_t)i * g.nv + j, epoch, g.ne) : -1;
      if (m >= 0) {
        int in, jn, dic, djc;
        float x, y;
        if (decide32(g, tayf, i, j, m, inv_Lv, in, jn, dic, djc, x, y) == 1) {
          kd = (unsigned char)(1 | (dic ? 4 : 0) | (djc ? 8 : 0));
          S.node[q] = make_int2(in, jn);
          S.xy[q] = make_float2(x, y);
          lo_i = min(lo_i, in - 1);
          hi_i = max(hi_i, in + 1);
          lo_j = min(lo_j, jn - 1);
          hi_j = max(hi_j, jn + 1);
        } else {
          kd = 2;
          S.node[q] = make_int2(m, 0);
        }
      }
    }
    S.kind[q] = kd;
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo_i = min(lo_i, __shfl_xor_sync(0xffffffffu, lo_i, o));
    hi_i = max(hi_i, __shfl_xor_sync(0xffffffffu, hi_i, o));
    lo_j = min(lo_j, __shfl_xor_sync(0xffffffffu, lo_j, o));
    hi_j = max(hi_j, __shfl_xor_sync(0xffffffffu, hi_j, o));
  }
  if ((tid & 31) == 0 && lo_i <= hi_i) {
    atomicMin(&S.bounds[0], lo_i);
    atomicMax(&S.bounds[1], hi_i);
    atomicMin(&S.bounds[2], lo_j);
    atomicMax(&S.bounds[3], hi_j);
  }
  __syncthreads();
  const int pi0 = S.bounds[0], pi1 = S.bounds[1];
  const int pj0 = (S.bounds[2] >> 2) << 2, pj1 = ((S.bounds[3] + 4) >> 2) << 2;  // [pj0, pj1), multiples of 4
  const bool fits = (g.nv % 4 == 0) && pi0 <= pi1 && (pi1 - pi0 + 1) <= RT_PR && (pj1 - pj0) <= RT_PC;
  if (fits) {
    const int nrows = pi1 - pi0 + 1, ncols = pj1 - pj0;
    // zeros where the patch leaves the grid
    for (int idx = tid; idx < nrows * ncols; idx += blockDim.x) {
      const int rr = idx / ncols, cc = idx - rr * ncols;
      const int ii = pi0 + rr, jj = pj0 + cc;
      if (ii < 0 || ii >= g.nx || jj < 0 || jj >= g.nv) S.patch[rr * RT_PC + cc] = 0.f;
    }
    const int c0 = max(pj0, 0), c1 = min(pj1, g.nv);
    const int r0 = max(pi0, 0), r1 = min(pi1, g.nx - 1);
    const unsigned row_bytes = (c1 > c0) ? (unsigned)(c1 - c0) * 4u : 0u;
    const unsigned total = (r1 >= r0) ? row_bytes * (unsigned)(r1 - r0 + 1) : 0u;
    if (tid == 0) mbar_init(&S.bar, 1);
    __syncthreads();
    if (tid == 0) {
      if (total > 0) {
        mbar_expect_tx(&S.bar, total);
        for (int ii = r0; ii <= r1; ii++)
          bulk_g2s(&S.patch[(ii - pi0) * RT_PC + (c0 - pj0)], fini + (size_t)ii * g.nv + c0, row_bytes, &S.bar);
      } else {
        mbar_arrive(&S.bar);
      }
    }
    // every copy completes unless a byte count were wrong: the wait is
    // bounded all the same, and a wait that runs out is reported
    bool ok = false;
    for (int it = 0; it < (1 << 22) && !ok; it++) ok = mbar_try_wait(&S.bar, 0);
    if (!ok) VM_BAD(dse, 41);
    __syncthreads();
    if (tid == 0) mbar_inval(&S.bar);
  }
  // phase 2: values, f, row sums
  double rs[RT_R];
#pragma unroll
  for (int r = 0; r < RT_R; r++) {
    const int i = i0 + r, q = r * RT_C + tid;
    const unsigned char kd = S.kind[q];
    float v = 0.f;
    if (kd & 1) {
      const int2 nd = S.node[q];
      const float2 xy = S.xy[q];
      const int in = nd.x, jn = nd.y, ic = in + ((kd & 4) ? -1 : 0), jc = jn + ((kd & 8) ? -1 : 0);
      if (fits) {
        const float* P = S.patch;
        auto at = [&](int a, int b) { return P[(a - pi0) * RT_PC + (b - pj0)]; };
        v = six_point(at(in, jn), at(in + 1, jn), at(in - 1, jn), at(in, jn + 1), at(in, jn - 1), at(ic, jc),
                      at(ic + 1, jc), at(ic, jc + 1), at(ic + 1, jc + 1), xy.x, xy.y);
      } else {
        v = six_point(F_at32(fini, g, in, jn), F_at32(fini, g, in + 1, jn), F_at32(fini, g, in - 1, jn),
                      F_at32(fini, g, in, jn + 1), F_at32(fini, g, in, jn - 1), F_at32(fini, g, ic, jc),
                      F_at32(fini, g, ic + 1, jc), F_at32(fini, g, ic, jc + 1), F_at32(fini, g, ic + 1, jc + 1),
                      xy.x, xy.y);
      }
    } else if (kd == 2) {
      v = recon_site32(g, tay, tayf, fini, i, j, S.node[q].x);
    }
    if (i < g.nx && j < g.nv) f[(size_t)i * g.nv + j] = v;
    double w = (double)v;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    rs[r] = w;
  }
  if ((tid & 31) == 0)
#pragma unroll
    for (int r = 0; r < RT_R; r++) S.rsum[r][tid >> 5] = rs[r];
  __syncthreads();
  if (tid < RT_R && i0 + tid < g.nx) {
    double t = 0.0;
    for (int w = 0; w < RT_C / 32; w++) t += S.rsum[tid][w];
    Mpart[(size_t)(i0 + tid) * ntj + tj] = t;
  }
}

__global__ void __launch_bounds__(RT_C) k_recon32_tiles(Grid g, const uint32_t* __restrict__ map, DevState* ds,
                                                        const double* __restrict__ tay, const float* __restrict__ tayf,
                                                        const float* __restrict__ fini, float* __restrict__ f,
                                                        double* __restrict__ Mpart) {
  recon32_tile_body(g, map, ds, tay, tayf, fini, f, Mpart, ds, blockIdx.x);
}

// M(i) = (sum of the row's tile sums, in tile order) dx dv.
__device__ __forceinline__ void row_mass_body(const Grid& g, const double* __restrict__ Mpart, double* __restrict__ M,
                                              int vb) {
  const int i = vb * blockDim.x + threadIdx.x;
  if (i >= g.nx) return;
  const int ntj = (g.nv + RT_C - 1) / RT_C;
  double t = 0.0;
  for (int k = 0; k < ntj; k++) t += Mpart[(size_t)i * ntj + k];
  M[i] = dmul(t, g.dxdv);
}

__global__ void k_row_mass(Grid g, const double* __restrict__ Mpart, double* __restrict__ M) {
  row_mass_body(g, Mpart, M, blockIdx.x);
}

__device__ __forceinline__ float W4f(float x) {
  if (x <= 1.f) return 1.f - 1.5f * x * x + 0.75f * x * x * x;
  if (x <= 2.f) {
    const float r = 2.f - x;
    return 0.25f * r * r * r;
  }
  return 0.f;
}

// beta range of one axis, 1: {-1,0}, 2: {-1,0,1}, 3: {0,1}, 0: cannot tell.
__device__ __forceinline__ int beta_range_f(float q, float e, float blo, float bhi) {
  if (q + e < -bhi) return 1;
  if (q - e >= -blo && q + e < blo) return 2;
  if (q - e >= bhi) return 3;
  return 0;
}

// Cubic B-spline at index coordinates (B + r) along each axis.
__device__ __forceinline__ float spline32(const float* __restrict__ eta, const Grid& g, int Bu, float ru, int Bw,
                                          float rw) {
  if (!(fabsf(ru) < 1e7f && fabsf(rw) < 1e7f)) return 0.f;
  const float fu = floorf(ru), fw = floorf(rw);
  const long long ku = (long long)Bu + (long long)fu, kw = (long long)Bw + (long long)fw;
  if (ku < -4 || ku > g.nx + 2 || kw < -4 || kw > g.nv + 2) return 0.f;
  const float tu = ru - fu, tw = rw - fw;
  float bu4[4], bw4[4];
  float s_ = 1.f - tu;
  bu4[0] = s_ * s_ * s_ * (1.f / 6.f);
  bu4[1] = (2.f / 3.f) - tu * tu + 0.5f * tu * tu * tu;
  bu4[2] = (2.f / 3.f) - s_ * s_ + 0.5f * s_ * s_ * s_;
  bu4[3] = tu * tu * tu * (1.f / 6.f);
  s_ = 1.f - tw;
  bw4[0] = s_ * s_ * s_ * (1.f / 6.f);
  bw4[1] = (2.f / 3.f) - tw * tw + 0.5f * tw * tw * tw;
  bw4[2] = (2.f / 3.f) - s_ * s_ + 0.5f * s_ * s_ * s_;
  bw4[3] = tw * tw * tw * (1.f / 6.f);
  float sum = 0.f;
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const long long gk = ghost(ku - 1 + a, g.nx);
    if (gk < 0) continue;
    float row = 0.f;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const long long gl = ghost(kw - 1 + b, g.nv);
      if (gl < 0) continue;
      row += __ldg(eta + gk * g.nv + gl) * bw4[b];
    }
    sum += row * bu4[a];
  }
  return sum;
}

__device__ __forceinline__ void k_remap32_body(const Grid& g, const uint32_t* __restrict__ map, const DevState* ds,
                                                 const double* __restrict__ tay, const float* __restrict__ tayf,
                                                 const float* __restrict__ eta, float* __restrict__ out, float blo,
                                                 float bhi, int vb) {
  const int i = vb;
  const float inv_s = 1.0f / (float)g.s, fs = (float)g.s;
  int js, je;
  row_span(g, ds, i, js, je);
  zero_outside(g, out + (size_t)i * g.nv, js, je);
  for (int j = js + threadIdx.x; j <= je; j += blockDim.x) {
    const size_t p = (size_t)i * g.nv + j;
    const int m = owner(map, p, ds_epoch(ds), g.ne);
    float val = 0.f;
    if (m >= 0) {
      const float* F = tayf + (size_t)m * TF_N;
      float px, pv;
      p_of(F, i, j, inv_s, px, pv);
      const QF q = qeval(F, px, pv);
      const int ra = beta_range_f(q.qx, q.ex, blo, bhi), rb = beta_range_f(q.qv, q.ev, blo, bhi);
      int Bu, Bw;
      float bu, bw;
      anchor(g, m < 0 ? 0 : m, Bu, bu, Bw, bw);
      float ru, rw;
      if (ra && rb) {
        // Q_r - Q_m in element units, blended over the beta set (Sec. 2.3.2)
        const int a0 = (ra == 3) ? 0 : -1, a1 = (ra == 1) ? 0 : 1;
        const int b0 = (rb == 3) ? 0 : -1, b1 = (rb == 1) ? 0 : 1;
        const bool full = (ra == 2) || (rb == 2);
        const int k = m / g.Lv, l = m - k * g.Lv;
        float nx_ = 0.f, nv_ = 0.f, den = 0.f;
        for (int a = a0; a <= a1; a++)
          for (int b = b0; b <= b1; b++) {
            if (full && a != 0 && b != 0) continue;
            const int kk = k + a, ll = l + b;
            if (!elem_exists(g, kk, ll)) continue;
            const float* Fn = tayf + (size_t)(kk * g.Lv + ll) * TF_N;
            float pxn, pvn;
            p_of(Fn, i, j, inv_s, pxn, pvn);
            const QF qn = (a == 0 && b == 0) ? q : qeval(Fn, pxn, pvn);
            const float wgt = W4f(2.f * sqrtf(qn.qx * qn.qx + qn.qv * qn.qv));
            nx_ += wgt * ((float)a + qn.qx);
            nv_ += wgt * ((float)b + qn.qv);
            den += wgt;
          }
        const float dx_ = (den > 0.f) ? nx_ / den : q.qx;
        const float dv_ = (den > 0.f) ? nv_ / den : q.qv;
        ru = bu + fs * dx_;
        rw = bw + fs * dv_;
      } else {
        double Qx, Qv;
        blended_q(g, tay, m, site_x(g, i), site_v(g, j), Qx, Qv);
        const double u = dmul(dsub(Qx, g.x_lo), g.inv_dx), w = dmul(dsub(Qv, g.v_lo), g.inv_dv);
        if (!(u > -3.0 && u < (double)(g.nx + 2) && w > -3.0 && w < (double)(g.nv + 2))) {
          out[p] = 0.f;
          continue;
        }
        const double fu = floor(u), fw = floor(w);
        Bu = (int)fu;
        Bw = (int)fw;
        ru = (float)(u - fu);
        rw = (float)(w - fw);
      }
      val = spline32(eta, g, Bu, ru, Bw, rw);
    }
    out[p] = val;
  }
}

__global__ void __launch_bounds__(256) k_remap32(Grid g, const uint32_t* __restrict__ map, const DevState* ds,
                                                 const double* __restrict__ tay, const float* __restrict__ tayf,
                                                 const float* __restrict__ eta, float* __restrict__ out, float blo,
                                                 float bhi) {
  if (gate_shut(g)) return;
  k_remap32_body(g, map, ds, tay, tayf, eta, out, blo, bhi, blockIdx.x);
}

// ---- group launches ----

__global__ void __launch_bounds__(256, 6) k_recon_group32(const SolveDesc* __restrict__ D, const int* __restrict__ off,
                                                        int ns, int total) {
  GROUP_LOOP(off, ns, total)
  k_recon32_body(gsh, d.map, d.ds, d.tay, d.tayf, (const float*)d.fini, (float*)d.f, d.M, vb);
  GROUP_END
}

__global__ void __launch_bounds__(256) k_recon_group64(const SolveDesc* __restrict__ D, const int* __restrict__ off,
                                                     int ns, int total) {
  GROUP_LOOP(off, ns, total)
  k_recon64_body(gsh, d.map, d.ds, d.tay, d.tayf, (const double*)d.fini, (double*)d.f, d.M, vb);
  GROUP_END
}

__global__ void __launch_bounds__(256) k_remap_group32(const SolveDesc* __restrict__ D, const int* __restrict__ off,
                                                     int ns, int total) {
  GROUP_LOOP(off, ns, total)
  k_remap32_body(gsh, d.map, d.ds, d.tay, d.tayf, (const float*)d.eta, (float*)d.tmp, d.blo, d.bhi, vb);
  GROUP_END
}

__global__ void __launch_bounds__(256) k_remap_group64(const SolveDesc* __restrict__ D, const int* __restrict__ off,
                                                     int ns, int total) {
  GROUP_LOOP(off, ns, total)
  k_remap64_body(gsh, d.map, d.ds, d.tay, (const double*)d.eta, (double*)d.tmp, vb);
  GROUP_END
}

__global__ void __launch_bounds__(RT_C) k_recon_tiles_group(const SolveDesc* __restrict__ D,
                                                            const int* __restrict__ off, int ns, int total) {
  GROUP_LOOP(off, ns, total)
  recon32_tile_body(gsh, d.map, d.ds, d.tay, d.tayf, (const float*)d.fini, (float*)d.f, d.Mpart, d.ds, vb);
  GROUP_END
}

__global__ void k_row_mass_group(const SolveDesc* __restrict__ D, const int* __restrict__ off, int ns, int total) {
  GROUP_LOOP(off, ns, total)
  row_mass_body(gsh, d.Mpart, d.M, vb);
  GROUP_END
}

// f_ini <- tmp (the resampled f of a remap), 4096 values per unit.
template <typename R>
__global__ void __launch_bounds__(256) k_copy_group(const SolveDesc* __restrict__ D, const int* __restrict__ off,
                                                  int ns, int total) {
  GROUP_LOOP(off, ns, total)
  const size_t n = (size_t)gsh.nx * gsh.nv;
  const size_t p0 = (size_t)vb * 4096;
  const R* src = (const R*)d.tmp;
  R* dst = (R*)d.fini;
  for (size_t p = p0 + threadIdx.x; p < p0 + 4096 && p < n; p += blockDim.x) dst[p] = src[p];
  GROUP_END
}

// tmp -> f_ini of one solve inside a gated remap (the copy a remap decided
// on the device may skip; element by element, any site count).
template <typename R>
__global__ void __launch_bounds__(256) k_copy_gated(Grid g, const R* __restrict__ src, R* __restrict__ dst) {
  if (gate_shut(g)) return;
  const size_t n = (size_t)g.nx * g.nv;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    dst[p] = src[p];
}

template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ src, D* __restrict__ dst, size_t n) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    dst[p] = (D)src[p];
}

inline unsigned grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)(b > 152 * 32 ? 152 * 32 : (b == 0 ? 1 : b));
}

}  // namespace

// The reconstruction's block size: the single-solve rule (it sets the row
// sums' association, so it is not a tuning parameter).
inline int recon_threads(int nv) { return nv >= 256 ? 256 : ((nv + 31) / 32) * 32; }

void group_reconstruct(const GroupPlan& G) {
  // every solve of a group has the same block size (the group is built so)
  const int nt = 256;
  if (G.fp32 && G.recon_tiles) {
    k_recon_tiles_group<<<group_grid(G, GP_RECON, G.tot_tiles), RT_C, sizeof(TileShared), G.stream>>>(
        G.D, G.off_tiles, G.ns, G.tot_tiles);
    k_row_mass_group<<<group_grid(G, GP_DIFF, G.tot_diff), 128, 0, G.stream>>>(G.D, G.off_diff, G.ns, G.tot_diff);
  } else if (G.fp32)
    k_recon_group32<<<group_grid(G, GP_RECON, G.tot_rows), nt, 0, G.stream>>>(G.D, G.off_rows, G.ns, G.tot_rows);
  else
    k_recon_group64<<<group_grid(G, GP_RECON, G.tot_rows), nt, 0, G.stream>>>(G.D, G.off_rows, G.ns, G.tot_rows);
}

void group_remap_resample(const GroupPlan& G) {
  const int nt = 256;
  if (G.fp32)
    k_remap_group32<<<group_grid(G, GP_REMAP, G.tot_rows), nt, 0, G.stream>>>(G.D, G.off_rows, G.ns, G.tot_rows);
  else
    k_remap_group64<<<group_grid(G, GP_REMAP, G.tot_rows), nt, 0, G.stream>>>(G.D, G.off_rows, G.ns, G.tot_rows);
}

void launch_copy_gated(vm_solver* s) {
  const unsigned nb = grid_for(s->n);
  if (s->fp32)
    k_copy_gated<float><<<nb, 256, 0, s->stream>>>(s->g, (const float*)s->tmp, (float*)s->fini);
  else
    k_copy_gated<double><<<nb, 256, 0, s->stream>>>(s->g, (const double*)s->tmp, (double*)s->fini);
  s->launches++;
}

void group_copy_tmp_to_fini(const GroupPlan& G) {
  if (G.fp32)
    k_copy_group<float><<<group_grid(G, GP_COPY, G.tot_copy), 256, 0, G.stream>>>(G.D, G.off_copy, G.ns, G.tot_copy);
  else
    k_copy_group<double><<<group_grid(G, GP_COPY, G.tot_copy), 256, 0, G.stream>>>(G.D, G.off_copy, G.ns, G.tot_copy);
}

int recon_tiles_of(const Grid& g) { return (g.nx + RT_R - 1) / RT_R * ((g.nv + RT_C - 1) / RT_C); }
size_t recon_tile_smem() { return sizeof(TileShared); }

bool recon_prepare() {
  static bool done = false;
  if (done) return true;
  cudaError_t e = cudaFuncSetAttribute(k_recon32_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(TileShared));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_recon_tiles_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(TileShared));
  if (e != cudaSuccess) {
    note_cuda(e);
    return false;
  }
  done = true;
  return true;
}

void launch_reconstruct(vm_solver* s) {
  const int nt = s->g.nv >= 256 ? 256 : ((s->g.nv + 31) / 32) * 32;
  const int ps_ = prof_begin(s, KID_RECON);
  if (s->fp32 && s->g.recon_tiles) {
    k_recon32_tiles<<<recon_tiles_of(s->g), RT_C, sizeof(TileShared), s->stream>>>(
        s->g, s->map, s->ds, s->tay, s->tayf, (const float*)s->fini, (float*)s->f, s->Mpart);
    k_row_mass<<<(s->g.nx + 127) / 128, 128, 0, s->stream>>>(s->g, s->Mpart, s->M);
    s->launches++;
  } else if (s->fp32)
    k_recon32<<<s->g.nx, nt, 0, s->stream>>>(s->g, s->map, s->ds, s->tay, s->tayf, (const float*)s->fini,
                                              (float*)s->f, s->M);
  else
    k_recon64<<<s->g.nx, nt, 0, s->stream>>>(s->g, s->map, s->ds, s->tay, s->tayf, (const double*)s->fini,
                                              (double*)s->f, s->M);
  prof_end(s, ps_);
  s->launches++;
}

void launch_remap_resample(vm_solver* s, void* out) {
  const int nt = s->g.nv >= 256 ? 256 : ((s->g.nv + 31) / 32) * 32;
  const int ps_ = prof_begin(s, KID_REMAP);
  if (s->fp32) {
    const float fb = (float)s->g.beta;
    const float blo = ((double)fb <= s->g.beta) ? fb : nextafterf(fb, -INFINITY);
    const float bhi = ((double)fb >= s->g.beta) ? fb : nextafterf(fb, INFINITY);
    k_remap32<<<s->g.nx, nt, 0, s->stream>>>(s->g, s->map, s->ds, s->tay, s->tayf, (const float*)s->eta,
                                              (float*)out, blo, bhi);
  } else {
    k_remap64<<<s->g.nx, nt, 0, s->stream>>>(s->g, s->map, s->ds, s->tay, (const double*)s->eta,
                                              (double*)out);
  }
  prof_end(s, ps_);
  s->launches++;
}

// Copy a stored-precision array into a double (dst_dtype 0) or float (1) one.
void launch_convert(vm_solver* s, const void* src, void* dst, int32_t dst_dtype, size_t count) {
  const unsigned nb = grid_for(count);
  if (s->fp32) {
    if (dst_dtype == VM_DTYPE_F64)
      k_convert<float, double><<<nb, 256, 0, s->stream>>>((const float*)src, (double*)dst, count);
    else
      k_convert<float, float><<<nb, 256, 0, s->stream>>>((const float*)src, (float*)dst, count);
  } else {
    if (dst_dtype == VM_DTYPE_F64)
      k_convert<double, double><<<nb, 256, 0, s->stream>>>((const double*)src, (double*)dst, count);
    else
      k_convert<double, float><<<nb, 256, 0, s->stream>>>((const double*)src, (float*)dst, count);
  }
  s->launches++;
}

// Store doubles into a stored-precision array.
void launch_store_real(vm_solver* s, const double* src, void* dst, size_t count) {
  const unsigned nb = grid_for(count);
  if (s->fp32)
    k_convert<double, float><<<nb, 256, 0, s->stream>>>(src, (float*)dst, count);
  else
    k_convert<double, double><<<nb, 256, 0, s->stream>>>(src, (double*)dst, count);
  s->launches++;
}

}  // namespace vm
