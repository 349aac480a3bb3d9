// Per-site reconstruction of f (Sec. 2.2, Liouville: f(P) = f_ini(Q(P))).
//
// Transport (Sec. 2.2.1): Q from the element that owns the site, six-point
// quadratic interpolation of f_ini, and the v-reduction of the row fused in
// the same block (pixel mass M(i), Sec. 2.5).  Remap (Secs. 2.2.2, 2.3.2):
// Q_r blended over the beta set of elements with the Monaghan kernel, then
// the cubic B-spline of f_ini at Q_r.
//
// Q, the interpolation node choice and the weights' arguments are FP64 in
// both precisions, evaluated in a fixed operation order; only the storage
// of f_ini / eta / f and the final interpolation sums follow the stored
// precision R.
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

// FP32 storage: nodes and weights as above (FP64), sums in float.
__device__ __forceinline__ double qinterp(const float* __restrict__ F, const Grid& g, double u, double w) {
  if (!(u > -2.0 && u < (double)g.nx + 1.0 && w > -2.0 && w < (double)g.nv + 1.0)) return 0.0;
  const long long in = (long long)floor(dadd(u, 0.5)), jn = (long long)floor(dadd(w, 0.5));
  const long long ic = (long long)floor(u), jc = (long long)floor(w);
  const float x = (float)dsub(u, (double)in), y = (float)dsub(w, (double)jn);
  float f = F_at(F, g, in, jn) * (1.0f - x * x - y * y);
  f += 0.5f * x * (F_at(F, g, in + 1, jn) * (1.0f + x) + F_at(F, g, in - 1, jn) * (x - 1.0f));
  f += 0.5f * y * (F_at(F, g, in, jn + 1) * (1.0f + y) + F_at(F, g, in, jn - 1) * (y - 1.0f));
  f += (F_at(F, g, ic + 1, jc + 1) + F_at(F, g, ic, jc) - F_at(F, g, ic + 1, jc) - F_at(F, g, ic, jc + 1)) * x * y;
  return (double)f;
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
template <typename R>
__global__ void __launch_bounds__(256) k_recon(Grid g, const int32_t* __restrict__ map,
                                               const double* __restrict__ tay, const R* __restrict__ fini,
                                               R* __restrict__ f, double* __restrict__ M) {
  __shared__ double sh[32];
  const int i = blockIdx.x;
  const double Px = site_x(g, i);
  double acc = 0.0;
  for (int j = threadIdx.x; j < g.nv; j += blockDim.x) {
    const size_t p = (size_t)i * g.nv + j;
    const int m = map[p];
    double val = 0.0;
    if (m >= 0) {
      const double* t = tay + (size_t)m * TY_N;
      double dqx, dqv;
      qofp_exact(t, Px, site_v(g, j), dqx, dqv);
      const double u = dmul(dsub(dadd(t[TY_QX], dqx), g.x_lo), g.inv_dx);
      const double w = dmul(dsub(dadd(t[TY_QV], dqv), g.v_lo), g.inv_dv);
      val = qinterp(fini, g, u, w);
    }
    const R out = (R)val;
    f[p] = out;
    acc += (double)out;
  }
  const double rowsum = block_sum(acc, sh);
  if (threadIdx.x == 0) M[i] = dmul(rowsum, g.dxdv);
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
      if (kk < 0 || kk >= g.Lx || ll < 0 || ll >= g.Lv) continue;
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

template <typename R>
__global__ void __launch_bounds__(256) k_remap(Grid g, const int32_t* __restrict__ map,
                                               const double* __restrict__ tay, const R* __restrict__ eta,
                                               R* __restrict__ out) {
  const int i = blockIdx.x;
  const double Px = site_x(g, i);
  for (int j = threadIdx.x; j < g.nv; j += blockDim.x) {
    const size_t p = (size_t)i * g.nv + j;
    const int m = map[p];
    double val = 0.0;
    if (m >= 0) {
      double Qx, Qv;
      blended_q(g, tay, m, Px, site_v(g, j), Qx, Qv);
      const double u = dmul(dsub(Qx, g.x_lo), g.inv_dx);
      const double w = dmul(dsub(Qv, g.v_lo), g.inv_dv);
      val = spline_eval(eta, g, u, w);
    }
    out[p] = (R)val;
  }
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

void launch_reconstruct(vm_solver* s) {
  const int nt = s->g.nv >= 256 ? 256 : ((s->g.nv + 31) / 32) * 32;
  const int ps_ = prof_begin(s, KID_RECON);
  if (s->fp32)
    k_recon<float><<<s->g.nx, nt, 0, s->stream>>>(s->g, s->map, s->tay, (const float*)s->fini,
                                                   (float*)s->f, s->M);
  else
    k_recon<double><<<s->g.nx, nt, 0, s->stream>>>(s->g, s->map, s->tay, (const double*)s->fini,
                                                    (double*)s->f, s->M);
  prof_end(s, ps_);
  s->launches++;
}

void launch_remap_resample(vm_solver* s, void* out) {
  const int nt = s->g.nv >= 256 ? 256 : ((s->g.nv + 31) / 32) * 32;
  const int ps_ = prof_begin(s, KID_REMAP);
  if (s->fp32)
    k_remap<float><<<s->g.nx, nt, 0, s->stream>>>(s->g, s->map, s->tay, (const float*)s->eta, (float*)out);
  else
    k_remap<double><<<s->g.nx, nt, 0, s->stream>>>(s->g, s->map, s->tay, (const double*)s->eta, (double*)out);
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
