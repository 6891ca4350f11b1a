// rt_grid.cu -- Krylov building blocks spread over the whole GPU, for single
// problems too large for one CTA (3D boxes).  The solve loop runs on the host
// (float64 Givens rotations and least squares there); each Arnoldi step is a
// few grid-wide kernels: operator, projections (per-CTA partial sums reduced
// by one CTA), fused update + normalisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rt_host.h"
#include "rt_internal.cuh"

namespace rt {

constexpr int kGT = 256;     // threads per CTA
constexpr int kGDots = 8;    // basis vectors per pass of the projection kernel
constexpr int kGMaxGroups = (kMaxKrylov + 2 + kGDots - 1) / kGDots;  // groups of one projection
static_assert((kGDots + 1) * kGMaxGroups <= kGridPartPerCta, "grid partial buffer too small");

int grid_ctas(const rt_handle *h) { return 2 * (h->n_sm > 0 ? h->n_sm : 152); }

// The vector kernels below stream whole basis vectors (up to 10 GB each for
// a 64^3 box): every thread takes kGE elements at a grid stride and issues
// the loads of all of them (and of a group of basis rows) before the
// arithmetic, so enough bytes are in flight to keep HBM busy; indices past n
// are clamped (re-reads of the last element, contributions dropped).
// Products are summed in TL over a thread's elements of kGWiden iterations
// before one float64 add (float64 adds run at 1/73 of the float32 rate).
constexpr int kGE = 4;      // elements per thread per iteration
constexpr int kGWiden = 4;  // iterations summed in TL before a float64 add
constexpr int kGRows = 4;   // basis rows per group in the update kernels

// partial[blockIdx][u] = sum over this CTA's elements of V_{i0+u} . w  (u < cnt),
// partial[blockIdx][kGDots] = w . w (when with_norm)
template <typename TL>
__global__ void __launch_bounds__(kGT) k_gdots(const TL *V, int64_t ldv, int i0, int cnt, const TL *w,
                                               int64_t n, int with_norm, double *partial) {
  __shared__ double red[(kGT / 32) * (kGDots + 1)];
  __shared__ double outb[kGDots + 1];
  double acc[kGDots + 1];
  TL part[kGDots + 1];
#pragma unroll
  for (int u = 0; u <= kGDots; ++u) {
    acc[u] = 0.0;
    part[u] = 0;
  }
  const TL *vp[kGDots];
#pragma unroll
  for (int u = 0; u < kGDots; ++u) vp[u] = V + (int64_t)(i0 + min(u, cnt - 1)) * ldv;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int it = 0;
  for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k0 < n; k0 += kGE * stride) {
    TL wv[kGE], vv[kGDots][kGE];
#pragma unroll
    for (int e = 0; e < kGE; ++e) {
      const int64_t k = min(k0 + e * stride, n - 1);
      wv[e] = w[k];
#pragma unroll
      for (int u = 0; u < kGDots; ++u) vv[u][e] = vp[u][k];
    }
#pragma unroll
    for (int e = 0; e < kGE; ++e)
      if (k0 + e * stride >= n) wv[e] = 0;
#pragma unroll
    for (int u = 0; u < kGDots; ++u)
#pragma unroll
      for (int e = 0; e < kGE; ++e) part[u] = fma(vv[u][e], wv[e], part[u]);
    if (with_norm) {
#pragma unroll
      for (int e = 0; e < kGE; ++e) part[kGDots] = fma(wv[e], wv[e], part[kGDots]);
    }
    if (++it == kGWiden) {
      it = 0;
#pragma unroll
      for (int u = 0; u <= kGDots; ++u) {
        acc[u] += (double)part[u];
        part[u] = 0;
      }
    }
  }
#pragma unroll
  for (int u = 0; u <= kGDots; ++u) acc[u] += (double)part[u];
  block_sum<kGDots + 1>(acc, red, outb);
  if (threadIdx.x <= kGDots) partial[(int64_t)blockIdx.x * (kGDots + 1) + threadIdx.x] = acc[threadIdx.x];
}

// out[g][u] = sum over CTAs of partial[g][cta][u], u <= kGDots: the sums of
// several k_gdots launches (one block per group of basis rows)
__global__ void k_greduce_groups(const double *partial, int nblk, double *out) {
  const int g = blockIdx.x, u = threadIdx.x;
  if (u > kGDots) return;
  const double *p = partial + (int64_t)g * nblk * (kGDots + 1) + u;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += p[(int64_t)b * (kGDots + 1)];
  out[g * (kGDots + 1) + u] = s;
}

__global__ void k_greduce(const double *partial, int nblk, int nv, double *out) {
  for (int u = threadIdx.x; u < nv; u += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * nv + u];
    out[u] = s;
  }
}

// acc[e] += sum_{i < cnt} cf[i] V_i[k0 + e stride] (rows in groups of
// kGRows, all loads of a group issued before its FMAs)
template <typename TL>
__device__ __forceinline__ void g_axpy(const TL *V, int64_t ldv, int cnt, const TL *cf, int64_t k0, int64_t stride,
                                       int64_t n, TL (&acc)[kGE]) {
  for (int r0 = 0; r0 < cnt; r0 += kGRows) {
    TL v[kGRows][kGE], c[kGRows];
#pragma unroll
    for (int u = 0; u < kGRows; ++u) {
      const int i = min(r0 + u, cnt - 1);
      c[u] = r0 + u < cnt ? cf[r0 + u] : TL(0);
      const TL *vi = V + (int64_t)i * ldv;
#pragma unroll
      for (int e = 0; e < kGE; ++e) v[u][e] = vi[min(k0 + e * stride, n - 1)];
    }
#pragma unroll
    for (int u = 0; u < kGRows; ++u)
#pragma unroll
      for (int e = 0; e < kGE; ++e) acc[e] = fma(c[u], v[u][e], acc[e]);
  }
}

// w = (w - sum_{i<cnt} coef[i] V_i) * scale; optional squared norm partials
template <typename TL>
__global__ void __launch_bounds__(kGT) k_gupdate(const TL *V, int64_t ldv, int cnt, const double *coef,
                                                 TL *w, int64_t n, double scale, double *partial) {
  __shared__ TL cf[1024];
  __shared__ double red[kGT / 32];
  __shared__ double outb[1];
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) cf[i] = (TL)(-coef[i]);
  __syncthreads();
  const TL sc = (TL)scale;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double a[1] = {0.0};
  TL part = 0;
  int it = 0;
  for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k0 < n; k0 += kGE * stride) {
    TL wv[kGE];
#pragma unroll
    for (int e = 0; e < kGE; ++e) wv[e] = w[min(k0 + e * stride, n - 1)];
    if (cnt > 0) g_axpy<TL>(V, ldv, cnt, cf, k0, stride, n, wv);
#pragma unroll
    for (int e = 0; e < kGE; ++e) {
      const int64_t k = k0 + e * stride;
      const TL v = wv[e] * sc;
      if (k < n) {
        w[k] = v;
        part = fma(v, v, part);
      }
    }
    if (++it == kGWiden) {
      it = 0;
      a[0] += (double)part;
      part = 0;
    }
  }
  a[0] += (double)part;
  if (partial) {
    block_sum<1>(a, red, outb);
    if (threadIdx.x == 0) partial[blockIdx.x] = a[0];
  }
}

// x += sum_{i<cnt} y[i] V_i  (correction summed in TL, added in float64)
template <typename TL>
__global__ void __launch_bounds__(kGT) k_gxupdate(const TL *V, int64_t ldv, int cnt, const double *y,
                                                  double *x, int64_t n) {
  __shared__ TL cf[1024];
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) cf[i] = (TL)y[i];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k0 < n; k0 += kGE * stride) {
    TL d[kGE];
#pragma unroll
    for (int e = 0; e < kGE; ++e) d[e] = 0;
    g_axpy<TL>(V, ldv, cnt, cf, k0, stride, n, d);
#pragma unroll
    for (int e = 0; e < kGE; ++e) {
      const int64_t k = k0 + e * stride;
      if (k < n) x[k] += cvt<double>(d[e]);
    }
  }
}

// r = b - y (in place in y) and squared-norm partials
__global__ void __launch_bounds__(kGT) k_gresid(const double *b, double *y, int64_t n, double *partial) {
  __shared__ double red[kGT / 32];
  __shared__ double outb[1];
  double a[1] = {0.0};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double r = b[k] - y[k];
    y[k] = r;
    a[0] += r * r;
  }
  block_sum<1>(a, red, outb);
  if (threadIdx.x == 0) partial[blockIdx.x] = a[0];
}

template <typename TL>
__global__ void k_gscale(const double *src, TL *dst, int64_t n, double s) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = cvt<TL>(src[k] * s);
}

__global__ void k_gnorm(const double *v, int64_t n, double *partial) {
  __shared__ double red[kGT / 32];
  __shared__ double outb[1];
  double a[1] = {0.0};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    a[0] += v[k] * v[k];
  block_sum<1>(a, red, outb);
  if (threadIdx.x == 0) partial[blockIdx.x] = a[0];
}

// ------------------------------------------------------------ host loop
struct GridCtx {
  rt_handle *h;
  cudaStream_t s;
  int G;
  double *part, *red, *coef;
  std::vector<double> host;
};

static int reduce_to_host(GridCtx &g, int nv, double *dst) {
  k_greduce<<<1, 64, 0, g.s>>>(g.part, g.G, nv, g.red);
  cudaError_t e = cudaMemcpyAsync(dst, g.red, nv * sizeof(double), cudaMemcpyDeviceToHost, g.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g.s);
  return (int)e;
}

// h = V[0..j]^T w and ww = w.w: the groups of kGDots rows run back to back
// into their own partial sums, one reduction and one copy to the host
template <typename TL>
static int dots(GridCtx &g, const TL *V, int64_t ldv, int j, const TL *w, int64_t n, std::vector<double> &h,
                double *ww) {
  h.assign(j + 1, 0.0);
  const int ng = (j + kGDots) / kGDots;
  if (ng > kGMaxGroups) return (int)cudaErrorInvalidValue;
  for (int gi = 0; gi < ng; ++gi) {
    const int i0 = gi * kGDots, cnt = std::min(kGDots, j + 1 - i0);
    k_gdots<TL><<<g.G, kGT, 0, g.s>>>(V, ldv, i0, cnt, w, n, gi == 0 ? 1 : 0,
                                      g.part + (int64_t)gi * g.G * (kGDots + 1));
  }
  k_greduce_groups<<<ng, 32, 0, g.s>>>(g.part, g.G, g.red);
  g.host.resize((size_t)ng * (kGDots + 1));
  cudaError_t e = cudaMemcpyAsync(g.host.data(), g.red, g.host.size() * sizeof(double), cudaMemcpyDeviceToHost, g.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g.s);
  if (e != cudaSuccess) return (int)e;
  for (int i = 0; i <= j; ++i) h[i] = g.host[(size_t)(i / kGDots) * (kGDots + 1) + i % kGDots];
  if (ww) *ww = g.host[kGDots];
  return 0;
}

template <typename TL>
static int update(GridCtx &g, const TL *V, int64_t ldv, const std::vector<double> &c, TL *w, int64_t n,
                  double scale, double *nrm2) {
  if (!c.empty()) {
    cudaError_t e = cudaMemcpyAsync(g.coef, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, g.s);
    if (e) return (int)e;
  }
  k_gupdate<TL><<<g.G, kGT, 0, g.s>>>(V, ldv, (int)c.size(), g.coef, w, n, scale, nrm2 ? g.part : nullptr);
  if (nrm2) {
    double v;
    int r = reduce_to_host(g, 1, &v);
    *nrm2 = v;
    return r;
  }
  return (int)cudaGetLastError();
}

// Restarted GMRES(m) with float64 refinement for one big problem (n_rhs == 1).
// apply64(x, y) writes y = A x in float64; applyL(v, w) writes w = A v in TL.
// mixed: applyL is the low-precision operator, each inner cycle stops at a
// reduction of tol_inner (else at the final tolerance).
template <typename TL, typename F64, typename FL>
static int grid_solve(rt_handle *h, const double *b, double *x, double tol, double tol_inner, int m,
                      int max_outer, int use_x0, cudaStream_t s, F64 apply64, FL applyL, bool mixed,
                      int &outer_out, int &inner_out, double &relres_out, int &status, double &bytes) {
  const int64_t n = h->E;
  const int64_t ldv = (n + 31) / 32 * 32;
  GridCtx g{h, s, grid_ctas(h), h->g_part, h->g_red, h->g_coef, {}};
  TL *V = static_cast<TL *>(h->ws.V);
  double *r = h->g_r;  // float64 residual
  const double sz = sizeof(TL);
  bytes = 0.0;
  k_gnorm<<<g.G, kGT, 0, s>>>(b, n, g.part);
  double bn2;
  int e = reduce_to_host(g, 1, &bn2);
  if (e) return e;
  const double bn = std::sqrt(bn2);
  bytes += 8.0 * n;
  status = 4;
  relres_out = 1.0;
  outer_out = 0;
  inner_out = 0;
  if (!std::isfinite(bn)) { status = 6; return 0; }
  if (!use_x0) cudaMemsetAsync(x, 0, n * sizeof(double), s);
  if (bn == 0.0) { status = 0; relres_out = 0.0; return 0; }
  std::vector<double> H((size_t)(m + 1) * m), cs(m + 1), sn(m + 1), gv(m + 2), hv, h2;
  for (int outer = 0;; ++outer) {
    outer_out = outer;
    double rn;
    const double *rsrc;
    if (outer == 0 && !use_x0) {
      rsrc = b;
      rn = bn;
    } else {
      if ((e = apply64(x, r))) return e;
      k_gresid<<<g.G, kGT, 0, s>>>(b, r, n, g.part);
      double rn2;
      if ((e = reduce_to_host(g, 1, &rn2))) return e;
      rn = std::sqrt(rn2);
      rsrc = r;
      bytes += (40.0 + 24.0) * n;
    }
    relres_out = rn / bn;
    if (!std::isfinite(rn)) { status = 6; return 0; }
    if (relres_out <= tol) { status = 0; return 0; }
    if (outer >= max_outer) { status = 4; return 0; }
    k_gscale<TL><<<g.G, kGT, 0, s>>>(rsrc, V, n, 1.0 / rn);
    bytes += (8.0 + sz) * n;
    gv.assign(m + 2, 0.0);
    gv[0] = rn;
    const double target = mixed ? std::max(tol_inner * rn, 0.5 * tol * bn) : 0.5 * tol * bn;
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      TL *vj = V + (int64_t)j * ldv;
      TL *w = V + (int64_t)(j + 1) * ldv;
      if ((e = applyL(vj, w))) return e;
      double ww = 0.0;
      if ((e = dots<TL>(g, V, ldv, j, w, n, hv, &ww))) return e;
      bytes += (5.0 * sz + sz * (j + 2)) * n;
      double hh = 0.0;
      for (double v : hv) hh += v * v;
      double hn;
      h2.assign(j + 1, 0.0);
      // second projection (DGKS) when ||w - V h||^2 <= eta2 ||w||^2: 1/2 for
      // float64 GMRES; 1e-4 for the float32 cycles of the mixed solve, whose
      // residual is recomputed in float64 at every restart (w = A v keeps most
      // of v on these operators, so the 1/2 test fires at nearly every step and
      // doubles the Arnoldi traffic)
      const double eta2 = mixed ? 1e-4 : 0.5;
      if (ww - hh > eta2 * ww) {
        hn = std::sqrt(ww - hh);
        if ((e = update<TL>(g, V, ldv, hv, w, n, hn > 0 ? 1.0 / hn : 0.0, nullptr))) return e;
        bytes += sz * (j + 3) * n;
      } else {
        if ((e = update<TL>(g, V, ldv, hv, w, n, 1.0, nullptr))) return e;
        if ((e = dots<TL>(g, V, ldv, j, w, n, h2, nullptr))) return e;
        double n2;
        if ((e = update<TL>(g, V, ldv, h2, w, n, 1.0, &n2))) return e;
        hn = std::sqrt(n2);
        std::vector<double> zero;
        if ((e = update<TL>(g, V, ldv, zero, w, n, hn > 0 ? 1.0 / hn : 0.0, nullptr))) return e;
        bytes += sz * (4.0 * j + 12.0) * n;
      }
      double *col = H.data() + (size_t)j * (m + 1);
      for (int i = 0; i <= j; ++i) col[i] = hv[i] + h2[i];
      col[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t0;
      }
      const double den = std::hypot(col[j], col[j + 1]);
      double cj = 1.0, sj = 0.0;
      if (den > 0.0) { cj = col[j] / den; sj = col[j + 1] / den; }
      cs[j] = cj;
      sn[j] = sj;
      col[j] = den;
      col[j + 1] = 0.0;
      gv[j + 1] = -sj * gv[j];
      gv[j] = cj * gv[j];
      jdone = j + 1;
      if (den == 0.0) { jdone = j; break; }
      if (!(hn > 1e-300 * rn)) break;
      if (std::fabs(gv[j + 1]) <= target) break;
    }
    inner_out += jdone;
    std::vector<double> yv(jdone);
    for (int i = jdone - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int k = i + 1; k < jdone; ++k) acc -= H[(size_t)k * (m + 1) + i] * yv[k];
      yv[i] = acc / H[(size_t)i * (m + 1) + i];
    }
    if (jdone > 0) {
      cudaMemcpyAsync(g.coef, yv.data(), jdone * sizeof(double), cudaMemcpyHostToDevice, s);
      k_gxupdate<TL><<<g.G, kGT, 0, s>>>(V, ldv, jdone, g.coef, x, n);
      bytes += (sz * jdone + 16.0) * n;
    }
    if ((e = (int)cudaGetLastError())) return e;
    if (jdone == 0) { status = 5; return 0; }
  }
}

// ------------------------------------------------------- BiCGStab (grid-wide)
// The float64 BiCGStab of k_solve_bicgstab for one big problem: the same
// recurrences, each fused vector pass one grid-wide kernel, the scalars on
// the host.  Partial sums per CTA, reduced by k_greduce.
__global__ void __launch_bounds__(kGT) k_gb_dir(double *p, const double *r, const double *v, double beta,
                                                double omega, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    p[k] = r[k] + beta * (p[k] - omega * v[k]);
}

// partial[blk][0] = (a, b), partial[blk][1] = (c, d) (0 when c is null)
__global__ void __launch_bounds__(kGT) k_gb_dots(const double *a, const double *b, const double *c,
                                                 const double *d, int64_t n, double *partial) {
  __shared__ double red[(kGT / 32) * 2];
  __shared__ double outb[2];
  double acc[2] = {0.0, 0.0};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    acc[0] = fma(a[k], b[k], acc[0]);
    if (c) acc[1] = fma(c[k], d[k], acc[1]);
  }
  block_sum<2>(acc, red, outb);
  if (threadIdx.x < 2) partial[(int64_t)blockIdx.x * 2 + threadIdx.x] = acc[threadIdx.x];
}

// s = r - alpha v, partial ||s||^2
__global__ void __launch_bounds__(kGT) k_gb_s(double *s, const double *r, const double *v, double alpha,
                                              int64_t n, double *partial) {
  __shared__ double red[kGT / 32];
  __shared__ double outb[1];
  double acc[1] = {0.0};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double sv = r[k] - alpha * v[k];
    s[k] = sv;
    acc[0] = fma(sv, sv, acc[0]);
  }
  block_sum<1>(acc, red, outb);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc[0];
}

// x += alpha p + omega s; r = s - omega t; partial ||r||^2, (r^, r)
__global__ void __launch_bounds__(kGT) k_gb_xr(double *x, const double *p, const double *s, const double *t,
                                               double *r, const double *rh, double alpha, double omega, int64_t n,
                                               double *partial) {
  __shared__ double red[(kGT / 32) * 2];
  __shared__ double outb[2];
  double acc[2] = {0.0, 0.0};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double sv = s[k];
    x[k] += alpha * p[k] + omega * sv;
    const double rv = sv - omega * t[k];
    r[k] = rv;
    acc[0] = fma(rv, rv, acc[0]);
    acc[1] = fma(rh[k], rv, acc[1]);
  }
  block_sum<2>(acc, red, outb);
  if (threadIdx.x < 2) partial[(int64_t)blockIdx.x * 2 + threadIdx.x] = acc[threadIdx.x];
}

__global__ void k_gb_axpy(double *x, const double *p, double alpha, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    x[k] += alpha * p[k];
}

int launch_grid_bicgstab(rt_handle *h, const double *b, double *x, double tol, int max_outer, int max_iter,
                         int use_x0, cudaStream_t s, int &restarts, int &iters, double &relres, int &status,
                         double &bytes) {
  const int64_t n = h->E;
  const int64_t ldv = (n + 31) / 32 * 32;
  GridCtx g{h, s, grid_ctas(h), h->g_part, h->g_red, h->g_coef, {}};
  double *r = static_cast<double *>(h->ws.V);
  double *rh = r + ldv, *pv = rh + ldv, *v = pv + ldv, *sv = v + ldv, *t = sv + ldv;
  auto apply = [&](const double *X, double *Y) -> int {
    return h->dims == 3 ? apply_box(h, 0, true, X, false, Y, false, s) : launch_apply(h, 0, true, X, Y, s, false);
  };
  auto true_resid = [&](double &rn) -> int {  // r = b - A x
    int e = apply(x, r);
    if (e) return e;
    k_gresid<<<g.G, kGT, 0, s>>>(b, r, n, g.part);
    double rn2 = 0.0;
    e = reduce_to_host(g, 1, &rn2);
    rn = std::sqrt(rn2);
    bytes += 64.0 * n;
    return e;
  };
  bytes = 0.0;
  restarts = iters = 0;
  status = 4;
  k_gnorm<<<g.G, kGT, 0, s>>>(b, n, g.part);
  double bn2 = 0.0;
  int e = reduce_to_host(g, 1, &bn2);
  if (e) return e;
  const double bn = std::sqrt(bn2);
  bytes += 8.0 * n;
  relres = 1.0;
  if (!std::isfinite(bn)) { status = 6; return 0; }
  if (!use_x0) cudaMemsetAsync(x, 0, n * sizeof(double), s);
  if (bn == 0.0) { status = 0; relres = 0.0; return 0; }
  double rn = bn;
  if (use_x0) {
    if ((e = true_resid(rn))) return e;
  } else {
    cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    bytes += 16.0 * n;
  }
  double rho = 0.0, rho_old = 1.0, alpha = 1.0, omega = 1.0;
  auto reset = [&]() {
    cudaMemcpyAsync(rh, r, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(pv, 0, n * sizeof(double), s);
    cudaMemsetAsync(v, 0, n * sizeof(double), s);
    rho = rn * rn;
    rho_old = alpha = omega = 1.0;
    bytes += 32.0 * n;
  };
  reset();
  const int cap = max_iter > 0 ? max_iter : 10000;
  bool rn_true = use_x0;
  for (;;) {
    if (!std::isfinite(rn)) { status = 6; break; }
    int restart = 0;
    if (rn <= tol * bn) {
      if ((e = true_resid(rn))) return e;
      rn_true = true;
      if (rn <= tol * bn) { status = 0; break; }
      restart = 1;
    } else if (iters >= cap) {
      break;
    } else if (!(rho != 0.0 && std::isfinite(rho)) || omega == 0.0) {
      if ((e = true_resid(rn))) return e;
      rn_true = true;
      restart = 2;
    }
    if (restart) {
      if (restarts >= max_outer) { status = restart == 2 ? 5 : 4; break; }
      ++restarts;
      reset();
      continue;
    }
    const double beta = (rho / rho_old) * (alpha / omega);
    k_gb_dir<<<g.G, kGT, 0, s>>>(pv, r, v, beta, omega, n);
    if ((e = apply(pv, v))) return e;
    double d2[2];
    k_gb_dots<<<g.G, kGT, 0, s>>>(rh, v, nullptr, nullptr, n, g.part);
    if ((e = reduce_to_host(g, 2, d2))) return e;
    bytes += (32.0 + 40.0 + 16.0) * n;
    ++iters;
    const double rv = d2[0];
    if (!(rv != 0.0 && std::isfinite(rv))) {
      if ((e = true_resid(rn))) return e;
      rn_true = true;
      if (rn <= tol * bn) { status = 0; break; }
      if (restarts >= max_outer) { status = 5; break; }
      ++restarts;
      reset();
      continue;
    }
    alpha = rho / rv;
    k_gb_s<<<g.G, kGT, 0, s>>>(sv, r, v, alpha, n, g.part);
    double sn2 = 0.0;
    if ((e = reduce_to_host(g, 1, &sn2))) return e;
    bytes += 24.0 * n;
    if (std::sqrt(sn2) <= tol * bn) {
      k_gb_axpy<<<g.G, kGT, 0, s>>>(x, pv, alpha, n);
      bytes += 24.0 * n;
      rn = std::sqrt(sn2);
      rn_true = false;
      continue;
    }
    if ((e = apply(sv, t))) return e;
    k_gb_dots<<<g.G, kGT, 0, s>>>(t, sv, t, t, n, g.part);
    if ((e = reduce_to_host(g, 2, d2))) return e;
    omega = d2[1] > 0.0 ? d2[0] / d2[1] : 0.0;
    k_gb_xr<<<g.G, kGT, 0, s>>>(x, pv, sv, t, r, rh, alpha, omega, n, g.part);
    if ((e = reduce_to_host(g, 2, d2))) return e;
    bytes += (40.0 + 16.0 + 56.0) * n;
    rn = std::sqrt(d2[0]);
    rn_true = false;
    rho_old = rho;
    rho = d2[1];
  }
  if (status != 0 && status != 6 && !rn_true)
    if ((e = true_resid(rn))) return e;
  relres = rn / bn;
  return (int)cudaGetLastError();
}

bool grid_bicgstab_fits(const rt_handle *h) {
  const int64_t ldv = (h->E + 31) / 32 * 32;
  return h->ws.cap_bytes >= 6 * ldv * 8;
}

// Nested solve for one 1D instance on the grid kernels (mixed handles):
// float64 flexible GMRES(kout) whose directions come from one GMRES(m_in)
// cycle on the float32 operator (stopped at a reduction of tol_inner), as the
// batched k_solve_nested does per CTA.  The operator reads and writes float64
// vectors, so all bases are float64 here: Vo [kout+1] | Z [kout] | U [m_in+1]
// in the handle's workspace (kout shrinks to what it holds).
static int grid_fgmres(rt_handle *h, const double *b, double *x, double tol, double tol_inner, int kout,
                       int m_in, int max_outer, int use_x0, cudaStream_t s, int &outer_out, int &inner_out,
                       double &relres_out, int &status, double &bytes) {
  const int64_t n = h->E;
  const int64_t ldv = (n + 31) / 32 * 32;
  const int64_t per = h->ws.cap_bytes / (8 * ldv);  // float64 vectors the workspace holds
  kout = (int)std::min<int64_t>(kout, (per - m_in - 2) / 2);
  if (kout < 1) return (int)cudaErrorInvalidValue;
  GridCtx g{h, s, grid_ctas(h), h->g_part, h->g_red, h->g_coef, {}};
  auto apply64 = [&](const double *xx, double *yy) -> int { return launch_apply(h, 0, true, xx, yy, s, false); };
  auto apply32 = [&](const double *xx, double *yy) -> int { return launch_apply(h, 0, false, xx, yy, s, false); };
  double *Vo = static_cast<double *>(h->ws.V);
  double *Z = Vo + (int64_t)(kout + 1) * ldv;
  double *U = Z + (int64_t)kout * ldv;
  double *r = h->g_r;
  bytes = 0.0;
  k_gnorm<<<g.G, kGT, 0, s>>>(b, n, g.part);
  double bn2;
  int e = reduce_to_host(g, 1, &bn2);
  if (e) return e;
  const double bn = std::sqrt(bn2);
  bytes += 8.0 * n;
  status = 4;
  relres_out = 1.0;
  outer_out = inner_out = 0;
  if (!std::isfinite(bn)) { status = 6; return 0; }
  if (!use_x0) cudaMemsetAsync(x, 0, n * sizeof(double), s);
  if (bn == 0.0) { status = 0; relres_out = 0.0; return 0; }
  // Givens least squares of one Hessenberg column (column-major, leading dim ld)
  auto givens = [](std::vector<double> &H, int ld, std::vector<double> &cs, std::vector<double> &sn,
                   std::vector<double> &gv, int j, const std::vector<double> &hv, const std::vector<double> &h2,
                   double hn) {
    double *col = H.data() + (size_t)j * ld;
    for (int i = 0; i <= j; ++i) col[i] = hv[i] + (h2.empty() ? 0.0 : h2[i]);
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
      col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
      col[i] = t0;
    }
    const double den = std::hypot(col[j], col[j + 1]);
    double cj = 1.0, sj = 0.0;
    if (den > 0.0) { cj = col[j] / den; sj = col[j + 1] / den; }
    cs[j] = cj;
    sn[j] = sj;
    col[j] = den;
    col[j + 1] = 0.0;
    gv[j + 1] = -sj * gv[j];
    gv[j] = cj * gv[j];
    return den;
  };
  auto trisolve = [](const std::vector<double> &H, int ld, const std::vector<double> &gv, int k) {
    std::vector<double> y(k);
    for (int i = k - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int q = i + 1; q < k; ++q) acc -= H[(size_t)q * ld + i] * y[q];
      y[i] = acc / H[(size_t)i * ld + i];
    }
    return y;
  };
  // one Gram-Schmidt step of w = V[j+1] against V[0..j]; second projection when
  // ||w - V h||^2 <= eta2 ||w||^2; returns ||w - V h|| and normalises w
  auto orth = [&](double *V, int j, std::vector<double> &hv, std::vector<double> &h2, double eta2,
                  double &hn) -> int {
    double *w = V + (int64_t)(j + 1) * ldv;
    double ww = 0.0;
    int e2 = dots<double>(g, V, ldv, j, w, n, hv, &ww);
    if (e2) return e2;
    double hh = 0.0;
    for (double v : hv) hh += v * v;
    h2.assign(j + 1, 0.0);
    bytes += 8.0 * (j + 2) * n;
    if (ww - hh > eta2 * ww) {
      hn = std::sqrt(ww - hh);
      bytes += 8.0 * (j + 3) * n;
      return update<double>(g, V, ldv, hv, w, n, hn > 0 ? 1.0 / hn : 0.0, nullptr);
    }
    if ((e2 = update<double>(g, V, ldv, hv, w, n, 1.0, nullptr))) return e2;
    if ((e2 = dots<double>(g, V, ldv, j, w, n, h2, nullptr))) return e2;
    double n2 = 0.0;
    if ((e2 = update<double>(g, V, ldv, h2, w, n, 1.0, &n2))) return e2;
    hn = std::sqrt(n2);
    std::vector<double> none;
    bytes += 8.0 * (3.0 * j + 10.0) * n;
    return update<double>(g, V, ldv, none, w, n, hn > 0 ? 1.0 / hn : 0.0, nullptr);
  };
  std::vector<double> Ho((size_t)(kout + 1) * kout), cso(kout + 1), sno(kout + 1), go(kout + 2);
  std::vector<double> Hi((size_t)(m_in + 1) * m_in), csi(m_in + 1), sni(m_in + 1), gi(m_in + 2), hv, h2;
  for (int cycle = 0;; ++cycle) {
    double rn;
    const double *rsrc;
    if (cycle == 0 && !use_x0) {
      rsrc = b;
      rn = bn;
    } else {
      if ((e = apply64(x, r))) return e;
      k_gresid<<<g.G, kGT, 0, s>>>(b, r, n, g.part);
      double rn2;
      if ((e = reduce_to_host(g, 1, &rn2))) return e;
      rn = std::sqrt(rn2);
      rsrc = r;
      bytes += 64.0 * n;
    }
    relres_out = rn / bn;
    if (!std::isfinite(rn)) { status = 6; return 0; }
    if (relres_out <= tol) { status = 0; return 0; }
    if (cycle >= max_outer) { status = 4; return 0; }
    k_gscale<double><<<g.G, kGT, 0, s>>>(rsrc, Vo, n, 1.0 / rn);
    bytes += 16.0 * n;
    go.assign(kout + 2, 0.0);
    go[0] = rn;
    int idone = 0;
    for (int i = 0; i < kout; ++i) {
      // inner: GMRES(m_in) on the float32 operator from Vo[i] (unit norm)
      double *vi = Vo + (int64_t)i * ldv;
      cudaMemcpyAsync(U, vi, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
      gi.assign(m_in + 2, 0.0);
      gi[0] = 1.0;
      int jdone = 0;
      for (int j = 0; j < m_in; ++j) {
        if ((e = apply32(U + (int64_t)j * ldv, U + (int64_t)(j + 1) * ldv))) return e;
        double hn = 0.0;
        if ((e = orth(U, j, hv, h2, 1e-4, hn))) return e;
        bytes += 40.0 * n;
        const double den = givens(Hi, m_in + 1, csi, sni, gi, j, hv, h2, hn);
        jdone = j + 1;
        if (den == 0.0) { jdone = j; break; }
        if (!(hn > 1e-30)) break;
        if (std::fabs(gi[j + 1]) <= tol_inner) break;
      }
      inner_out += jdone;
      double *zi = Z + (int64_t)i * ldv;
      cudaMemsetAsync(zi, 0, n * sizeof(double), s);
      if (jdone > 0) {
        const std::vector<double> y = trisolve(Hi, m_in + 1, gi, jdone);
        cudaMemcpyAsync(g.coef, y.data(), jdone * sizeof(double), cudaMemcpyHostToDevice, s);
        k_gxupdate<double><<<g.G, kGT, 0, s>>>(U, ldv, jdone, g.coef, zi, n);
        bytes += (8.0 * jdone + 16.0) * n;
      }
      // outer: w = A z_i in float64, orthogonalised against Vo (DGKS)
      if ((e = apply64(zi, Vo + (int64_t)(i + 1) * ldv))) return e;
      double hn = 0.0;
      if ((e = orth(Vo, i, hv, h2, 0.5, hn))) return e;
      bytes += 40.0 * n;
      const double den = givens(Ho, kout + 1, cso, sno, go, i, hv, h2, hn);
      idone = i + 1;
      ++outer_out;
      if (den == 0.0) { idone = i; break; }
      if (!(hn > 1e-300 * rn)) break;
      if (std::fabs(go[i + 1]) <= 0.3 * tol * bn) break;
    }
    if (idone > 0) {
      const std::vector<double> y = trisolve(Ho, kout + 1, go, idone);
      cudaMemcpyAsync(g.coef, y.data(), idone * sizeof(double), cudaMemcpyHostToDevice, s);
      k_gxupdate<double><<<g.G, kGT, 0, s>>>(Z, ldv, idone, g.coef, x, n);
      bytes += (8.0 * idone + 16.0) * n;
    }
    if ((e = (int)cudaGetLastError())) return e;
    if (idone == 0) { status = 5; return 0; }
  }
}

// ------------------------------------------------------ Arnoldi (spectra)
// m steps of the Arnoldi process on the float64 operator of one instance
// (a box or a single 1D column), classical Gram-Schmidt with the DGKS second
// projection; H (host, column-major (m+1) x m) receives the Hessenberg
// matrix, m_done the steps taken (fewer on an invariant subspace).
int launch_grid_arnoldi(rt_handle *h, const double *v0, int m, double *H, int &m_done, cudaStream_t s) {
  const int64_t n = h->E;
  const int64_t ldv = (n + 31) / 32 * 32;
  GridCtx g{h, s, grid_ctas(h), h->g_part, h->g_red, h->g_coef, {}};
  double *V = static_cast<double *>(h->ws.V);
  auto apply = [&](const double *X, double *Y) -> int {
    return h->dims == 3 ? apply_box(h, 0, true, X, false, Y, false, s) : launch_apply(h, 0, true, X, Y, s, false);
  };
  std::fill(H, H + (size_t)(m + 1) * m, 0.0);
  m_done = 0;
  k_gnorm<<<g.G, kGT, 0, s>>>(v0, n, g.part);
  double nv2 = 0.0;
  int e = reduce_to_host(g, 1, &nv2);
  if (e) return e;
  const double nv = std::sqrt(nv2);
  if (!(nv > 0.0) || !std::isfinite(nv)) return -1;
  k_gscale<double><<<g.G, kGT, 0, s>>>(v0, V, n, 1.0 / nv);
  std::vector<double> hv, h2;
  for (int j = 0; j < m; ++j) {
    double *w = V + (int64_t)(j + 1) * ldv;
    if ((e = apply(V + (int64_t)j * ldv, w))) return e;
    double ww = 0.0;
    if ((e = dots<double>(g, V, ldv, j, w, n, hv, &ww))) return e;
    double hh = 0.0, hmax = 0.0;
    for (double v : hv) {
      hh += v * v;
      hmax = std::max(hmax, std::fabs(v));
    }
    double hn;
    h2.assign(j + 1, 0.0);
    if (ww - hh > 0.5 * ww) {
      hn = std::sqrt(ww - hh);
      if ((e = update<double>(g, V, ldv, hv, w, n, hn > 0 ? 1.0 / hn : 0.0, nullptr))) return e;
    } else {
      if ((e = update<double>(g, V, ldv, hv, w, n, 1.0, nullptr))) return e;
      if ((e = dots<double>(g, V, ldv, j, w, n, h2, nullptr))) return e;
      double n2 = 0.0;
      if ((e = update<double>(g, V, ldv, h2, w, n, 1.0, &n2))) return e;
      hn = std::sqrt(n2);
      std::vector<double> none;
      if ((e = update<double>(g, V, ldv, none, w, n, hn > 0 ? 1.0 / hn : 0.0, nullptr))) return e;
    }
    double *col = H + (size_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = hv[i] + h2[i];
    col[j + 1] = hn;
    m_done = j + 1;
    if (!(hn > 1e-14 * hmax)) break;
  }
  return (int)cudaGetLastError();
}

int launch_grid_solve(rt_handle *h, const double *b, double *x, double tol, double tol_inner, int m,
                      int max_outer, int use_x0, cudaStream_t s, int &outer, int &inner, double &relres,
                      int &status, double &bytes, int m_in) {
  if (h->dims == 1 && h->precision != 0)  // one 1D instance, mixed: nested solve on the grid kernels
    return grid_fgmres(h, b, x, tol, tol_inner, m, m_in, max_outer, use_x0, s, outer, inner, relres, status,
                       bytes);
  if (h->dims == 1) {  // one 1D instance, float64 GMRES: the batched apply kernels over the whole GPU
    const int64_t ldv = (h->E + 31) / 32 * 32;
    m = std::min<int64_t>(m, h->ws.cap_bytes / (8 * ldv) - 1);
    if (m < 1) return (int)cudaErrorInvalidValue;
    auto apply64 = [&](const double *xx, double *yy) -> int { return launch_apply(h, 0, true, xx, yy, s, false); };
    return grid_solve<double>(h, b, x, tol, tol_inner, m, max_outer, use_x0, s, apply64, apply64, false, outer,
                              inner, relres, status, bytes);
  }
  auto apply64 = [&](const double *xx, double *yy) -> int { return apply_box(h, 0, true, xx, false, yy, false, s); };
  if (h->precision == 0) {
    auto applyL = [&](const double *v, double *w) -> int { return apply_box(h, 0, true, v, false, w, false, s); };
    return grid_solve<double>(h, b, x, tol, tol_inner, m, max_outer, use_x0, s, apply64, applyL, false, outer,
                              inner, relres, status, bytes);
  }
  auto applyL = [&](const float *v, float *w) -> int { return apply_box(h, 0, false, v, true, w, true, s); };
  return grid_solve<float>(h, b, x, tol, tol_inner, m, max_outer, use_x0, s, apply64, applyL, true, outer, inner,
                           relres, status, bytes);
}

}  // namespace rt
