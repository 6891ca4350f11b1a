// rt_column.cu -- kernels for batches of 1D columns (Sec. 3.1-3.3):
//   k_coefficients    : per-layer step coefficients in float64 (SC-L, implicit
//                       Euler, quadratic SC), with float32 copies
//   k_solve<double>   : float64 restarted GMRES(m) per (column, rhs) instance
//                       (classical Gram-Schmidt with DGKS, Givens rotations)
//   k_solve_nested    : mixed precision: float64 flexible GMRES whose
//                       directions come from float32 GMRES cycles on a
//                       binary16 basis
//   k_solve_bicgstab  : float64 BiCGStab per instance
//
// Every solve kernel walks a work queue of (column, rhs) instances with one
// CTA per instance at a time; all synchronisation is inside the CTA, no CTA
// ever waits for another.
#include <algorithm>

#include <cuda_runtime.h>

#include "rt_async.cuh"
#include "rt_host.h"
#include "rt_internal.cuh"

namespace rt {

constexpr int kNT = 512;      // threads per CTA of the solve kernel (one CTA per SM)
constexpr int kDots = 4;      // basis vectors per block reduction in Gram-Schmidt

int solve_block_threads() { return kNT; }

// ------------------------------------------------------------ coefficients
// One thread per (layer, |mu| class, nu) of one column (blockIdx.y).  The
// optical depth of layer l is 0.5 (chi_l + chi_{l+1}) (z_{l+1} - z_l) / |mu|.
// SC-L step: e = e^-d, w0 = -expm1(-d), beta = w1/d (series below d = 0.1),
// alpha = w0 - beta.  Implicit Euler: e = 1/(1+d), alpha = 0, beta = d/(1+d).
// Quadratic SC (fs == 2): the parabola through upwind u, current c and
// downwind point at path depths 0, du, du + dd, integrated against
// e^-(du - s) with the moments W1/du^2 and W2/du^3 (series below 0.1):
//   psi_c = du ((du + dd) W1/du^2 - du W2/du^3) / dd
//   psi_d = du^3 (W2/du^3 - W1/du^2) / (dd (du + dd)),  psi_u = w0 - psi_c - psi_d;
// a ray's last step (no downwind point) is SC-L with psi_d = 0.  Rays going
// down take dd from layer l+1, rays going up from layer l-1.
struct CoefOut {
  double *E, *A, *B, *C, *A2, *B2, *C2;
  float *Ef, *Af, *Bf, *Cf, *A2f, *B2f, *C2f;
};

__device__ __forceinline__ void scl_step(double d, double &e, double &a, double &b) {
  e = exp(-d);
  const double w0 = -expm1(-d);
  double beta;
  if (d < 0.1) {
    // w1/d = sum_{k>=1} (-1)^(k+1) d^k/(k+1)! = (d/2)(1 - (d/3)(1 - (d/4)(1 - ...)))
    // 16 terms, nested from the innermost factor d/17
    double s = 1.0;
    for (int j = 17; j >= 3; --j) s = 1.0 - (d / j) * s;
    beta = 0.5 * d * s;
  } else {
    beta = (d - w0) / d;
  }
  b = beta;
  a = w0 - beta;
}

// quadratic step weights for depths du (u -> c) and dd (c -> d)
__device__ __forceinline__ void qsc_step(double du, double dd, double &pu, double &pc, double &pd) {
  double m1, m2;  // W1/du^2, W2/du^3
  if (du < 0.1) {
    // W1/du^2 = sum_{k>=0} (-1)^k du^k/(k+2)!,  W2/du^3 = 2 sum_{k>=0} (-1)^k du^k/(k+3)!
    // nested: 1/2 (1 - du/3 (1 - du/4 (...))), 1/3 (1 - du/4 (1 - du/5 (...)))
    double s1 = 1.0, s2 = 1.0;
    for (int j = 19; j >= 3; --j) s1 = 1.0 - (du / j) * s1;
    for (int j = 20; j >= 4; --j) s2 = 1.0 - (du / j) * s2;
    m1 = 0.5 * s1;
    m2 = s2 / 3.0;
  } else {
    const double w1 = du + expm1(-du);
    m1 = w1 / (du * du);
    m2 = (du * du - 2.0 * w1) / (du * du * du);
  }
  const double w0 = -expm1(-du);
  pc = du * ((du + dd) * m1 - du * m2) / dd;
  pd = du * du * du * (m2 - m1) / (dd * (du + dd));
  pu = w0 - pc - pd;
}

__global__ void k_coefficients(const ColDev *__restrict__ cols, const double *__restrict__ z,
                               const int64_t *__restrict__ zoff, const double *__restrict__ chi,
                               const double *__restrict__ mu_cls, const int32_t *__restrict__ cls_off,
                               CoefOut o) {
  const int col = blockIdx.y;
  const ColDev c = cols[col];
  const int64_t count = (int64_t)(c.nz - 1) * c.ncls * c.nn;
  auto dtau = [&](int layer, int f, int cl) {
    const double dz = z[zoff[col] + layer + 1] - z[zoff[col] + layer];
    const double cbar = 0.5 * (chi[c.g_off + (int64_t)layer * c.nn + f] +
                               chi[c.g_off + (int64_t)(layer + 1) * c.nn + f]);
    return cbar * dz / mu_cls[cls_off[col] + cl];
  };
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(i % c.nn);
    const int cl = (int)((i / c.nn) % c.ncls);
    const int layer = (int)(i / ((int64_t)c.nn * c.ncls));
    const double d = dtau(layer, f, cl);
    double e, a, b;
    if (c.fs == 1) {
      e = 1.0 / (1.0 + d);
      a = 0.0;
      b = d * e;
    } else {
      scl_step(d, e, a, b);
    }
    const int64_t k = c.c_off + i;
    o.E[k] = e;
    o.Ef[k] = (float)e;
    if (c.fs != 2) {
      o.A[k] = a;
      o.B[k] = b;
      o.Af[k] = (float)a;
      o.Bf[k] = (float)b;
      continue;
    }
    double pu, pc, pd;
    // going down: u = layer, c = layer + 1, downwind layer + 2
    if (layer + 1 < c.nz - 1) qsc_step(d, dtau(layer + 1, f, cl), pu, pc, pd);
    else { pu = a; pc = b; pd = 0.0; }
    o.A[k] = pu; o.B[k] = pc; o.C[k] = pd;
    o.Af[k] = (float)pu; o.Bf[k] = (float)pc; o.Cf[k] = (float)pd;
    // going up: u = layer + 1, c = layer, downwind layer - 1
    if (layer >= 1) qsc_step(d, dtau(layer - 1, f, cl), pu, pc, pd);
    else { pu = a; pc = b; pd = 0.0; }
    o.A2[k] = pu; o.B2[k] = pc; o.C2[k] = pd;
    o.A2f[k] = (float)pu; o.B2f[k] = (float)pc; o.C2f[k] = (float)pd;
  }
}

int launch_coefficients(rt_handle *h, const double *d_z, const int64_t *d_zoff,
                        const double *d_chi, const double *d_mu_cls, const int32_t *d_cls_off, cudaStream_t s) {
  int64_t most = 1;
  for (const ColDev &c : h->h_cols) most = std::max<int64_t>(most, (int64_t)(c.nz - 1) * c.ncls * c.nn);
  const int bx = (int)std::min<int64_t>((most + 255) / 256, 4096);
  dim3 grid(bx, h->n_cols);
  const int64_t nc = h->n_coef;
  CoefOut o{h->E64, h->A64, h->B64, nullptr, nullptr, nullptr, nullptr,
            h->E32, h->A32, h->B32, nullptr, nullptr, nullptr, nullptr};
  if (h->Q64) {
    o.C = h->Q64; o.A2 = h->Q64 + nc; o.B2 = h->Q64 + 2 * nc; o.C2 = h->Q64 + 3 * nc;
    o.Cf = h->Q32; o.A2f = h->Q32 + nc; o.B2f = h->Q32 + 2 * nc; o.C2f = h->Q32 + 3 * nc;
  }
  k_coefficients<<<grid, 256, 0, s>>>(h->d_cols, d_z, d_zoff, d_chi, d_mu_cls, d_cls_off, o);
  return (int)cudaGetLastError();
}

__device__ __forceinline__ int next_instance(int *queue, int *s_q) {
  if (threadIdx.x == 0) *s_q = atomicAdd(queue, 1);
  __syncthreads();
  const int q = *s_q;
  __syncthreads();
  return q;
}

// ------------------------------------------------------------------ solve
struct SolveParams {
  Common cm;
  Tables<double> t64;
  Tables<float> t32;
  const int32_t *order;
  int n_cols, n_inst;
  int64_t E;
  const double *b;      // [n_rhs][E]
  int b_shared;         // 1: b has one rhs vector shared by every rhs
  double *x;            // [n_rhs][E]
  double tol, tol_inner;
  int m, max_outer, use_x0;
  int m_in;             // mixed precision: inner float32 GMRES cycle length
  int max_iter;         // BiCGStab: iteration cap
  void *V;              // [slots][cap] Krylov bases of one slot
  int64_t cap;          // fp64 path: basis capacity of one slot in elements; mixed: bytes
  double *S;            // [slots][ld] float64 scratch: source function / residual
  int64_t ld;
  double *H;            // [slots][hld] Hessenberg (column-major), cs, sn, g
  int64_t hld;
  int *queue;
  SolveOut out;
};

constexpr int kU = 8;  // independent elements per thread in the vector loops
constexpr int kRwCache = 128 * 128;  // floats of frequency kernel kept in shared memory by the mixed solve
constexpr int kUwlCache = 256;       // floats of each angular factor kept in shared memory

__device__ __forceinline__ double cta_norm2(const double *v, int64_t n, double *red, double *outb) {
  double a[1] = {0.0};
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) a[0] += v[k] * v[k];
  block_sum<1>(a, red, outb);
  return a[0];
}

// h[0..j] = V[0..j]^T w and ||w||^2 (returned).  Products and the running sums
// over 8 consecutive elements of a thread are taken in TL, then accumulated
// in float64, then summed over the block in float64.
template <typename TL>
__device__ __noinline__ double cta_dots(const TL *V, int64_t ldv, int j, const TL *w, int64_t n, double *h,
                           double *red, double *outb) {
  double nrm = 0.0;
  constexpr int kWiden = 8;  // loop iterations summed in TL before one float64 add
  for (int i0 = 0; i0 <= j; i0 += kDots) {
    const int cnt = min(kDots, j + 1 - i0);
    // unconditional loads: vectors past the last one re-read the last (cache hit)
    const TL *vp[kDots];
#pragma unroll
    for (int u = 0; u < kDots; ++u) vp[u] = V + (int64_t)min(i0 + u, j) * ldv;
    double acc[kDots + 1];
#pragma unroll
    for (int u = 0; u <= kDots; ++u) acc[u] = 0.0;
    TL part[kDots + 1];
#pragma unroll
    for (int u = 0; u <= kDots; ++u) part[u] = 0;
    int it = 0;
    for (int64_t k0 = threadIdx.x; k0 < n; k0 += (int64_t)kU * blockDim.x) {
      TL wv[kU], vv[kDots][kU];
#pragma unroll
      for (int e = 0; e < kU; ++e) {
        const int64_t k = min(k0 + (int64_t)e * blockDim.x, n - 1);
        wv[e] = w[k];
#pragma unroll
        for (int u = 0; u < kDots; ++u) vv[u][e] = vp[u][k];
      }
#pragma unroll
      for (int e = 0; e < kU; ++e)
        if (k0 + (int64_t)e * blockDim.x >= n) wv[e] = 0;
#pragma unroll
      for (int u = 0; u < kDots; ++u)
#pragma unroll
        for (int e = 0; e < kU; ++e) part[u] = fma(vv[u][e], wv[e], part[u]);
#pragma unroll
      for (int e = 0; e < kU; ++e) part[kDots] = fma(wv[e], wv[e], part[kDots]);
      if (++it == kWiden) {
        it = 0;
#pragma unroll
        for (int u = 0; u <= kDots; ++u) {
          acc[u] += (double)part[u];
          part[u] = 0;
        }
      }
    }
#pragma unroll
    for (int u = 0; u <= kDots; ++u) acc[u] += (double)part[u];
    block_sum<kDots + 1>(acc, red, outb);
    if (threadIdx.x < cnt) h[i0 + threadIdx.x] = outb[threadIdx.x];
    if (i0 == 0) nrm = acc[kDots];
  }
  __syncthreads();
  return nrm;
}

// acc[e] += sum_{i < cnt} coef[i] * V_i[k0 + e*blockDim] for kU elements; the
// basis is walked kDots vectors at a time with all their loads issued before
// the FMAs (kDots*kU independent loads in flight per thread).  coef is in TL.
template <typename TL>
__device__ __forceinline__ void axpy_block(const TL *V, int64_t ldv, int cnt, const TL *coef, int64_t k0,
                                           int64_t n, TL (&acc)[kU]) {
  for (int i0 = 0; i0 < cnt; i0 += kDots) {
    TL v[kDots][kU], hu[kDots];
#pragma unroll
    for (int u = 0; u < kDots; ++u) {
      // unconditional loads: rows past cnt re-read row cnt-1 with a zero coefficient
      const int i = min(i0 + u, cnt - 1);
      hu[u] = (i0 + u < cnt) ? coef[i0 + u] : (TL)0;
      const TL *vi = V + (int64_t)i * ldv;
#pragma unroll
      for (int e = 0; e < kU; ++e) v[u][e] = vi[min(k0 + (int64_t)e * blockDim.x, n - 1)];
    }
#pragma unroll
    for (int u = 0; u < kDots; ++u)
#pragma unroll
      for (int e = 0; e < kU; ++e) acc[e] = fma(hu[u], v[u][e], acc[e]);
  }
}

// coefficients -> TL in shared memory (sign applied), then a barrier
template <typename TL>
__device__ __forceinline__ void stage_coef(const double *h, int cnt, double sgn, TL *hf) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) hf[i] = (TL)(sgn * h[i]);
  __syncthreads();
}

// w = (w - V[0..j] h) * scale; returns ||result||^2 when want_norm (else 0).
// hf: shared scratch of at least j+1 TL.
template <typename TL>
__device__ __noinline__ double cta_update(const TL *V, int64_t ldv, int j, TL *w, int64_t n, const double *h,
                             double scale, bool want_norm, TL *hf, double *red, double *outb) {
  stage_coef<TL>(h, j + 1, -1.0, hf);
  const TL sc = (TL)scale;
  double a[1] = {0.0};
  for (int64_t k0 = threadIdx.x; k0 < n; k0 += (int64_t)kU * blockDim.x) {
    TL wv[kU];
#pragma unroll
    for (int e = 0; e < kU; ++e) {
      const int64_t k = k0 + (int64_t)e * blockDim.x;
      wv[e] = k < n ? w[k] : (TL)0;
    }
    axpy_block<TL>(V, ldv, j + 1, hf, k0, n, wv);
    TL part = 0;
#pragma unroll
    for (int e = 0; e < kU; ++e) {
      const int64_t k = k0 + (int64_t)e * blockDim.x;
      const TL v = wv[e] * sc;
      if (k < n) w[k] = v;
      part = fma(v, v, part);
    }
    if (want_norm) a[0] += (double)part;
  }
  if (want_norm) block_sum<1>(a, red, outb);
  else __syncthreads();
  return want_norm ? a[0] : 0.0;
}

enum InstStatus : int { kConverged = 0, kNoConv = 4, kBreakdown = 5, kNonFinite = 6 };

constexpr int kMaxM = 512;  // largest Krylov basis per instance

// One CTA solves one (column, rhs) instance at a time, to completion:
//   outer loop (float64): r = b - A x, stop when ||r|| <= tol ||b||;
//   inner GMRES(m) on the operator in TL (float: mixed, double: plain fp64),
//   basis stored in TL, m = min(requested, kMaxM, slot capacity / instance size);
//   Arnoldi: classical Gram-Schmidt with the DGKS test: when ||w - V h|| >=
//   ||w||/sqrt(2) (known from ||w||^2 - ||h||^2 without another pass) one
//   update pass also normalises; otherwise a second projection is made;
//   Givens rotations and the triangular solve in float64 by thread 0;
//   x += V y with the correction summed in TL.
template <typename TL>
__global__ void __launch_bounds__(kNT, 1) k_solve(SolveParams p) {
  __shared__ double sm[4 * kSigBuf];
  __shared__ double red[(kNT / 32) * (kDots + 1)];
  __shared__ double outb[kDots + 1];
  __shared__ double hbuf[2 * (kMaxM + 8)];
  __shared__ TL hf[kMaxM + 8];
  __shared__ int s_q;
  __shared__ double s_val[4];
  TL *Vslot = reinterpret_cast<TL *>(p.V) + (int64_t)blockIdx.x * p.cap;
  double *S64 = p.S + (int64_t)blockIdx.x * p.ld;
  TL *SL = reinterpret_cast<TL *>(S64);
  double *Hc = p.H + (int64_t)blockIdx.x * p.hld;
  double *h = hbuf;
  double *h2 = hbuf + kMaxM + 8;
  const Tables<TL> &tl = *reinterpret_cast<const Tables<TL> *>(
      sizeof(TL) == 8 ? (const void *)&p.t64 : (const void *)&p.t32);
  const bool mixed = sizeof(TL) == 4;
  const double sz = (double)sizeof(TL);
  for (;;) {
    const int q = next_instance(p.queue, &s_q);
    if (q >= p.n_inst) break;
    const int inst = p.order[q];
    const int ci = inst % p.n_cols, rhs = inst / p.n_cols;
    const ColDev c = p.cm.cols[ci];
    const int64_t n = (int64_t)c.nz * c.nr;
    const int64_t ldv = (n + 31) / 32 * 32;
    const int64_t fit = p.cap / ldv - 1;
    const int m = (int)(fit < (int64_t)min(p.m, kMaxM) ? fit : (int64_t)min(p.m, kMaxM));
    double *cs = Hc + (int64_t)(m + 1) * m;
    double *sn = cs + (m + 1);
    double *g = sn + (m + 1);
    const double *bv = p.b + (p.b_shared ? 0 : rhs * p.E) + c.x_off;
    double *x = p.x + rhs * p.E + c.x_off;
    const double bn = sqrt(cta_norm2(bv, n, red, outb));
    if (!p.use_x0) {
      for (int64_t k = threadIdx.x; k < n; k += blockDim.x) x[k] = 0.0;
      __syncthreads();
    }
    int status = kNoConv, outer = 0, inner_total = 0;
    double relres = 1.0;
    double bpe = p.use_x0 ? 8.0 : 16.0;  // algorithmic bytes per element: ||b||, x = 0
    const bool bad_b = !(bn == bn) || bn > 1e300;
    if (bad_b) {
      status = kNonFinite;
    } else if (bn == 0.0) {
      for (int64_t k = threadIdx.x; k < n; k += blockDim.x) x[k] = 0.0;
      status = kConverged;
      relres = 0.0;
    }
    for (; bn > 0.0 && !bad_b; ++outer) {
      // ---- r = b - A x in float64, then V_0 = r / ||r|| in TL ----------------
      double rn;
      const double *rsrc;
      if (outer == 0 && !p.use_x0) {
        rn = bn;
        rsrc = bv;
        bpe += 0.0;
      } else {
        sigma_column<double, double>(c, p.t64, x, S64, sm, 4 * kSigBuf);
        double a[1] = {sweep_column<double, double, double, 2, kOutResid>(c, p.t64, p.cm, S64, nullptr, x, bv,
                                                                           S64, false)};
        block_sum<1>(a, red, outb);
        rn = sqrt(a[0]);
        rsrc = S64;
        bpe += 48.0;  // x, S, S, x, b, r
      }
      relres = rn / bn;
      if (!(rn == rn) || rn > 1e300) { status = kNonFinite; break; }
      if (relres <= p.tol) { status = kConverged; break; }
      if (outer >= p.max_outer) { status = kNoConv; break; }
      for (int64_t k = threadIdx.x; k < n; k += blockDim.x) Vslot[k] = (TL)(rsrc[k] / rn);
      __syncthreads();
      bpe += 8.0 + sz;
      if (threadIdx.x == 0) g[0] = rn;
      const double target = mixed ? fmax(p.tol_inner * rn, 0.5 * p.tol * bn) : 0.5 * p.tol * bn;
      int jdone = 0;
      bool breakdown = false;
      for (int j = 0; j < m; ++j) {
        TL *vj = Vslot + (int64_t)j * ldv;
        TL *w = Vslot + (int64_t)(j + 1) * ldv;
        sigma_column<TL, TL>(c, tl, vj, SL, reinterpret_cast<TL *>(sm), 4 * kSigBuf * (int)(8 / sizeof(TL)));
        sweep_column<TL, TL, TL, sizeof(TL) == 8 ? 2 : 4, kOutAminus>(c, tl, p.cm, SL, nullptr, vj, nullptr, w, false);
        __syncthreads();
        bpe += 5.0 * sz;  // v, S, S, v, w
        const double ww = cta_dots<TL>(Vslot, ldv, j, w, n, h, red, outb);
        double hh = 0.0;
        for (int i = 0; i <= j; ++i) hh += h[i] * h[i];
        double hn;
        bpe += sz * (j + 2);
        if (ww - hh > 0.5 * ww) {
          hn = sqrt(ww - hh);
          cta_update<TL>(Vslot, ldv, j, w, n, h, hn > 0.0 ? 1.0 / hn : 0.0, false, hf, red, outb);
          bpe += sz * (j + 3);
          for (int i = threadIdx.x; i <= j; i += blockDim.x) h2[i] = 0.0;
        } else {
          // second projection: w' = w - V h, h2 = V^T w', w'' = w' - V h2
          cta_update<TL>(Vslot, ldv, j, w, n, h, 1.0, false, hf, red, outb);
          cta_dots<TL>(Vslot, ldv, j, w, n, h2, red, outb);
          const double hn2 = cta_update<TL>(Vslot, ldv, j, w, n, h2, 1.0, true, hf, red, outb);
          hn = sqrt(hn2);
          for (int64_t k = threadIdx.x; k < n; k += blockDim.x) w[k] = (TL)((double)w[k] / hn);
          __syncthreads();
          bpe += sz * (3.0 * j + 10.0);
        }
        if (threadIdx.x == 0) {
          double *col = Hc + (int64_t)j * (m + 1);
          for (int i = 0; i <= j; ++i) col[i] = h[i] + h2[i];
          col[j + 1] = hn;
          for (int i = 0; i < j; ++i) {
            const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
            col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
            col[i] = t0;
          }
          const double den = hypot(col[j], col[j + 1]);
          double cj = 1.0, sj = 0.0;
          if (den > 0.0) { cj = col[j] / den; sj = col[j + 1] / den; }
          cs[j] = cj;
          sn[j] = sj;
          col[j] = den;
          col[j + 1] = 0.0;
          g[j + 1] = -sj * g[j];
          g[j] = cj * g[j];
          s_val[0] = fabs(g[j + 1]);
          s_val[1] = den;
        }
        __syncthreads();
        const double est = s_val[0];
        const double den = s_val[1];
        jdone = j + 1;
        if (den == 0.0) { breakdown = true; jdone = j; break; }
        if (!(hn > 1e-300 * fmax(1.0, rn))) break;  // invariant subspace: exact in it
        if (!(est == est)) break;
        if (est <= target) break;
      }
      inner_total += jdone;
      // ---- y = R^-1 g (float64), x += V y -------------------------------------
      if (threadIdx.x == 0) {
        for (int i = jdone - 1; i >= 0; --i) {
          double acc = g[i];
          for (int k = i + 1; k < jdone; ++k) acc -= Hc[(int64_t)k * (m + 1) + i] * h[k];
          h[i] = acc / Hc[(int64_t)i * (m + 1) + i];
        }
      }
      __syncthreads();
      stage_coef<TL>(h, jdone, 1.0, hf);
      for (int64_t k0 = threadIdx.x; k0 < n; k0 += (int64_t)kU * blockDim.x) {
        TL d[kU];
#pragma unroll
        for (int e = 0; e < kU; ++e) d[e] = 0;
        axpy_block<TL>(Vslot, ldv, jdone, hf, k0, n, d);
#pragma unroll
        for (int e = 0; e < kU; ++e) {
          const int64_t k = k0 + (int64_t)e * blockDim.x;
          if (k < n) x[k] += (double)d[e];
        }
      }
      bpe += sz * jdone + 16.0;
      __syncthreads();
      if (breakdown && jdone == 0) { status = kBreakdown; break; }
    }
    if (threadIdx.x == 0) {
      p.out.outer[inst] = outer;
      p.out.inner[inst] = inner_total;
      p.out.status[inst] = status;
      p.out.relres[inst] = relres;
      p.out.bytes[inst] = bpe * (double)n;
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------- mixed solve
// Givens update of column j of a Hessenberg matrix stored column-major with
// leading dimension ld (thread 0 only); returns |g_{j+1}| and den via s_val.
// shifted: the Arnoldi step ran on K = Id - A (same Krylov space), so the
// column of A's Hessenberg is e_j - (h + h2) with subdiagonal -hn.
__device__ __forceinline__ void givens_step(double *Hc, int ld, double *cs, double *sn, double *g, int j,
                                            const double *h, const double *h2, double hn, double *s_val,
                                            double sign = 1.0, double diag = 0.0) {
  // the Arnoldi step ran on a shifted operator: column j of A's Hessenberg is
  // diag e_j + sign (h + h2) with subdiagonal sign hn (sign -1, diag 1: K =
  // Id - A; sign 1, diag 1: the direction A z minus the basis vector v_j)
  double *col = Hc + (int64_t)j * ld;
  for (int i = 0; i <= j; ++i) col[i] = (i == j ? diag : 0.0) + sign * (h[i] + h2[i]);
  col[j + 1] = sign * hn;
  for (int i = 0; i < j; ++i) {
    const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t0;
  }
  const double den = hypot(col[j], col[j + 1]);
  double cj = 1.0, sj = 0.0;
  if (den > 0.0) { cj = col[j] / den; sj = col[j + 1] / den; }
  cs[j] = cj;
  sn[j] = sj;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -sj * g[j];
  g[j] = cj * g[j];
  s_val[0] = fabs(g[j + 1]);
  s_val[1] = den;
}

// One Arnoldi step on basis V[0..j] (TL) with w = V[j+1] unnormalised:
// classical Gram-Schmidt with the DGKS test (second projection when
// ||w - V h||^2 <= eta2 ||w||^2, eta2 = 1/2 by default) and a fused
// normalisation (see k_solve).
// Leaves h (+ h2) and returns ||w - V h||; bytes per element in bpe.
template <typename TL>
__device__ double arnoldi_orth(TL *V, int64_t ldv, int j, int64_t n, double *h, double *h2, TL *hf,
                               double *red, double *outb, double &bpe, double eta2 = 0.5) {
  TL *w = V + (int64_t)(j + 1) * ldv;
  const double sz = sizeof(TL);
  const double ww = cta_dots<TL>(V, ldv, j, w, n, h, red, outb);
  double hh = 0.0;
  for (int i = 0; i <= j; ++i) hh += h[i] * h[i];
  bpe += sz * (j + 2);
  double hn;
  if (ww - hh > eta2 * ww) {
    hn = sqrt(ww - hh);
    cta_update<TL>(V, ldv, j, w, n, h, hn > 0.0 ? 1.0 / hn : 0.0, false, hf, red, outb);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h2[i] = 0.0;
    bpe += sz * (j + 3);
  } else {
    cta_update<TL>(V, ldv, j, w, n, h, 1.0, false, hf, red, outb);
    cta_dots<TL>(V, ldv, j, w, n, h2, red, outb);
    hn = sqrt(cta_update<TL>(V, ldv, j, w, n, h2, 1.0, true, hf, red, outb));
    const TL inv = (TL)(hn > 0.0 ? 1.0 / hn : 0.0);
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) w[k] *= inv;
    bpe += sz * (3.0 * j + 10.0);
  }
  __syncthreads();
  return hn;
}

// ------------------------------------- Sigma of an inner cycle (binary16 input)
// Separable kernel, X in binary16 (a basis row of the inner cycle), S in
// float32.  Each warp takes points warp, warp + nw, ...; the X block and the
// Gamma row of its next point are copied into the warp's shared buffer by
// cp.async while the current point's frequency-kernel and expansion steps
// run, so the global latency is hidden behind compute.  Per-warp buffer
// (16-byte aligned parts): wm [rp][nn] float | wz [rp][nn] float | xs [nr]
// binary16 | gs [nn] float.  The angular factors Uw, Ul come from shared
// memory when the caller staged them.
constexpr int kSig16WarpBytes = 7168;  // shared bytes per warp (16 warps: 112 KB)

__host__ __device__ inline int sig16_part(int elems, int bytes) { return (elems * bytes + 15) / 16 * 16; }

__device__ inline bool sig16_ok(const ColDev &c) {
  const int need = 2 * sig16_part(c.rp * c.nn, 4) + sig16_part(c.nr, 2) + sig16_part(c.nn, 4);
  return c.psi_off < 0 && c.nr % 8 == 0 && c.rp <= 8 && need <= kSig16WarpBytes;
}

template <int KR>
__device__ __noinline__ void sigma_points_h16(const ColDev &c, const Tables<float> &tb,
                                              const __half *__restrict__ X, float *__restrict__ S,
                                              unsigned char *wbuf, const float *Rw, const float *Uw,
                                              const float *Ul, const float *lrA) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nd = c.nd, nn = c.nn, nr = c.nr, rp = c.rp;
  const float *gam = tb.gamma + c.g_off;
  const int pz = sig16_part(rp * nn, 4);
  float *wm = reinterpret_cast<float *>(wbuf);
  float *wz = reinterpret_cast<float *>(wbuf + pz);
  __half *xs = reinterpret_cast<__half *>(wbuf + 2 * pz);
  float *gs = reinterpret_cast<float *>(wbuf + 2 * pz + sig16_part(nr, 2));
  const int nvec = nr / 8;
  auto fetch = [&](int p) {  // X block and Gamma row of point p -> xs, gs (asynchronous)
    const uint4 *src = reinterpret_cast<const uint4 *>(X + (int64_t)p * nr);
    for (int i = lane; i < nvec; i += 32) cp_async16(reinterpret_cast<uint4 *>(xs) + i, src + i, 16u);
    const float *g = gam + (int64_t)p * nn;
    for (int f = lane; f < nn; f += 32) cp_async4(gs + f, g + f);
    cp_async_commit();
  };
  if (warp < c.nz) fetch(warp);
  for (int p = warp; p < c.nz; p += nw) {
    cp_async_wait<0>();
    __syncwarp();
    // 1. moments m_k(f) = sum_d Uw[d][k] X(d, f), lanes over f
    for (int f = lane; f < nn; f += 32) {
      float m[KR];
#pragma unroll
      for (int k = 0; k < KR; ++k) m[k] = 0.f;
      for (int d = 0; d < nd; ++d) {
        const float xv = __half2float(xs[d * nn + f]);
        const float *u = Uw + d * rp;
#pragma unroll
        for (int k = 0; k < KR; ++k)
          if (k < rp) m[k] = fmaf(u[k], xv, m[k]);
      }
#pragma unroll
      for (int k = 0; k < KR; ++k)
        if (k < rp) wm[k * nn + f] = m[k];
    }
    __syncwarp();
    const float *zw = wz;
    if (lrA) {
      // truncated frequency kernel: t = A^T m into wz, z = B t back into wm
      lowrank_frequency_warp<float>(lrA, lrA + nn * c.lr_rank, c.lr_rank, nn, rp, wm, wz, wm);
      zw = wm;
    } else
    // 2. frequency kernel z_k(f) = sum_q RwT[q][f] m_k(q), two frequencies per lane
    for (int fb = 0; fb < nn; fb += 64) {
      const int fa = fb + lane, fc = fa + 32;
      const bool va = fa < nn, vc = fc < nn;
      const int fa_ = va ? fa : 0, fc_ = vc ? fc : 0;
      float aa[KR], ac[KR];
#pragma unroll
      for (int k = 0; k < KR; ++k) aa[k] = ac[k] = 0.f;
      if (c.rdiag) {
#pragma unroll
        for (int k = 0; k < KR; ++k)
          if (k < rp) {
            aa[k] = Rw[fa_] * wm[k * nn + fa_];
            ac[k] = Rw[fc_] * wm[k * nn + fc_];
          }
      } else {
        for (int q = 0; q < nn; ++q) {
          const float ra = Rw[q * nn + fa_], rc = Rw[q * nn + fc_];
#pragma unroll
          for (int k = 0; k < KR; ++k)
            if (k < rp) {
              const float mv = wm[k * nn + q];
              aa[k] = fmaf(ra, mv, aa[k]);
              ac[k] = fmaf(rc, mv, ac[k]);
            }
        }
      }
#pragma unroll
      for (int k = 0; k < KR; ++k)
        if (k < rp) {
          if (va) wz[k * nn + fa] = aa[k];
          if (vc) wz[k * nn + fc] = ac[k];
        }
    }
    __syncwarp();
    // 3. expansion S(d, f) = gamma(f) sum_k Ul[d][k] z_k(f): lanes over f
    //    (coalesced stores), the lane's z and gamma in registers, loop over d
    float *sp = S + (int64_t)p * nr;
    for (int f = lane; f < nn; f += 32) {
      float zf[KR];
#pragma unroll
      for (int k = 0; k < KR; ++k) zf[k] = k < rp ? zw[k * nn + f] : 0.f;
      const float gf = gs[f];
      for (int d = 0; d < nd; ++d) {
        const float *u = Ul + d * rp;
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < KR; ++k)
          if (k < rp) acc = fmaf(u[k], zf[k], acc);
        sp[d * nn + f] = gf * acc;
      }
    }
    __syncwarp();
    if (p + nw < c.nz) fetch(p + nw);  // xs, gs are free again
  }
  cp_async_wait<0>();
}

// Every point of one column (one CTA); wbase: nw * kSig16WarpBytes of shared
// memory; Rw, Uw, Ul: the column's float32 factors (shared or global).
// lrA: the column's truncated frequency kernel A | B (shared memory), or null
__device__ __noinline__ void sigma_column_h16(const ColDev &c, const Tables<float> &tb, const __half *X,
                                              float *S, unsigned char *wbase, const float *Rw, const float *Uw,
                                              const float *Ul, const float *lrA) {
  unsigned char *wbuf = wbase + (threadIdx.x >> 5) * kSig16WarpBytes;
  if (c.rp <= 2) sigma_points_h16<2>(c, tb, X, S, wbuf, Rw, Uw, Ul, lrA);
  else sigma_points_h16<8>(c, tb, X, S, wbuf, Rw, Uw, Ul, lrA);
  __syncthreads();
}

// ------------------------------------------- inner cycles with a binary16 basis
// The float32 inner GMRES cycles of the mixed solve keep their basis rows U_i
// in IEEE binary16.  The rows have unit norm, so every entry is at most 1 in
// magnitude; entries below 6e-8 flush to zero, an absolute error far below
// what a preconditioner solved to a relative 0.1 can notice, and the 2^-11
// relative rounding of the rest perturbs the Arnoldi relation by ~5e-4.  The
// outer float64 FGMRES is exact for whatever direction the cycle returns, so
// the final accuracy does not depend on it; the basis traffic halves.
// Rows are ldv (a multiple of 32) long and their entries n..ldv-1 are kept
// zero; the unnormalised direction w is float32 and its entries past n are
// ignored.  Vector loops walk quads (4 consecutive entries): 8-byte loads of
// U, 16-byte loads of w.
constexpr int kQ = 4;    // quads per thread per loop iteration (measured best with kD16 = 8)
constexpr int kD16 = 8;  // basis rows per streaming group

__device__ __forceinline__ void h4_to_f(uint2 raw, float (&f)[4]) {
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
  f[0] = a.x;
  f[1] = a.y;
  f[2] = b.x;
  f[3] = b.y;
}

__device__ __forceinline__ void st_h4(__half *p, const float (&f)[4]) {
  const __half2 a = __floats2half2_rn(f[0], f[1]), b = __floats2half2_rn(f[2], f[3]);
  uint2 raw;
  raw.x = *reinterpret_cast<const uint32_t *>(&a);
  raw.y = *reinterpret_cast<const uint32_t *>(&b);
  *reinterpret_cast<uint2 *>(p) = raw;
}

// entries k..k+3 of w, zero where k + t >= n or the quad is a clamped duplicate
__device__ __forceinline__ void ld_w4(const float *w, int64_t k, int64_t n, bool live, float (&f)[4]) {
  const float4 v = *reinterpret_cast<const float4 *>(w + k);
  f[0] = live && k < n ? v.x : 0.f;
  f[1] = live && k + 1 < n ? v.y : 0.f;
  f[2] = live && k + 2 < n ? v.z : 0.f;
  f[3] = live && k + 3 < n ? v.w : 0.f;
}

// h[0..j] = U[0..j]^T w, returns ||w||^2.  Sums are float32 over a thread's
// 8 loop steps, then float64, then one block reduction per group of kD16 rows.
__device__ __noinline__ double cta_dots16(const __half *U, int64_t ldv, int j, const float *w, int64_t n,
                                          double *h, double *red, double *outb) {
  const int64_t nq = ldv / 4;
  double nrm = 0.0;
  constexpr int kWiden = 8;
  for (int i0 = 0; i0 <= j; i0 += kD16) {
    const int cnt = min(kD16, j + 1 - i0);
    const __half *up[kD16];
#pragma unroll
    for (int u = 0; u < kD16; ++u) up[u] = U + (int64_t)min(i0 + u, j) * ldv;
    double acc[kD16 + 1];
    float part[kD16 + 1];
#pragma unroll
    for (int u = 0; u <= kD16; ++u) {
      acc[u] = 0.0;
      part[u] = 0.f;
    }
    int it = 0;
    for (int64_t q0 = threadIdx.x; q0 < nq; q0 += (int64_t)kQ * blockDim.x) {
      float wv[kQ][4];
      uint2 raw[kD16][kQ];
#pragma unroll
      for (int e = 0; e < kQ; ++e) {
        const int64_t q = q0 + (int64_t)e * blockDim.x;
        const int64_t qc = min(q, nq - 1);
        ld_w4(w, 4 * qc, n, q < nq, wv[e]);
#pragma unroll
        for (int u = 0; u < kD16; ++u) raw[u][e] = *reinterpret_cast<const uint2 *>(up[u] + 4 * qc);
      }
#pragma unroll
      for (int u = 0; u < kD16; ++u)
#pragma unroll
        for (int e = 0; e < kQ; ++e) {
          float f[4];
          h4_to_f(raw[u][e], f);
#pragma unroll
          for (int t = 0; t < 4; ++t) part[u] = fmaf(f[t], wv[e][t], part[u]);
        }
#pragma unroll
      for (int e = 0; e < kQ; ++e)
#pragma unroll
        for (int t = 0; t < 4; ++t) part[kD16] = fmaf(wv[e][t], wv[e][t], part[kD16]);
      if (++it == kWiden) {
        it = 0;
#pragma unroll
        for (int u = 0; u <= kD16; ++u) {
          acc[u] += (double)part[u];
          part[u] = 0.f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u <= kD16; ++u) acc[u] += (double)part[u];
    block_sum<kD16 + 1>(acc, red, outb);
    if (threadIdx.x < cnt) h[i0 + threadIdx.x] = outb[threadIdx.x];
    if (i0 == 0) nrm = acc[kD16];
  }
  __syncthreads();
  return nrm;
}

// acc[e][t] += sum_{i < cnt} coef[i] U_i[quad q_e]; kD16 rows' loads in flight
__device__ __forceinline__ void axpy16(const __half *U, int64_t ldv, int cnt, const float *coef,
                                       const int64_t (&qc)[kQ], float (&acc)[kQ][4]) {
  for (int i0 = 0; i0 < cnt; i0 += kD16) {
    uint2 raw[kD16][kQ];
    float hu[kD16];
#pragma unroll
    for (int u = 0; u < kD16; ++u) {
      const int i = min(i0 + u, cnt - 1);  // rows past cnt: re-read with a zero coefficient
      hu[u] = (i0 + u < cnt) ? coef[i0 + u] : 0.f;
      const __half *ui = U + (int64_t)i * ldv;
#pragma unroll
      for (int e = 0; e < kQ; ++e) raw[u][e] = *reinterpret_cast<const uint2 *>(ui + 4 * qc[e]);
    }
#pragma unroll
    for (int u = 0; u < kD16; ++u)
#pragma unroll
      for (int e = 0; e < kQ; ++e) {
        float f[4];
        h4_to_f(raw[u][e], f);
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[e][t] = fmaf(hu[u], f[t], acc[e][t]);
      }
  }
}

// r = (w - U[0..j] h) * scale.  out16: write r to that binary16 row (zero past
// n), else r overwrites w.  Returns ||r||^2 when want_norm (else 0).
__device__ __noinline__ double cta_update16(const __half *U, int64_t ldv, int j, float *w, int64_t n,
                                            const double *h, double scale, __half *out16, bool want_norm,
                                            float *hf, double *red, double *outb) {
  stage_coef<float>(h, j + 1, -1.0, hf);
  const int64_t nq = ldv / 4;
  const float sc = (float)scale;
  double a[1] = {0.0};
  for (int64_t q0 = threadIdx.x; q0 < nq; q0 += (int64_t)kQ * blockDim.x) {
    int64_t qc[kQ];
    bool live[kQ];
    float acc[kQ][4];
#pragma unroll
    for (int e = 0; e < kQ; ++e) {
      const int64_t q = q0 + (int64_t)e * blockDim.x;
      live[e] = q < nq;
      qc[e] = min(q, nq - 1);
      ld_w4(w, 4 * qc[e], n, live[e], acc[e]);
    }
    axpy16(U, ldv, j + 1, hf, qc, acc);
    float part = 0.f;
#pragma unroll
    for (int e = 0; e < kQ; ++e) {
      const int64_t k = 4 * qc[e];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        acc[e][t] = k + t < n ? acc[e][t] * sc : 0.f;
        part = fmaf(acc[e][t], acc[e][t], part);
      }
      if (live[e]) {
        if (out16) st_h4(out16 + k, acc[e]);
        else *reinterpret_cast<float4 *>(w + k) = make_float4(acc[e][0], acc[e][1], acc[e][2], acc[e][3]);
      }
    }
    if (want_norm) a[0] += (double)part;
  }
  if (want_norm) block_sum<1>(a, red, outb);
  else __syncthreads();
  return want_norm ? a[0] : 0.0;
}

// One Arnoldi step of an inner cycle: w (float32) against U[0..j] (binary16),
// the normalised result written to U[j+1].  Classical Gram-Schmidt; a second
// projection only when ||w - U h||^2 <= 1e-4 ||w||^2.  On these operators the
// DGKS bound of 1/2 is crossed at nearly every step (w = A u keeps most of u),
// which would double the traffic, while a preconditioner solved to 0.1 needs
// the basis orthogonal only to ~1e-3: single-pass loss measured ~2e-5.
// Leaves h (+ h2), returns ||w - U h||; bytes per element in bpe.
__device__ double arnoldi16(__half *U, int64_t ldv, int j, float *w, int64_t n, double *h, double *h2,
                            float *hf, double *red, double *outb, double &bpe) {
  __half *out = U + (int64_t)(j + 1) * ldv;
  const double ww = cta_dots16(U, ldv, j, w, n, h, red, outb);
  double hh = 0.0;
  for (int i = 0; i <= j; ++i) hh += h[i] * h[i];
  bpe += 2.0 * (j + 1) + 4.0;
  double hn;
  if (ww - hh > 1e-4 * ww) {
    hn = sqrt(ww - hh);
    cta_update16(U, ldv, j, w, n, h, hn > 0.0 ? 1.0 / hn : 0.0, out, false, hf, red, outb);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h2[i] = 0.0;
    bpe += 2.0 * (j + 1) + 6.0;
  } else {
    cta_update16(U, ldv, j, w, n, h, 1.0, nullptr, false, hf, red, outb);
    const double w1 = cta_dots16(U, ldv, j, w, n, h2, red, outb);
    double hh2 = 0.0;
    for (int i = 0; i <= j; ++i) hh2 += h2[i] * h2[i];
    hn = sqrt(fmax(w1 - hh2, 0.0));
    cta_update16(U, ldv, j, w, n, h2, hn > 0.0 ? 1.0 / hn : 0.0, out, false, hf, red, outb);
    bpe += 6.0 * (j + 1) + 18.0;
  }
  __syncthreads();
  return hn;
}

// y = R^-1 g for the leading k x k triangle of H (thread 0), result in y
__device__ __forceinline__ void tri_solve(const double *Hc, int ld, const double *g, int k, double *y) {
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double acc = g[i];
      for (int q = i + 1; q < k; ++q) acc -= Hc[(int64_t)q * ld + i] * y[q];
      y[i] = acc / Hc[(int64_t)i * ld + i];
    }
  }
  __syncthreads();
}

// Mixed precision (RT_P_MIXED): flexible GMRES(kout) with the Arnoldi basis,
// Givens rotations, residual and x in float64, preconditioned by one cycle of
// float32 GMRES(m_in) on the float32 operator (relative tolerance tol_inner):
//   z_i ~ A^-1 v_i (float32), w = A z_i (float64 operator), orthogonalise w,
//   x += Z y at the end of a cycle; cycles restart from the true residual.
// One CTA per (column, rhs) instance, as k_solve.  NT threads per CTA: 512
// (one CTA per SM) or 256 (two per SM, so one instance's latency-bound phases
// overlap another's streaming); shared memory scales with the warps, the
// frequency kernel is staged when it fits RWC floats (else read from L2).
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_solve_nested(SolveParams p) {
  constexpr int kSmD = (NT / 32) * kSig16WarpBytes / 8;  // doubles of Sigma work buffers
  constexpr int kRWC = NT == 512 ? kRwCache : kRwCache / 2;
  __shared__ __align__(16) double sm[kSmD];  // Sigma work buffers (inner: a kSig16WarpBytes part per warp)
  constexpr int kRed = (kDots > kD16 ? kDots : kD16) + 1;  // widest block_sum
  __shared__ double red[(NT / 32) * kRed];
  __shared__ double outb[kRed];
  __shared__ double hbuf[2 * (kMaxM + 8)];
  __shared__ double ybuf[kMaxM + 8];
  __shared__ float hf32[kMaxM + 8];
  __shared__ double hf64[kMaxM + 8];
  __shared__ int s_q;
  __shared__ double s_val[4];
  __shared__ float rw_s[kRWC];  // float32 frequency kernel of the current column
  __shared__ float uwl_s[2 * kUwlCache];  // float32 angular factors Uw | Ul of the current column
  uint8_t *slot = reinterpret_cast<uint8_t *>(p.V) + (int64_t)blockIdx.x * p.cap;
  double *S64 = p.S + (int64_t)blockIdx.x * p.ld;
  float *S32 = reinterpret_cast<float *>(S64);
  float *W32 = S32 + p.ld;  // inner cycles: the new direction (second half of the float64 scratch)
  double *Hbase = p.H + (int64_t)blockIdx.x * p.hld;
  double *h = hbuf;
  double *h2 = hbuf + kMaxM + 8;
  for (;;) {
    const int q = next_instance(p.queue, &s_q);
    if (q >= p.n_inst) break;
    const int inst = p.order[q];
    const int ci = inst % p.n_cols, rhs = inst / p.n_cols;
    const ColDev c = p.cm.cols[ci];
    const int64_t n = (int64_t)c.nz * c.nr;
    const int64_t ldv = (n + 31) / 32 * 32;
    const int m_in = min(p.m_in, kMaxM);
    // slot: Vout [(kout+1) ldv] double | Z [kout ldv] float | U [(m_in+1) ldv] binary16
    const int64_t per = p.cap / ldv;  // bytes per vector element available
    const int64_t kfit = (per - 8 - 2 * (int64_t)(m_in + 1)) / 12;
    const int kout = (int)(kfit < (int64_t)min(p.m, kMaxM) ? kfit : (int64_t)min(p.m, kMaxM));
    double *Vo = reinterpret_cast<double *>(slot);
    float *Z = reinterpret_cast<float *>(Vo + (int64_t)(kout + 1) * ldv);
    __half *U = reinterpret_cast<__half *>(Z + (int64_t)kout * ldv);
    double *Ho = Hbase;
    double *cso = Ho + (int64_t)(kout + 1) * kout, *sno = cso + (kout + 1), *go = sno + (kout + 1);
    double *Hi = go + (kout + 2);
    double *csi = Hi + (int64_t)(m_in + 1) * m_in, *sni = csi + (m_in + 1), *gi = sni + (m_in + 1);
    const double *bv = p.b + (p.b_shared ? 0 : rhs * p.E) + c.x_off;
    double *x = p.x + rhs * p.E + c.x_off;
    const double bn = sqrt(cta_norm2(bv, n, red, outb));
    const bool h16 = sig16_ok(c) && (blockDim.x >> 5) * kSig16WarpBytes <= (int)sizeof(sm);
    // stage the float32 frequency kernel of this column (dense, up to 128 x
    // 128), or its truncated factors A | B when the handle has them
    const float *rw_c = nullptr, *lr_c = nullptr;
    if (p.t32.LR && c.lr_rank > 0 && !c.rdiag && c.psi_off < 0) {
      const int len = 2 * c.nn * c.lr_rank;
      for (int k = threadIdx.x; k < len; k += blockDim.x) rw_s[k] = p.t32.LR[c.lr_off + k];
      __syncthreads();
      lr_c = rw_s;
    } else if (!c.rdiag && c.psi_off < 0 && c.nn * c.nn <= kRWC) {
      for (int k = threadIdx.x; k < c.nn * c.nn; k += blockDim.x) rw_s[k] = p.t32.RwT[c.r_off + k];
      __syncthreads();
      rw_c = rw_s;
    }
    const float *uw_c = p.t32.Uw + c.u_off, *ul_c = p.t32.Ul + c.u_off;
    if (c.nd * c.rp <= kUwlCache) {
      for (int k = threadIdx.x; k < c.nd * c.rp; k += blockDim.x) {
        uwl_s[k] = uw_c[k];
        uwl_s[kUwlCache + k] = ul_c[k];
      }
      __syncthreads();
      uw_c = uwl_s;
      ul_c = uwl_s + kUwlCache;
    }
    if (!p.use_x0) {
      for (int64_t k = threadIdx.x; k < n; k += blockDim.x) x[k] = 0.0;
      __syncthreads();
    }
    int status = kNoConv, cycles = 0, outer_total = 0, inner_total = 0;
    double relres = 1.0;
    double bpe = p.use_x0 ? 8.0 : 16.0;
    const bool bad_b = !(bn == bn) || bn > 1e300;
    if (bad_b) {
      status = kNonFinite;
    } else if (bn == 0.0) {
      status = kConverged;
      relres = 0.0;
    }
    for (; bn > 0.0 && !bad_b && kout >= 1; ++cycles) {
      double rn;
      const double *rsrc;
      if (cycles == 0 && !p.use_x0) {
        rn = bn;
        rsrc = bv;
      } else {
        sigma_column<double, double>(c, p.t64, x, S64, sm, kSmD < 4 * kSigBuf ? kSmD : 4 * kSigBuf);
        double a[1] = {sweep_column<double, double, double, 2, kOutResid>(c, p.t64, p.cm, S64, nullptr, x, bv,
                                                                           S64, false)};
        block_sum<1>(a, red, outb);
        rn = sqrt(a[0]);
        rsrc = S64;
        bpe += 48.0;
      }
      relres = rn / bn;
      if (!(rn == rn) || rn > 1e300) { status = kNonFinite; break; }
      if (relres <= p.tol) { status = kConverged; break; }
      if (cycles >= p.max_outer) { status = kNoConv; break; }
      for (int64_t k = threadIdx.x; k < n; k += blockDim.x) Vo[k] = rsrc[k] / rn;
      __syncthreads();
      bpe += 16.0;
      if (threadIdx.x == 0) go[0] = rn;
      int idone = 0;
      for (int i = 0; i < kout; ++i) {
        // ---- inner: one float32 GMRES(m_in) cycle, z_i ~ A^-1 v_i -----------
        const double *vi = Vo + (int64_t)i * ldv;
        float *zi = Z + (int64_t)i * ldv;
        double a0[1] = {0.0};
        for (int64_t k = threadIdx.x; k < n; k += blockDim.x) a0[0] += vi[k] * vi[k];
        block_sum<1>(a0, red, outb);
        const double beta = sqrt(a0[0]);
        {
          const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
          for (int64_t q = threadIdx.x; q < ldv / 4; q += blockDim.x) {
            float f[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) f[t] = 4 * q + t < n ? narrow_f32(vi[4 * q + t] * inv) : 0.f;
            st_h4(U + 4 * q, f);
          }
          __syncthreads();
        }
        bpe += 8.0 + 8.0 + 2.0;
        if (threadIdx.x == 0) gi[0] = beta;
        int jdone = 0;
        for (int j = 0; j < m_in; ++j) {
          const __half *uj = U + (int64_t)j * ldv;
          if (h16)
            sigma_column_h16(c, p.t32, uj, S32, reinterpret_cast<unsigned char *>(sm),
                             rw_c ? rw_c : p.t32.RwT + c.r_off, uw_c, ul_c, lr_c);
          else
            sigma_column<float, __half>(c, p.t32, uj, S32, reinterpret_cast<float *>(sm),
                                        2 * kSmD < 8 * kSigBuf ? 2 * kSmD : 8 * kSigBuf, rw_c);
          // Arnoldi on K = Lambda Sigma (A = Id - K, same Krylov space): the
          // sweep emits K u_j and needs no read of u_j
          sweep_column<float, __half, float, 4, kOutI>(c, p.t32, p.cm, S32, nullptr, uj, nullptr, W32, false);
          __syncthreads();
          bpe += 14.0;
          const double hn = arnoldi16(U, ldv, j, W32, n, h, h2, hf32, red, outb, bpe);
          if (threadIdx.x == 0) givens_step(Hi, m_in + 1, csi, sni, gi, j, h, h2, hn, s_val, -1.0, 1.0);
          __syncthreads();
          const double est = s_val[0], den = s_val[1];
          jdone = j + 1;
          if (den == 0.0) { jdone = j; break; }
          if (!(hn > 1e-30 * beta)) break;
          if (!(est == est) || est <= p.tol_inner * beta) break;
        }
        inner_total += jdone;
        tri_solve(Hi, m_in + 1, gi, jdone, ybuf);
        stage_coef<float>(ybuf, jdone, 1.0, hf32);
        for (int64_t q0 = threadIdx.x; q0 < ldv / 4; q0 += (int64_t)kQ * blockDim.x) {
          int64_t qc[kQ];
          float d[kQ][4];
#pragma unroll
          for (int e = 0; e < kQ; ++e) {
            qc[e] = min(q0 + (int64_t)e * blockDim.x, ldv / 4 - 1);
#pragma unroll
            for (int t = 0; t < 4; ++t) d[e][t] = 0.f;
          }
          axpy16(U, ldv, jdone, hf32, qc, d);
#pragma unroll
          for (int e = 0; e < kQ; ++e)
            if (q0 + (int64_t)e * blockDim.x < ldv / 4)
              *reinterpret_cast<float4 *>(zi + 4 * qc[e]) = make_float4(d[e][0], d[e][1], d[e][2], d[e][3]);
        }
        __syncthreads();
        bpe += 2.0 * jdone + 4.0;
        // ---- outer: w = A z_i - v_i in float64, orthogonalised in float64 ---
        // (z_i nearly solves A z = v_i, so A z_i keeps most of v_i and its
        // projection cancels; the difference -- the inner residual -- is far
        // from span(V), one Gram-Schmidt pass keeps V orthogonal to rounding
        // (projected/original norm >= 0.3 measured), and A's Hessenberg column
        // is e_i + h)
        double *w = Vo + (int64_t)(i + 1) * ldv;
        sigma_column<double, float>(c, p.t64, zi, S64, sm, kSmD < 4 * kSigBuf ? kSmD : 4 * kSigBuf);
        sweep_column<double, float, double, 2, kOutAminusB>(c, p.t64, p.cm, S64, nullptr, zi, vi, w, false);
        __syncthreads();
        bpe += 4.0 + 8.0 + 8.0 + 4.0 + 8.0 + 8.0;
        const double hn = arnoldi_orth<double>(Vo, ldv, i, n, h, h2, hf64, red, outb, bpe, 0.05);
        if (threadIdx.x == 0) givens_step(Ho, kout + 1, cso, sno, go, i, h, h2, hn, s_val, 1.0, 1.0);
        __syncthreads();
        const double est = s_val[0], den = s_val[1];
        idone = i + 1;
        if (den == 0.0) { idone = i; break; }
        if (!(hn > 1e-300 * rn)) break;
        if (!(est == est) || est <= 0.3 * p.tol * bn) break;
      }
      outer_total += idone;
      // ---- x += Z y ----------------------------------------------------------
      tri_solve(Ho, kout + 1, go, idone, ybuf);
      for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        double acc = x[k];
        for (int i = 0; i < idone; ++i) acc = fma(ybuf[i], widen_f64(Z[(int64_t)i * ldv + k]), acc);
        x[k] = acc;
      }
      __syncthreads();
      bpe += 4.0 * idone + 16.0;
      if (idone == 0) { status = kBreakdown; break; }
    }
    if (threadIdx.x == 0) {
      p.out.outer[inst] = outer_total;
      p.out.inner[inst] = inner_total;
      p.out.status[inst] = status;
      p.out.relres[inst] = relres;
      p.out.bytes[inst] = bpe * (double)n;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------- BiCGStab
// BiCGStab (van der Vorst), float64 vectors and the float64 operator, one CTA
// per (column, rhs) instance as k_solve.  Per iteration two operator
// applications and four fused vector passes:
//   p = r + beta (p - omega v)            (bicg_dir)
//   v = A p;  alpha = rho / (r^, v)
//   s = r - alpha v, ||s||^2              (bicg_s)
//   t = A s;  omega = (t, s) / (t, t)
//   x += alpha p + omega s; r = s - omega t; ||r||^2 and (r^, r)  (bicg_xr)
// Convergence is declared only on the true residual b - A x; when the
// recursive residual has drifted, or rho / (r^, v) / omega break down, the
// iteration restarts from the true residual (at most max_outer times).
// Every loop handles kU elements per thread with all loads issued first.
__device__ __noinline__ void bicg_dir(double *__restrict__ p, const double *__restrict__ r,
                                      const double *__restrict__ v, double beta, double omega, int64_t n) {
  for (int64_t k0 = threadIdx.x; k0 < n; k0 += (int64_t)kU * blockDim.x) {
    double a[kU], b[kU], c[kU];
#pragma unroll
    for (int e = 0; e < kU; ++e) {
      const int64_t k = k0 + (int64_t)e * blockDim.x;
      const bool in = k < n;
      a[e] = in ? r[k] : 0.0;
      b[e] = in ? p[k] : 0.0;
      c[e] = in ? v[k] : 0.0;
    }
#pragma unroll
    for (int e = 0; e < kU; ++e) {
      const int64_t k = k0 + (int64_t)e * blockDim.x;
      if (k < n) p[k] = a[e] + beta * (b[e] - omega * c[e]);
    }
  }
  __syncthreads();
}

// (a, b) and, when c is given, (c, d), float64 block sums
__device__ __noinline__ void bicg_dots(const double *__restrict__ a, const double *__restrict__ b,
                                       const double *__restrict__ c, const double *__restrict__ d, int64_t n,
                                       double *red, double *outb, double &ab, double &cd) {
  double acc[2] = {0.0, 0.0};
  for (int64_t k0 = threadIdx.x; k0 < n; k0 += (int64_t)kU * blockDim.x) {
    double x0[kU], x1[kU], y0[kU], y1[kU];
#pragma unroll
    for (int e = 0; e < kU; ++e) {
      const int64_t k = k0 + (int64_t)e * blockDim.x;
      const bool in = k < n;
      x0[e] = in ? a[k] : 0.0;
      x1[e] = in ? b[k] : 0.0;
      y0[e] = in && c ? c[k] : 0.0;
      y1[e] = in && c ? d[k] : 0.0;
    }
#pragma unroll
    for (int e = 0; e < kU; ++e) {
      acc[0] = fma(x0[e], x1[e], acc[0]);
      acc[1] = fma(y0[e], y1[e], acc[1]);
    }
  }
  block_sum<2>(acc, red, outb);
  ab = acc[0];
  cd = acc[1];
}

// s = r - alpha v; returns ||s||^2
__device__ __noinline__ double bicg_s(double *__restrict__ s, const double *__restrict__ r,
                                      const double *__restrict__ v, double alpha, int64_t n, double *red,
                                      double *outb) {
  double acc[1] = {0.0};
  for (int64_t k0 = threadIdx.x; k0 < n; k0 += (int64_t)kU * blockDim.x) {
    double a[kU], c[kU];
#pragma unroll
    for (int e = 0; e < kU; ++e) {
      const int64_t k = k0 + (int64_t)e * blockDim.x;
      const bool in = k < n;
      a[e] = in ? r[k] : 0.0;
      c[e] = in ? v[k] : 0.0;
    }
#pragma unroll
    for (int e = 0; e < kU; ++e) {
      const int64_t k = k0 + (int64_t)e * blockDim.x;
      const double sv = a[e] - alpha * c[e];
      if (k < n) s[k] = sv;
      acc[0] = fma(sv, sv, acc[0]);
    }
  }
  block_sum<1>(acc, red, outb);
  return acc[0];
}

// x += alpha p + omega s (p only when s is null); r = s - omega t (when t is
// given) with ||r||^2 and (r^, r) returned through rr, rhr
__device__ __noinline__ void bicg_xr(double *__restrict__ x, const double *__restrict__ p,
                                     const double *__restrict__ s, const double *__restrict__ t,
                                     double *__restrict__ r, const double *__restrict__ rh, double alpha,
                                     double omega, int64_t n, double *red, double *outb, double &rr,
                                     double &rhr) {
  double acc[2] = {0.0, 0.0};
  for (int64_t k0 = threadIdx.x; k0 < n; k0 += (int64_t)kU * blockDim.x) {
    double xv[kU], pv[kU], sv[kU], tv[kU], hv[kU];
#pragma unroll
    for (int e = 0; e < kU; ++e) {
      const int64_t k = k0 + (int64_t)e * blockDim.x;
      const bool in = k < n;
      xv[e] = in ? x[k] : 0.0;
      pv[e] = in ? p[k] : 0.0;
      sv[e] = in && s ? s[k] : 0.0;
      tv[e] = in && t ? t[k] : 0.0;
      hv[e] = in && t ? rh[k] : 0.0;
    }
#pragma unroll
    for (int e = 0; e < kU; ++e) {
      const int64_t k = k0 + (int64_t)e * blockDim.x;
      if (k < n) x[k] = xv[e] + alpha * pv[e] + omega * sv[e];
      if (t) {
        const double rv = sv[e] - omega * tv[e];
        if (k < n) r[k] = rv;
        acc[0] = fma(rv, rv, acc[0]);
        acc[1] = fma(hv[e], rv, acc[1]);
      }
    }
  }
  block_sum<2>(acc, red, outb);
  rr = acc[0];
  rhr = acc[1];
}

__global__ void __launch_bounds__(kNT, 1) k_solve_bicgstab(SolveParams p) {
  __shared__ double sm[4 * kSigBuf];
  __shared__ double red[(kNT / 32) * (kDots + 1)];
  __shared__ double outb[kDots + 1];
  __shared__ int s_q;
  double *slot = reinterpret_cast<double *>(p.V) + (int64_t)blockIdx.x * p.cap;  // cap in float64 elements
  double *S64 = p.S + (int64_t)blockIdx.x * p.ld;
  for (;;) {
    const int q = next_instance(p.queue, &s_q);
    if (q >= p.n_inst) break;
    const int inst = p.order[q];
    const int ci = inst % p.n_cols, rhs = inst / p.n_cols;
    const ColDev c = p.cm.cols[ci];
    const int64_t n = (int64_t)c.nz * c.nr;
    const int64_t ldv = (n + 31) / 32 * 32;
    double *r = slot, *rh = r + ldv, *pv = rh + ldv, *v = pv + ldv, *sv = v + ldv, *t = sv + ldv;
    const double *bv = p.b + (p.b_shared ? 0 : rhs * p.E) + c.x_off;
    double *x = p.x + rhs * p.E + c.x_off;
    auto apply = [&](const double *X, double *Y) {  // Y = A X, float64
      sigma_column<double, double>(c, p.t64, X, S64, sm, 4 * kSigBuf);
      sweep_column<double, double, double, 2, kOutAminus>(c, p.t64, p.cm, S64, nullptr, X, nullptr, Y, false);
      __syncthreads();
    };
    auto true_resid = [&]() -> double {  // r = b - A x, returns ||r||
      sigma_column<double, double>(c, p.t64, x, S64, sm, 4 * kSigBuf);
      double a[1] = {sweep_column<double, double, double, 2, kOutResid>(c, p.t64, p.cm, S64, nullptr, x, bv, r, false)};
      block_sum<1>(a, red, outb);
      return sqrt(a[0]);
    };
    const double bn = sqrt(cta_norm2(bv, n, red, outb));
    double bpe = 8.0;
    int status = kNoConv, it = 0, restarts = 0;
    double rn;
    if (!p.use_x0) {
      for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        x[k] = 0.0;
        r[k] = bv[k];
      }
      __syncthreads();
      rn = bn;
      bpe += 24.0;
    } else {
      rn = true_resid();
      bpe += 48.0;
    }
    double rho = 0.0, rho_old = 1.0, alpha = 1.0, omega = 1.0;
    auto reset = [&]() {  // shadow residual = current residual, empty search space
      for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        rh[k] = r[k];
        pv[k] = 0.0;
        v[k] = 0.0;
      }
      __syncthreads();
      rho = rn * rn;
      rho_old = alpha = omega = 1.0;
      bpe += 32.0;
    };
    const int max_iter = p.max_iter > 0 ? p.max_iter : 10000;
    const bool bad_b = !(bn == bn) || bn > 1e300;
    if (bad_b) status = kNonFinite;
    else if (bn == 0.0) { status = kConverged; rn = 0.0; }
    else reset();
    bool rn_true = false;  // rn is the true residual norm (not the recursive one)
    while (!bad_b && bn > 0.0) {
      if (!(rn == rn) || rn > 1e300) { status = kNonFinite; break; }
      int restart = 0;  // 1: recursive residual drifted, 2: a coefficient broke down
      if (rn <= p.tol * bn) {  // confirm on the true residual
        rn = true_resid();
        rn_true = true;
        bpe += 48.0;
        if (rn <= p.tol * bn) { status = kConverged; break; }
        restart = 1;
      } else if (it >= max_iter) {
        break;
      } else if (!(rho != 0.0 && rho == rho) || !(omega != 0.0)) {
        rn = true_resid();
        rn_true = true;
        bpe += 48.0;
        restart = 2;
      }
      if (restart) {
        if (restarts >= p.max_outer) { status = restart == 2 ? kBreakdown : kNoConv; break; }
        ++restarts;
        reset();
        continue;
      }
      const double beta = (rho / rho_old) * (alpha / omega);
      bicg_dir(pv, r, v, beta, omega, n);
      apply(pv, v);
      double rv = 0.0, unused = 0.0;
      bicg_dots(rh, v, nullptr, nullptr, n, red, outb, rv, unused);
      bpe += 32.0 + 40.0 + 16.0;
      ++it;
      if (!(rv != 0.0 && rv == rv)) {
        rn = true_resid();
        rn_true = true;
        bpe += 48.0;
        if (rn <= p.tol * bn) { status = kConverged; break; }
        if (restarts >= p.max_outer) { status = kBreakdown; break; }
        ++restarts;
        reset();
        continue;
      }
      alpha = rho / rv;
      const double sn = sqrt(bicg_s(sv, r, v, alpha, n, red, outb));
      bpe += 24.0;
      if (sn <= p.tol * bn) {  // half step: x += alpha p, then the true-residual check
        double d0 = 0.0, d1 = 0.0;
        bicg_xr(x, pv, nullptr, nullptr, nullptr, nullptr, alpha, 0.0, n, red, outb, d0, d1);
        bpe += 24.0;
        rn = sn;
        rn_true = false;
        continue;
      }
      apply(sv, t);
      double ts = 0.0, tt = 0.0;
      bicg_dots(t, sv, t, t, n, red, outb, ts, tt);
      omega = tt > 0.0 ? ts / tt : 0.0;
      double rr = 0.0, rhr = 0.0;
      bicg_xr(x, pv, sv, t, r, rh, alpha, omega, n, red, outb, rr, rhr);
      bpe += 40.0 + 16.0 + 56.0;
      rn = sqrt(rr);
      rn_true = false;
      rho_old = rho;
      rho = rhr;
    }
    if (status != kConverged && status != kNonFinite && !rn_true && bn > 0.0) {  // report the true residual
      rn = true_resid();
      bpe += 48.0;
    }
    if (threadIdx.x == 0) {
      p.out.outer[inst] = restarts;
      p.out.inner[inst] = it;
      p.out.status[inst] = status;
      p.out.relres[inst] = bn > 0.0 ? rn / bn : 0.0;
      p.out.bytes[inst] = bpe * (double)n;
    }
    __syncthreads();
  }
}

int launch_bicgstab(rt_handle *h, const double *b, double *x, double tol, int max_outer, int max_iter,
                    int use_x0, cudaStream_t s) {
  SolveParams p;
  p.cm = Common{h->d_cols, h->d_dir_cls, h->d_dir_up, h->d_tsrc, h->d_Itop, h->d_Ibot};
  p.t64 = tables64(h);
  p.t32 = tables32(h);
  p.order = h->d_order;
  p.n_cols = h->n_cols;
  p.n_inst = h->n_cols * h->n_rhs;
  p.E = h->E;
  p.b = b ? b : h->b_int;
  p.b_shared = b ? 0 : 1;
  p.x = x;
  p.tol = tol;
  p.tol_inner = 0.0;
  p.m = 0;
  p.max_outer = max_outer;
  p.max_iter = max_iter;
  p.use_x0 = use_x0;
  p.V = h->ws.V;
  p.cap = h->ws.cap_bytes / 8;  // float64 elements per slot
  p.m_in = 0;
  p.S = h->ws.S;
  p.ld = h->ws.ld;
  p.H = h->ws.H;
  p.hld = h->ws.hld;
  p.queue = h->d_queue + 1;
  p.out = h->so;
  cudaError_t e = cudaMemsetAsync(h->d_queue + 1, 0, sizeof(int), s);
  if (e != cudaSuccess) return (int)e;
  k_solve_bicgstab<<<h->ws.slots, kNT, 0, s>>>(p);
  return (int)cudaGetLastError();
}

bool bicgstab_fits(const rt_handle *h) { return h->ws.cap_bytes >= 6 * h->ws.ld * 8; }

int launch_solve(rt_handle *h, const double *b, double *x, double tol, double tol_inner, int m,
                 int max_outer, int use_x0, cudaStream_t s, int m_in) {
  SolveParams p;
  p.cm = Common{h->d_cols, h->d_dir_cls, h->d_dir_up, h->d_tsrc, h->d_Itop, h->d_Ibot};
  p.t64 = tables64(h);
  p.t32 = tables32(h);
  p.order = h->d_order;
  p.n_cols = h->n_cols;
  p.n_inst = h->n_cols * h->n_rhs;
  p.E = h->E;
  p.b = b ? b : h->b_int;
  p.b_shared = b ? 0 : 1;
  p.x = x;
  p.tol = tol;
  p.tol_inner = tol_inner;
  p.m = m;
  p.max_outer = max_outer;
  p.use_x0 = use_x0;
  p.V = h->ws.V;
  p.cap = h->precision == 0 ? h->ws.cap_bytes / 8 : h->ws.cap_bytes;
  p.m_in = m_in;
  p.max_iter = 0;
  p.S = h->ws.S;
  p.ld = h->ws.ld;
  p.H = h->ws.H;
  p.hld = h->ws.hld;
  p.queue = h->d_queue + 1;
  p.out = h->so;
  cudaError_t e = cudaMemsetAsync(h->d_queue + 1, 0, sizeof(int), s);
  if (e != cudaSuccess) return (int)e;
  if (h->precision == 0) k_solve<double><<<h->ws.slots, kNT, 0, s>>>(p);
  else if (h->ws.per_sm == 2) k_solve_nested<256><<<h->ws.slots, 256, 0, s>>>(p);
  else k_solve_nested<512><<<h->ws.slots, 512, 0, s>>>(p);
  return (int)cudaGetLastError();
}

int max_krylov() { return kMaxM; }

}  // namespace rt
