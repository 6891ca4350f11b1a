// rt_box.cu -- 3D boxes (Sec. 3.4): the scattering contraction and the
// short-characteristics formal solution between consecutive z-planes,
// periodic in x and y, with bilinear interpolation of I, S and chi at the
// upwind point (the interpolation operators T_RC, T_CR of Sec. 3.4, rows
// summing to one).
//
// Data layout of the apply.  x and y keep the space-based ordering of
// Sec. 3.1 (point, direction, frequency fastest).  The source function S
// between the two kernels is internal scratch and is written by the Sigma
// kernel in the layout the sweep streams: [direction][frequency block][point]
// [FB frequencies], so one sweep CTA reads one contiguous run per plane.  The
// opacity is stored in blocks of 4 frequencies: [f / 4][point][f % 4].
//
//   k_sigma_box : one warp per point, S = Gamma (factored P (x) R) X
//                 (eq. Sigma) -- angular moments, frequency kernel, expansion
//   k_sweep3d   : one CTA per (direction, block of FB frequencies) marches
//                 the planes.  The previous plane's I, S and chi live in
//                 shared memory (FB values per cell); each thread owns CPT
//                 cells, loads their current-plane S, chi and x in batches
//                 of CB cells, interpolates the upwind values from shared
//                 memory, steps the recurrence and writes y; the new plane
//                 replaces the old one between two barriers.
// The float32 step coefficients use e = exp(-d) (fast exponential), and for
// d < 0.5 the series of 1 - e^-d and of w1/d (no cancellation); the float64
// ones use exp, expm1 and the series of w1/d below 0.1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

#include "rt_host.h"
#include "rt_internal.cuh"

namespace rt {

template <typename T, int FB>
struct alignas(sizeof(T) * FB) Pack {
  T v[FB];
};

// casts between the vector and arithmetic types, without float64 cvt
template <typename T, typename X> __device__ __forceinline__ T cast_to(X v) { return (T)v; }
template <> __device__ __forceinline__ float cast_to<float, double>(double v) { return narrow_f32(v); }
template <> __device__ __forceinline__ double cast_to<double, float>(float v) { return widen_f64(v); }

// ------------------------------------------------------------ coefficients
template <typename T>
__device__ __forceinline__ void step_coef(T d, int ie, T &e, T &a, T &b);

template <>
__device__ __forceinline__ void step_coef<float>(float d, int ie, float &e, float &a, float &b) {
  if (ie) {
    e = __fdividef(1.f, 1.f + d);
    a = 0.f;
    b = d * e;
    return;
  }
  e = __expf(-d);
  float w0, beta;
  if (d < 0.5f) {
    // series, no cancellation: 1 - e^-d = d (1 - d/2 (1 - d/3 (...))) and
    // w1/d = (d/2)(1 - (d/3)(1 - (d/4)(...))), 8 factors each (the first
    // dropped terms, d^8/9! and 2 d^8/10!, stay below 1.1e-8 for d < 0.5)
    float s0 = 1.f, s1 = 1.f;
#pragma unroll
    for (int j = 9; j >= 2; --j) s0 = 1.f - d * (1.f / (float)j) * s0;
#pragma unroll
    for (int j = 10; j >= 3; --j) s1 = 1.f - d * (1.f / (float)j) * s1;
    w0 = d * s0;
    beta = 0.5f * d * s1;
  } else {
    w0 = 1.f - e;
    beta = 1.f - __fdividef(w0, d);
  }
  b = beta;
  a = w0 - beta;
}

template <>
__device__ __forceinline__ void step_coef<double>(double d, int ie, double &e, double &a, double &b) {
  if (ie) {
    e = 1.0 / (1.0 + d);
    a = 0.0;
    b = d * e;
    return;
  }
  e = exp(-d);
  const double w0 = -expm1(-d);
  double beta;
  if (d < 0.1) {
    // w1/d = (d/2)(1 - (d/3)(1 - (d/4)(1 - ...))): 16 factors
    double s = 1.0;
#pragma unroll
    for (int j = 17; j >= 3; --j) s = 1.0 - d * (1.0 / j) * s;
    beta = 0.5 * d * s;
  } else {
    beta = (d - w0) / d;
  }
  b = beta;
  a = w0 - beta;
}

// Quadratic short-characteristics step (Sec. 5.3 integrator): S is the
// parabola through the upwind, current and downwind points, at optical path
// -du, 0 and +dd from the current point, integrated exactly against the
// attenuation:  I_c = e I_u + pu S_u + pc S_c + pd S_d  with the moments
// W1 = du - w0 and W2 = du^2 - 2 W1 taken as a = W1 / du^2 and
// m = a - W2 / du^3 = (W1 (du + 2) - du^2) / du^3:
//   pc = du a + du^2 m / dd,  pd = -du^3 m / (dd (du + dd)),
//   pu = w0 - du a - du^2 m / (du + dd)      (the three sum to w0).
// Below the cut a and m come from their series, a = sum (-du)^k / (k+2)! and
// m = sum (-du)^k (k+1) / (k+3)!, which do not cancel.
template <typename T>
__device__ __forceinline__ void qsc_coef(T du, T dd, T &e, T &pu, T &pc, T &pd);

template <>
__device__ __forceinline__ void qsc_coef<float>(float du, float dd, float &e, float &pu, float &pc, float &pd) {
  e = __expf(-du);
  float w0, a, m;
  if (du < 0.5f) {
    // 8 terms each: the first dropped ones, du^8/10! and 9 du^8/11!, stay below 1.2e-9
    float s0 = 1.f;
#pragma unroll
    for (int j = 9; j >= 2; --j) s0 = 1.f - du * (1.f / (float)j) * s0;
    w0 = du * s0;
    a = 0.f, m = 0.f;
    float ik = 1.f / 362880.f;  // 1/(k+2)! at k = 7
#pragma unroll
    for (int k = 7; k >= 0; --k) {
      a = fmaf(-du, a, ik);
      m = fmaf(-du, m, ik * (float)(k + 1) / (float)(k + 3));
      ik *= (float)(k + 2);
    }
  } else {
    w0 = 1.f - e;
    const float w1 = du - w0;
    const float r = 1.f / du;
    a = w1 * r * r;
    m = (w1 * (du + 2.f) - du * du) * r * r * r;
  }
  const float q = du * du * m;
  pc = du * a + q / dd;
  pd = -q * du / (dd * (du + dd));
  pu = w0 - du * a - q / (du + dd);
}

template <>
__device__ __forceinline__ void qsc_coef<double>(double du, double dd, double &e, double &pu, double &pc,
                                                 double &pd) {
  e = exp(-du);
  const double w0 = -expm1(-du);
  double a, m;
  if (du < 0.1) {
    // 18 terms each
    a = 0.0, m = 0.0;
    double ik = 1.0 / 121645100408832000.0;  // 1/(k+2)! at k = 17 (1/19!)
#pragma unroll
    for (int k = 17; k >= 0; --k) {
      a = fma(-du, a, ik);
      m = fma(-du, m, ik * (double)(k + 1) / (double)(k + 3));  // (k+1)/(k+3)!
      ik *= (double)(k + 2);
    }
  } else {
    const double w1 = du - w0;
    a = w1 / (du * du);
    m = (w1 * (du + 2.0) - du * du) / (du * du * du);
  }
  const double q = du * du * m;
  pc = du * a + q / dd;
  pd = -q * du / (dd * (du + dd));
  pu = w0 - du * a - q / (du + dd);
}

// ------------------------------------------------------------------ Sigma
constexpr int kBoxSigNT = 256;     // threads per Sigma CTA (8 warps, one point each)
constexpr int kBoxRwCache = 32768;  // bytes of frequency kernel staged in shared memory (else global)

// Index of (point p, direction d, frequency f) in the sweep layout
// [d][f / FB][p][f % FB]; fb_out == 0 selects the space-based layout.
__device__ __forceinline__ int64_t box_out_index(int64_t p, int d, int f, int nn, int nr, int64_t npts, int fb_out,
                                                 int nfb) {
  if (fb_out == 0) return p * nr + (int64_t)d * nn + f;
  const int fb = f / fb_out;
  return (((int64_t)d * nfb + fb) * npts + p) * fb_out + (f - fb * fb_out);
}

// Separable kernel: one warp per point (grid-stride).  Lane l owns the
// frequencies l, l + 32, ..., FL of them, and keeps their KR >= rank moments
// and frequency-kernel outputs in registers through the three stages, so a
// shared-memory load of a factor entry feeds FL FMAs.  Shared memory: Uw | Ul
// (nd * KR each, zero past the rank), the frequency kernel RwT when it fits
// kBoxRwCache, and per warp the moments (KR * nn) that stage 2 broadcasts.
template <typename T, typename TX, int KR, int FL>
__global__ void __launch_bounds__(kBoxSigNT) k_sigma_box(ColDev c, Tables<T> tb, int64_t npts, const TX *__restrict__ X,
                                                         T *__restrict__ S, int fb_out) {
  extern __shared__ __align__(16) unsigned char sig_smem[];
  const int nd = c.nd, nn = c.nn, nr = c.nr, rp = c.rp;
  const int nfb = fb_out ? (nn + fb_out - 1) / fb_out : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T *sUw = reinterpret_cast<T *>(sig_smem);
  T *sUl = sUw + nd * KR;
  T *sRw = sUl + nd * KR;
  const bool rw_cached = !c.rdiag && (int64_t)nn * nn * sizeof(T) <= kBoxRwCache;
  const int rw_len = c.rdiag ? nn : (rw_cached ? nn * nn : 0);
  T *wm = sRw + ((rw_len + 1) & ~1) + (int64_t)warp * KR * nn;
  for (int i = threadIdx.x; i < nd * KR; i += blockDim.x) {
    const int d = i / KR, k = i - d * KR;
    sUw[i] = k < rp ? tb.Uw[c.u_off + d * rp + k] : T(0);
    sUl[i] = k < rp ? tb.Ul[c.u_off + d * rp + k] : T(0);
  }
  for (int i = threadIdx.x; i < rw_len; i += blockDim.x) sRw[i] = tb.RwT[c.r_off + i];
  __syncthreads();
  const T *Rw = (c.rdiag || rw_cached) ? sRw : tb.RwT + c.r_off;
  const T *gam = tb.gamma + c.g_off;
  int fl[FL];
  bool on[FL];
#pragma unroll
  for (int j = 0; j < FL; ++j) {
    on[j] = lane + 32 * j < nn;
    fl[j] = on[j] ? lane + 32 * j : 0;
  }
  for (int64_t p = (int64_t)blockIdx.x * nw + warp; p < npts; p += (int64_t)gridDim.x * nw) {
    const TX *xp = X + p * nr;
    // 1. moments m_k(f) = sum_d Uw[d][k] X(d, f)
    T m[FL][KR];
#pragma unroll
    for (int j = 0; j < FL; ++j)
#pragma unroll
      for (int k = 0; k < KR; ++k) m[j][k] = 0;
    int d = 0;
    constexpr int kDL = FL <= 2 ? 8 : 4;  // directions whose loads are issued together
    for (; d + kDL <= nd; d += kDL) {
      T xv[kDL][FL];
#pragma unroll
      for (int e = 0; e < kDL; ++e)
#pragma unroll
        for (int j = 0; j < FL; ++j) xv[e][j] = on[j] ? cast_to<T>(xp[(d + e) * nn + fl[j]]) : T(0);
#pragma unroll
      for (int e = 0; e < kDL; ++e) {
        const T *u = sUw + (d + e) * KR;
#pragma unroll
        for (int k = 0; k < KR; ++k) {
          const T uk = u[k];
#pragma unroll
          for (int j = 0; j < FL; ++j) m[j][k] = fma(uk, xv[e][j], m[j][k]);
        }
      }
    }
    for (; d < nd; ++d) {
      const T *u = sUw + d * KR;
#pragma unroll
      for (int j = 0; j < FL; ++j) {
        const T xv = on[j] ? cast_to<T>(xp[d * nn + fl[j]]) : T(0);
#pragma unroll
        for (int k = 0; k < KR; ++k) m[j][k] = fma(u[k], xv, m[j][k]);
      }
    }
    // 2. frequency kernel z_k(f) = sum_q RwT[q][f] m_k(q)
    T z[FL][KR];
    if (c.rdiag) {
#pragma unroll
      for (int j = 0; j < FL; ++j)
#pragma unroll
        for (int k = 0; k < KR; ++k) z[j][k] = Rw[fl[j]] * m[j][k];
    } else {
#pragma unroll
      for (int j = 0; j < FL; ++j)
        if (on[j]) {
#pragma unroll
          for (int k = 0; k < KR; ++k) wm[k * nn + fl[j]] = m[j][k];
        }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < FL; ++j)
#pragma unroll
        for (int k = 0; k < KR; ++k) z[j][k] = 0;
      for (int q = 0; q < nn; ++q) {
        T mq[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) mq[k] = wm[k * nn + q];
#pragma unroll
        for (int j = 0; j < FL; ++j) {
          const T r = Rw[q * nn + fl[j]];
#pragma unroll
          for (int k = 0; k < KR; ++k) z[j][k] = fma(r, mq[k], z[j][k]);
        }
      }
      __syncwarp();
    }
    // 3. expansion S(d, f) = gamma(f) sum_k Ul[d][k] z_k(f)
    T gf[FL];
#pragma unroll
    for (int j = 0; j < FL; ++j) {
      gf[j] = gam[p * nn + fl[j]];
#pragma unroll
      for (int k = 0; k < KR; ++k) z[j][k] *= gf[j];
    }
    for (int dd = 0; dd < nd; ++dd) {
      const T *u = sUl + dd * KR;
      T acc[FL];
#pragma unroll
      for (int j = 0; j < FL; ++j) acc[j] = 0;
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const T uk = u[k];
#pragma unroll
        for (int j = 0; j < FL; ++j) acc[j] = fma(uk, z[j][k], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < FL; ++j)
        if (on[j]) S[box_out_index(p, dd, fl[j], nn, nr, npts, fb_out, nfb)] = acc[j];
    }
  }
}

// Four consecutive values of a float32 / float64 array (16-byte aligned).
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  static __device__ __forceinline__ void ld(const float *p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
  }
  static __device__ __forceinline__ void st(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Vec4<double> {
  static __device__ __forceinline__ void ld(const double *p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
  static __device__ __forceinline__ void st(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
  }
};

// Separable kernel, sweep-layout output with FBO in {1, 2, 4} frequencies per
// block and nn a multiple of 4: LP lanes per point, each owning 4 consecutive
// frequencies (16- or 32-byte loads of X, one vector load of the frequency
// kernel row per q), 32 / LP consecutive points per warp, so the points'
// FBO-value runs of one (direction, block) are adjacent in the output and a
// warp's store fills whole sectors.  Output offsets are formed once per point
// (no division per store).  Same stages and shared memory as k_sigma_box.
template <typename T, typename TX, int KR, int LP, int FBO>
__global__ void __launch_bounds__(kBoxSigNT) k_sigma_box4(ColDev c, Tables<T> tb, int64_t npts,
                                                          const TX *__restrict__ X, T *__restrict__ S,
                                                          T *__restrict__ XS) {
  extern __shared__ __align__(16) unsigned char sig_smem[];
  constexpr int PPW = 32 / LP;
  const int nd = c.nd, nn = c.nn, nr = c.nr, rp = c.rp;
  const int nfb = nn / FBO;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ps = lane / LP, f0 = 4 * (lane % LP);
  const bool on = f0 < nn;
  T *sUw = reinterpret_cast<T *>(sig_smem);
  T *sUl = sUw + nd * KR;
  T *sRw = sUl + nd * KR;
  const bool rw_cached = !c.rdiag && (int64_t)nn * nn * sizeof(T) <= kBoxRwCache;
  const int rw_len = c.rdiag ? nn : (rw_cached ? nn * nn : 0);
  const int wstride = KR * nn + 4;  // per point of a warp: moments, offset so points hit other banks
  T *wm = sRw + ((rw_len + 3) & ~3) + (int64_t)warp * PPW * wstride + ps * wstride;
  for (int i = threadIdx.x; i < nd * KR; i += blockDim.x) {
    const int d = i / KR, k = i - d * KR;
    sUw[i] = k < rp ? tb.Uw[c.u_off + d * rp + k] : T(0);
    sUl[i] = k < rp ? tb.Ul[c.u_off + d * rp + k] : T(0);
  }
  for (int i = threadIdx.x; i < rw_len; i += blockDim.x) sRw[i] = tb.RwT[c.r_off + i];
  __syncthreads();
  const T *Rw = (c.rdiag || rw_cached) ? sRw : tb.RwT + c.r_off;
  const T *gam = tb.gamma + c.g_off;
  const int64_t dstride = (int64_t)nfb * npts * FBO;  // output stride of one direction
  for (int64_t p0 = ((int64_t)blockIdx.x * nw + warp) * PPW; p0 < npts; p0 += (int64_t)gridDim.x * nw * PPW) {
    const int64_t p = p0 + ps;
    const bool act = on && p < npts;
    const TX *xp = X + p * nr + f0;
    const int64_t obase = ((int64_t)(f0 / FBO) * npts + p) * FBO;  // direction 0, first block of this lane
    const int64_t bstride = npts * FBO;                            // next frequency block
    // X in the sweep's layout and precision, for the sweep's y = x - I
    auto put_x = [&](int dd, const TX (&v)[4]) {
      T t[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) t[j] = cast_to<T>(v[j]);
      T *o = XS + obase + (int64_t)dd * dstride;
      if (FBO == 4) {
        Vec4<T>::st(o, t);
      } else if (FBO == 2) {
        o[0] = t[0], o[1] = t[1];
        o[bstride] = t[2], o[bstride + 1] = t[3];
      } else {
        o[0] = t[0], o[bstride] = t[1], o[2 * bstride] = t[2], o[3 * bstride] = t[3];
      }
    };
    // 1. moments m_k(f) = sum_d Uw[d][k] X(d, f)
    T m[4][KR];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < KR; ++k) m[j][k] = 0;
    constexpr int kDL = 4;  // directions whose loads are issued together
    int d = 0;
    for (; d + kDL <= nd; d += kDL) {
      TX xv[kDL][4];
#pragma unroll
      for (int e = 0; e < kDL; ++e) {
        if (act) {
          Vec4<TX>::ld(xp + (int64_t)(d + e) * nn, xv[e]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) xv[e][j] = TX(0);
        }
      }
      if (XS && act) {
#pragma unroll
        for (int e = 0; e < kDL; ++e) put_x(d + e, xv[e]);
      }
#pragma unroll
      for (int e = 0; e < kDL; ++e) {
        const T *u = sUw + (d + e) * KR;
        T xt[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) xt[j] = cast_to<T>(xv[e][j]);
#pragma unroll
        for (int k = 0; k < KR; ++k) {
          const T uk = u[k];
#pragma unroll
          for (int j = 0; j < 4; ++j) m[j][k] = fma(uk, xt[j], m[j][k]);
        }
      }
    }
    for (; d < nd; ++d) {
      TX xv[4] = {TX(0), TX(0), TX(0), TX(0)};
      if (act) Vec4<TX>::ld(xp + (int64_t)d * nn, xv);
      if (XS && act) put_x(d, xv);
      const T *u = sUw + d * KR;
#pragma unroll
      for (int k = 0; k < KR; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) m[j][k] = fma(u[k], cast_to<T>(xv[j]), m[j][k]);
    }
    // 2. frequency kernel z_k(f) = sum_q RwT[q][f] m_k(q)
    T z[4][KR];
    if (c.rdiag) {
      T r[4] = {T(0), T(0), T(0), T(0)};
      if (on) Vec4<T>::ld(Rw + f0, r);
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < KR; ++k) z[j][k] = r[j] * m[j][k];
    } else {
      if (on) {
#pragma unroll
        for (int k = 0; k < KR; ++k) {
          const T v[4] = {m[0][k], m[1][k], m[2][k], m[3][k]};
          Vec4<T>::st(wm + k * nn + f0, v);
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < KR; ++k) z[j][k] = 0;
      if (on) {
        for (int q = 0; q < nn; ++q) {
          T r[4];
          Vec4<T>::ld(Rw + (int64_t)q * nn + f0, r);
#pragma unroll
          for (int k = 0; k < KR; ++k) {
            const T mq = wm[k * nn + q];
#pragma unroll
            for (int j = 0; j < 4; ++j) z[j][k] = fma(r[j], mq, z[j][k]);
          }
        }
      }
      __syncwarp();
    }
    if (!act) continue;
    // 3. expansion S(d, f) = gamma(f) sum_k Ul[d][k] z_k(f), into the blocks
    //    of FBO frequencies: f0 / FBO .. (f0 + 3) / FBO
    T g[4];
    Vec4<T>::ld(gam + p * nn + f0, g);
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < KR; ++k) z[j][k] *= g[j];
    T *out = S + obase;
    for (int dd = 0; dd < nd; ++dd, out += dstride) {
      const T *u = sUl + dd * KR;
      T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const T uk = u[k];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] = fma(uk, z[j][k], acc[j]);
      }
      if (FBO == 4) {
        Vec4<T>::st(out, acc);
      } else if (FBO == 2) {
        out[0] = acc[0], out[1] = acc[1];
        out[bstride] = acc[2], out[bstride + 1] = acc[3];
      } else {
        out[0] = acc[0], out[bstride] = acc[1], out[2 * bstride] = acc[2], out[3 * bstride] = acc[3];
      }
    }
  }
}

// Dense kernel Psi (n_r x n_r): S(p, r) = gamma sum_q PsiwT[q][r] X(p, q),
// lanes over r, one warp per point (small problems only).
template <typename T, typename TX>
__global__ void __launch_bounds__(kBoxSigNT) k_sigma_box_dense(ColDev c, Tables<T> tb, int64_t npts,
                                                               const TX *__restrict__ X, T *__restrict__ S,
                                                               int fb_out) {
  const int nn = c.nn, nr = c.nr;
  const int nfb = fb_out ? (nn + fb_out - 1) / fb_out : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T *Pw = tb.PsiwT + c.psi_off;
  const T *gam = tb.gamma + c.g_off;
  for (int64_t p = (int64_t)blockIdx.x * nw + warp; p < npts; p += (int64_t)gridDim.x * nw) {
    const TX *xp = X + p * nr;
    for (int r = lane; r < nr; r += 32) {
      T acc = 0;
      for (int q = 0; q < nr; ++q) acc = fma(Pw[(int64_t)q * nr + r], cast_to<T>(xp[q]), acc);
      const int d = r / nn, f = r - d * nn;
      S[box_out_index(p, d, f, nn, nr, npts, fb_out, nfb)] = gam[p * nn + f] * acc;
    }
  }
}

// x (space-based layout, float64) -> the sweep layout in T (Lambda x alone)
// (one CTA per point, threads over its rays)
template <typename T>
__global__ void k_box_to_sweep(const double *__restrict__ x, T *__restrict__ S, int64_t npts, int nd, int nn,
                               int fb) {
  const int nfb = (nn + fb - 1) / fb, nr = nd * nn;
  for (int64_t p = blockIdx.x; p < npts; p += gridDim.x)
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const int d = r / nn, f = r - d * nn;
      S[box_out_index(p, d, f, nn, nr, npts, fb, nfb)] = cast_to<T>(x[p * nr + r]);
    }
}

// sweep layout T -> space-based float64 (Sigma x alone)
template <typename T>
__global__ void k_box_from_sweep(const T *__restrict__ S, double *__restrict__ y, int64_t npts, int nd, int nn,
                                 int fb) {
  const int nfb = (nn + fb - 1) / fb, nr = nd * nn;
  for (int64_t p = blockIdx.x; p < npts; p += gridDim.x)
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const int d = r / nn, f = r - d * nn;
      y[p * nr + r] = cast_to<double>(S[box_out_index(p, d, f, nn, nr, npts, fb, nfb)]);
    }
}

// ------------------------------------------------------------------ sweep
// geo per direction (6 doubles): fx, fy (integer upwind shift in cells,
// reduced modulo nx, ny: the box is periodic), ax, ay (fractional parts),
// ds (path length between planes), up (1: Omega_z > 0).
// chiN: opacity [npad / 4][npts][4] (npad = nn rounded up to 4, zero past nn),
// so a CTA's FB <= 4 frequencies of consecutive cells are contiguous.
// SL: source in the sweep layout, or null when the source is the thermal
// term tsrc [npts][nn] (float64) broadcast over directions.
// x, y: space-based layout; x unused for kOutI.
// MODE: how the step weights are formed.  kSwChi: from the opacity chiN
// (interpolated at the upwind point); kSwPre: precomputed (1 - e^-d, w1/d)
// in cW0, cB (float64 boxes); kSwKap: the opacity is kappa(p) phi(nu)
// (detected at creation), so shared memory holds one kappa per cell (kap)
// instead of FB opacities and d = ds/2 phi (kappa_u + kappa_c); kSwQsc:
// quadratic short characteristics, the opacity as kSwChi, plus S and chi
// at the downwind point (the upwind stencil mirrored, in the next plane,
// gathered from global memory: that plane is not in shared memory) and the
// qsc_coef weights; the last plane of the sweep takes the linear step.
enum { kSwChi = 0, kSwPre = 1, kSwKap = 2, kSwQsc = 3, kSwLc = 4 };

template <typename T, int FB, int CPT, int CB, typename TX, typename TY, int MODE>
__global__ void __launch_bounds__(512) k_sweep3d(BoxDev bx, const double *__restrict__ geo,
                                                 const T *__restrict__ chiN, int npad,
                                                 const Pack<T, FB> *__restrict__ SL,
                                                 const double *__restrict__ tsrc, const TX *__restrict__ x,
                                                 TY *__restrict__ y, int out, int inflow,
                                                 const double *__restrict__ I_top,
                                                 const double *__restrict__ I_bot,
                                                 const T *__restrict__ cW0, const T *__restrict__ cB,
                                                 const T *__restrict__ kap, const T *__restrict__ phi,
                                                 const T *__restrict__ xs) {
  using P = Pack<T, FB>;
  extern __shared__ __align__(16) unsigned char sw_smem[];
  const int nx = bx.nx, ny = bx.ny, nz = bx.nz, nn = bx.nn, nd = bx.nd;
  const int plane = nx * ny;
  const int nfb = (nn + FB - 1) / FB;
  // kSwKap double-buffers I (the new plane's intensity is written as it is
  // computed, so it needs no registers): sI and sIn swap every plane
  constexpr bool dbl = MODE == kSwKap;
  P *sI = reinterpret_cast<P *>(sw_smem);
  P *sIn = dbl ? sI + plane : sI;
  P *const sS = sI + (dbl ? 2 : 1) * plane;
  P *sC = sS + plane;                          // kSwChi: opacity of the previous plane
  T *sK = reinterpret_cast<T *>(sS + plane);   // kSwKap: kappa of the previous plane
  const int d = blockIdx.x / nfb, fb = blockIdx.x - d * nfb, f0 = fb * FB;
  const int64_t npts = (int64_t)plane * nz;
  const int64_t nr = (int64_t)nd * nn;
  const double *g = geo + 6 * d;
  const int fx = (int)g[0], fy = (int)g[1];
  const T ax = (T)g[2], ay = (T)g[3];
  const T hds = (T)(0.5 * g[4]);
  const bool up = g[5] > 0.5;
  const T w00 = ((T)1 - ay) * ((T)1 - ax), w01 = ((T)1 - ay) * ax, w10 = ay * ((T)1 - ax), w11 = ay * ax;
  const int step = up ? -1 : 1, k0 = up ? nz - 1 : 0;
  const P *Sd = SL ? SL + ((int64_t)d * nfb + fb) * npts : nullptr;
  // x already cast to T in the sweep layout (written by the Sigma kernel),
  // or null: x read in the space-based layout
  const P *Xd = xs ? reinterpret_cast<const P *>(xs) + ((int64_t)d * nfb + fb) * npts : nullptr;
  const int ie = bx.ie;
  // this thread's cells and their four upwind neighbours (the shift is the
  // same for every plane), packed two 16-bit cell indices per word
  constexpr bool qsc = MODE == kSwQsc;
  uint32_t nb0[CPT], nb1[CPT];
  uint32_t nd0[qsc ? CPT : 1], nd1[qsc ? CPT : 1];  // kSwQsc: the downwind stencil
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int c = threadIdx.x + i * blockDim.x;
    nb0[i] = nb1[i] = 0;
    if (qsc) nd0[i] = nd1[i] = 0;
    if (c < plane) {
      const int yy = c / nx, xx = c - yy * nx;
      int x0 = xx - fx, y0 = yy - fy;
      if (x0 < 0) x0 += nx;
      if (y0 < 0) y0 += ny;
      const int x1 = x0 == 0 ? nx - 1 : x0 - 1;
      const int y1 = y0 == 0 ? ny - 1 : y0 - 1;
      nb0[i] = (uint32_t)(y0 * nx + x0) | ((uint32_t)(y0 * nx + x1) << 16);
      nb1[i] = (uint32_t)(y1 * nx + x0) | ((uint32_t)(y1 * nx + x1) << 16);
      if (qsc) {
        // the point (xx + fx + ax, yy + fy + ay): cells +0 / +1, same weights
        int u0 = xx + fx, v0 = yy + fy;
        if (u0 >= nx) u0 -= nx;
        if (v0 >= ny) v0 -= ny;
        const int u1 = u0 + 1 == nx ? 0 : u0 + 1;
        const int v1 = v0 + 1 == ny ? 0 : v0 + 1;
        nd0[qsc ? i : 0] = (uint32_t)(v0 * nx + u0) | ((uint32_t)(v0 * nx + u1) << 16);
        nd1[qsc ? i : 0] = (uint32_t)(v1 * nx + u0) | ((uint32_t)(v1 * nx + u1) << 16);
      }
    }
  }
  auto load_src = [&](int64_t p) -> P {
    if (Sd) return Sd[p];
    P r;
#pragma unroll
    for (int j = 0; j < FB; ++j) r.v[j] = f0 + j < nn ? cast_to<T>(tsrc[p * nn + f0 + j]) : T(0);
    return r;
  };
  const T *chiB = chiN + (int64_t)(f0 >> 2) * npts * 4 + (f0 & 3);
  auto load_chi = [&](int64_t p) -> P { return *reinterpret_cast<const P *>(chiB + p * 4); };
  // precomputed step weights (1 - e^-d, w1/d) in blocks of 2 frequencies:
  // [d][f / 2][p][f % 2]; the plane's opacity is then not needed
  constexpr bool pre = MODE == kSwPre;
  const int64_t cbase = pre ? ((int64_t)d * ((nn + 1) / 2) + (f0 >> 1)) * npts * 2 + (f0 & 1) : 0;
  T hphi[FB];  // kSwKap: ds/2 phi(nu) of the CTA's frequencies
#pragma unroll
  for (int j = 0; j < FB; ++j) hphi[j] = MODE == kSwKap ? hds * phi[f0 + j] : T(0);
  // x and y of a cell: FB consecutive values, one vector access when aligned
  const bool vec = nn % FB == 0;
  using PX = Pack<TX, FB>;
  using PY = Pack<TY, FB>;
  // first plane: inflow (or zero)
  {
    P I0;
#pragma unroll
    for (int j = 0; j < FB; ++j)
      I0.v[j] = (inflow && f0 + j < nn) ? (T)(up ? I_bot[f0 + j] : I_top[f0 + j]) : T(0);
    const int64_t pk = (int64_t)k0 * plane;
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
      const int c = threadIdx.x + i * blockDim.x;
      if (c >= plane) continue;
      sI[c] = I0;
      sS[c] = load_src(pk + c);
      if (MODE == kSwChi || qsc) sC[c] = load_chi(pk + c);
      if (MODE == kSwKap) sK[c] = kap[pk + c];
      const int64_t k = (pk + c) * nr + (int64_t)d * nn + f0;
#pragma unroll
      for (int j = 0; j < FB; ++j) {
        if (f0 + j >= nn) continue;
        if (out == kOutI) y[k + j] = cast_to<TY>(I0.v[j]);
        else y[k + j] = cast_to<TY>(cast_to<T>(x[k + j]) - I0.v[j]);
      }
    }
  }
  __syncthreads();
  for (int s = 1; s < nz; ++s) {
    const int kp = k0 + s * step;
    const int64_t pk = (int64_t)kp * plane;
    P In[dbl ? 1 : CPT];
#pragma unroll
    for (int i0 = 0; i0 < CPT; i0 += CB) {
      // loads of CB cells issued together
      P Sc[CB], Cc[CB];
      T Kc[CB];
      T xv[CB][FB];
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const int c = threadIdx.x + (i0 + u) * blockDim.x;
        const int cc = c < plane ? c : 0;
        Sc[u] = load_src(pk + cc);
        if (MODE == kSwPre) {  // Cc holds 1 - e^-d
          Cc[u] = *reinterpret_cast<const P *>(cW0 + cbase + (pk + cc) * 2);
        } else if (MODE == kSwKap) {
          Kc[u] = kap[pk + cc];
        } else {
          Cc[u] = load_chi(pk + cc);
        }
        if (out != kOutI) {
          const int64_t k = (pk + cc) * nr + (int64_t)d * nn + f0;
          if (Xd) {
            const P v = Xd[pk + cc];
#pragma unroll
            for (int j = 0; j < FB; ++j) xv[u][j] = v.v[j];
          } else if (vec) {
            const PX v = *reinterpret_cast<const PX *>(x + k);
#pragma unroll
            for (int j = 0; j < FB; ++j) xv[u][j] = cast_to<T>(v.v[j]);
          } else {
#pragma unroll
            for (int j = 0; j < FB; ++j) xv[u][j] = f0 + j < nn ? cast_to<T>(x[k + j]) : T(0);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const int i = i0 + u;
        const int c = threadIdx.x + i * blockDim.x;
        if (c >= plane) continue;
        const int c00 = nb0[i] & 0xffff, c01 = nb0[i] >> 16, c10 = nb1[i] & 0xffff, c11 = nb1[i] >> 16;
        const P I00 = sI[c00], I01 = sI[c01], I10 = sI[c10], I11 = sI[c11];
        const P S00 = sS[c00], S01 = sS[c01], S10 = sS[c10], S11 = sS[c11];
        P C00, C01, C10, C11, Bc;
        T Ku = 0;
        if (MODE == kSwPre) {
          Bc = *reinterpret_cast<const P *>(cB + cbase + (pk + c) * 2);
        } else if (MODE == kSwKap) {
          Ku = w00 * sK[c00] + w01 * sK[c01] + w10 * sK[c10] + w11 * sK[c11] + Kc[u];
        } else {
          C00 = sC[c00], C01 = sC[c01], C10 = sC[c10], C11 = sC[c11];
        }
        const int64_t k = (pk + c) * nr + (int64_t)d * nn + f0;
        // kSwQsc away from the last plane: S and chi at the downwind point
        P Sdw, Cdw;
        const bool quad = qsc && s + 1 < nz;
        if (quad) {
          const int64_t pd = pk + (int64_t)step * plane;
          const int e00 = nd0[qsc ? i : 0] & 0xffff, e01 = nd0[qsc ? i : 0] >> 16;
          const int e10 = nd1[qsc ? i : 0] & 0xffff, e11 = nd1[qsc ? i : 0] >> 16;
          const P A00 = load_src(pd + e00), A01 = load_src(pd + e01), A10 = load_src(pd + e10),
                  A11 = load_src(pd + e11);
          const P B00 = load_chi(pd + e00), B01 = load_chi(pd + e01), B10 = load_chi(pd + e10),
                  B11 = load_chi(pd + e11);
#pragma unroll
          for (int j = 0; j < FB; ++j) {
            Sdw.v[j] = w00 * A00.v[j] + w01 * A01.v[j] + w10 * A10.v[j] + w11 * A11.v[j];
            Cdw.v[j] = w00 * B00.v[j] + w01 * B01.v[j] + w10 * B10.v[j] + w11 * B11.v[j];
          }
        }
        PY yv;
#pragma unroll
        for (int j = 0; j < FB; ++j) {
          const T Iu = w00 * I00.v[j] + w01 * I01.v[j] + w10 * I10.v[j] + w11 * I11.v[j];
          const T Su = w00 * S00.v[j] + w01 * S01.v[j] + w10 * S10.v[j] + w11 * S11.v[j];
          T e, a, b, pdS = T(0);
          if (MODE == kSwPre) {
            const T w0 = Cc[u].v[j];
            e = (T)1 - w0;
            b = Bc.v[j];
            a = w0 - b;
          } else if (MODE == kSwKap) {
            step_coef<T>(hphi[j] * Ku, ie, e, a, b);
          } else {
            const T Cu = w00 * C00.v[j] + w01 * C01.v[j] + w10 * C10.v[j] + w11 * C11.v[j];
            if (quad) {  // weights of the upwind, current and downwind source
              T wd;
              qsc_coef<T>(hds * (Cu + Cc[u].v[j]), hds * (Cc[u].v[j] + Cdw.v[j]), e, a, b, wd);
              pdS = wd * Sdw.v[j];
            } else {
              step_coef<T>(hds * (Cu + Cc[u].v[j]), qsc ? 0 : ie, e, a, b);
            }
          }
          const T I = quad ? fma(e, Iu, fma(a, Su, fma(b, Sc[u].v[j], pdS))) : fma(e, Iu, fma(a, Su, b * Sc[u].v[j]));
          In[dbl ? 0 : i].v[j] = I;
          yv.v[j] = out == kOutI ? cast_to<TY>(I) : cast_to<TY>(xv[u][j] - I);
        }
        if (vec) {
          *reinterpret_cast<PY *>(y + k) = yv;
        } else {
#pragma unroll
          for (int j = 0; j < FB; ++j)
            if (f0 + j < nn) y[k + j] = yv.v[j];
        }
        if (dbl) sIn[c] = In[0];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
      const int c = threadIdx.x + i * blockDim.x;
      if (c >= plane) continue;
      if (!dbl) sI[c] = In[i];
      sS[c] = load_src(pk + c);
      if (MODE == kSwChi || qsc) sC[c] = load_chi(pk + c);
      if (MODE == kSwKap) sK[c] = kap[pk + c];
    }
    __syncthreads();
    if (dbl) {
      P *t = sI;
      sI = sIn;
      sIn = t;
    }
  }
}

// Long characteristics (RT_FS_LC, kSwLc): every point's value from its own
// straight ray traced back to the inflow plane.  The ray through cell c of
// plane k crosses plane k' at c shifted back by (k - k') (sx, sy) cells; S and
// chi are interpolated there (bilinear, periodic) and the linear step of
// eqs. ie_1/ie_2 is taken from crossing to crossing; the intensity is never
// interpolated.  One thread per (direction, frequency, cell of a plane), all
// target planes in sweep order, O(nz) steps per point; no shared memory, no
// barriers.  SL: the source in the sweep layout with one frequency per block,
// [d][f][p], or null for the thermal term tsrc.
template <typename T, typename TX, typename TY>
__global__ void __launch_bounds__(256) k_box_lc(BoxDev bx, const double *__restrict__ geo,
                                                const T *__restrict__ chiN, const T *__restrict__ SL,
                                                const double *__restrict__ tsrc, const TX *__restrict__ x,
                                                TY *__restrict__ y, int out, int inflow,
                                                const double *__restrict__ I_top,
                                                const double *__restrict__ I_bot) {
  const int nx = bx.nx, ny = bx.ny, nz = bx.nz, nn = bx.nn, nd = bx.nd;
  const int plane = nx * ny;
  const int64_t npts = (int64_t)plane * nz, nr = (int64_t)nd * nn;
  const int64_t total = (int64_t)nd * nn * plane;
  for (int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gid < total;
       gid += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(gid % plane);
    const int64_t df = gid / plane;
    const int f = (int)(df % nn), d = (int)(df / nn);
    const double *g = geo + 6 * d;
    const int fx = (int)g[0], fy = (int)g[1];
    const T ax = (T)g[2], ay = (T)g[3], hds = (T)(0.5 * g[4]);
    const bool up = g[5] > 0.5;
    const int k0 = up ? nz - 1 : 0, step = up ? -1 : 1;
    const int yy = c / nx, xx = c - yy * nx;
    const T *Sd = SL ? SL + ((int64_t)d * nn + f) * npts : nullptr;
    const T *chiB = chiN + (int64_t)(f >> 2) * npts * 4 + (f & 3);
    // S and chi of plane km at cell c shifted back by t segments
    auto at = [&](int km, int t, T &sv, T &cv) {
      const T tx = (T)t * ax, ty = (T)t * ay;
      const T flx = floor(tx), fly = floor(ty);
      const T wx = tx - flx, wy = ty - fly;
      const int shx = (int)(((int64_t)t * fx + (int64_t)flx) % nx);
      const int shy = (int)(((int64_t)t * fy + (int64_t)fly) % ny);
      int x0 = xx - shx, y0 = yy - shy;
      if (x0 < 0) x0 += nx;
      if (y0 < 0) y0 += ny;
      const int x1 = x0 == 0 ? nx - 1 : x0 - 1;
      const int y1 = y0 == 0 ? ny - 1 : y0 - 1;
      const int64_t b = (int64_t)km * plane;
      const int64_t p00 = b + y0 * nx + x0, p01 = b + y0 * nx + x1, p10 = b + y1 * nx + x0, p11 = b + y1 * nx + x1;
      const T w00 = ((T)1 - wy) * ((T)1 - wx), w01 = ((T)1 - wy) * wx, w10 = wy * ((T)1 - wx), w11 = wy * wx;
      if (Sd) {
        sv = w00 * Sd[p00] + w01 * Sd[p01] + w10 * Sd[p10] + w11 * Sd[p11];
      } else {
        sv = w00 * cast_to<T>(tsrc[p00 * nn + f]) + w01 * cast_to<T>(tsrc[p01 * nn + f]) +
             w10 * cast_to<T>(tsrc[p10 * nn + f]) + w11 * cast_to<T>(tsrc[p11 * nn + f]);
      }
      cv = w00 * chiB[p00 * 4] + w01 * chiB[p01 * 4] + w10 * chiB[p10 * 4] + w11 * chiB[p11 * 4];
    };
    auto put = [&](int k, T I) {
      const int64_t q = ((int64_t)k * plane + c) * nr + (int64_t)d * nn + f;
      y[q] = out == kOutI ? cast_to<TY>(I) : cast_to<TY>(cast_to<T>(x[q]) - I);
    };
    const T I0 = inflow ? (T)(up ? I_bot[f] : I_top[f]) : T(0);
    put(k0, I0);
    for (int s = 1; s < nz; ++s) {
      T I = I0, Sa, ca;
      at(k0, s, Sa, ca);
      for (int m = 1; m <= s; ++m) {
        T Sm, cm, e, a, b;
        at(k0 + m * step, s - m, Sm, cm);
        step_coef<T>(hds * (ca + cm), 0, e, a, b);
        I = fma(e, I, fma(a, Sa, b * Sm));
        Sa = Sm;
        ca = cm;
      }
      put(k0 + s * step, I);
    }
  }
}


// Step weights of the float64 sweep, once per handle: for every (direction,
// point, frequency) the optical depth of the step from the upwind plane,
// 0.5 (chi_u + chi_c) ds with chi_u bilinear at the upwind point, and from it
// w0 = 1 - e^-d (expm1) and w1/d (series below 0.1), or the implicit-Euler
// pair (d/(1+d), d/(1+d)).  Layout [d][f / 2][p][f % 2]; the first plane of
// each direction (no step) holds zeros.
__global__ void k_box_coef64(BoxDev bx, const double *__restrict__ geo, const double *__restrict__ chiN,
                             double *__restrict__ W0, double *__restrict__ Bt) {
  const int nx = bx.nx, ny = bx.ny, nz = bx.nz, nn = bx.nn, nd = bx.nd;
  const int plane = nx * ny;
  const int64_t npts = (int64_t)plane * nz;
  const int nfb2 = (nn + 1) / 2;
  const int64_t total = (int64_t)nd * npts * nfb2 * 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i & 1);
    const int64_t r = i >> 1;
    const int64_t p = r % npts;
    const int64_t db = r / npts;
    const int fb2 = (int)(db % nfb2), d = (int)(db / nfb2);
    const int f = 2 * fb2 + j;
    double w0 = 0.0, bt = 0.0;
    const double *g = geo + 6 * d;
    const bool up = g[5] > 0.5;
    const int kp = (int)(p / plane), c = (int)(p - (int64_t)kp * plane);
    const int k0 = up ? nz - 1 : 0, step = up ? -1 : 1;
    if (f < nn && kp != k0) {
      const int fx = (int)g[0], fy = (int)g[1];
      const double ax = g[2], ay = g[3];
      const int yy = c / nx, xx = c - yy * nx;
      int x0 = xx - fx, y0 = yy - fy;
      if (x0 < 0) x0 += nx;
      if (y0 < 0) y0 += ny;
      const int x1 = x0 == 0 ? nx - 1 : x0 - 1, y1 = y0 == 0 ? ny - 1 : y0 - 1;
      const int64_t pu = (int64_t)(kp - step) * plane;
      auto chi = [&](int64_t q) { return chiN[((int64_t)(f >> 2) * npts + q) * 4 + (f & 3)]; };
      const double cu = (1 - ay) * (1 - ax) * chi(pu + y0 * nx + x0) + (1 - ay) * ax * chi(pu + y0 * nx + x1) +
                        ay * (1 - ax) * chi(pu + y1 * nx + x0) + ay * ax * chi(pu + y1 * nx + x1);
      const double dt = 0.5 * g[4] * (cu + chi(p));
      double e, a, b;
      step_coef<double>(dt, bx.ie, e, a, b);
      w0 = bx.ie ? b : -expm1(-dt);
      bt = b;
    }
    W0[i] = w0;
    Bt[i] = bt;
  }
}

// ------------------------------------------------------------ host side
// Step-weight mode of the sweep for one precision (see k_sweep3d).
static int box_mode(const rt_handle *h, bool fp64) {
  if (h->box.lc) return kSwLc;
  if (h->box.qsc) return kSwQsc;
  if (fp64) return h->box_w064 ? kSwPre : kSwChi;
  return h->box_kap32 ? kSwKap : kSwChi;
}

// Shared memory of one sweep CTA: I and S of the plane (FB values per cell)
// and the previous plane's opacity (FB values, or one kappa, or nothing).
static size_t box_smem(const rt_handle *h, bool fp64, int fb) {
  const size_t plane = (size_t)h->box.nx * h->box.ny, esz = fp64 ? 8 : 4;
  const int mode = box_mode(h, fp64);
  return plane * esz * (2 * fb + ((mode == kSwChi || mode == kSwQsc) ? fb : mode == kSwKap ? fb + 1 : 0));
}

// Launch shape of the sweep for one precision: FB frequencies per CTA and
// CPT cells per thread (at most 512 threads).  The shapes are those whose
// registers stay within 128 per thread without spills (float32: FB = 4 up to
// CPT = 4 with the opacity, 8 with kappa, FB <= 2 up to 8; float64: FB = 2 up
// to 2 with the opacity, 8 with precomputed weights, FB = 1 up to 8).  FB is
// the largest whose plane arrays fit the shared memory and whose plane fits
// 512 threads, not wider than the frequencies need; rt_autotune may cap FB
// and raise CPT.
static int box_cpt_max(bool fp64, int fb, int mode) {
  if (mode == kSwQsc) return fb == 1 ? 4 : 2;
  if (fp64) return fb == 2 && mode != kSwPre ? 2 : 8;
  return fb == 4 && mode != kSwKap ? 4 : 8;
}

static void box_shape(const rt_handle *h, bool fp64, int &fb, int &cpt) {
  const int plane = h->box.nx * h->box.ny;
  const int mode = box_mode(h, fp64);
  if (mode == kSwLc) {  // one frequency per source block, no plane sweep
    fb = cpt = 1;
    return;
  }
  const int fbmax = fp64 ? 2 : 4;
  fb = h->tune.box_fb > 0 ? std::min(fbmax, h->tune.box_fb) : fbmax;
  while (fb > 1 && (fb / 2 >= h->box.nn || box_smem(h, fp64, fb) > (size_t)kBoxSmemMax ||
                    plane > 512 * box_cpt_max(fp64, fb, mode)))
    fb /= 2;
  cpt = 1;
  while ((plane + cpt - 1) / cpt > 512) cpt *= 2;
  if (h->tune.box_cpt > cpt) cpt = std::min(h->tune.box_cpt, box_cpt_max(fp64, fb, mode));
}

void box_effective_shape(const rt_handle *h, bool fp64, int &fb, int &cpt) { box_shape(h, fp64, fb, cpt); }

static int box_fb(const rt_handle *h, bool fp64) {
  int fb, cpt;
  box_shape(h, fp64, fb, cpt);
  return fb;
}

bool box_plane_fits(int nx, int ny) {
  const int64_t plane = (int64_t)nx * ny;
  return plane <= 8 * 512 && plane < 65536 && 3 * plane * 8 <= kBoxSmemMax;
}

int64_t box_scratch_elems(const rt_handle *h, bool fp64) {
  const int fb = box_fb(h, fp64);
  const int64_t npts = (int64_t)h->box.nx * h->box.ny * h->box.nz;
  const int64_t nfb = (h->box.nn + fb - 1) / fb;
  return npts * h->box.nd * nfb * fb;
}

template <typename T, int FB, int CPT, int MODE, typename TX, typename TY>
static int sweep3d_run(rt_handle *h, const T *chiN, const void *S, const double *tsrc, const TX *x, TY *y, int out,
                       bool inflow, cudaStream_t s, const T *xs) {
  const BoxDev &bx = h->box;
  const int plane = bx.nx * bx.ny;
  const int nfb = (bx.nn + FB - 1) / FB;
  const int nt = std::min(512, ((plane + CPT - 1) / CPT + 31) / 32 * 32);
  if ((int64_t)nt * CPT < plane) return (int)cudaErrorInvalidConfiguration;
  const size_t smem = box_smem(h, sizeof(T) == 8, FB);
  constexpr int CB = (8 / FB) < CPT ? (8 / FB) : CPT;  // cells whose loads are issued together
  auto kern = k_sweep3d<T, FB, CPT, CB, TX, TY, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const T *cw = nullptr, *cb = nullptr, *kap = nullptr, *phi = nullptr;
  if (MODE == kSwPre) {
    cw = reinterpret_cast<const T *>(h->box_w064);
    cb = reinterpret_cast<const T *>(h->box_bt64);
  }
  if (MODE == kSwKap) {
    kap = reinterpret_cast<const T *>(h->box_kap32);
    phi = reinterpret_cast<const T *>(h->box_phi32);
  }
  kern<<<bx.nd * nfb, nt, smem, s>>>(bx, h->d_geo, chiN, h->box_npad, static_cast<const Pack<T, FB> *>(S), tsrc, x,
                                     y, out, inflow ? 1 : 0, h->d_Itop, h->d_Ibot, cw, cb, kap, phi, xs);
  return (int)cudaGetLastError();
}

template <typename T, int FB, int MODE, typename TX, typename TY>
static int sweep3d_cpt(rt_handle *h, int cpt, const T *chiN, const void *S, const double *tsrc, const TX *x, TY *y,
                       int out, bool inflow, cudaStream_t s, const T *xs) {
  constexpr bool f64 = sizeof(T) == 8;
  constexpr int cmax = MODE == kSwQsc ? (FB == 1 ? 4 : 2)
                                      : f64 ? (FB == 2 && MODE != kSwPre ? 2 : 8) : (FB == 4 && MODE != kSwKap ? 4 : 8);
  if (cpt <= 1) return sweep3d_run<T, FB, 1, MODE>(h, chiN, S, tsrc, x, y, out, inflow, s, xs);
  if (cpt == 2 || cmax == 2) return sweep3d_run<T, FB, 2, MODE>(h, chiN, S, tsrc, x, y, out, inflow, s, xs);
  if constexpr (cmax >= 4) {
    if (cpt == 4 || cmax == 4) return sweep3d_run<T, FB, 4, MODE>(h, chiN, S, tsrc, x, y, out, inflow, s, xs);
  }
  if constexpr (cmax >= 8) return sweep3d_run<T, FB, 8, MODE>(h, chiN, S, tsrc, x, y, out, inflow, s, xs);
  return (int)cudaErrorInvalidConfiguration;
}

template <typename T, int MODE, typename TX, typename TY>
static int sweep3d_fb(rt_handle *h, int fb, int cpt, const T *chiN, const void *S, const double *tsrc, const TX *x,
                      TY *y, int out, bool inflow, cudaStream_t s, const T *xs) {
  if constexpr (sizeof(T) == 4) {
    if (fb == 4) return sweep3d_cpt<T, 4, MODE>(h, cpt, chiN, S, tsrc, x, y, out, inflow, s, xs);
  }
  if (fb == 2) return sweep3d_cpt<T, 2, MODE>(h, cpt, chiN, S, tsrc, x, y, out, inflow, s, xs);
  return sweep3d_cpt<T, 1, MODE>(h, cpt, chiN, S, tsrc, x, y, out, inflow, s, xs);
}

template <typename T, typename TX, typename TY>
static int sweep3d(rt_handle *h, const void *S, const double *tsrc, const TX *x, TY *y, int out, bool inflow,
                   cudaStream_t s, const T *xs = nullptr) {
  constexpr bool f64 = sizeof(T) == 8;
  const T *chiN = reinterpret_cast<const T *>(f64 ? (const void *)h->chi64 : (const void *)h->chi32);
  int fb, cpt;
  box_shape(h, f64, fb, cpt);
  const int mode = box_mode(h, f64);
  if (mode == kSwLc) {
    const int64_t total = (int64_t)h->box.nd * h->box.nn * h->box.nx * h->box.ny;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)(h->n_sm > 0 ? h->n_sm : 152) * 32);
    k_box_lc<T, TX, TY><<<grid, 256, 0, s>>>(h->box, h->d_geo, chiN, static_cast<const T *>(S), tsrc, x, y, out,
                                             inflow ? 1 : 0, h->d_Itop, h->d_Ibot);
    return (int)cudaGetLastError();
  }
  if (mode == kSwQsc) return sweep3d_fb<T, kSwQsc>(h, fb, cpt, chiN, S, tsrc, x, y, out, inflow, s, xs);
  if constexpr (f64) {
    if (mode == kSwPre) return sweep3d_fb<T, kSwPre>(h, fb, cpt, chiN, S, tsrc, x, y, out, inflow, s, xs);
  } else {
    if (mode == kSwKap) return sweep3d_fb<T, kSwKap>(h, fb, cpt, chiN, S, tsrc, x, y, out, inflow, s, xs);
  }
  return sweep3d_fb<T, kSwChi>(h, fb, cpt, chiN, S, tsrc, x, y, out, inflow, s, xs);
}

// XS (may be null): also write x, cast to T, in the sweep layout there; set
// to null when the kernel taken does not (the sweep then reads x itself).
template <typename T, typename TX>
static int sigma_box(rt_handle *h, const Tables<T> &tb, const TX *x, T *S, int fb_out, cudaStream_t s,
                     T *&XS) {
  const ColDev &c = h->h_cols[0];
  const int64_t npts = (int64_t)h->box.nx * h->box.ny * h->box.nz;
  const int nw = kBoxSigNT / 32;
  const int grid = (int)std::min<int64_t>((npts + nw - 1) / nw, (int64_t)h->n_sm * 16);
  if (c.psi_off >= 0) {
    XS = nullptr;
    k_sigma_box_dense<T, TX><<<grid, kBoxSigNT, 0, s>>>(c, tb, npts, x, S, fb_out);
    return (int)cudaGetLastError();
  }
  const bool rw_cached = !c.rdiag && (int64_t)c.nn * c.nn * sizeof(T) <= kBoxRwCache;
  const int rw_len = c.rdiag ? c.nn : (rw_cached ? c.nn * c.nn : 0);
  auto launch = [&](auto kern, int kr) -> int {
    const size_t smem = sizeof(T) * ((size_t)2 * c.nd * kr + ((rw_len + 1) & ~1) + (size_t)nw * kr * c.nn);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    kern<<<grid, kBoxSigNT, smem, s>>>(c, tb, npts, x, S, fb_out);
    return (int)cudaGetLastError();
  };
  // four frequencies per lane into sweep blocks of 1, 2 or 4 (nn a multiple
  // of 4, at most 128; Gamma rows 16-byte aligned)
  if (fb_out > 0 && 4 % fb_out == 0 && c.nn % 4 == 0 && c.nn <= 128 && c.g_off % 4 == 0) {
    const int lp = c.nn <= 32 ? 8 : (c.nn <= 64 ? 16 : 32);
    const int pts_per_cta = nw * (32 / lp);
    const int grid4 = (int)std::min<int64_t>((npts + pts_per_cta - 1) / pts_per_cta, (int64_t)h->n_sm * 16);
    auto launch4 = [&](auto kern, int kr) -> int {
      const size_t smem = sizeof(T) * ((size_t)2 * c.nd * kr + ((rw_len + 3) & ~3) +
                                       (size_t)nw * (32 / lp) * (kr * c.nn + 4));
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return (int)e;
      kern<<<grid4, kBoxSigNT, smem, s>>>(c, tb, npts, x, S, XS);
      return (int)cudaGetLastError();
    };
#define RT_SIGMA_BOX4(KR)                                                                        \
  {                                                                                              \
    if (lp == 8) {                                                                               \
      if (fb_out == 4) return launch4(k_sigma_box4<T, TX, KR, 8, 4>, KR);                        \
      if (fb_out == 2) return launch4(k_sigma_box4<T, TX, KR, 8, 2>, KR);                        \
      return launch4(k_sigma_box4<T, TX, KR, 8, 1>, KR);                                         \
    }                                                                                            \
    if (lp == 16) {                                                                              \
      if (fb_out == 4) return launch4(k_sigma_box4<T, TX, KR, 16, 4>, KR);                       \
      if (fb_out == 2) return launch4(k_sigma_box4<T, TX, KR, 16, 2>, KR);                       \
      return launch4(k_sigma_box4<T, TX, KR, 16, 1>, KR);                                        \
    }                                                                                            \
    if (fb_out == 4) return launch4(k_sigma_box4<T, TX, KR, 32, 4>, KR);                         \
    if (fb_out == 2) return launch4(k_sigma_box4<T, TX, KR, 32, 2>, KR);                         \
    return launch4(k_sigma_box4<T, TX, KR, 32, 1>, KR);                                          \
  }
    if (c.rp <= 2) RT_SIGMA_BOX4(2)
    RT_SIGMA_BOX4(6)
#undef RT_SIGMA_BOX4
  }
  XS = nullptr;
  const int fl = (c.nn + 31) / 32;
  if (c.rp <= 2) {
    if (fl <= 1) return launch(k_sigma_box<T, TX, 2, 1>, 2);
    if (fl <= 2) return launch(k_sigma_box<T, TX, 2, 2>, 2);
    return launch(k_sigma_box<T, TX, 2, 4>, 2);
  }
  if (fl <= 1) return launch(k_sigma_box<T, TX, 6, 1>, 6);
  if (fl <= 2) return launch(k_sigma_box<T, TX, 6, 2>, 6);
  return launch(k_sigma_box<T, TX, 6, 4>, 6);
}

// the box Sigma holds the rank and frequencies in registers: rank <= 6 and
// n_nu <= 128 (four frequencies per lane)
bool box_sigma_fits(const rt_desc *d, int rp) {
  const size_t esz = 8;
  const int nn = d->n_nu;
  const bool rw_cached = (int64_t)nn * nn * esz <= kBoxRwCache;
  const size_t smem = esz * ((size_t)2 * d->n_dir * 6 + (rw_cached ? nn * nn + 1 : 1) + (size_t)(kBoxSigNT / 32) * 6 * nn);
  return rp <= 6 && nn <= 128 && smem <= 200 * 1024;
}

template <typename T, typename TX, typename TY>
static int box_apply_t(rt_handle *h, const Tables<T> &tb, int op, const TX *x, TY *y, cudaStream_t s, void *S) {
  const int fb = box_fb(h, sizeof(T) == 8);
  const int64_t npts = (int64_t)h->box.nx * h->box.ny * h->box.nz;
  const int64_t len = h->E;
  const int cgrid = (int)std::min<int64_t>((len + 255) / 256, 16 * 152);
  T *St = static_cast<T *>(S);
  int e = 0;
  switch (op) {
    case 0: {  // y = x - Lambda Sigma x
      // float32 operator on the handle's scratch (room for two float32
      // arrays): Sigma also writes x in the sweep layout behind S
      T *XS = sizeof(T) == 4 && S == h->apply_S ? St + npts * h->box.nd * h->box_npad : nullptr;
      if ((e = sigma_box<T, TX>(h, tb, x, St, fb, s, XS))) return e;
      return sweep3d<T, TX, TY>(h, St, nullptr, x, y, kOutAminus, false, s, XS);
    }
    case 1:  // y = Lambda x
      if constexpr (sizeof(TX) != 8) return (int)cudaErrorInvalidValue;
      else {
        k_box_to_sweep<T><<<(int)std::min<int64_t>(npts, 65535), 256, 0, s>>>(x, St, npts, h->box.nd, h->box.nn, fb);
        return sweep3d<T, TX, TY>(h, St, nullptr, nullptr, y, kOutI, false, s);
      }
    case 2:  // y = Sigma x (space-based layout, float64 out)
      if constexpr (sizeof(TY) != 8) return (int)cudaErrorInvalidValue;
      else {
        T *no_xs = nullptr;
        if ((e = sigma_box<T, TX>(h, tb, x, St, fb, s, no_xs))) return e;
        k_box_from_sweep<T><<<(int)std::min<int64_t>(npts, 65535), 256, 0, s>>>(St, y, npts, h->box.nd, h->box.nn, fb);
        return (int)cudaGetLastError();
      }
    default:  // y = Lambda t + I_in
      if (h->d_tsrc) return sweep3d<T, TX, TY>(h, nullptr, h->d_tsrc, nullptr, y, kOutI, true, s);
      cudaMemsetAsync(St, 0, box_scratch_elems(h, sizeof(T) == 8) * sizeof(T), s);
      return sweep3d<T, TX, TY>(h, St, nullptr, nullptr, y, kOutI, true, s);
  }
}

// Operators of a 3D box; x (and y) are float32 when xf (yf), else float64;
// the float64 operator needs both in float64.  scratch: the source function
// (box_scratch_elems of the operator's precision), or null for the handle's.
int box_apply(rt_handle *h, int op, bool fp64, const void *x, bool xf, void *y, bool yf, cudaStream_t s,
              void *scratch) {
  void *S = scratch ? scratch : h->apply_S;
  if (fp64 || h->precision == 0) {
    if (xf || yf) return (int)cudaErrorInvalidValue;
    return box_apply_t<double, double, double>(h, tables64(h), op, static_cast<const double *>(x),
                                               static_cast<double *>(y), s, S);
  }
  const Tables<float> tb = tables32(h);
  if (xf && yf)
    return box_apply_t<float, float, float>(h, tb, op, static_cast<const float *>(x), static_cast<float *>(y), s, S);
  if (!xf && !yf)
    return box_apply_t<float, double, double>(h, tb, op, static_cast<const double *>(x), static_cast<double *>(y),
                                              s, S);
  return (int)cudaErrorInvalidValue;
}

// Opacity in the sweep's padded per-point layout, both precisions.
int box_prepare(rt_handle *h, const double *chi) {
  // RT_BOX_FB = 1, 2 or 4 fixes the plane sweep's frequencies per CTA (the
  // choice rt_autotune makes by timing; it may override it later)
  const char *efb = std::getenv("RT_BOX_FB");
  if (efb && (efb[0] == '1' || efb[0] == '2' || efb[0] == '4') && efb[1] == 0) h->tune.box_fb = efb[0] - '0';
  const int nn = h->box.nn;
  const int npad = (nn + 3) / 4 * 4;
  const int64_t npts = (int64_t)h->box.nx * h->box.ny * h->box.nz;
  h->box_npad = npad;
  std::vector<double> c64((size_t)npts * npad, 0.0);
  std::vector<float> c32((size_t)npts * npad, 0.f);
  for (int64_t p = 0; p < npts; ++p)
    for (int f = 0; f < nn; ++f) {
      const size_t k = ((size_t)(f >> 2) * npts + p) * 4 + (f & 3);  // [f / 4][p][f % 4]
      c64[k] = chi[(size_t)p * nn + f];
      c32[k] = (float)chi[(size_t)p * nn + f];
    }
  cudaError_t e = cudaMalloc(&h->chi64, c64.size() * 8);
  if (e == cudaSuccess) e = cudaMemcpy(h->chi64, c64.data(), c64.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&h->chi32, c32.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(h->chi32, c32.data(), c32.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return (int)e;
  // separable opacity chi(p, nu) = kappa(p) phi(nu) (to 1e-14): the float32
  // sweep then keeps one kappa per cell; phi from the point of largest
  // opacity, kappa(p) = chi(p, f*) / phi(f*) at that point's largest frequency
  {
    int64_t pr = 0;
    int fr = 0;
    double cmax = -1.0;
    for (int64_t p = 0; p < npts; ++p)
      for (int f = 0; f < nn; ++f)
        if (chi[(size_t)p * nn + f] > cmax) {
          cmax = chi[(size_t)p * nn + f];
          pr = p;
          fr = f;
        }
    bool sep = cmax > 0.0 && !h->box.qsc && !h->box.lc;  // these two read the full opacity
    std::vector<double> phi(nn), kap(npts);
    for (int f = 0; f < nn && sep; ++f) phi[f] = chi[(size_t)pr * nn + f];
    for (int64_t p = 0; p < npts && sep; ++p) {
      kap[p] = chi[(size_t)p * nn + fr] / cmax;
      for (int f = 0; f < nn; ++f) {
        const double c = chi[(size_t)p * nn + f];
        if (std::fabs(kap[p] * phi[f] - c) > 1e-14 * std::fabs(c) + 1e-300) { sep = false; break; }
      }
    }
    if (sep) {
      std::vector<float> k32(kap.begin(), kap.end()), p32((size_t)npad, 0.f);
      for (int f = 0; f < nn; ++f) p32[f] = (float)phi[f];
      e = cudaMalloc(&h->box_kap32, k32.size() * 4);
      if (e == cudaSuccess) e = cudaMemcpy(h->box_kap32, k32.data(), k32.size() * 4, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMalloc(&h->box_phi32, p32.size() * 4);
      if (e == cudaSuccess) e = cudaMemcpy(h->box_phi32, p32.data(), p32.size() * 4, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return (int)e;
    }
  }
  // float64 step weights, when they take at most a quarter of the free memory
  // and RT_BOX_COEF64 is not "0" (then the float64 sweep forms them on the fly)
  const int64_t ncoef = (int64_t)h->box.nd * npts * ((nn + 1) / 2) * 2;
  const char *env = std::getenv("RT_BOX_COEF64");
  const bool allow = !(env && env[0] == '0' && env[1] == 0) && !h->box.qsc && !h->box.lc;
  size_t free_b = 0, total_b = 0;
  if (allow && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && (double)ncoef * 16.0 <= 0.25 * (double)free_b) {
    e = cudaMalloc(&h->box_w064, (size_t)ncoef * 8);
    if (e == cudaSuccess) e = cudaMalloc(&h->box_bt64, (size_t)ncoef * 8);
    if (e != cudaSuccess) return (int)e;
    const int grid = (int)std::min<int64_t>((ncoef + 255) / 256, 152 * 32);
    k_box_coef64<<<grid, 256>>>(h->box, h->d_geo, h->chi64, h->box_w064, h->box_bt64);
    e = cudaGetLastError();
  }
  return (int)e;
}

}  // namespace rt
