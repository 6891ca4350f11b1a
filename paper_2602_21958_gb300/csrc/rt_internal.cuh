// rt_internal.cuh -- device data layout and per-column device routines shared by
// the 1D apply and solve kernels.
//
// A handle holds a batch of 1D columns (Sec. 3.1) in concatenated device arrays.
// Per column: step coefficients per (layer, |mu| class, nu), the factored
// scattering kernel, Gamma, the thermal term and the inflow.  Vectors follow the
// space-based ordering of Sec. 3.1 (point, direction, frequency fastest).
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace rt {

constexpr int kSigBuf = 2048;  // elements of each shared buffer of the Sigma stage

// Per-column metadata (device resident, one entry per column).
struct ColDev {
  int64_t x_off;    // offset of the column inside one right-hand-side vector
  int64_t g_off;    // offset in per-(point, nu) arrays: gamma, t_src, chi
  int64_t c_off;    // offset in step-coefficient arrays [nz-1][ncls][nn]
  int64_t r_off;    // offset in the frequency-kernel storage
  int64_t psi_off;  // offset in the dense-kernel storage, -1 when separable
  int32_t u_off;    // offset in angular-factor arrays [nd][rp]
  int32_t d_off;    // offset in per-direction arrays [nd]
  int32_t in_off;   // offset in inflow arrays [nn]
  int32_t nz, nd, nn, nr;
  int32_t ncls;     // number of distinct |mu|
  int32_t rp;       // rank of the angular factor
  int32_t rdiag;    // 1: frequency kernel is diagonal (coherent scattering)
  int32_t fs;       // formal solver: 0 SC-L, 1 implicit Euler, 2 quadratic SC
  int32_t lr_rank;  // float32 operator: rank of the truncated frequency kernel (0: exact)
  int64_t lr_off;   // offset of its factors A | B ([nn][lr_rank] each) in Tables::LR
};

constexpr int kLrMax = 32;  // largest rank of a truncated frequency kernel

// Arrays in one arithmetic precision T (double: fp64 path; float: mixed path).
template <typename T>
struct Tables {
  const T *E, *A, *B;   // step coefficients: I_c = E I_u + A S_u + B S_c
  const T *Uw;          // [nd][rp] moment weights  (eigvecs of P times w_dir)
  const T *Ul;          // [nd][rp] expansion       (eigvecs of P times eigvals)
  const T *RwT;         // [nn'][nn] (R w_nu)^T, or [nn] diagonal when rdiag
  const T *PsiwT;       // [nr'][nr] (Psi diag(w_r))^T for dense kernels
  const T *gamma;       // [nz][nn]
  // quadratic short characteristics (fs == 2): I_c = E I_u + A S_u + B S_c + C S_d
  // with (A, B, C) for rays going down (mu < 0) and (A2, B2, C2) going up,
  // indexed like E by the layer between u and c (C = 0 on a ray's last step)
  const T *C = nullptr, *A2 = nullptr, *B2 = nullptr, *C2 = nullptr;
  // truncated frequency kernel (float32 operator, columns with lr_rank > 0):
  // R W ~ B A^T with A[q][s] = U[q][s] w_q^(1/2), B[f][s] = U[f][s] l_s w_f^(-1/2)
  const T *LR = nullptr;
};

// Frequency kernel of one point in low-rank form: z_k(f) = sum_s B[f][s]
// t_k(s), t_k(s) = sum_q A[q][s] m_k(q), for the rp ranks k of the angular
// factor.  m: [rp][nn] moments (read), t: [rp][r] scratch, z: [rp][nn] out
// (z may be m: m is not read after the first half).  Lanes of one warp.
template <typename T>
__device__ __forceinline__ void lowrank_frequency_warp(const T *A, const T *B, int r, int nn, int rp, const T *m,
                                                       T *t, T *z) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < rp * r; i += 32) {
    const int k = i / r, sidx = i - k * r;
    const T *mk = m + k * nn;
    T acc = 0;
    for (int q = 0; q < nn; ++q) acc = fma(A[q * r + sidx], mk[q], acc);
    t[i] = acc;
  }
  __syncwarp();
  for (int i = lane; i < rp * nn; i += 32) {
    const int k = i / nn, f = i - k * nn;
    const T *tk = t + k * r;
    const T *bf = B + f * r;
    T acc = 0;
    for (int sidx = 0; sidx < r; ++sidx) acc = fma(bf[sidx], tk[sidx], acc);
    z[i] = acc;
  }
  __syncwarp();
}

struct Common {
  const ColDev *cols;
  const int32_t *dir_cls;   // [sum nd] |mu| class of each direction
  const int32_t *dir_up;    // [sum nd] 1 if mu > 0 (sweeps towards the surface)
  const double *tsrc;       // [sum nz*nn] thermal term, or nullptr
  const double *I_top;      // [sum nn]
  const double *I_bot;      // [sum nn]
};

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// ------------------------------------------------------------ block reductions
// Sum NV per-thread values over the block; every thread receives the totals.
// `red` must hold (blockDim/32)*NV doubles; `out` NV doubles (shared).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *red, double *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    v[k] = s;
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp * NV + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * NV + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = out[k];
  __syncthreads();
}

// ------------------------------------------------- float64 <-> float32 casts
// On GB300 the conversion instructions between float64 and float32 run on the
// float64 pipe (about 0.6 T/s per GPU, measured), slower than streaming the
// values from HBM.  These casts work on the IEEE-754 bit fields with integer
// operations instead; values outside the float32 normal range (and zeros,
// subnormals, inf, nan) take the conversion instruction.
// narrow_f32: round to nearest even, as the cvt.rn.f32.f64 it replaces.
// In the normal float32 range the top 32 bits of (bits << 3) hold the low 9
// exponent bits and the 23 leading mantissa bits; subtracting 896 << 23
// rebiases the exponent (modulo 2^9 it is exact for biased exponents
// 897..1150); the 29 dropped bits round the result, a carry moving into the
// exponent as it should.  Zero and subnormal doubles give a signed zero.
__device__ __forceinline__ float narrow_f32(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (e - 897u > 253u) return e == 0u ? __uint_as_float(hi & 0x80000000u) : (float)v;
  uint32_t r = __funnelshift_l(lo, hi, 3) - (896u << 23);
  r += ((lo & 0x1fffffffu) + 0x0fffffffu + (r & 1u)) >> 29;
  return __uint_as_float(r | (hi & 0x80000000u));
}
// widen_f64: exact, as cvt.f64.f32.
__device__ __forceinline__ double widen_f64(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e - 1u > 253u) return (double)v;  // zero, subnormal, inf, nan
  const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// cvt<TO>(v): a cast that never issues a float64 <-> float32 conversion instruction
template <typename TO, typename FROM> __device__ __forceinline__ TO cvt(FROM v) { return (TO)v; }
template <> __device__ __forceinline__ float cvt<float, double>(double v) { return narrow_f32(v); }
template <> __device__ __forceinline__ double cvt<double, float>(float v) { return widen_f64(v); }

template <typename T> __device__ __forceinline__ T to(double v) { return cvt<T>(v); }
template <typename T> __device__ __forceinline__ T to(float v) { return cvt<T>(v); }
template <typename T> __device__ __forceinline__ T to(__half v) { return cvt<T>(__half2float(v)); }
__device__ __forceinline__ float as_f32(float v) { return v; }
__device__ __forceinline__ float as_f32(double v) { return narrow_f32(v); }
__device__ __forceinline__ float as_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ double as_f64(double v) { return v; }
__device__ __forceinline__ double as_f64(float v) { return widen_f64(v); }
__device__ __forceinline__ double as_f64(__half v) { return widen_f64(__half2float(v)); }

// ------------------------------------------------------------------ Sigma
// S_p = Gamma_p Psi W X_p for every point of one column (eq. Sigma), the
// separable kernel Phi = P (x) R taken in factored form:
//   m_k(nu')  = sum_d Uw[d][k] X(d, nu')                (angular moments)
//   z_k(nu)   = sum_nu' RwT[nu'][nu] m_k(nu')           (frequency kernel)
//   S(d, nu)  = gamma(nu) sum_k Ul[d][k] z_k(nu)        (+ t(nu) if tsrc)
// X is read in its own type and rounded to T; S is written in T.  Shared buffers:
// sm0, sm1 each kSigBuf elements of T.
// Points [p0, p0+np) of one column; np * rp * nn (separable) or np * nr
// (dense) must not exceed kSigBuf.  Ends with __syncthreads().  KR: ranks kept
// in registers per pass (a compile-time bound, so no dead predicated work).
template <typename T, typename TX, int KR>
__device__ void sigma_block_kr(const ColDev &c, const Tables<T> &tb, const TX *__restrict__ X,
                               T *__restrict__ S, int p0, int np, T *sm0, T *sm1) {
  const int nd = c.nd, nn = c.nn, nr = c.nr, rp = c.rp;
  const T *gam = tb.gamma + c.g_off;
  if (c.psi_off >= 0) {
    // Dense kernel: S = gamma * (PsiwT^T X_p); X_p staged in shared memory.
    const T *Pw = tb.PsiwT + c.psi_off;
    for (int i = threadIdx.x; i < np * nr; i += blockDim.x) sm0[i] = to<T>(X[(int64_t)p0 * nr + i]);
    __syncthreads();
    for (int i = threadIdx.x; i < np * nr; i += blockDim.x) {
      const int b = i / nr, r = i - b * nr;
      const T *xp = sm0 + b * nr;
      T acc = 0;
      for (int q = 0; q < nr; ++q) acc = fma(Pw[(int64_t)q * nr + r], xp[q], acc);
      S[(int64_t)(p0 + b) * nr + r] = gam[(int64_t)(p0 + b) * nn + (r % nn)] * acc;
    }
    __syncthreads();
    return;
  }
  const T *Uw = tb.Uw + c.u_off;
  const T *Ul = tb.Ul + c.u_off;
  const T *Rw = tb.RwT + c.r_off;
  const int per_pt = rp * nn;
  // 1. angular moments, one thread per (point, nu'), KR ranks in registers per pass
  for (int i = threadIdx.x; i < np * nn; i += blockDim.x) {
    const int b = i / nn, f = i - b * nn;
    const TX *xp = X + (int64_t)(p0 + b) * nr + f;
    for (int k0 = 0; k0 < rp; k0 += KR) {
      const int kn = min(KR, rp - k0);
      T m[KR];
#pragma unroll
      for (int k = 0; k < KR; ++k) m[k] = 0;
      int d = 0;
      for (; d + 4 <= nd; d += 4) {  // four independent loads in flight
        T xv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) xv[e] = to<T>(xp[(d + e) * nn]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const T *u = Uw + (d + e) * rp + k0;
#pragma unroll
          for (int k = 0; k < KR; ++k)
            if (k < kn) m[k] = fma(u[k], xv[e], m[k]);
        }
      }
      for (; d < nd; ++d) {
        const T xv = to<T>(xp[d * nn]);
        const T *u = Uw + d * rp + k0;
#pragma unroll
        for (int k = 0; k < KR; ++k)
          if (k < kn) m[k] = fma(u[k], xv, m[k]);
      }
#pragma unroll
      for (int k = 0; k < KR; ++k)
        if (k < kn) sm0[(b * rp + k0 + k) * nn + f] = m[k];
    }
  }
  __syncthreads();
  // 2. frequency kernel, one thread per (point, rank, nu)
  T *zbuf = sm1;
  if (tb.LR && c.lr_rank > 0 && !c.rdiag) {
    // low rank: t = A^T m into sm1, then z = B t into sm0 (moments consumed)
    const int lr = c.lr_rank;
    const T *A = tb.LR + c.lr_off, *Bf = A + (int64_t)nn * lr;
    for (int i = threadIdx.x; i < np * rp * lr; i += blockDim.x) {
      const int row = i / lr, sidx = i - row * lr;
      const T *mrow = sm0 + row * nn;
      T acc = 0;
      for (int q = 0; q < nn; ++q) acc = fma(A[q * lr + sidx], mrow[q], acc);
      sm1[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np * per_pt; i += blockDim.x) {
      const int row = i / nn, f = i - row * nn;
      const T *trow = sm1 + row * lr;
      T acc = 0;
      for (int sidx = 0; sidx < lr; ++sidx) acc = fma(Bf[f * lr + sidx], trow[sidx], acc);
      sm0[i] = acc;
    }
    zbuf = sm0;
  } else {
    for (int i = threadIdx.x; i < np * per_pt; i += blockDim.x) {
      const int f = i % nn;
      const T *mrow = sm0 + (i - f);
      T acc;
      if (c.rdiag) {
        acc = Rw[f] * mrow[f];
      } else {
        acc = 0;
        for (int q = 0; q < nn; ++q) acc = fma(Rw[q * nn + f], mrow[q], acc);
      }
      sm1[i] = acc;
    }
  }
  __syncthreads();
  // 3. expansion over directions, scaled by Gamma: one thread per (point, nu)
  //    with its ranks' z and Gamma in registers, looping over the directions
  //    (stores of a warp stay contiguous in nu); same sums, same order
  if (rp <= KR) {
    for (int i = threadIdx.x; i < np * nn; i += blockDim.x) {
      const int b = i / nn, f = i - b * nn;
      const T *zb = zbuf + b * per_pt + f;
      T z[KR];
#pragma unroll
      for (int k = 0; k < KR; ++k) z[k] = k < rp ? zb[k * nn] : T(0);
      const T g = gam[(int64_t)(p0 + b) * nn + f];
      T *out = S + (int64_t)(p0 + b) * nr + f;
      for (int d = 0; d < nd; ++d) {
        const T *u = Ul + d * rp;
        T acc = 0;
#pragma unroll
        for (int k = 0; k < KR; ++k)
          if (k < rp) acc = fma(u[k], z[k], acc);
        out[(int64_t)d * nn] = g * acc;
      }
    }
  } else {
    for (int i = threadIdx.x; i < np * nr; i += blockDim.x) {
      const int b = i / nr, r = i - b * nr, d = r / nn, f = r - d * nn;
      const T *zb = zbuf + b * per_pt + f;
      const T *u = Ul + d * rp;
      T acc = 0;
      for (int k = 0; k < rp; ++k) acc = fma(u[k], zb[k * nn], acc);
      S[(int64_t)(p0 + b) * nr + r] = gam[(int64_t)(p0 + b) * nn + f] * acc;
    }
  }
  __syncthreads();
}

template <typename T, typename TX>
__device__ void sigma_block(const ColDev &c, const Tables<T> &tb, const TX *__restrict__ X,
                            T *__restrict__ S, int p0, int np, T *sm0, T *sm1) {
  if (c.rp <= 2) sigma_block_kr<T, TX, 2>(c, tb, X, S, p0, np, sm0, sm1);
  else sigma_block_kr<T, TX, 8>(c, tb, X, S, p0, np, sm0, sm1);
}

// ---- separable Sigma, one warp per point --------------------------------
constexpr int kWarpBuf = 1024;  // elements of each per-warp shared buffer

// True when the per-warp form applies (separable kernel, rank*n_nu small).
__host__ __device__ inline bool sigma_warp_ok(const ColDev &c) {
  return c.psi_off < 0 && c.rp * c.nn <= kWarpBuf;
}

// S_p = Gamma_p (factored P (x) R) X_p for points p = p_begin + warp, stepping
// by the number of warps in the block.  wm, wz: this warp's two shared
// buffers of kWarpBuf T.  Only __syncwarp inside: warps progress on their own,
// so the loads of many points are in flight at once.
template <typename T, typename TX, int KR>
__device__ void sigma_points_warp(const ColDev &c, const Tables<T> &tb, const TX *__restrict__ X,
                                  T *__restrict__ S, int p_begin, int p_end, T *wm, T *wz,
                                  const T *rw_cached = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nd = c.nd, nn = c.nn, nr = c.nr, rp = c.rp;
  const T *Uw = tb.Uw + c.u_off;
  const T *Ul = tb.Ul + c.u_off;
  const T *Rw = rw_cached ? rw_cached : tb.RwT + c.r_off;
  const T *gam = tb.gamma + c.g_off;
  for (int p = p_begin + warp; p < p_end; p += nw) {
    const TX *xp = X + (int64_t)p * nr;
    // 1. moments m_k(f) = sum_d Uw[d][k] X(d, f); lanes over f, KR ranks per pass
    for (int f = lane; f < nn; f += 32) {
      for (int k0 = 0; k0 < rp; k0 += KR) {
        const int kn = min(KR, rp - k0);
        T m[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) m[k] = 0;
        int d = 0;
        for (; d + 8 <= nd; d += 8) {
          T xv[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) xv[e] = to<T>(xp[(d + e) * nn + f]);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const T *u = Uw + (d + e) * rp + k0;
#pragma unroll
            for (int k = 0; k < KR; ++k)
              if (k < kn) m[k] = fma(u[k], xv[e], m[k]);
          }
        }
        for (; d < nd; ++d) {
          const T xv = to<T>(xp[d * nn + f]);
          const T *u = Uw + d * rp + k0;
#pragma unroll
          for (int k = 0; k < KR; ++k)
            if (k < kn) m[k] = fma(u[k], xv, m[k]);
        }
#pragma unroll
        for (int k = 0; k < KR; ++k)
          if (k < kn) wm[(k0 + k) * nn + f] = m[k];
      }
    }
    __syncwarp();
    const T *zw = wz;
    if (tb.LR && c.lr_rank > 0 && !c.rdiag) {
      // low rank: t into wz, z back into wm (moments consumed)
      const T *A = tb.LR + c.lr_off;
      lowrank_frequency_warp<T>(A, A + (int64_t)nn * c.lr_rank, c.lr_rank, nn, rp, wm, wz, wm);
      zw = wm;
    } else
    // 2. frequency kernel z_k(f) = sum_q RwT[q][f] m_k(q): each lane owns two
    //    frequencies (f, f+32) and KR ranks, so a RwT load feeds KR FMAs and a
    //    moment load feeds two
    for (int fb = 0; fb < nn; fb += 64) {
      const int fa = fb + lane, fc = fa + 32;
      const bool va = fa < nn, vc = fc < nn;
      const int fa_ = va ? fa : 0, fc_ = vc ? fc : 0;
      for (int k0 = 0; k0 < rp; k0 += KR) {
        const int kn = min(KR, rp - k0);
        const T *mk = wm + k0 * nn;
        T aa[KR], ac[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) aa[k] = ac[k] = 0;
        if (c.rdiag) {
#pragma unroll
          for (int k = 0; k < KR; ++k)
            if (k < kn) {
              aa[k] = Rw[fa_] * mk[k * nn + fa_];
              ac[k] = Rw[fc_] * mk[k * nn + fc_];
            }
        } else {
          for (int q = 0; q < nn; ++q) {
            const T ra = Rw[q * nn + fa_], rc = Rw[q * nn + fc_];
#pragma unroll
            for (int k = 0; k < KR; ++k)
              if (k < kn) {
                const T mv = mk[k * nn + q];
                aa[k] = fma(ra, mv, aa[k]);
                ac[k] = fma(rc, mv, ac[k]);
              }
          }
        }
#pragma unroll
        for (int k = 0; k < KR; ++k)
          if (k < kn) {
            if (va) wz[(k0 + k) * nn + fa] = aa[k];
            if (vc) wz[(k0 + k) * nn + fc] = ac[k];
          }
      }
    }
    __syncwarp();
    // 3. expansion S(d, f) = gamma(f) sum_k Ul[d][k] z_k(f)
    const T *g = gam + (int64_t)p * nn;
    T *sp = S + (int64_t)p * nr;
    for (int r = lane; r < nr; r += 32) {
      const int d = r / nn, f = r - d * nn;
      const T *u = Ul + d * rp;
      T acc = 0;
      for (int k = 0; k < rp; ++k) acc = fma(u[k], zw[k * nn + f], acc);
      sp[r] = g[f] * acc;
    }
    __syncwarp();
  }
}

// Points per Sigma tile of the apply kernel (256 threads): what fits the two
// block buffers, at most max_pts.
__host__ __device__ inline int sigma_points_per_block(const ColDev &c, int max_pts = 1 << 30) {
  const int per_pt = c.psi_off >= 0 ? c.nr : c.rp * c.nn;
  int pb = kSigBuf / per_pt;
  if (pb > max_pts) pb = max_pts;
  return pb < 1 ? 1 : pb;
}

// Every point of one column, block by block (one CTA).
// smbuf holds cap elements of T (cap >= 2*kSigBuf); warps take equal shares
// of it when the per-warp form fits, else it is split into the two block buffers.
// rw_cached: this column's RwT already staged in shared memory, or nullptr.
template <typename T, typename TX>
__device__ __noinline__ void sigma_column(const ColDev &c, const Tables<T> &tb, const TX *__restrict__ X,
                             T *__restrict__ S, T *smbuf, int cap, const T *rw_cached = nullptr) {
  const int nw = blockDim.x >> 5;
  const int per_warp = cap / nw / 2;
  if (sigma_warp_ok(c) && c.rp * c.nn <= per_warp) {
    T *wm = smbuf + (threadIdx.x >> 5) * 2 * per_warp;
    if (c.rp <= 2) sigma_points_warp<T, TX, 2>(c, tb, X, S, 0, c.nz, wm, wm + per_warp, rw_cached);
    else sigma_points_warp<T, TX, 8>(c, tb, X, S, 0, c.nz, wm, wm + per_warp, rw_cached);
    __syncthreads();
    return;
  }
  const int pb = sigma_points_per_block(c);
  for (int p0 = 0; p0 < c.nz; p0 += pb)
    sigma_block<T, TX>(c, tb, X, S, p0, min(pb, c.nz - p0), smbuf, smbuf + kSigBuf);
}

// ------------------------------------------------------------------ sweep
enum SweepOut : int {
  kOutAminus = 0,  // y = x - I            (A x with I = Lambda Sigma x)
  kOutI = 1,       // y = I                (Lambda S, or the right-hand side)
  kOutResid = 2,   // y = b - x + I        (b - A x), returns the squared norm
  kOutAminusB = 3  // y = x - I - b        (A x - b: a direction minus a known vector)
};

// Formal solution along every ray of one column (eqs. ie_1, ie_2 with the
// coefficients of the chosen step): mu < 0 from the surface down, mu > 0 from
// the deep boundary up.  The source is S[p][r] (T), or the thermal term
// broadcast over directions when `tsrc` is non-null.  With `inflow` the first
// point of each ray holds I_top / I_bot, else 0.  Loads run ahead of the
// recurrence by kAhead depth points.  Returns this thread's partial sum of y^2
// for kOutResid (0 otherwise).  y may alias S: each thread reads S and writes y
// only at the points of its own rays, the source value is read before the
// output at the same point is written.  OUT >= 0 fixes the output mode at
// compile time (then `out` is ignored): the x and b values a mode does not
// use hold no registers, and b is loaded ahead with the other values.
template <typename T, typename TX, typename TY, int kAhead = 4, bool kQuad = false, int OUT = -1>
__device__ double sweep_ray(const ColDev &c, const Tables<T> &tb, const Common &cm, const T *S,
                            const double *__restrict__ tsrc, const TX *__restrict__ x,
                            const double *__restrict__ bv, TY *y, int out_rt, bool inflow, int r) {
  const int out = OUT >= 0 ? OUT : out_rt;
  constexpr bool pre_b = OUT == kOutResid || OUT == kOutAminusB;  // b prefetched (compile-time modes)
  const int nz = c.nz, nn = c.nn, nr = c.nr, ncls = c.ncls;
  const int d = r / nn, f = r - d * nn;
  const int up = cm.dir_up[c.d_off + d];
  constexpr bool quad = kQuad;  // quadratic SC (c.fs == 2): a downwind source term
  const T *E = tb.E + c.c_off;
  const T *A = (quad && up ? tb.A2 : tb.A) + c.c_off, *B = (quad && up ? tb.B2 : tb.B) + c.c_off;
  const T *Cq = quad ? (up ? tb.C2 : tb.C) + c.c_off : nullptr;
  double ss = 0.0;
  const int cls = cm.dir_cls[c.d_off + d];
  const int step = up ? -1 : 1;
  const int i0 = up ? nz - 1 : 0;
  const bool want_x = out != kOutI;
  T Iu = 0;
  if (inflow) Iu = cvt<T>(up ? cm.I_bot[c.in_off + f] : cm.I_top[c.in_off + f]);
  auto src = [&](int i) -> T {
    return tsrc ? cvt<T>(tsrc[(int64_t)i * nn + f]) : S[(int64_t)i * nr + r];
  };
  // y at point i from the intensity I and the prefetched x (and b) values
  // (the float32 operator, T = float, subtracts in float32: x is rounded to
  // float32 first, and no float64 instruction is issued)
  auto emit = [&](int i, T I, TX xi, double bi) {
    const int64_t k = (int64_t)i * nr + r;
    if (out == kOutResid) {
      const double v = (pre_b ? bi : bv[k]) - as_f64(xi) + as_f64(I);
      y[k] = cvt<TY>(v);
      ss += v * v;
    } else if (out == kOutAminusB) {
      y[k] = cvt<TY>(as_f64(xi) - as_f64(I) - (pre_b ? bi : bv[k]));
    } else if (out == kOutI) {
      y[k] = cvt<TY>(I);
    } else if (sizeof(T) == 4) {
      y[k] = cvt<TY>(as_f32(xi) - (float)I);
    } else {
      y[k] = cvt<TY>(as_f64(xi) - as_f64(I));
    }
  };
  // loads of the points i+step .. i+cnt*step (cnt <= kAhead); indices past
  // the column are clamped to its last point (the values are not used)
  auto load = [&](int i, int cnt, T (&e)[kAhead], T (&a)[kAhead], T (&b)[kAhead], T (&cq)[kAhead],
                  T (&sc)[kAhead], TX (&xv)[kAhead], double (&bb)[kAhead]) {
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      int ic = i + (u + 1) * step;
      ic = u < cnt ? ic : i0 + (nz - 1) * step;
      const int layer = up ? ic : ic - 1;  // layer between ic and its upwind point
      const int64_t ci = ((int64_t)layer * ncls + cls) * nn + f;
      e[u] = E[ci];
      a[u] = A[ci];
      b[u] = B[ci];
      cq[u] = quad ? Cq[ci] : T(0);
      sc[u] = src(ic);
      xv[u] = want_x ? x[(int64_t)ic * nr + r] : TX(0);
      bb[u] = pre_b ? bv[(int64_t)ic * nr + r] : 0.0;
    }
  };
  T Su = src(i0);
  emit(i0, Iu, want_x ? x[(int64_t)i0 * nr + r] : TX(0), pre_b ? bv[(int64_t)i0 * nr + r] : 0.0);
  // chunks of kAhead points; the next chunk's loads are issued before the
  // current chunk's recurrence (2 kAhead points of loads in flight)
  T e0[kAhead], a0[kAhead], b0[kAhead], c0[kAhead], s0[kAhead];
  TX x0[kAhead];
  double bb0[kAhead];
  int i = i0;
  int cnt = min(kAhead, nz - 1);
  if (cnt > 0) load(i, cnt, e0, a0, b0, c0, s0, x0, bb0);
  for (int done = 1; done < nz; done += kAhead) {
    const int inext = i + cnt * step;
    const int cnext = min(kAhead, nz - done - cnt);
    T e1[kAhead], a1[kAhead], b1[kAhead], c1[kAhead], s1[kAhead];
    TX x1[kAhead];
    double bb1[kAhead];
    if (cnext > 0) load(inext, cnext, e1, a1, b1, c1, s1, x1, bb1);
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      if (u < cnt) {
        T Ic = fma(e0[u], Iu, fma(a0[u], Su, b0[u] * s0[u]));
        if (quad) {  // downwind source: next point of this chunk, or the next chunk's first
          const T Sd = u + 1 < cnt ? s0[u + 1 < kAhead ? u + 1 : 0] : (cnext > 0 ? s1[0] : T(0));
          Ic = fma(c0[u], Sd, Ic);
        }
        emit(i + (u + 1) * step, Ic, x0[u], bb0[u]);
        Iu = Ic;
        Su = s0[u];
      }
    }
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      e0[u] = e1[u];
      a0[u] = a1[u];
      b0[u] = b1[u];
      c0[u] = c1[u];
      s0[u] = s1[u];
      x0[u] = x1[u];
      bb0[u] = bb1[u];
    }
    i = inext;
    cnt = cnext;
  }
  return out == kOutResid ? ss : 0.0;
}

// Formal solution along every ray of one column (eqs. ie_1, ie_2 with the
// coefficients of the chosen step): mu < 0 from the surface down, mu > 0 from
// the deep boundary up.  The source is S[p][r] (T), or the thermal term
// broadcast over directions when `tsrc` is non-null.  With `inflow` the first
// point of each ray holds I_top / I_bot, else 0.  Loads run ahead of the
// recurrence by kAhead depth points.  Returns this thread's partial sum of y^2
// for kOutResid (0 otherwise).  y may alias S: each thread reads S and writes y
// only at the points of its own rays, the source value is read before the
// output at the same point is written.
// The output mode OUT (kOutAminus, kOutI, kOutResid, kOutAminusB) is a
// compile-time parameter; the quadratic and linear steps are separate
// non-inlined functions, each with its own register allocation.
template <typename T, typename TX, typename TY, int kAhead, int OUT, bool kQuad>
__device__ __noinline__ double sweep_rays(const ColDev &c, const Tables<T> &tb, const Common &cm, const T *S,
                                          const double *__restrict__ tsrc, const TX *__restrict__ x,
                                          const double *__restrict__ bv, TY *y, bool inflow) {
  double ss = 0.0;
  for (int r = threadIdx.x; r < c.nr; r += blockDim.x)
    ss += sweep_ray<T, TX, TY, kAhead, kQuad, OUT>(c, tb, cm, S, tsrc, x, bv, y, OUT, inflow, r);
  return ss;
}

template <typename T, typename TX, typename TY, int kAhead, int OUT>
__device__ __forceinline__ double sweep_column(const ColDev &c, const Tables<T> &tb, const Common &cm,
                                               const T *S, const double *__restrict__ tsrc,
                                               const TX *__restrict__ x, const double *__restrict__ bv, TY *y,
                                               bool inflow) {
  if (c.fs == 2) return sweep_rays<T, TX, TY, kAhead, OUT, true>(c, tb, cm, S, tsrc, x, bv, y, inflow);
  return sweep_rays<T, TX, TY, kAhead, OUT, false>(c, tb, cm, S, tsrc, x, bv, y, inflow);
}

}  // namespace rt
