// rt_box.cu -- 3D boxes (Sec. 3.4): short-characteristics formal solution
// between consecutive z-planes, periodic in x and y, with bilinear
// interpolation of I, S and chi at the upwind point (the interpolation
// operators T_RC, T_CR of Sec. 3.4, rows summing to one).
//
// k_sweep3d: one CTA per (direction, block of frequencies spanning 32 bytes)
// marches the planes; the previous plane's intensity lives in shared memory,
// the upwind source and opacity are gathered from global memory (L1/L2), the
// optical depth 0.5 (chi_u + chi_c) ds and the step coefficients are formed on
// the fly (float32 path: expf / expm1f; float64 path: exp / expm1 and the
// alternating series for w1/dtau below 0.1).
#include <cuda_runtime.h>

#include "rt_host.h"
#include "rt_internal.cuh"

namespace rt {

template <typename T>
__device__ __forceinline__ void step_coef(T d, int ie, T &e, T &a, T &b) {
  if (ie) {
    e = (T)1 / ((T)1 + d);
    a = 0;
    b = d * e;
    return;
  }
  T w0;
  if (sizeof(T) == 8) {
    e = (T)exp((double)-d);
    w0 = (T)-expm1((double)-d);
  } else {
    e = (T)expf((float)-d);
    w0 = (T)-expm1f((float)-d);
  }
  T beta;
  if (d < (T)0.1) {
    // w1/d = (d/2)(1 - (d/3)(1 - (d/4)(1 - ...))): 16 terms (fp64), 8 (fp32)
    T s = 1;
    const int top = sizeof(T) == 8 ? 17 : 9;
    for (int j = top; j >= 3; --j) s = (T)1 - (d / (T)j) * s;
    beta = (T)0.5 * d * s;
  } else {
    beta = (d - w0) / d;
  }
  b = beta;
  a = w0 - beta;
}

// geo per direction (6 doubles): fx, fy (integer upwind shift in cells,
// reduced modulo nx, ny: the box is periodic), ax, ay (fractional parts),
// ds (path length between planes), up (1: Omega_z > 0)
template <typename T, int VPT>
__global__ void __launch_bounds__(1024, 1) k_sweep3d(BoxDev bx, const double *__restrict__ geo,
                                                  const T *__restrict__ chi, const T *S,
                                                  const double *__restrict__ tsrc, const void *xin,
                                                  int x_is_float, void *yout, int y_is_float, int out,
                                                  int inflow, const double *__restrict__ I_top,
                                                  const double *__restrict__ I_bot) {
  constexpr int FB = 32 / sizeof(T);
  extern __shared__ __align__(16) unsigned char sw_smem[];
  T *Ip = reinterpret_cast<T *>(sw_smem);  // [plane][FB]
  const int nd = bx.nd, nn = bx.nn, nx = bx.nx, ny = bx.ny, nz = bx.nz;
  const int plane = nx * ny;
  const int nfb = (nn + FB - 1) / FB;
  const int d = blockIdx.x / nfb, f0 = (blockIdx.x % nfb) * FB;
  const int nr = nd * nn;
  const double *g = geo + 6 * d;
  const int fx = (int)g[0], fy = (int)g[1];
  const T ax = (T)g[2], ay = (T)g[3];
  const T hds = (T)(0.5 * g[4]);
  const int up = g[5] > 0.5;
  const T w00 = ((T)1 - ay) * ((T)1 - ax), w01 = ((T)1 - ay) * ax, w10 = ay * ((T)1 - ax), w11 = ay * ax;
  const int step = up ? -1 : 1;
  const int k0 = up ? nz - 1 : 0;
  const int nval = plane * FB;
  const double *xd = static_cast<const double *>(xin);
  const float *xf = static_cast<const float *>(xin);
  double *yd = static_cast<double *>(yout);
  float *yf = static_cast<float *>(yout);
  auto emit = [&](int64_t k, T I) {
    if (out == kOutI) {
      if (y_is_float) yf[k] = (float)I;
      else yd[k] = (double)I;
    } else if (y_is_float && x_is_float) {
      yf[k] = xf[k] - (float)I;
    } else {
      const double v = (x_is_float ? (double)xf[k] : xd[k]) - (double)I;
      if (y_is_float) yf[k] = (float)v;
      else yd[k] = v;
    }
  };
  auto src = [&](int64_t p, int f) -> T {
    return tsrc ? (T)tsrc[p * nn + f] : S[p * nr + (int64_t)d * nn + f];
  };
  const bool pow2 = (nx & (nx - 1)) == 0;
  const int lgx = __ffs(nx) - 1;
  // first plane: inflow (or zero)
  for (int v = threadIdx.x; v < nval; v += blockDim.x) {
    const int c = v / FB, fl = v - c * FB, f = f0 + fl;
    T I0 = 0;
    if (inflow && f < nn) I0 = (T)(up ? I_bot[f] : I_top[f]);
    Ip[v] = I0;
    if (f < nn) emit(((int64_t)k0 * plane + c) * nr + (int64_t)d * nn + f, I0);
  }
  __syncthreads();
  for (int s = 1; s < nz; ++s) {
    const int k = k0 + s * step, ku = k - step;
    const int64_t pu = (int64_t)ku * plane, pk = (int64_t)k * plane;
    T In[VPT];
#pragma unroll
    for (int i = 0; i < VPT; ++i) {
      In[i] = 0;
      const int v = threadIdx.x + i * blockDim.x;
      if (v >= nval) continue;
      const int c = v / FB, fl = v - c * FB, f = f0 + fl;
      if (f >= nn) continue;
      const int y = pow2 ? (c >> lgx) : c / nx, x = c - y * nx;
      int x0 = x - fx, y0 = y - fy;
      if (x0 < 0) x0 += nx;
      if (y0 < 0) y0 += ny;
      const int x1 = x0 == 0 ? nx - 1 : x0 - 1;
      const int y1 = y0 == 0 ? ny - 1 : y0 - 1;
      const int c00 = y0 * nx + x0, c01 = y0 * nx + x1, c10 = y1 * nx + x0, c11 = y1 * nx + x1;
      const int64_t pc = pk + c;
      const T Iu = w00 * Ip[c00 * FB + fl] + w01 * Ip[c01 * FB + fl] + w10 * Ip[c10 * FB + fl] +
                   w11 * Ip[c11 * FB + fl];
      const T Su = w00 * src(pu + c00, f) + w01 * src(pu + c01, f) + w10 * src(pu + c10, f) +
                   w11 * src(pu + c11, f);
      const T cu = w00 * chi[(pu + c00) * nn + f] + w01 * chi[(pu + c01) * nn + f] +
                   w10 * chi[(pu + c10) * nn + f] + w11 * chi[(pu + c11) * nn + f];
      T e, a, b;
      step_coef<T>(hds * (cu + chi[pc * nn + f]), bx.ie, e, a, b);
      In[i] = e * Iu + a * Su + b * src(pc, f);
      emit(pc * nr + (int64_t)d * nn + f, In[i]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < VPT; ++i) {
      const int v = threadIdx.x + i * blockDim.x;
      if (v < nval) Ip[v] = In[i];
    }
    __syncthreads();
  }
}

// Launch the 3D sweep; x/y may be float or double (the float64 path passes
// double for both).  32 values per thread; threads per CTA = plane*FB/32.
template <typename T>
static int sweep3d_launch(rt_handle *h, const T *chi, const T *S, const double *tsrc, const void *x,
                          bool xf, void *y, bool yf, int out, bool inflow, cudaStream_t s) {
  const BoxDev &bx = h->box;
  constexpr int FB = 32 / sizeof(T);
  constexpr int VPT = 32;
  const int plane = bx.nx * bx.ny;
  const int nval = plane * FB;
  const int nfb = (bx.nn + FB - 1) / FB;
  const int grid = bx.nd * nfb;
  const size_t smem = (size_t)nval * sizeof(T);
  int nt = (nval + VPT - 1) / VPT;
  nt = (nt + 31) / 32 * 32;
  if (nt > 1024 || plane >= 65536) return (int)cudaErrorInvalidConfiguration;
  cudaFuncSetAttribute(k_sweep3d<T, VPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_sweep3d<T, VPT><<<grid, nt, smem, s>>>(bx, h->d_geo, chi, S, tsrc, x, xf ? 1 : 0, y, yf ? 1 : 0, out,
                                           inflow ? 1 : 0, h->d_Itop, h->d_Ibot);
  return (int)cudaGetLastError();
}

int launch_sweep3d(rt_handle *h, bool fp64, const void *S, const double *tsrc, const void *x, bool xf,
                   void *y, bool yf, int out, bool inflow, cudaStream_t s) {
  if (fp64)
    return sweep3d_launch<double>(h, h->chi64, static_cast<const double *>(S), tsrc, x, xf, y, yf, out,
                                  inflow, s);
  return sweep3d_launch<float>(h, h->chi32, static_cast<const float *>(S), tsrc, x, xf, y, yf, out, inflow,
                               s);
}

}  // namespace rt
