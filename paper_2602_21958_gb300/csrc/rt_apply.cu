// rt_apply.cu -- the operators of rt_apply over a batch of 1D columns, as two
// fully parallel kernels:
//   k_sigma_tiles : Sigma on (instance, block of points) tiles      (eq. Sigma)
//   k_sweep_tiles : one thread per ray on (instance, block of rays)  (eqs. ie_1, ie_2)
// The source function makes one round trip through HBM between them.
#include <cuda_runtime.h>

#include <mutex>

#include "rt_host.h"
#include "rt_internal.cuh"

namespace rt {

constexpr int kSigNT = 256;

// skip_tc: columns handled by the tensor-core kernel are left to it
template <typename T, typename TX>
__global__ void __launch_bounds__(kSigNT) k_sigma_tiles(Common cm, Tables<T> tb, const int3 *tiles,
                                                        int n_cols, int64_t E, const TX *X, T *S,
                                                        int skip_tc) {
  __shared__ T sm[2 * kSigBuf];
  const int3 t = tiles[blockIdx.x];
  const int ci = t.x % n_cols, rhs = t.x / n_cols;
  const ColDev c = cm.cols[ci];
  if (skip_tc && c.psi_off >= 0 && c.nr % 16 == 0) return;
  const int64_t base = rhs * E + c.x_off;
  sigma_block<T, TX>(c, tb, X + base, S + base, t.y, t.z, sm, sm + kSigBuf);
}

// out: kOutAminus (y = x - Lambda S), kOutI (y = Lambda S, or Lambda t + I_in
// when tsrc is set and inflow is on).  RB rays per tile (threads), AH depth
// points of loads issued ahead (both picked by rt_autotune).
template <typename T, int RB, int AH>
__global__ void __launch_bounds__(RB) k_sweep_tiles(Common cm, Tables<T> tb, const int2 *tiles,
                                                    int n_cols, int64_t E, const T *S,
                                                    const double *x, double *y, int out,
                                                    int use_tsrc, int inflow) {
  const int2 t = tiles[blockIdx.x];
  const int ci = t.x % n_cols, rhs = t.x / n_cols;
  const ColDev c = cm.cols[ci];
  const int r = t.y + threadIdx.x;
  if (r >= c.nr) return;
  const int64_t base = rhs * E + c.x_off;
  const double *ts = use_tsrc ? cm.tsrc + c.g_off : nullptr;
  if (c.fs == 2)
    sweep_ray<T, double, double, AH, true>(c, tb, cm, S ? S + base : nullptr, ts, x ? x + base : nullptr, nullptr,
                                           y + base, out, inflow != 0, r);
  else
    sweep_ray<T, double, double, AH, false>(c, tb, cm, S ? S + base : nullptr, ts, x ? x + base : nullptr,
                                            nullptr, y + base, out, inflow != 0, r);
}

template <typename T>
__global__ void k_convert(const double *a, T *b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = cvt<T>(a[i]);
}

template <typename T>
__global__ void k_widen(const T *a, double *b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = cvt<double>(a[i]);
}

// sweep launch with the handle's tuned (ray block, loads ahead)
template <typename T>
static void sweep_launch(rt_handle *h, int nsw, const Common &cm, const Tables<T> &tb, const T *S,
                         const double *x, double *y, int out, int use_tsrc, int inflow, cudaStream_t s) {
#define RT_SW(RB, AH)                                                                                      \
  k_sweep_tiles<T, RB, AH><<<nsw, RB, 0, s>>>(cm, tb, h->d_sw_tiles, h->n_cols, h->E, S, x, y, out, use_tsrc, \
                                             inflow)
  const int rb = h->tune.ray_block, ah = h->tune.ahead;
  if (rb == 64) {
    if (ah == 2) RT_SW(64, 2); else if (ah == 8) RT_SW(64, 8); else RT_SW(64, 4);
  } else if (rb == 256) {
    if (ah == 2) RT_SW(256, 2); else if (ah == 8) RT_SW(256, 8); else RT_SW(256, 4);
  } else {
    if (ah == 2) RT_SW(128, 2); else if (ah == 8) RT_SW(128, 8); else RT_SW(128, 4);
  }
#undef RT_SW
}

template <typename T>
static int run_apply(rt_handle *h, const Tables<T> &tb, int op, const double *x, double *y, cudaStream_t s,
                     bool first_rhs_only, void *scratch) {
  const Common cm{h->d_cols, h->d_dir_cls, h->d_dir_up, h->d_tsrc, h->d_Itop, h->d_Ibot};
  const int nsig = first_rhs_only ? h->n_sig_tiles_rhs0 : h->n_sig_tiles;
  const int nsw = first_rhs_only ? h->n_sw_tiles_rhs0 : h->n_sw_tiles;
  const int64_t len = (first_rhs_only ? 1 : h->n_rhs) * h->E;
  T *S = reinterpret_cast<T *>(scratch ? scratch : h->apply_S);
  const bool tc = sizeof(T) == 4 && h->n_tc_jobs > 0 && !first_rhs_only;
  auto sigma = [&]() -> int {
    k_sigma_tiles<T, double><<<nsig, kSigNT, 0, s>>>(cm, tb, h->d_sig_tiles, h->n_cols, h->E, x, S, tc ? 1 : 0);
    if (tc) return launch_sigma_dense_tc(h, false, x, S, false, s);
    return 0;
  };
  const int cgrid = (int)std::min<int64_t>((len + 255) / 256, 16 * 152);
  switch (op) {
    case 0:  // y = x - Lambda Sigma x
      sigma();
      sweep_launch<T>(h, nsw, cm, tb, S, x, y, kOutAminus, 0, 0, s);
      break;
    case 1:  // y = Lambda x
      k_convert<T><<<cgrid, 256, 0, s>>>(x, S, len);
      sweep_launch<T>(h, nsw, cm, tb, S, nullptr, y, kOutI, 0, 0, s);
      break;
    case 2:  // y = Sigma x
      if (tc && tc_all_columns(h)) {  // every column on the tensor cores: straight into y
        const int e = launch_sigma_dense_tc(h, false, x, y, true, s);
        if (e) return e;
        break;
      }
      sigma();
      k_widen<T><<<cgrid, 256, 0, s>>>(S, y, len);
      break;
    default:  // y = Lambda t + I_in
      if (h->d_tsrc) {
        sweep_launch<T>(h, nsw, cm, tb, nullptr, nullptr, y, kOutI, 1, 1, s);
      } else {
        cudaMemsetAsync(S, 0, len * sizeof(T), s);
        sweep_launch<T>(h, nsw, cm, tb, S, nullptr, y, kOutI, 0, 1, s);
      }
  }
  return (int)cudaGetLastError();
}

static int launch_apply_s(rt_handle *h, int op, bool fp64, const double *x, double *y, cudaStream_t s,
                          bool first_rhs_only, void *scratch) {
  if (h->dims == 3) return box_apply(h, op, fp64, x, false, y, false, s, scratch);
  if (fp64 || h->precision == 0) {
    const Tables<double> tb = tables64(h);
    return run_apply<double>(h, tb, op, x, y, s, first_rhs_only, scratch);
  }
  const Tables<float> tb = tables32(h);
  return run_apply<float>(h, tb, op, x, y, s, first_rhs_only, scratch);
}

int launch_apply(rt_handle *h, int op, bool fp64, const double *x, double *y, cudaStream_t s,
                 bool first_rhs_only) {
  return launch_apply_s(h, op, fp64, x, y, s, first_rhs_only, nullptr);
}

// ------------------------------------------------ allocation-free apply
// Scratch of rt_apply_noalloc: the source function S of one apply lives in
// this file-scope device array instead of handle-owned memory.  Every GPU that
// loads the library holds it until the process exits.  Host code must not
// pass the symbol itself to a kernel (it is a host-side stand-in); the device
// address is taken with cudaGetSymbolAddress once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[256] = {};
}  // namespace

// Device address of the scratch array on the current device (set-up on the
// first call per device, with that device current).  Returns a cudaError_t.
static int noalloc_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= 256) return (int)cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return (int)e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return 0;
}

int launch_apply_noalloc(rt_handle *h, int op, bool fp64, const double *x, double *y, cudaStream_t s) {
  void *scratch = nullptr;
  const int e = noalloc_scratch(&scratch);
  if (e) return e;
  return launch_apply_s(h, op, fp64, x, y, s, false, scratch);
}

}  // namespace rt
