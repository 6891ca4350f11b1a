// rt_api.cu -- C ABI entry points (include/rt_gb300.h): validation, host-side
// factorisation of the separable scattering kernel, device tables, workspaces.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <numeric>
#include <thread>
#include <utility>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rt_gb300.h"
#include "rt_host.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

// Host-side fault injection for failure-detection tests (no GPU fault is
// ever made): the environment variable RT_FAULT, read at each call, set to
//   alloc     -> rt_create / rt_create_batch fail with RT_ERR_OOM before any
//                device call,
//   launch    -> rt_apply, rt_apply_noalloc, rt_solve and rt_arnoldi fail with
//                RT_ERR_CUDA before launching anything,
//   nan_input -> rt_solve reports a non-finite input (RT_ERR_NONFINITE, info
//                filled) without launching,
//   stall     -> the bounded waits of the tensor-core Sigma poll once, so they
//                give up and the call returns RT_ERR_TIMEOUT (the kernel
//                drains its own work and frees its tensor memory first).
enum Fault { kFaultNone = 0, kFaultAlloc, kFaultLaunch, kFaultNan, kFaultStall };

int fault_now() {
  const char *f = std::getenv("RT_FAULT");
  if (!f || !*f) return kFaultNone;
  if (!std::strcmp(f, "alloc")) return kFaultAlloc;
  if (!std::strcmp(f, "launch")) return kFaultLaunch;
  if (!std::strcmp(f, "nan_input")) return kFaultNan;
  if (!std::strcmp(f, "stall")) return kFaultStall;
  return kFaultNone;
}

// RT_FAULT=stall for the duration of one call: pipeline waits poll once
struct StallScope {
  rt_handle *h;
  long long saved;
  explicit StallScope(rt_handle *hh) : h(hh), saved(hh->wait_limit) {
    if (fault_now() == kFaultStall) h->wait_limit = 1;
  }
  ~StallScope() { h->wait_limit = saved; }
};

#define RT_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      g_err = std::string(#call) + ": " + cudaGetErrorString(e_);                            \
      return e_ == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;                     \
    }                                                                                        \
  } while (0)

template <typename T>
int dev_upload(T **dst, const std::vector<T> &src) {
  *dst = nullptr;
  if (src.empty()) return RT_OK;
  RT_CUDA(cudaMalloc((void **)dst, src.size() * sizeof(T)));
  RT_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return RT_OK;
}

template <typename T>
std::vector<float> to_f32(const std::vector<T> &v) {
  std::vector<float> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
  return o;
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major).
// Returns eigenvalues in w and eigenvectors as columns of Q.
void jacobi_eig(int n, std::vector<double> a, std::vector<double> &w, std::vector<double> &Q) {
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double v = a[(size_t)i * n + j] * a[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-34 * tot || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // rotate columns p, q
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rotate rows p, q
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
          Q[(size_t)k * n + p] = c * qkp - s * qkq;
          Q[(size_t)k * n + q] = s * qkp + c * qkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
}

bool finite_all(const double *v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void free_handle(rt_handle *h) {
  if (!h) return;
  void *ptrs[] = {h->d_cols, h->d_dir_cls, h->d_dir_up, h->d_tsrc, h->d_Itop, h->d_Ibot,
                  h->E64, h->A64, h->B64, h->Uw64, h->Ul64, h->Rw64, h->Psi64, h->gam64,
                  h->E32, h->A32, h->B32, h->Uw32, h->Ul32, h->Rw32, h->Psi32, h->gam32,
                  h->b_int, h->d_order, h->d_queue, h->ws.V, h->ws.S, h->ws.H,
                  h->so.outer, h->so.inner, h->so.status, h->so.relres, h->so.bytes,
                  h->stage_x, h->stage_y, h->d_sig_tiles, h->d_sw_tiles, h->apply_S,
                  h->d_tc_jobs, h->d_tc_off, h->d_tc_tiles, h->d_tc_xb, h->d_tc_maps, h->d_err, h->d_geo,
                  h->chi64, h->chi32, h->box_w064, h->box_bt64, h->box_kap32, h->box_phi32, h->g_part, h->g_red, h->g_coef, h->g_r, h->Q64, h->Q32, h->lr32};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (h->solve_graph) cudaGraphExecDestroy(h->solve_graph);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  for (cudaEvent_t e : h->tc_ev) cudaEventDestroy(e);
  delete h;
}

struct ColumnHost {
  rt::ColDev c{};
  std::vector<double> mu_cls;
  std::vector<int32_t> dir_cls, dir_up;
  std::vector<double> Uw, Ul, Rw, Psi;
};

int check_desc(const rt_desc *d, int idx) {
  char pre[64];
  std::snprintf(pre, sizeof pre, "column %d: ", idx);
  if (!d) return fail(RT_ERR_ARG, std::string(pre) + "null descriptor");
  if (d->dims != 1) return fail(RT_ERR_ARG, std::string(pre) + "only dims == 1 is supported by this entry point");
  if (d->nx != 1 || d->ny != 1) return fail(RT_ERR_ARG, std::string(pre) + "1D columns need nx = ny = 1");
  if (d->nz < 2 || d->n_dir < 1 || d->n_nu < 1)
    return fail(RT_ERR_ARG, std::string(pre) + "need nz >= 2, n_dir >= 1, n_nu >= 1");
  if ((int64_t)d->n_dir * d->n_nu > 8192) return fail(RT_ERR_ARG, std::string(pre) + "n_dir*n_nu > 8192");
  if (!d->z || !d->dir || !d->w_dir || !d->w_nu || !d->chi || !d->gamma)
    return fail(RT_ERR_ARG, std::string(pre) + "missing z, dir, w_dir, w_nu, chi or gamma");
  if (!d->Psi && (!d->P || !d->R)) return fail(RT_ERR_ARG, std::string(pre) + "need Psi or both P and R");
  if (d->formal_solver == RT_FS_LC)
    return fail(RT_ERR_ARG, std::string(pre) + "long characteristics (RT_FS_LC) are for 3D boxes");
  if (d->formal_solver != RT_FS_SCL && d->formal_solver != RT_FS_IE && d->formal_solver != RT_FS_QSC)
    return fail(RT_ERR_ARG, std::string(pre) + "unknown formal_solver");
  for (int i = 0; i + 1 < d->nz; ++i)
    if (!(d->z[i + 1] > d->z[i])) return fail(RT_ERR_ARG, std::string(pre) + "z must increase strictly");
  for (int k = 0; k < d->n_dir; ++k)
    if (!(std::fabs(d->dir[3 * k + 2]) > 0.0)) return fail(RT_ERR_ARG, std::string(pre) + "mu = 0 direction");
  const size_t np = (size_t)d->nz * d->n_nu;
  if (!finite_all(d->chi, np) || !finite_all(d->gamma, np) || !finite_all(d->z, d->nz))
    return fail(RT_ERR_NONFINITE, std::string(pre) + "non-finite chi, gamma or z");
  for (size_t i = 0; i < np; ++i)
    if (d->chi[i] < 0.0) return fail(RT_ERR_ARG, std::string(pre) + "negative opacity");
  return RT_OK;
}

// Factor the separable kernel: P = Q diag(lam) Q^T (symmetric) truncated at
// |lam| <= 1e-13 max|lam|; otherwise the full-rank identity factor.
void factor_angular(const rt_desc *d, ColumnHost &ch) {
  const int nd = d->n_dir;
  bool sym = true;
  double pmax = 0.0;
  for (int i = 0; i < nd * nd; ++i) pmax = std::max(pmax, std::fabs(d->P[i]));
  for (int i = 0; i < nd && sym; ++i)
    for (int j = 0; j < nd; ++j)
      if (std::fabs(d->P[i * nd + j] - d->P[j * nd + i]) > 1e-14 * pmax) { sym = false; break; }
  ch.Uw.clear();
  ch.Ul.clear();
  if (sym) {
    std::vector<double> w, Q;
    jacobi_eig(nd, std::vector<double>(d->P, d->P + nd * nd), w, Q);
    double wmax = 0.0;
    for (double v : w) wmax = std::max(wmax, std::fabs(v));
    std::vector<int> keep;
    for (int k = 0; k < nd; ++k)
      if (std::fabs(w[k]) > 1e-13 * wmax) keep.push_back(k);
    if (keep.empty()) keep.push_back(0);
    const int rp = (int)keep.size();
    ch.c.rp = rp;
    ch.Uw.resize((size_t)nd * rp);
    ch.Ul.resize((size_t)nd * rp);
    for (int dd = 0; dd < nd; ++dd)
      for (int k = 0; k < rp; ++k) {
        const double q = Q[(size_t)dd * nd + keep[k]];
        ch.Uw[(size_t)dd * rp + k] = q * d->w_dir[dd];
        ch.Ul[(size_t)dd * rp + k] = q * w[keep[k]];
      }
  } else {
    ch.c.rp = nd;
    ch.Uw.assign((size_t)nd * nd, 0.0);
    ch.Ul.assign(d->P, d->P + nd * nd);
    for (int dd = 0; dd < nd; ++dd) ch.Uw[(size_t)dd * nd + dd] = d->w_dir[dd];
  }
}

int build_column(const rt_desc *d, ColumnHost &ch) {
  const int nd = d->n_dir, nn = d->n_nu;
  ch.c.nz = d->nz;
  ch.c.nd = nd;
  ch.c.nn = nn;
  ch.c.nr = nd * nn;
  // |mu| classes
  ch.mu_cls.clear();
  ch.dir_cls.assign(nd, 0);
  ch.dir_up.assign(nd, 0);
  for (int k = 0; k < nd; ++k) {
    const double mu = d->dir[3 * k + 2], am = std::fabs(mu);
    ch.dir_up[k] = mu > 0.0 ? 1 : 0;
    int found = -1;
    for (size_t c = 0; c < ch.mu_cls.size(); ++c)
      if (std::fabs(ch.mu_cls[c] - am) <= 1e-15 * am) { found = (int)c; break; }
    if (found < 0) {
      found = (int)ch.mu_cls.size();
      ch.mu_cls.push_back(am);
    }
    ch.dir_cls[k] = found;
  }
  ch.c.ncls = (int)ch.mu_cls.size();
  ch.c.rdiag = 0;
  ch.Rw.clear();
  ch.Psi.clear();
  if (d->Psi) {
    const int nr = nd * nn;
    ch.c.rp = 1;
    ch.Uw.assign(nd, 0.0);
    ch.Ul.assign(nd, 0.0);
    ch.Psi.resize((size_t)nr * nr);
    for (int r = 0; r < nr; ++r)
      for (int q = 0; q < nr; ++q)
        ch.Psi[(size_t)q * nr + r] = d->Psi[(size_t)r * nr + q] * d->w_dir[q / nn] * d->w_nu[q % nn];
    if (!finite_all(ch.Psi.data(), ch.Psi.size())) return fail(RT_ERR_NONFINITE, "non-finite Psi");
    ch.Rw.assign(1, 0.0);
    if (nr > rt::kSigBuf) return fail(RT_ERR_ARG, "dense kernel needs n_dir*n_nu <= 2048");
  } else {
    if (!finite_all(d->P, (size_t)nd * nd) || !finite_all(d->R, (size_t)nn * nn))
      return fail(RT_ERR_NONFINITE, "non-finite P or R");
    factor_angular(d, ch);
    if ((int64_t)ch.c.rp * nn > rt::kSigBuf)
      return fail(RT_ERR_ARG, "rank(P) * n_nu must not exceed 2048");
    bool diag = true;
    for (int i = 0; i < nn && diag; ++i)
      for (int j = 0; j < nn; ++j)
        if (i != j && d->R[i * nn + j] != 0.0) { diag = false; break; }
    ch.c.rdiag = diag ? 1 : 0;
    if (diag) {
      ch.Rw.resize(nn);
      for (int i = 0; i < nn; ++i) ch.Rw[i] = d->R[i * nn + i] * d->w_nu[i];
    } else {
      ch.Rw.resize((size_t)nn * nn);
      for (int f = 0; f < nn; ++f)
        for (int q = 0; q < nn; ++q) ch.Rw[(size_t)q * nn + f] = d->R[(size_t)f * nn + q] * d->w_nu[q];
    }
  }
  return RT_OK;
}

// Workspace: one slot per resident CTA of the solve kernel.  A slot's basis
// bytes are shared by whatever instance runs there, so the restart length of an
// instance is (slot bytes / instance bytes) - 1, capped by the request.
// per_sm: concurrently resident CTAs of the mixed batched solve per SM (1 or
// 2); a second call replaces the previous workspace.
int alloc_workspace(rt_handle *h, int max_restart, int per_sm = 1) {
  const int m = std::max(1, std::min(max_restart, rt::max_krylov()));
  int dev = 0;
  RT_CUDA(cudaGetDevice(&dev));
  RT_CUDA(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));
  if (h->ws.V) cudaFree(h->ws.V);
  if (h->ws.S) cudaFree(h->ws.S);
  if (h->ws.H) cudaFree(h->ws.H);
  h->ws.V = nullptr;
  h->ws.S = h->ws.H = nullptr;
  const int n_inst = h->n_cols * h->n_rhs;
  const int64_t ld = (h->nmax + 31) / 32 * 32;
  const int64_t elt = h->precision == RT_P_FP64 ? 8 : 4;
  size_t free_b = 0, total_b = 0;
  RT_CUDA(cudaMemGetInfo(&free_b, &total_b));
  // Hessenberg + Givens storage for an outer and an inner basis of up to m
  const int64_t hld = 2 * ((int64_t)(m + 1) * m + 3 * (m + 2));
  // fp64: basis of m+1 float64 vectors.  mixed: outer float64 basis (m+1), its
  // float32 preconditioned vectors (m), the inner float32 basis (m+1).  The
  // largest instance must fit with at least min(m, 8) vectors of each.
  auto bytes_per_elt = [&](int mm) -> int64_t {
    return elt == 8 ? (int64_t)(mm + 1) * 8 : (int64_t)(mm + 1) * 8 + (int64_t)mm * 4 + (int64_t)(mm + 1) * 4;
  };
  const int64_t min_cap = bytes_per_elt(std::min(m, 8)) * ld;
  const int64_t want_cap = bytes_per_elt(m) * ld;
  const double fixed = (double)(ld * 8 + hld * 8);
  const double budget = 0.6 * (double)free_b;
  // one 512-thread CTA per SM (a heavy instance gets a whole SM's bandwidth),
  // or two 256-thread CTAs
  int slots = std::min(n_inst, h->n_sm * per_sm);
  while (slots > 1 && budget / slots < fixed + (double)min_cap) --slots;
  if (budget < fixed + (double)min_cap) return fail(RT_ERR_OOM, "not enough device memory for one Krylov workspace");
  int64_t cap = (int64_t)std::min<double>((double)want_cap, budget / slots - fixed);
  cap = cap / 256 * 256;
  h->ws.slots = slots;
  h->ws.per_sm = per_sm;
  h->ws.m = m;
  h->ws.ld = ld;
  h->ws.cap_bytes = cap;
  h->ws.hld = hld;
  RT_CUDA(cudaMalloc(&h->ws.V, (size_t)slots * cap));
  RT_CUDA(cudaMalloc(&h->ws.S, (size_t)slots * ld * sizeof(double)));
  RT_CUDA(cudaMalloc(&h->ws.H, (size_t)slots * hld * sizeof(double)));
  if (!h->so.outer) {
    RT_CUDA(cudaMalloc(&h->so.outer, n_inst * sizeof(int32_t)));
    RT_CUDA(cudaMalloc(&h->so.inner, n_inst * sizeof(int32_t)));
    RT_CUDA(cudaMalloc(&h->so.status, n_inst * sizeof(int32_t)));
    RT_CUDA(cudaMalloc(&h->so.relres, n_inst * sizeof(double)));
    RT_CUDA(cudaMalloc(&h->so.bytes, n_inst * sizeof(double)));
  }
  if (h->solve_graph) {  // captured with the old workspace
    cudaGraphExecDestroy(h->solve_graph);
    h->solve_graph = nullptr;
  }
  return RT_OK;
}

// Sigma tiles (instance, first point, points) and sweep tiles (instance, first
// ray) of a batch, rhs 0 first, longest columns first; replaces the handle's.
int build_apply_tiles(rt_handle *h, int ray_block, int sigma_pts) {
  const auto &cols = h->h_cols;
  const int n_cols = h->n_cols, n_rhs = h->n_rhs;
  std::vector<int3> sig;
  std::vector<int2> sw;
  std::vector<int> by_depth(n_cols);
  std::iota(by_depth.begin(), by_depth.end(), 0);
  // longest columns first: their sweeps are the longest sequential chains
  std::stable_sort(by_depth.begin(), by_depth.end(), [&](int a, int b) { return cols[a].nz > cols[b].nz; });
  for (int r = 0; r < n_rhs; ++r) {
    for (int ci : by_depth) {
      const rt::ColDev &c = cols[ci];
      const int inst = r * n_cols + ci;
      const int pb = rt::sigma_points_per_block(c, sigma_pts > 0 ? sigma_pts : 1 << 30);
      for (int p0 = 0; p0 < c.nz; p0 += pb) sig.push_back(make_int3(inst, p0, std::min(pb, c.nz - p0)));
      for (int r0 = 0; r0 < c.nr; r0 += ray_block) sw.push_back(make_int2(inst, r0));
    }
    if (r == 0) {
      h->n_sig_tiles_rhs0 = (int)sig.size();
      h->n_sw_tiles_rhs0 = (int)sw.size();
    }
  }
  if (sig.size() > 0x7fffffff || sw.size() > 0x7fffffff) return fail(RT_ERR_ARG, "batch too large for the apply tiling");
  if (h->d_sig_tiles) cudaFree(h->d_sig_tiles);
  if (h->d_sw_tiles) cudaFree(h->d_sw_tiles);
  h->d_sig_tiles = nullptr;
  h->d_sw_tiles = nullptr;
  h->n_sig_tiles = (int)sig.size();
  h->n_sw_tiles = (int)sw.size();
  int rc = dev_upload(&h->d_sig_tiles, sig);
  if (rc == RT_OK) rc = dev_upload(&h->d_sw_tiles, sw);
  return rc;
}

int create_columns(const rt_desc *descs, int n_cols, int n_rhs, int precision, int max_restart,
                   rt_handle **out) {
  if (!out) return fail(RT_ERR_ARG, "out is null");
  *out = nullptr;
  if (n_cols < 1 || n_rhs < 1) return fail(RT_ERR_ARG, "need n_cols >= 1 and n_rhs >= 1");
  if (n_cols > 65535) return fail(RT_ERR_ARG, "at most 65535 columns per batch");
  if ((int64_t)n_cols * n_rhs > (1 << 30)) return fail(RT_ERR_ARG, "too many instances");
  if (precision != RT_P_FP64 && precision != RT_P_MIXED) return fail(RT_ERR_ARG, "unknown precision");
  if (max_restart < 1 || max_restart > rt::max_krylov())
    return fail(RT_ERR_ARG, "max_restart must be in [1, 512]");
  for (int i = 0; i < n_cols; ++i) {
    const int rc = check_desc(&descs[i], i);
    if (rc != RT_OK) return rc;
  }
  rt_handle *h = new rt_handle();
  h->dims = 1;
  h->n_cols = n_cols;
  h->n_rhs = n_rhs;
  h->precision = precision;
  h->max_restart = max_restart;
  std::vector<rt::ColDev> cols(n_cols);
  std::vector<int32_t> dir_cls, dir_up, cls_off, fs;
  std::vector<double> z, mu_cls, chi, gam, tsrc, itop, ibot, Uw, Ul, Rw, Psi, wnu;
  std::vector<int64_t> zoff;
  bool any_t = false;
  for (int i = 0; i < n_cols; ++i) any_t = any_t || descs[i].t_src;
  int64_t x_off = 0, g_off = 0, c_off = 0, r_off = 0, psi_off = 0;
  int32_t u_off = 0, d_off = 0, in_off = 0;
  for (int i = 0; i < n_cols; ++i) {
    const rt_desc *d = &descs[i];
    ColumnHost ch{};
    int rc = build_column(d, ch);
    if (rc != RT_OK) {
      free_handle(h);
      return rc;
    }
    rt::ColDev &c = ch.c;
    c.x_off = x_off;
    c.g_off = g_off;
    c.c_off = c_off;
    c.r_off = r_off;
    c.psi_off = d->Psi ? psi_off : -1;
    c.u_off = u_off;
    c.d_off = d_off;
    c.in_off = in_off;
    c.fs = d->formal_solver;
    cols[i] = c;
    const int64_t ncol = (int64_t)c.nz * c.nr;
    h->nmax = std::max(h->nmax, ncol);
    x_off += ncol;
    zoff.push_back((int64_t)z.size());
    z.insert(z.end(), d->z, d->z + d->nz);
    cls_off.push_back((int32_t)mu_cls.size());
    mu_cls.insert(mu_cls.end(), ch.mu_cls.begin(), ch.mu_cls.end());
    fs.push_back(d->formal_solver);
    const size_t np = (size_t)d->nz * d->n_nu;
    chi.insert(chi.end(), d->chi, d->chi + np);
    gam.insert(gam.end(), d->gamma, d->gamma + np);
    if (any_t) {
      if (d->t_src) tsrc.insert(tsrc.end(), d->t_src, d->t_src + np);
      else tsrc.insert(tsrc.end(), np, 0.0);
    }
    for (int f = 0; f < d->n_nu; ++f) {
      itop.push_back(d->I_top ? d->I_top[f] : 0.0);
      ibot.push_back(d->I_bot ? d->I_bot[f] : 0.0);
    }
    wnu.insert(wnu.end(), d->w_nu, d->w_nu + d->n_nu);
    dir_cls.insert(dir_cls.end(), ch.dir_cls.begin(), ch.dir_cls.end());
    dir_up.insert(dir_up.end(), ch.dir_up.begin(), ch.dir_up.end());
    Uw.insert(Uw.end(), ch.Uw.begin(), ch.Uw.end());
    Ul.insert(Ul.end(), ch.Ul.begin(), ch.Ul.end());
    Rw.insert(Rw.end(), ch.Rw.begin(), ch.Rw.end());
    Psi.insert(Psi.end(), ch.Psi.begin(), ch.Psi.end());
    if (d->Psi) h->has_dense = true;
    g_off += np;
    c_off += (int64_t)(c.nz - 1) * c.ncls * c.nn;
    r_off += (int64_t)ch.Rw.size();
    psi_off += (int64_t)ch.Psi.size();
    u_off += (int32_t)ch.Uw.size();
    d_off += c.nd;
    in_off += c.nn;
  }
  h->E = x_off;
  h->h_cols = cols;
  h->h_rw = Rw;
  h->h_wnu = wnu;
  int rc = RT_OK;
#define UP(dst, src)                          \
  if ((rc = dev_upload(&(dst), src)) != RT_OK) { \
    free_handle(h);                           \
    return rc;                                \
  }
  UP(h->d_cols, cols);
  UP(h->d_dir_cls, dir_cls);
  UP(h->d_dir_up, dir_up);
  if (any_t) UP(h->d_tsrc, tsrc);
  UP(h->d_Itop, itop);
  UP(h->d_Ibot, ibot);
  UP(h->Uw64, Uw);
  UP(h->Ul64, Ul);
  UP(h->Rw64, Rw);
  UP(h->gam64, gam);
  std::vector<float> Uwf = to_f32(Uw), Ulf = to_f32(Ul), Rwf = to_f32(Rw), gamf = to_f32(gam);
  UP(h->Uw32, Uwf);
  UP(h->Ul32, Ulf);
  UP(h->Rw32, Rwf);
  UP(h->gam32, gamf);
  if (!Psi.empty()) {
    UP(h->Psi64, Psi);
    std::vector<float> Psif = to_f32(Psi);
    UP(h->Psi32, Psif);
  }
  {
    cudaError_t e2 = cudaMalloc(&h->d_err, sizeof(int));
    if (e2 == cudaSuccess) e2 = cudaMemset(h->d_err, 0, sizeof(int));
    if (e2 == cudaSuccess && precision == RT_P_MIXED && !Psi.empty()) e2 = (cudaError_t)rt::tc_prepare(h, Psi);
    if (e2 != cudaSuccess) {
      free_handle(h);
      return fail(RT_ERR_CUDA, std::string("tensor-core tables: ") + cudaGetErrorString(e2));
    }
  }
  // step coefficients on the device (float64 exp / expm1)
  double *d_z = nullptr, *d_chi = nullptr, *d_mu = nullptr;
  int64_t *d_zoff = nullptr;
  int32_t *d_clsoff = nullptr;
  auto cleanup_tmp = [&]() {
    cudaFree(d_z); cudaFree(d_chi); cudaFree(d_mu); cudaFree(d_zoff); cudaFree(d_clsoff);
  };
  if ((rc = dev_upload(&d_z, z)) || (rc = dev_upload(&d_chi, chi)) || (rc = dev_upload(&d_mu, mu_cls)) ||
      (rc = dev_upload(&d_zoff, zoff)) || (rc = dev_upload(&d_clsoff, cls_off))) {
    cleanup_tmp();
    free_handle(h);
    return rc;
  }
  const size_t nc = (size_t)std::max<int64_t>(c_off, 1);
  h->n_coef = (int64_t)nc;
  const bool any_qsc = std::find(fs.begin(), fs.end(), (int32_t)RT_FS_QSC) != fs.end();
  cudaError_t ce = cudaSuccess;
  if (any_qsc && ce == cudaSuccess) ce = cudaMalloc(&h->Q64, 4 * nc * 8);
  if (any_qsc && ce == cudaSuccess) ce = cudaMalloc(&h->Q32, 4 * nc * 4);
  if (ce == cudaSuccess) ce = cudaMalloc(&h->E64, nc * 8);
  if (ce == cudaSuccess) ce = cudaMalloc(&h->A64, nc * 8);
  if (ce == cudaSuccess) ce = cudaMalloc(&h->B64, nc * 8);
  if (ce == cudaSuccess) ce = cudaMalloc(&h->E32, nc * 4);
  if (ce == cudaSuccess) ce = cudaMalloc(&h->A32, nc * 4);
  if (ce == cudaSuccess) ce = cudaMalloc(&h->B32, nc * 4);
  if (ce == cudaSuccess) ce = (cudaError_t)rt::launch_coefficients(h, d_z, d_zoff, d_chi, d_mu, d_clsoff, 0);
  if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  cleanup_tmp();
  if (ce != cudaSuccess) {
    free_handle(h);
    return fail(ce == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA,
                std::string("coefficients: ") + cudaGetErrorString(ce));
  }
  // instance order: largest columns first (dynamic queue balances the tail)
  const int n_inst = n_cols * n_rhs;
  std::vector<int32_t> order(n_inst);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const auto &ca = cols[a % n_cols], &cb = cols[b % n_cols];
    return (int64_t)ca.nz * ca.nr > (int64_t)cb.nz * cb.nr;
  });
  UP(h->d_order, order);
#undef UP
  ce = cudaMalloc(&h->d_queue, 4 * sizeof(int));
  if (ce != cudaSuccess) {
    free_handle(h);
    return fail(RT_ERR_OOM, "queue allocation failed");
  }
  if ((rc = alloc_workspace(h, max_restart)) != RT_OK) {
    free_handle(h);
    return rc;
  }
  // apply tiles (rhs 0 first) and the source-function scratch of rt_apply
  if ((rc = build_apply_tiles(h, h->tune.ray_block, h->tune.sigma_pts)) != RT_OK) {
    free_handle(h);
    return rc;
  }
  ce = cudaMalloc(&h->apply_S, (size_t)h->E * n_rhs * sizeof(double));
  if (ce != cudaSuccess) {
    free_handle(h);
    return fail(RT_ERR_OOM, "apply scratch allocation failed");
  }
  ce = cudaMalloc(&h->b_int, (size_t)h->E * sizeof(double));
  if (ce == cudaSuccess) ce = (cudaError_t)rt::launch_apply(h, RT_OP_RHS, true, h->b_int, h->b_int, 0, true);
  if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  if (ce != cudaSuccess) {
    free_handle(h);
    return fail(RT_ERR_CUDA, std::string("internal rhs: ") + cudaGetErrorString(ce));
  }
  if (rt::single_instance(h)) {  // one (column, rhs): solved by the grid-wide kernels
    const int G = rt::grid_ctas(h);
    ce = cudaMalloc(&h->g_r, (size_t)h->ws.ld * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc(&h->g_part, (size_t)G * rt::kGridPartPerCta * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc(&h->g_red, rt::kGridPartPerCta * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc(&h->g_coef, 1024 * sizeof(double));
    if (ce != cudaSuccess) {
      free_handle(h);
      return fail(RT_ERR_OOM, "grid solve buffers");
    }
  }
  *out = h;
  return RT_OK;
}


// 3D box: Sigma tables as one "column" of n_pts points; plane-sweep geometry.
int create_box(const rt_desc *d, int n_rhs, int precision, int max_restart, rt_handle **out) {
  if (!out) return fail(RT_ERR_ARG, "out is null");
  *out = nullptr;
  if (n_rhs != 1) return fail(RT_ERR_ARG, "3D boxes take one right-hand side per handle");
  if (precision != RT_P_FP64 && precision != RT_P_MIXED) return fail(RT_ERR_ARG, "unknown precision");
  if (max_restart < 1 || max_restart > rt::max_krylov()) return fail(RT_ERR_ARG, "max_restart must be in [1, 512]");
  if (d->nx < 1 || d->ny < 1 || d->nz < 2 || d->n_dir < 1 || d->n_nu < 1)
    return fail(RT_ERR_ARG, "box: need nx, ny >= 1, nz >= 2, n_dir, n_nu >= 1");
  if (!d->z || !d->dir || !d->w_dir || !d->w_nu || !d->chi || !d->gamma)
    return fail(RT_ERR_ARG, "box: missing z (spacings), dir, w_dir, w_nu, chi or gamma");
  if (!(d->z[0] > 0 && d->z[1] > 0 && d->z[2] > 0)) return fail(RT_ERR_ARG, "box: spacings must be positive");
  if (!d->Psi && (!d->P || !d->R)) return fail(RT_ERR_ARG, "box: need Psi or both P and R");
  if (d->formal_solver != RT_FS_SCL && d->formal_solver != RT_FS_IE && d->formal_solver != RT_FS_QSC &&
      d->formal_solver != RT_FS_LC)
    return fail(RT_ERR_ARG, "unknown formal_solver");
  const int64_t npts = (int64_t)d->nx * d->ny * d->nz;
  if (!rt::box_plane_fits(d->nx, d->ny)) return fail(RT_ERR_ARG, "box: nx*ny must be at most 4096 (a z-plane in shared memory)");
  for (int k = 0; k < d->n_dir; ++k)
    if (!(std::fabs(d->dir[3 * k + 2]) > 0.0)) return fail(RT_ERR_ARG, "box: direction with Omega_z = 0");
  const size_t np = (size_t)npts * d->n_nu;
  if (!finite_all(d->chi, np) || !finite_all(d->gamma, np)) return fail(RT_ERR_NONFINITE, "box: non-finite chi or gamma");
  for (size_t i = 0; i < np; ++i)
    if (d->chi[i] < 0.0) return fail(RT_ERR_ARG, "box: negative opacity");
  ColumnHost ch{};
  rt_desc dd = *d;
  int rc = build_column(&dd, ch);
  if (rc != RT_OK) return rc;
  if (!d->Psi && !rt::box_sigma_fits(d, ch.c.rp))
    return fail(RT_ERR_ARG, "box: the separable kernel needs rank(P) <= 6 and n_nu <= 128");
  rt_handle *h = new rt_handle();
  h->dims = 3;
  h->n_cols = 1;
  h->n_rhs = 1;
  h->precision = precision;
  h->max_restart = max_restart;
  rt::ColDev c = ch.c;
  if (npts > 0x7fffffff) { free_handle(h); return fail(RT_ERR_ARG, "box too large"); }
  c.nz = (int32_t)npts;
  c.x_off = 0; c.g_off = 0; c.c_off = 0; c.r_off = 0; c.psi_off = d->Psi ? 0 : -1;
  c.u_off = 0; c.d_off = 0; c.in_off = 0;
  h->h_cols = {c};
  h->E = npts * c.nr;
  h->nmax = h->E;
  h->box = rt::BoxDev{d->nx, d->ny, d->nz, d->n_dir, d->n_nu, d->formal_solver == RT_FS_IE ? 1 : 0,
                      d->formal_solver == RT_FS_QSC ? 1 : 0, d->formal_solver == RT_FS_LC ? 1 : 0};
  // per direction: integer upwind shift reduced modulo the periodic plane,
  // its fractional part, the path length between planes, the sweep sense
  std::vector<double> geo(6 * (size_t)d->n_dir);
  for (int k = 0; k < d->n_dir; ++k) {
    const double ox = d->dir[3 * k], oy = d->dir[3 * k + 1], oz = d->dir[3 * k + 2];
    const double ds = d->z[2] / std::fabs(oz);
    const double sx = ox * ds / d->z[0], sy = oy * ds / d->z[1];
    const double fx = std::floor(sx), fy = std::floor(sy);
    geo[6 * k + 0] = (double)((((long long)fx % d->nx) + d->nx) % d->nx);
    geo[6 * k + 1] = (double)((((long long)fy % d->ny) + d->ny) % d->ny);
    geo[6 * k + 2] = sx - fx;
    geo[6 * k + 3] = sy - fy;
    geo[6 * k + 4] = ds;
    geo[6 * k + 5] = oz > 0 ? 1.0 : 0.0;
  }
  std::vector<double> chi(d->chi, d->chi + np), gam(d->gamma, d->gamma + np), itop, ibot, tsrc;
  for (int f = 0; f < d->n_nu; ++f) {
    itop.push_back(d->I_top ? d->I_top[f] : 0.0);
    ibot.push_back(d->I_bot ? d->I_bot[f] : 0.0);
  }
  if (d->t_src) tsrc.assign(d->t_src, d->t_src + np);
  std::vector<rt::ColDev> cols = {c};
#define UPB(dst, src)                           \
  if ((rc = dev_upload(&(dst), src)) != RT_OK) { \
    free_handle(h);                             \
    return rc;                                  \
  }
  UPB(h->d_cols, cols);
  UPB(h->d_dir_cls, ch.dir_cls);
  UPB(h->d_dir_up, ch.dir_up);
  UPB(h->d_geo, geo);
  {
    const cudaError_t be = (cudaError_t)rt::box_prepare(h, chi.data());
    if (be != cudaSuccess) {
      free_handle(h);
      return fail(be == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, std::string("box opacity: ") + cudaGetErrorString(be));
    }
  }
  std::vector<float> gamf = to_f32(gam);
  UPB(h->gam64, gam);
  UPB(h->gam32, gamf);
  UPB(h->d_Itop, itop);
  UPB(h->d_Ibot, ibot);
  if (!tsrc.empty()) UPB(h->d_tsrc, tsrc);
  UPB(h->Uw64, ch.Uw);
  UPB(h->Ul64, ch.Ul);
  UPB(h->Rw64, ch.Rw);
  std::vector<float> Uwf = to_f32(ch.Uw), Ulf = to_f32(ch.Ul), Rwf = to_f32(ch.Rw);
  UPB(h->Uw32, Uwf);
  UPB(h->Ul32, Ulf);
  UPB(h->Rw32, Rwf);
  if (!ch.Psi.empty()) {
    UPB(h->Psi64, ch.Psi);
    std::vector<float> Psif = to_f32(ch.Psi);
    UPB(h->Psi32, Psif);
  }
  std::vector<int3> sig;
  const int pb = rt::sigma_points_per_block(c);
  for (int64_t p0 = 0; p0 < npts; p0 += pb) sig.push_back(make_int3(0, (int)p0, (int)std::min<int64_t>(pb, npts - p0)));
  h->n_sig_tiles = h->n_sig_tiles_rhs0 = (int)sig.size();
  UPB(h->d_sig_tiles, sig);
#undef UPB
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int G = 2 * h->n_sm;
  // source-function scratch in the sweep layout: frequencies padded up to the
  // sweep's block (at most to a multiple of 4), float64 at most
  const size_t s_bytes = (size_t)npts * d->n_dir * h->box_npad * sizeof(double);
  if (ce == cudaSuccess) ce = cudaMalloc(&h->apply_S, std::max(s_bytes, (size_t)h->E * sizeof(double)));
  if (ce == cudaSuccess) ce = cudaMalloc(&h->g_r, (size_t)h->E * sizeof(double));
  if (ce == cudaSuccess) ce = cudaMalloc(&h->g_part, (size_t)G * rt::kGridPartPerCta * sizeof(double));
  if (ce == cudaSuccess) ce = cudaMalloc(&h->g_red, rt::kGridPartPerCta * sizeof(double));
  if (ce == cudaSuccess) ce = cudaMalloc(&h->g_coef, 1024 * sizeof(double));
  if (ce == cudaSuccess) ce = cudaMalloc(&h->d_err, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMemset(h->d_err, 0, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMalloc(&h->b_int, (size_t)h->E * sizeof(double));
  if (ce != cudaSuccess) {
    free_handle(h);
    return fail(ce == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, std::string("box buffers: ") + cudaGetErrorString(ce));
  }
  // Krylov basis: as many vectors as 60% of the free memory holds, up to max_restart
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const int64_t ldv = (h->E + 31) / 32 * 32;
  const int64_t elt = precision == RT_P_FP64 ? 8 : 4;
  int m = max_restart;
  while (m > 1 && (double)(m + 1) * ldv * elt > 0.6 * (double)free_b) --m;
  if ((double)(m + 1) * ldv * elt > 0.6 * (double)free_b) { free_handle(h); return fail(RT_ERR_OOM, "box: no room for a Krylov basis"); }
  h->ws.slots = 1;
  h->ws.m = m;
  h->ws.ld = ldv;
  h->ws.cap_bytes = (m + 1) * ldv * elt;
  ce = cudaMalloc(&h->ws.V, (size_t)h->ws.cap_bytes);
  if (ce == cudaSuccess) ce = (cudaError_t)rt::apply_box(h, RT_OP_RHS, true, nullptr, false, h->b_int, false, 0);
  if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  if (ce != cudaSuccess) {
    free_handle(h);
    return fail(ce == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, std::string("box setup: ") + cudaGetErrorString(ce));
  }
  *out = h;
  return RT_OK;
}

int ensure_stage(rt_handle *h, int64_t len) {
  if (h->stage_len >= len) return RT_OK;
  if (h->stage_x) cudaFree(h->stage_x);
  if (h->stage_y) cudaFree(h->stage_y);
  h->stage_x = h->stage_y = nullptr;
  h->stage_len = 0;
  RT_CUDA(cudaMalloc(&h->stage_x, len * sizeof(double)));
  RT_CUDA(cudaMalloc(&h->stage_y, len * sizeof(double)));
  h->stage_len = len;
  return RT_OK;
}

// Plane-sweep launch shape of a 3D box (frequencies per CTA, cells per
// thread): every distinct feasible combination timed on rt_apply(RT_OP_A) in
// the handle's precision, the fastest kept; RT_TUNE_CACHE as for batches.
int autotune_box(rt_handle *h, int flags, rt_tune_info *out, cudaStream_t s, const char *sig, const char *path,
                 rt_tune_info loc) {
  const bool f64 = h->precision == RT_P_FP64;
  auto report = [&](double best, double first, int from_cache) {
    int fb = 0, cpt = 0;
    rt::box_effective_shape(h, f64, fb, cpt);
    loc.box_fb = fb;
    loc.box_cpt = cpt;
    loc.ms_best = best;
    loc.ms_default = first;
    loc.from_cache = from_cache;
    if (out) *out = loc;
    return RT_OK;
  };
  if (path && !(flags & 1)) {
    if (FILE *f = std::fopen(path, "r")) {
      char line[512];
      int fb = 0, cpt = 0;
      double ms = 0;
      bool hit = false;
      while (std::fgets(line, sizeof line, f)) {
        const char *q = std::strstr(line, "\"sig\": \"");
        if (!q || std::strncmp(q + 8, sig, std::strlen(sig)) != 0 || q[8 + std::strlen(sig)] != '"') continue;
        const char *r = std::strstr(line, "\"box_fb\":");
        if (r && std::sscanf(r, "\"box_fb\": %d, \"box_cpt\": %d, \"ms\": %lf", &fb, &cpt, &ms) == 3) hit = true;
      }
      std::fclose(f);
      if (hit) {
        h->tune.box_fb = fb;
        h->tune.box_cpt = cpt;
        h->tune.ms = ms;
        h->tune.from_cache = 1;
        return report(ms, 0.0, 1);
      }
    }
  }
  const int64_t len = h->E;
  double *x = nullptr, *y = nullptr;
  RT_CUDA(cudaMalloc(&x, len * sizeof(double)));
  cudaError_t ce = cudaMalloc(&y, len * sizeof(double));
  if (ce != cudaSuccess) {
    cudaFree(x);
    return fail(RT_ERR_OOM, "autotune buffers");
  }
  cudaMemsetAsync(x, 0, len * sizeof(double), s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300, first = 0.0;
  int best_fb = 0, best_cpt = 0;
  std::vector<std::pair<int, int>> seen;
  int rc = RT_OK;
  const int fbs[3] = {4, 2, 1}, cpts[4] = {1, 2, 4, 8};
  for (int a = 0; a < 3 && rc == RT_OK; ++a)
    for (int b = 0; b < 4 && rc == RT_OK; ++b) {
      h->tune.box_fb = fbs[a];
      h->tune.box_cpt = cpts[b];
      int fb = 0, cpt = 0;
      rt::box_effective_shape(h, f64, fb, cpt);
      if (std::find(seen.begin(), seen.end(), std::make_pair(fb, cpt)) != seen.end()) continue;
      seen.emplace_back(fb, cpt);
      if (rt::launch_apply(h, RT_OP_A, f64, x, y, s) != 0) { rc = fail(RT_ERR_CUDA, "autotune launch"); break; }
      cudaEventRecord(e0, s);
      for (int k = 0; k < 3; ++k) rt::launch_apply(h, RT_OP_A, f64, x, y, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(RT_ERR_CUDA, "autotune launch"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double t = ms / 3.0;
      if (seen.size() == 1) first = t;
      if (t < best) {
        best = t;
        best_fb = fb;
        best_cpt = cpt;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (rc != RT_OK) return rc;
  h->tune.box_fb = best_fb;
  h->tune.box_cpt = best_cpt;
  h->tune.ms = best;
  h->tune.from_cache = 0;
  if (path) {
    if (FILE *f = std::fopen(path, "a")) {
      std::fprintf(f, "{\"sig\": \"%s\", \"box_fb\": %d, \"box_cpt\": %d, \"ms\": %.6f}\n", sig, best_fb, best_cpt,
                   best);
      std::fclose(f);
    }
  }
  return report(best, first, 0);
}

// Persistent mixed solve of a 1D batch: CTAs per SM (1 x 512 or 2 x 256
// threads; the workspace is re-allocated to match) and the inner float32
// cycle length, timed on full solves of the handle's own batch with the
// internal right-hand side (tolerance 1e-10, tol_inner 0.1): first the two CTA
// shapes at cycle length 20, then cycle lengths 12 and 30 with the faster
// shape.  RT_TUNE_CACHE as for the apply shapes.
int autotune_solve(rt_handle *h, int flags, cudaStream_t s, const char *sig, const char *path,
                   rt_tune_info &loc) {
  if (path && !(flags & 1)) {
    if (FILE *f = std::fopen(path, "r")) {
      char line[512];
      int ps = 0, mi = 0;
      double ms = 0;
      bool hit = false;
      while (std::fgets(line, sizeof line, f)) {
        const char *q = std::strstr(line, "\"sig\": \"");
        if (!q || std::strncmp(q + 8, sig, std::strlen(sig)) != 0 || q[8 + std::strlen(sig)] != '"') continue;
        const char *r = std::strstr(line, "\"solve_per_sm\":");
        if (r && std::sscanf(r, "\"solve_per_sm\": %d, \"solve_inner\": %d, \"solve_ms\": %lf", &ps, &mi, &ms) == 3)
          hit = true;
      }
      std::fclose(f);
      if (hit) {
        if (ps != h->ws.per_sm) {
          const int rc = alloc_workspace(h, h->max_restart, ps);
          if (rc != RT_OK) return rc;
        }
        h->tune.solve_m_in = mi;
        loc.solve_per_sm = ps;
        loc.solve_inner = mi;
        loc.solve_ms = ms;
        return RT_OK;
      }
    }
  }
  const int64_t len = h->E * h->n_rhs;
  double *x = nullptr;
  RT_CUDA(cudaMalloc(&x, len * sizeof(double)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int m = std::min(32, h->ws.m);
  int rc = RT_OK;
  auto time_solve = [&](int m_in, double &ms) -> int {
    cudaEventRecord(e0, s);
    int e = rt::launch_solve(h, nullptr, x, 1e-10, 0.1, m, 60, 0, s, std::min(m_in, h->ws.m));
    cudaEventRecord(e1, s);
    if (e || cudaEventSynchronize(e1) != cudaSuccess) return fail(RT_ERR_CUDA, "autotune solve launch");
    float f = 0.f;
    cudaEventElapsedTime(&f, e0, e1);
    ms = f;
    return RT_OK;
  };
  double best = 1e300;
  int best_ps = h->ws.per_sm, best_mi = 20;
  for (int ps = 1; ps <= 2 && rc == RT_OK; ++ps) {
    if (ps != h->ws.per_sm && (rc = alloc_workspace(h, h->max_restart, ps)) != RT_OK) break;
    double ms = 0;
    if ((rc = time_solve(20, ms)) != RT_OK) break;
    if (ms < best) {
      best = ms;
      best_ps = ps;
    }
  }
  if (rc == RT_OK && best_ps != h->ws.per_sm) rc = alloc_workspace(h, h->max_restart, best_ps);
  for (int mi : {12, 30}) {
    if (rc != RT_OK || mi > h->ws.m) break;
    double ms = 0;
    if ((rc = time_solve(mi, ms)) != RT_OK) break;
    if (ms < best) {
      best = ms;
      best_mi = mi;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  if (rc != RT_OK) return rc;
  h->tune.solve_m_in = best_mi;
  loc.solve_per_sm = best_ps;
  loc.solve_inner = best_mi;
  loc.solve_ms = best;
  if (path) {
    if (FILE *f = std::fopen(path, "a")) {
      std::fprintf(f, "{\"sig\": \"%s\", \"solve_per_sm\": %d, \"solve_inner\": %d, \"solve_ms\": %.3f}\n", sig,
                   best_ps, best_mi, best);
      std::fclose(f);
    }
  }
  return RT_OK;
}

}  // namespace

extern "C" {

const char *rt_last_error(void) { return g_err.c_str(); }

const char *rt_version(void) { return "rt_gb300 0.1 (sm_103a)"; }

int rt_create(const rt_desc *desc, int32_t n_rhs, int32_t precision, int32_t max_restart,
              rt_handle **out) {
  if (out) *out = nullptr;
  if (fault_now() == kFaultAlloc) return fail(RT_ERR_OOM, "RT_FAULT=alloc: injected device allocation failure");
  if (!desc) return fail(RT_ERR_ARG, "null descriptor");
  if (desc->dims == 3) return create_box(desc, n_rhs, precision, max_restart, out);
  return create_columns(desc, 1, n_rhs, precision, max_restart, out);
}

int rt_create_batch(const rt_desc *cols, int32_t n_cols, int32_t n_rhs, int32_t precision,
                    int32_t max_restart, rt_handle **out) {
  if (out) *out = nullptr;
  if (fault_now() == kFaultAlloc) return fail(RT_ERR_OOM, "RT_FAULT=alloc: injected device allocation failure");
  if (!cols) return fail(RT_ERR_ARG, "null descriptor array");
  return create_columns(cols, n_cols, n_rhs, precision, max_restart, out);
}

int64_t rt_vector_length(const rt_handle *h) { return h ? h->E * h->n_rhs : 0; }

int rt_apply(rt_handle *h, int32_t op, int32_t fp64, const double *x, double *y, void *stream) {
  if (!h) return fail(RT_ERR_ARG, "null handle");
  if (fault_now() == kFaultLaunch) return fail(RT_ERR_CUDA, "RT_FAULT=launch: injected launch failure");
  StallScope stall(h);
  if (op < RT_OP_A || op > RT_OP_RHS) return fail(RT_ERR_ARG, "unknown op");
  if (!y || (!x && op != RT_OP_RHS)) return fail(RT_ERR_ARG, "null vector");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t len = h->E * h->n_rhs;
  const bool xd = x ? is_device_ptr(x) : true, yd = is_device_ptr(y);
  const double *xin = x;
  double *yout = y;
  if (!xd || !yd) {
    int rc = ensure_stage(h, len);
    if (rc != RT_OK) return rc;
    if (x && !xd) {
      RT_CUDA(cudaMemcpyAsync(h->stage_x, x, len * sizeof(double), cudaMemcpyHostToDevice, s));
      xin = h->stage_x;
    }
    if (!yd) yout = h->stage_y;
  }
  if (!xin) xin = yout;  // RT_OP_RHS ignores x
  const int e = rt::launch_apply(h, op, fp64 != 0, xin, yout, s);
  if (e != 0) return fail(RT_ERR_CUDA, std::string("apply launch: ") + cudaGetErrorString((cudaError_t)e));
  if (h->n_tc_jobs > 0 && !fp64 && (op == RT_OP_A || op == RT_OP_SIGMA)) {
    int err = 0;
    RT_CUDA(cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    if (err) {
      cudaMemsetAsync(h->d_err, 0, sizeof(int), s);
      return fail(RT_ERR_TIMEOUT, "tensor-core Sigma: a bounded wait gave up");
    }
  }
  if (!yd) {
    RT_CUDA(cudaMemcpyAsync(y, yout, len * sizeof(double), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
  } else if (!xd) {
    RT_CUDA(cudaStreamSynchronize(s));
  }
  return RT_OK;
}

int rt_apply_noalloc(rt_handle *h, int32_t op, int32_t fp64, const double *x, double *y, void *stream) {
  if (!h) return fail(RT_ERR_ARG, "null handle");
  if (fault_now() == kFaultLaunch) return fail(RT_ERR_CUDA, "RT_FAULT=launch: injected launch failure");
  StallScope stall(h);
  if (op < RT_OP_A || op > RT_OP_RHS) return fail(RT_ERR_ARG, "unknown op");
  if (!y || (!x && op != RT_OP_RHS)) return fail(RT_ERR_ARG, "null vector");
  if ((x && !is_device_ptr(x)) || !is_device_ptr(y))
    return fail(RT_ERR_ARG, "rt_apply_noalloc takes device pointers only");
  const bool f64 = fp64 || h->precision == RT_P_FP64;
  const long long need = (h->dims == 3 ? (long long)rt::box_scratch_elems(h, f64) : (long long)h->E * h->n_rhs) *
                         (f64 ? 8 : 4);
  if (need > rt::kNoAllocScratchBytes) {
    char msg[200];
    std::snprintf(msg, sizeof msg, "rt_apply_noalloc: the apply needs %lld bytes of scratch, the static "
                  "array holds %lld", need, (long long)rt::kNoAllocScratchBytes);
    return fail(RT_ERR_ARG, msg);
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int e = rt::launch_apply_noalloc(h, op, fp64 != 0, x ? x : y, y, s);
  if (e != 0) return fail(RT_ERR_CUDA, std::string("rt_apply_noalloc: ") + cudaGetErrorString((cudaError_t)e));
  if (h->n_tc_jobs > 0 && !fp64 && (op == RT_OP_A || op == RT_OP_SIGMA)) {
    int err = 0;
    RT_CUDA(cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    if (err) {
      cudaMemsetAsync(h->d_err, 0, sizeof(int), s);
      return fail(RT_ERR_TIMEOUT, "tensor-core Sigma: a bounded wait gave up");
    }
  }
  return RT_OK;
}

int rt_set_sigma_rank(rt_handle *h, double tol, int32_t *max_rank) {
  if (!h) return fail(RT_ERR_ARG, "null handle");
  if (h->dims != 1 || h->precision != RT_P_MIXED)
    return fail(RT_ERR_ARG, "rt_set_sigma_rank: the truncated kernel acts on the float32 operator of mixed 1D handles");
  if (!(tol >= 0.0) || !(tol < 1.0)) return fail(RT_ERR_ARG, "rt_set_sigma_rank: need 0 <= tol < 1");
  const int n_cols = h->n_cols;
  std::vector<std::vector<float>> fac(n_cols);
  std::vector<int> rank(n_cols, 0);
  if (tol > 0.0) {
    // per column: M = W^1/2 R W^1/2 (symmetric), eigen-decomposed; keep
    // |l| >= tol max |l|; A[q][s] = U[q][s] w_q^1/2, B[f][s] = U[f][s] l_s w_f^-1/2
    auto work = [&](int ci) {
      const rt::ColDev &c = h->h_cols[ci];
      if (c.psi_off >= 0 || c.rdiag) return;
      const int nn = c.nn;
      const double *RwT = h->h_rw.data() + c.r_off;   // RwT[q][f] = R(f, q) w_q
      const double *w = h->h_wnu.data() + c.in_off;
      std::vector<double> M((size_t)nn * nn), lam, Q;
      for (int f = 0; f < nn; ++f)
        for (int q = 0; q < nn; ++q)
          M[(size_t)f * nn + q] = std::sqrt(w[f] / w[q]) * RwT[(size_t)q * nn + f];
      for (int f = 0; f < nn; ++f)  // symmetrise the rounding
        for (int q = f + 1; q < nn; ++q) {
          const double v = 0.5 * (M[(size_t)f * nn + q] + M[(size_t)q * nn + f]);
          M[(size_t)f * nn + q] = M[(size_t)q * nn + f] = v;
        }
      jacobi_eig(nn, M, lam, Q);
      double lmax = 0.0;
      for (double v : lam) lmax = std::max(lmax, std::fabs(v));
      std::vector<int> keep;
      for (int k = 0; k < nn; ++k)
        if (std::fabs(lam[k]) >= tol * lmax && lam[k] != 0.0) keep.push_back(k);
      const int r = (int)keep.size();
      if (r == 0 || r > rt::kLrMax) return;  // exact kernel for this column
      std::vector<float> &F = fac[ci];
      F.assign((size_t)2 * nn * r, 0.f);
      for (int q = 0; q < nn; ++q)
        for (int k = 0; k < r; ++k) {
          const double u = Q[(size_t)q * nn + keep[k]];
          F[(size_t)q * r + k] = (float)(u * std::sqrt(w[q]));
          F[(size_t)nn * r + (size_t)q * r + k] = (float)(u * lam[keep[k]] / std::sqrt(w[q]));
        }
      rank[ci] = r;
    };
    const int nt = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), 32));
    std::vector<std::thread> pool;
    std::atomic<int> next{0};
    for (int t = 0; t < nt; ++t)
      pool.emplace_back([&]() {
        for (int ci = next++; ci < n_cols; ci = next++) work(ci);
      });
    for (auto &th : pool) th.join();
  }
  std::vector<float> all;
  int rmax = 0;
  for (int ci = 0; ci < n_cols; ++ci) {
    h->h_cols[ci].lr_rank = rank[ci];
    h->h_cols[ci].lr_off = (int64_t)all.size();
    all.insert(all.end(), fac[ci].begin(), fac[ci].end());
    rmax = std::max(rmax, rank[ci]);
  }
  if (h->lr32) cudaFree(h->lr32);
  h->lr32 = nullptr;
  if (!all.empty()) {
    int rc = dev_upload(&h->lr32, all);
    if (rc != RT_OK) return rc;
  }
  RT_CUDA(cudaMemcpy(h->d_cols, h->h_cols.data(), h->h_cols.size() * sizeof(rt::ColDev), cudaMemcpyHostToDevice));
  h->lr_tol = tol;
  if (h->solve_graph) {  // the captured solve holds the old table pointers
    cudaGraphExecDestroy(h->solve_graph);
    h->solve_graph = nullptr;
  }
  if (max_rank) *max_rank = rmax;
  return RT_OK;
}

int rt_tc_timer(rt_handle *h, int32_t on, double *ms, int64_t *launches) {
  if (!h) return fail(RT_ERR_ARG, "null handle");
  if (on) {
    constexpr int kPairs = 4096;
    for (cudaEvent_t e : h->tc_ev) cudaEventDestroy(e);
    h->tc_ev.clear();
    h->tc_ev_used = 0;
    for (int i = 0; i < 2 * kPairs; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        for (cudaEvent_t f : h->tc_ev) cudaEventDestroy(f);
        h->tc_ev.clear();
        return fail(RT_ERR_CUDA, "rt_tc_timer: event creation failed");
      }
      h->tc_ev.push_back(e);
    }
    return RT_OK;
  }
  if (h->tc_ev.empty()) return fail(RT_ERR_ARG, "rt_tc_timer: no timing session");
  double total = 0.0;
  int rc = RT_OK;
  for (int i = 0; i + 1 < h->tc_ev_used; i += 2) {
    float t = 0.f;
    if (cudaEventSynchronize(h->tc_ev[i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, h->tc_ev[i], h->tc_ev[i + 1]) != cudaSuccess) {
      rc = fail(RT_ERR_CUDA, "rt_tc_timer: event read failed");
      break;
    }
    total += t;
  }
  if (ms) *ms = total;
  if (launches) *launches = h->tc_ev_used / 2;
  for (cudaEvent_t e : h->tc_ev) cudaEventDestroy(e);
  h->tc_ev.clear();
  h->tc_ev_used = 0;
  return rc;
}

int rt_autotune(rt_handle *h, int32_t flags, rt_tune_info *out, void *stream) {
  if (!h) return fail(RT_ERR_ARG, "null handle");
  cudaStream_t s = (cudaStream_t)stream;
  char sig[256];
  int nzmax = 0, nrmax = 0;
  for (const rt::ColDev &c : h->h_cols) {
    nzmax = std::max(nzmax, c.nz);
    nrmax = std::max(nrmax, c.nr);
  }
  std::snprintf(sig, sizeof sig, "dims=%d cols=%d rhs=%d E=%lld nzmax=%d nrmax=%d prec=%d", h->dims, h->n_cols,
                h->n_rhs, (long long)h->E, nzmax, nrmax, h->precision);
  rt_tune_info loc{};
  loc.ray_block = h->tune.ray_block;
  loc.ahead = h->tune.ahead;
  loc.sigma_points = h->tune.sigma_pts;
  const char *path = std::getenv("RT_TUNE_CACHE");
  if (h->dims == 3) return autotune_box(h, flags, out, s, sig, path, loc);
  if (path && !(flags & 1)) {
    if (FILE *f = std::fopen(path, "r")) {
      char line[512];
      while (std::fgets(line, sizeof line, f)) {
        int rb = 0, ah = 0, pts = 0;
        double ms = 0;
        const char *q = std::strstr(line, "\"sig\": \"");
        if (!q || std::strncmp(q + 8, sig, std::strlen(sig)) != 0 || q[8 + std::strlen(sig)] != '"') continue;
        const char *r = std::strstr(line, "\"ray_block\":");
        if (r && std::sscanf(r, "\"ray_block\": %d, \"ahead\": %d, \"sigma_points\": %d, \"ms\": %lf", &rb, &ah,
                             &pts, &ms) == 4) {
          h->tune.ray_block = rb;
          h->tune.ahead = ah;
          h->tune.sigma_pts = pts;
          h->tune.ms = ms;
          h->tune.from_cache = 1;
        }
      }
      std::fclose(f);
      if (h->tune.from_cache) {
        int rc = build_apply_tiles(h, h->tune.ray_block, h->tune.sigma_pts);
        loc.ray_block = h->tune.ray_block;
        loc.ahead = h->tune.ahead;
        loc.sigma_points = h->tune.sigma_pts;
        loc.ms_best = h->tune.ms;
        loc.from_cache = 1;
        if (rc == RT_OK && (flags & 2) && h->precision == RT_P_MIXED && h->n_cols * h->n_rhs > 1)
          rc = autotune_solve(h, flags, s, sig, path, loc);
        if (out) *out = loc;
        return rc;
      }
    }
  }
  const int64_t len = h->E * h->n_rhs;
  double *x = nullptr, *y = nullptr;
  RT_CUDA(cudaMalloc(&x, len * sizeof(double)));
  cudaError_t ce = cudaMalloc(&y, len * sizeof(double));
  if (ce != cudaSuccess) {
    cudaFree(x);
    return fail(RT_ERR_OOM, "autotune buffers");
  }
  cudaMemsetAsync(x, 0, len * sizeof(double), s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300, first = 0;
  rt::Tune best_t = h->tune;
  const int rbs[3] = {64, 128, 256}, ahs[3] = {2, 4, 8}, pts[3] = {4, 8, 0};
  int rc = RT_OK;
  for (int a = 0; a < 3 && rc == RT_OK; ++a)
    for (int b = 0; b < 3 && rc == RT_OK; ++b)
      for (int c = 0; c < 3 && rc == RT_OK; ++c) {
        h->tune.ray_block = rbs[a];
        h->tune.ahead = ahs[b];
        h->tune.sigma_pts = pts[c];
        if ((rc = build_apply_tiles(h, rbs[a], pts[c])) != RT_OK) break;
        rt::launch_apply(h, RT_OP_A, false, x, y, s);
        cudaEventRecord(e0, s);
        for (int k = 0; k < 3; ++k) rt::launch_apply(h, RT_OP_A, false, x, y, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(RT_ERR_CUDA, "autotune launch"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double t = ms / 3.0;
        if (rbs[a] == 128 && ahs[b] == 8 && pts[c] == 0) first = t;
        if (t < best) {
          best = t;
          best_t = h->tune;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (rc != RT_OK) return rc;
  h->tune = best_t;
  h->tune.ms = best;
  h->tune.from_cache = 0;
  if ((rc = build_apply_tiles(h, best_t.ray_block, best_t.sigma_pts)) != RT_OK) return rc;
  if (path) {
    if (FILE *f = std::fopen(path, "a")) {
      std::fprintf(f, "{\"sig\": \"%s\", \"ray_block\": %d, \"ahead\": %d, \"sigma_points\": %d, \"ms\": %.6f}\n",
                   sig, best_t.ray_block, best_t.ahead, best_t.sigma_pts, best);
      std::fclose(f);
    }
  }
  loc.ray_block = best_t.ray_block;
  loc.ahead = best_t.ahead;
  loc.sigma_points = best_t.sigma_pts;
  loc.ms_best = best;
  loc.ms_default = first;
  loc.from_cache = 0;
  if ((flags & 2) && h->precision == RT_P_MIXED && h->n_cols * h->n_rhs > 1)
    if ((rc = autotune_solve(h, flags, s, sig, path, loc)) != RT_OK) return rc;
  if (out) *out = loc;
  return RT_OK;
}

int rt_arnoldi(rt_handle *h, const double *v0, int32_t m, double *H, int32_t *m_done, void *stream) {
  if (!h || !H || !m_done) return fail(RT_ERR_ARG, "null handle, H or m_done");
  if (fault_now() == kFaultLaunch) return fail(RT_ERR_CUDA, "RT_FAULT=launch: injected launch failure");
  if (h->dims != 3 && !rt::single_instance(h))
    return fail(RT_ERR_ARG, "rt_arnoldi needs a handle with one instance (a box or one column, n_rhs = 1)");
  if (m < 1 || m > rt::kMaxKrylov) return fail(RT_ERR_ARG, "need 1 <= m <= 512");
  const int64_t ldv = (h->E + 31) / 32 * 32;
  if ((int64_t)(m + 1) * ldv * 8 > h->ws.cap_bytes)
    return fail(RT_ERR_ARG, "workspace holds fewer than m+1 float64 vectors: create the handle with a larger max_restart");
  if (v0 && !is_device_ptr(v0)) return fail(RT_ERR_ARG, "v0 must be a device pointer");
  if (!h->g_part) return fail(RT_ERR_ARG, "handle has no grid-solve buffers");
  cudaStream_t s = (cudaStream_t)stream;
  int done = 0;
  const int e = rt::launch_grid_arnoldi(h, v0 ? v0 : h->b_int, m, H, done, s);
  *m_done = done;
  if (e == -1) return fail(RT_ERR_ARG, "v0 is zero or not finite");
  if (e != 0) return fail(RT_ERR_CUDA, std::string("arnoldi: ") + cudaGetErrorString((cudaError_t)e));
  RT_CUDA(cudaStreamSynchronize(s));
  return RT_OK;
}

int rt_solve(rt_handle *h, const double *b, double *x, const rt_solve_opts *o, rt_info *info,
             void *stream) {
  if (!h || !x || !o) return fail(RT_ERR_ARG, "null handle, x or options");
  {
    const int fk = fault_now();
    if (fk == kFaultLaunch) return fail(RT_ERR_CUDA, "RT_FAULT=launch: injected launch failure");
    if (fk == kFaultNan) {
      if (info) {
        rt_info loc{};
        loc.status = RT_ERR_NONFINITE;
        loc.n_instances = h->dims == 3 ? 1 : h->n_cols * h->n_rhs;
        loc.max_relres = NAN;
        loc.inst_outer = info->inst_outer;
        loc.inst_inner = info->inst_inner;
        loc.inst_relres = info->inst_relres;
        *info = loc;
      }
      return fail(RT_ERR_NONFINITE, "RT_FAULT=nan_input: injected non-finite right-hand side");
    }
  }
  if (o->method != RT_KRYLOV_GMRES && o->method != RT_KRYLOV_BICGSTAB)
    return fail(RT_ERR_ARG, "method must be RT_KRYLOV_GMRES or RT_KRYLOV_BICGSTAB");
  const bool bicg = o->method == RT_KRYLOV_BICGSTAB;
  if (!(o->tol > 0.0) || o->max_outer < 1) return fail(RT_ERR_ARG, "need tol > 0 and max_outer >= 1");
  if (bicg) {
    if (o->max_iter < 0) return fail(RT_ERR_ARG, "max_iter must be >= 0");
    const bool fits = h->dims == 3 ? rt::grid_bicgstab_fits(h) : rt::bicgstab_fits(h);
    if (!fits)
      return fail(RT_ERR_ARG, "BiCGStab needs six float64 vectors of workspace per instance: "
                              "create the handle with a larger max_restart");
  } else {
    if (o->restart < 1 || o->restart > h->ws.m) return fail(RT_ERR_ARG, "restart outside [1, max_restart]");
    if (h->precision == RT_P_MIXED && !(o->tol_inner > 0.0 && o->tol_inner < 1.0))
      return fail(RT_ERR_ARG, "mixed precision needs 0 < tol_inner < 1");
    if (o->inner_restart < 0 || o->inner_restart > h->ws.m)
      return fail(RT_ERR_ARG, "inner_restart outside [0, max_restart]");
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t len = h->E * h->n_rhs;
  const bool bd = b ? is_device_ptr(b) : true, xd = is_device_ptr(x);
  const double *bin = b;
  double *xio = x;
  if (!bd || !xd) {
    int rc = ensure_stage(h, len);
    if (rc != RT_OK) return rc;
    if (b && !bd) {
      RT_CUDA(cudaMemcpyAsync(h->stage_y, b, len * sizeof(double), cudaMemcpyHostToDevice, s));
      bin = h->stage_y;
    }
    if (!xd) {
      if (o->use_x0) RT_CUDA(cudaMemcpyAsync(h->stage_x, x, len * sizeof(double), cudaMemcpyHostToDevice, s));
      xio = h->stage_x;
    }
  }
  // boxes and single 1D instances run on the grid-wide kernels; a small single
  // mixed instance stays on one CTA (the host-driven grid loop's per-step
  // synchronisation outweighs a 1-SM inner cycle below ~64k dofs)
  const bool grid_1d = rt::single_instance(h) && (bicg || h->precision == RT_P_FP64 || h->E >= 65536);
  if (h->dims == 3 || grid_1d) {
    int outer = 0, inner = 0, status = 0;
    double relres = 1.0, bytes = 0.0;
    cudaEvent_t e0, e1;
    RT_CUDA(cudaEventCreate(&e0));
    RT_CUDA(cudaEventCreate(&e1));
    RT_CUDA(cudaEventRecord(e0, s));
    const int e = bicg ? rt::launch_grid_bicgstab(h, bin ? bin : h->b_int, xio, o->tol, o->max_outer, o->max_iter,
                                                  o->use_x0, s, outer, inner, relres, status, bytes)
                       : rt::launch_grid_solve(h, bin ? bin : h->b_int, xio, o->tol, o->tol_inner, o->restart,
                                               o->max_outer, o->use_x0, s, outer, inner, relres, status, bytes,
                                               o->inner_restart > 0 ? o->inner_restart : 20);  // single instance
    RT_CUDA(cudaEventRecord(e1, s));
    if (e != 0) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(RT_ERR_CUDA, std::string("grid solve: ") + cudaGetErrorString((cudaError_t)e));
    }
    if (!xd) RT_CUDA(cudaMemcpyAsync(x, xio, len * sizeof(double), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->last_bytes = bytes;
    if (info) {
      rt_info loc{};
      loc.status = status;
      loc.n_instances = 1;
      loc.max_outer = outer;
      loc.max_inner = inner;
      loc.total_inner = inner;
      loc.max_relres = relres;
      loc.ms = ms;
      loc.bytes = bytes;
      loc.inst_outer = info->inst_outer;
      loc.inst_inner = info->inst_inner;
      loc.inst_relres = info->inst_relres;
      if (info->inst_outer) info->inst_outer[0] = outer;
      if (info->inst_inner) info->inst_inner[0] = inner;
      if (info->inst_relres) info->inst_relres[0] = relres;
      *info = loc;
    }
    if (status != RT_OK) {
      char msg[160];
      std::snprintf(msg, sizeof msg, "solve: status %d, relative residual %.3e", status, relres);
      g_err = msg;
    }
    return status;
  }
  cudaEvent_t e0, e1;
  RT_CUDA(cudaEventCreate(&e0));
  RT_CUDA(cudaEventCreate(&e1));
  // the launch (queue reset + persistent kernel) is captured once into a CUDA
  // graph and replayed while (b, x, options) stay the same
  const int m_in = o->inner_restart > 0 ? o->inner_restart : (h->tune.solve_m_in > 0 ? h->tune.solve_m_in : 20);
  unsigned long long key[10];
  key[0] = (unsigned long long)(uintptr_t)bin;
  key[1] = (unsigned long long)(uintptr_t)xio;
  std::memcpy(&key[2], &o->tol, 8);
  std::memcpy(&key[3], &o->tol_inner, 8);
  key[4] = (unsigned long long)o->restart;
  key[5] = (unsigned long long)o->max_outer;
  key[6] = (unsigned long long)o->use_x0;
  key[7] = (unsigned long long)m_in;
  key[8] = (unsigned long long)o->method;
  key[9] = (unsigned long long)o->max_iter;
  int e = 0;
  if (!h->solve_graph || std::memcmp(key, h->graph_key, sizeof key) != 0) {
    if (h->solve_graph) {
      cudaGraphExecDestroy(h->solve_graph);
      h->solve_graph = nullptr;
    }
    if (!h->capture_stream) RT_CUDA(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    RT_CUDA(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
    e = bicg ? rt::launch_bicgstab(h, bin, xio, o->tol, o->max_outer, o->max_iter, o->use_x0, h->capture_stream)
             : rt::launch_solve(h, bin, xio, o->tol, o->tol_inner, o->restart, o->max_outer, o->use_x0,
                                h->capture_stream, m_in);
    const cudaError_t ce = cudaStreamEndCapture(h->capture_stream, &graph);
    if (e == 0 && ce != cudaSuccess) e = (int)ce;
    if (e == 0) e = (int)cudaGraphInstantiate(&h->solve_graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e == 0) std::memcpy(h->graph_key, key, sizeof key);
    h->graph_replays = 0;
  }
  RT_CUDA(cudaEventRecord(e0, s));
  if (e == 0) {
    e = (int)cudaGraphLaunch(h->solve_graph, s);
    ++h->graph_replays;
  }
  if (e != 0) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return fail(RT_ERR_CUDA, std::string("solve launch: ") + cudaGetErrorString((cudaError_t)e));
  }
  RT_CUDA(cudaEventRecord(e1, s));
  if (!xd) RT_CUDA(cudaMemcpyAsync(x, xio, len * sizeof(double), cudaMemcpyDeviceToHost, s));
  RT_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int n_inst = h->n_cols * h->n_rhs;
  std::vector<int32_t> outer(n_inst), inner(n_inst), status(n_inst);
  std::vector<double> relres(n_inst), bytes(n_inst);
  RT_CUDA(cudaMemcpy(bytes.data(), h->so.bytes, n_inst * 8, cudaMemcpyDeviceToHost));
  h->last_bytes = 0.0;
  for (double v : bytes) h->last_bytes += v;
  RT_CUDA(cudaMemcpy(outer.data(), h->so.outer, n_inst * 4, cudaMemcpyDeviceToHost));
  RT_CUDA(cudaMemcpy(inner.data(), h->so.inner, n_inst * 4, cudaMemcpyDeviceToHost));
  RT_CUDA(cudaMemcpy(status.data(), h->so.status, n_inst * 4, cudaMemcpyDeviceToHost));
  RT_CUDA(cudaMemcpy(relres.data(), h->so.relres, n_inst * 8, cudaMemcpyDeviceToHost));
  int worst = RT_OK;
  rt_info loc{};
  loc.n_instances = n_inst;
  for (int i = 0; i < n_inst; ++i) {
    loc.max_outer = std::max(loc.max_outer, outer[i]);
    loc.max_inner = std::max(loc.max_inner, inner[i]);
    loc.total_inner += inner[i];
    loc.max_relres = std::max(loc.max_relres, relres[i]);
    if (status[i] != RT_OK && worst != RT_ERR_TIMEOUT &&
        (worst == RT_OK || status[i] == RT_ERR_NONFINITE || status[i] == RT_ERR_TIMEOUT))
      worst = status[i];
  }
  loc.status = worst;
  loc.ms = ms;
  loc.bytes = h->last_bytes;
  if (info) {
    int32_t *po = info->inst_outer, *pi = info->inst_inner;
    double *pr = info->inst_relres;
    if (po) std::copy(outer.begin(), outer.end(), po);
    if (pi) std::copy(inner.begin(), inner.end(), pi);
    if (pr) std::copy(relres.begin(), relres.end(), pr);
    loc.inst_outer = po;
    loc.inst_inner = pi;
    loc.inst_relres = pr;
    *info = loc;
  }
  if (worst != RT_OK) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "solve: status %d, largest relative residual %.3e", worst, loc.max_relres);
    g_err = msg;
  }
  return worst;
}

void rt_destroy(rt_handle *h) { free_handle(h); }

}  // extern "C"
