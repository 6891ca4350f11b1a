// rt_host.h -- host-side handle and launch interface shared by the C-ABI
// translation unit and the kernel translation units.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rt_gb300.h"
#include "rt_async.cuh"
#include "rt_internal.cuh"

namespace rt {

struct SolveOut {
  int32_t *outer, *inner, *status;  // device [n_inst]
  double *relres;                   // device [n_inst]
  double *bytes;                    // device [n_inst] algorithmic HBM bytes of the solve
};

struct Workspace {
  int slots = 0;           // concurrently resident instances (persistent CTAs)
  int per_sm = 1;          // mixed batched solve: CTAs per SM (1: 512 threads, 2: 256)
  int m = 0;               // largest Krylov basis length a solve may ask for
  int64_t ld = 0;          // float64 scratch length per slot (>= largest column)
  int64_t cap_bytes = 0;   // Krylov basis bytes per slot (shared by whatever instance runs there)
  int64_t hld = 0;         // doubles per slot of Hessenberg + Givens storage
  void *V = nullptr;       // [slots][cap_bytes]
  double *S = nullptr;     // [slots][ld] source-function / residual scratch
  double *H = nullptr;     // [slots][hld]
};

// Launch shapes of the apply kernels (rt_autotune)
struct Tune {
  int ray_block = 128;   // rays per sweep tile (threads per CTA): 64, 128, 256
  int ahead = 4;         // depth points per load chunk of a ray (2 chunks in flight): 2, 4, 8
  int sigma_pts = 0;     // cap on points per Sigma tile: 4, 8, or 0 (as many as fit)
  double ms = 0.0;       // apply time measured for this choice
  int from_cache = 0;
  int box_fb = 0;        // 3D sweep: cap on frequencies per CTA (0: largest that fits)
  int box_cpt = 0;       // 3D sweep: cells per thread (0: 8, adjusted to the plane)
  int solve_m_in = 0;    // mixed batched solve: inner cycle length (0: 20)
};

constexpr int kBoxSmemMax = 220 * 1024;  // shared-memory budget of one 3D sweep CTA

// 3D box geometry (device-side copy of the scalars)
struct BoxDev {
  int nx, ny, nz, nd, nn, ie, qsc, lc;  // qsc: quadratic short characteristics, lc: long characteristics
};

}  // namespace rt

struct rt_handle {
  int dims = 1;
  int n_cols = 0, n_rhs = 1, precision = 0, max_restart = 0;
  int64_t E = 0;       // length of one right-hand side (all columns)
  int64_t nmax = 0;    // largest column length
  int n_sm = 0;
  std::vector<rt::ColDev> h_cols;
  rt::ColDev *d_cols = nullptr;
  int32_t *d_dir_cls = nullptr, *d_dir_up = nullptr;
  double *d_tsrc = nullptr, *d_Itop = nullptr, *d_Ibot = nullptr;
  // float64 tables
  double *E64 = nullptr, *A64 = nullptr, *B64 = nullptr, *Uw64 = nullptr, *Ul64 = nullptr,
         *Rw64 = nullptr, *Psi64 = nullptr, *gam64 = nullptr;
  // float32 tables (mixed precision)
  float *E32 = nullptr, *A32 = nullptr, *B32 = nullptr, *Uw32 = nullptr, *Ul32 = nullptr,
        *Rw32 = nullptr, *Psi32 = nullptr, *gam32 = nullptr;
  // quadratic short characteristics: C | A2 | B2 | C2, each n_coef long (null
  // when no column uses it)
  double *Q64 = nullptr;
  float *Q32 = nullptr;
  int64_t n_coef = 0;           // entries of each step-coefficient array
  double *b_int = nullptr;       // internal right-hand side [E]
  int32_t *d_order = nullptr;    // instance order, largest first
  int *d_queue = nullptr;        // work-queue counters (2 ints)
  rt::Workspace ws;
  rt::SolveOut so{};
  double last_bytes = 0.0;           // algorithmic bytes of the last solve (all instances)
  double *stage_x = nullptr, *stage_y = nullptr;  // device staging for host vectors
  // tiled apply: Sigma tiles (instance, first point, points) and sweep tiles
  // (instance, first ray), rhs 0 first; scratch for the source function
  int3 *d_sig_tiles = nullptr;
  int2 *d_sw_tiles = nullptr;
  int n_sig_tiles = 0, n_sig_tiles_rhs0 = 0, n_sw_tiles = 0, n_sw_tiles_rhs0 = 0;
  void *apply_S = nullptr;
  // dense-kernel Sigma on tcgen05 (mixed precision, columns with n_r % 16 == 0)
  int n_tc_jobs = 0;
  void *d_tc_jobs = nullptr;          // TcJob[n_tc_jobs]
  int64_t *d_tc_off = nullptr;        // per column offset into the bf16 tiles
  uint16_t *d_tc_tiles = nullptr;     // pre-tiled bf16 PsiW
  uint32_t *d_tc_xb = nullptr;        // X packed to bf16 (A operand), rows stacked per column
  void *d_tc_maps = nullptr;          // TMA tensor maps over d_tc_xb, one per column
  int *d_err = nullptr;               // device error word (bounded waits)
  long long wait_limit = rt::kSpinLimit;  // polls of a pipeline wait of the tensor-core Sigma
  // rt_tc_timer session: event pairs around launches of the tensor-core Sigma
  std::vector<cudaEvent_t> tc_ev;
  int tc_ev_used = 0;
  // 3D boxes: geometry, per-direction (sx, sy, ds, up), opacity, grid-solve scratch
  // CUDA graph of the batched solve (queue reset + persistent kernel), reused
  // while the call signature (b, x, options) repeats
  cudaGraphExec_t solve_graph = nullptr;
  cudaStream_t capture_stream = nullptr;
  unsigned long long graph_key[10] = {};
  int graph_replays = 0;
  rt::Tune tune{};
  rt::BoxDev box{};
  double *d_geo = nullptr;
  double *chi64 = nullptr;   // 3D: opacity [n_pts][box_npad], zero past n_nu
  float *chi32 = nullptr;
  int box_npad = 0;          // 3D: frequencies rounded up to a multiple of 4
  // truncated frequency kernels of the float32 operator (rt_set_sigma_rank):
  // factors A | B per column, null when every column is exact
  float *lr32 = nullptr;
  double lr_tol = 0.0;
  std::vector<double> h_rw, h_wnu;   // host copies: R w (as RwT) and w_nu per column
  double *box_w064 = nullptr, *box_bt64 = nullptr;  // 3D: float64 step weights, or null
  float *box_kap32 = nullptr, *box_phi32 = nullptr; // 3D: separable opacity kappa [n_pts], phi [npad], or null
  double *g_part = nullptr, *g_red = nullptr, *g_coef = nullptr, *g_r = nullptr;
  int64_t stage_len = 0;
  bool has_dense = false;
};

namespace rt {
// launchers (defined in rt_column.cu); all return a cudaError_t as int
int launch_coefficients(rt_handle *h, const double *d_z, const int64_t *d_zoff,
                        const double *d_chi, const double *d_mu_cls, const int32_t *d_cls_off, cudaStream_t s);
// the handle's tables in one precision (quadratic-SC arrays when present)
inline Tables<double> tables64(const rt_handle *h) {
  Tables<double> t{h->E64, h->A64, h->B64, h->Uw64, h->Ul64, h->Rw64, h->Psi64, h->gam64};
  if (h->Q64) {
    t.C = h->Q64;
    t.A2 = h->Q64 + h->n_coef;
    t.B2 = h->Q64 + 2 * h->n_coef;
    t.C2 = h->Q64 + 3 * h->n_coef;
  }
  return t;
}
inline Tables<float> tables32(const rt_handle *h) {
  Tables<float> t{h->E32, h->A32, h->B32, h->Uw32, h->Ul32, h->Rw32, h->Psi32, h->gam32};
  t.LR = h->lr32;
  if (h->Q32) {
    t.C = h->Q32;
    t.A2 = h->Q32 + h->n_coef;
    t.B2 = h->Q32 + 2 * h->n_coef;
    t.C2 = h->Q32 + 3 * h->n_coef;
  }
  return t;
}
int launch_apply(rt_handle *h, int op, bool fp64, const double *x, double *y, cudaStream_t s,
                 bool first_rhs_only = false);
int launch_solve(rt_handle *h, const double *b, double *x, double tol, double tol_inner, int m,
                 int max_outer, int use_x0, cudaStream_t s, int m_in);
int solve_block_threads();
int launch_sigma_dense_tc(rt_handle *h, bool x_is_float, const void *x, void *S, bool s_is_double,
                          cudaStream_t s);
int tc_all_columns(const rt_handle *h);
struct TcJob;
int tc_prepare(rt_handle *h, const std::vector<double> &psiwT);
// 3D boxes (rt_box.cu)
int box_apply(rt_handle *h, int op, bool fp64, const void *x, bool xf, void *y, bool yf, cudaStream_t s,
              void *scratch);
inline int apply_box(rt_handle *h, int op, bool fp64, const void *x, bool xf, void *y, bool yf, cudaStream_t s) {
  return box_apply(h, op, fp64, x, xf, y, yf, s, nullptr);
}
int box_prepare(rt_handle *h, const double *chi);
int64_t box_scratch_elems(const rt_handle *h, bool fp64);
bool box_plane_fits(int nx, int ny);
bool box_sigma_fits(const rt_desc *d, int rp);
void box_effective_shape(const rt_handle *h, bool fp64, int &fb, int &cpt);
int launch_bicgstab(rt_handle *h, const double *b, double *x, double tol, int max_outer, int max_iter,
                    int use_x0, cudaStream_t s);
bool bicgstab_fits(const rt_handle *h);
int launch_grid_bicgstab(rt_handle *h, const double *b, double *x, double tol, int max_outer, int max_iter,
                         int use_x0, cudaStream_t s, int &restarts, int &iters, double &relres, int &status,
                         double &bytes);
bool grid_bicgstab_fits(const rt_handle *h);
int launch_grid_arnoldi(rt_handle *h, const double *v0, int m, double *H, int &m_done, cudaStream_t s);
// One 1D (column, rhs) instance: its solves run on the grid-wide kernels (all
// SMs) instead of one CTA.
inline bool single_instance(const rt_handle *h) { return h->dims == 1 && h->n_cols * h->n_rhs == 1; }
int launch_grid_solve(rt_handle *h, const double *b, double *x, double tol, double tol_inner, int m,
                      int max_outer, int use_x0, cudaStream_t s, int &outer, int &inner, double &relres,
                      int &status, double &bytes, int m_in = 20);
int grid_ctas(const rt_handle *h);
// allocation-free apply: scratch in a static device array of this many bytes
constexpr long long kNoAllocScratchBytes = 16ll << 20;
int launch_apply_noalloc(rt_handle *h, int op, bool fp64, const double *x, double *y, cudaStream_t s);
constexpr int kRayBlock = 128;  // default rays (threads) per sweep tile
int max_krylov();
constexpr int kMaxKrylov = 512;          // largest Krylov basis (max_restart, rt_arnoldi's m)
constexpr int kGridPartPerCta = 9 * 65;  // float64 partial sums per grid-solve CTA: one projection
                                         // over kMaxKrylov + 2 rows in groups of 8 (+ the norm)
int apply_slots(rt_handle *h);
}  // namespace rt
