/*
 * rt_gb300.h -- C ABI of the GB300 (sm_103a) matrix-free S_N radiative-transfer
 * operator and its Krylov solve.
 *
 * The operator is the discretised linear polychromatic RT system of
 * Benedusi, Riva, Belluzzi, Serra-Capizzano, "Analysis of eigenvalue clustering
 * leads to optimal scaling in numerical radiative transfer" (arXiv 2602.21958):
 *
 *     A_N I = b,   A_N = Id - Lambda_N Sigma_N,   b = Lambda_N t + I_in
 *                                         (Sec. 3.1, eq. RT_sys_algebraic)
 *
 * Lambda_N is the formal solution along every ray (Sec. 3.2, eqs. ie_1, ie_2,
 * lambda_block; Sec. 3.4 for 3D); Sigma_N = Gamma_N Psi_N W_N is the scattering
 * contraction, block diagonal over spatial points (Sec. 3.3, eqs. S, Sigma).
 *
 * Vector layout (every x, y, b below).  Space-based lexicographic ordering of
 * Sec. 3.1: point-major, then direction, then frequency fastest.  A batch of
 * columns stores, for each right-hand side, the columns one after another; the
 * n_rhs vectors follow each other:  index = ((rhs * E) + off[col]) + (p*n_dir + d)*n_nu + f
 * with E = sum of the columns' sizes nz*n_dir*n_nu.  All values are float64.
 *
 * Memory and ownership.  Descriptor arrays (rt_desc) are HOST pointers that
 * rt_create copies; the caller may free them when it returns.  Vector arguments
 * of rt_apply / rt_solve may be device pointers (used in place, stream-ordered)
 * or host pointers (staged through handle-owned device buffers; the call then
 * synchronises the stream before returning).  The handle owns every workspace;
 * no call frees caller memory.
 *
 * Errors.  Every int-returning call returns RT_OK (0) or an RT_ERR_* code and
 * records a message retrievable by rt_last_error() (thread-local).  On error
 * the output buffers are unspecified; the handle stays valid unless rt_create
 * failed (then *out is NULL).
 *
 * Fault injection (failure-detection tests; implementation property, the paper
 * has none).  The environment variable RT_FAULT, read at each call:
 *   alloc     rt_create / rt_create_batch return RT_ERR_OOM before any device call;
 *   launch    rt_apply, rt_apply_noalloc, rt_solve, rt_arnoldi return RT_ERR_CUDA
 *             before launching;
 *   nan_input rt_solve returns RT_ERR_NONFINITE (info->status too) without launching;
 *   stall     the bounded device waits of the tensor-core Sigma (mixed handles with a
 *             dense kernel) poll once, give up, drain their own copies and MMAs, free
 *             their tensor memory, and the call returns RT_ERR_TIMEOUT; the handle
 *             stays usable.
 *
 * Memory option.  RT_BOX_COEF64=0, read by rt_create for 3D boxes, keeps the
 * float64 sweep's step weights on the fly instead of precomputing them (16
 * bytes per dof, taken only when they fit in a quarter of the free memory).
 * Shape option.  RT_BOX_FB=1, 2 or 4, read by rt_create for 3D boxes, fixes
 * the frequencies per plane-sweep CTA (capped at 2 for the float64 sweep and
 * by shared memory) until rt_autotune picks one by timing.
 */
#ifndef RT_GB300_H
#define RT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
enum {
  RT_OK = 0,
  RT_ERR_ARG = 1,        /* invalid argument (shape, pointer, option)          */
  RT_ERR_CUDA = 2,       /* a CUDA runtime call or kernel launch failed         */
  RT_ERR_OOM = 3,        /* device allocation failed                            */
  RT_ERR_NOCONV = 4,     /* solve stopped before the tolerance; info is filled  */
  RT_ERR_BREAKDOWN = 5,  /* Arnoldi breakdown before convergence                */
  RT_ERR_NONFINITE = 6,  /* NaN or Inf met in inputs or residuals               */
  RT_ERR_TIMEOUT = 7     /* a bounded device wait gave up                       */
};

/* ---- enumerations ---------------------------------------------------- */
enum { RT_FS_SCL = 0,    /* linear short-characteristics exponential step       */
       RT_FS_IE = 1,     /* implicit Euler, eqs. ie_1, ie_2                      */
       RT_FS_QSC = 2,    /* quadratic short characteristics (upwind, current and
                            downwind points; the last step of a ray is linear) --
                            the quadratic exponential integrator of the paper's 3D
                            runs (Sec. 5.3), restated; in 3D boxes the downwind
                            point is the upwind stencil mirrored into the next
                            plane                                                */
       RT_FS_LC = 3 };   /* 3D boxes only: long characteristics (Sec. 3.4 rays,
                            TRIP's choice named in Sec. 5.3) -- each point's ray
                            traced back to the inflow plane, S and chi interpolated
                            at every plane crossing, linear steps; O(nz) steps per
                            point                                                */
enum { RT_P_FP64 = 0,    /* every stage in float64                              */
       RT_P_MIXED = 1 }; /* Sigma and sweep in float32 (bf16 tensor cores for the
                            dense kernel), Krylov and refinement in float64     */
enum { RT_OP_A = 0,      /* y = x - Lambda Sigma x          (eq. RT_sys_algebraic) */
       RT_OP_LAMBDA = 1, /* y = Lambda x, zero inflow       (eq. lambda_block)     */
       RT_OP_SIGMA = 2,  /* y = Sigma x, no thermal term    (eq. Sigma)            */
       RT_OP_RHS = 3 };  /* y = Lambda t + I_in; x unused   (eq. RT_sys_algebraic) */
enum { RT_KRYLOV_GMRES = 0,      /* GMRES (fp64) / flexible GMRES + inner cycles (mixed) */
       RT_KRYLOV_BICGSTAB = 1 }; /* BiCGStab in float64, either handle precision     */

/* ---- one problem: a 1D column or a 3D box ----------------------------- */
typedef struct rt_desc {
  int32_t dims;          /* 1 (plane-parallel column, Sec. 3.1) or 3 (box, Sec. 3.4)   */
  int32_t nx, ny, nz;    /* points; 1D: nx = ny = 1.  3D: nz planes of ny*nx cells,
                            point p = (k*ny + j)*nx + i, plane 0 at the top; periodic
                            in x and y, inflow through the top and bottom planes       */
  int32_t n_dir, n_nu;   /* directions and frequencies; n_r = n_dir*n_nu rays         */
  const double *z;       /* 1D: depth coordinate [nz], strictly increasing from the
                            surface; 3D: spacings {dx, dy, dz}                         */
  const double *dir;     /* [n_dir*3] unit vectors; component 2 is mu = Omega_z,
                            mu > 0 points to the surface (Sec. 3)                    */
  const double *w_dir;   /* [n_dir] direction weights (Sigma uses them as given)      */
  const double *w_nu;    /* [n_nu] frequency weights                                  */
  const double *chi;     /* [n_pts*n_nu] opacity per unit of z; the optical depth of a
                            step is 0.5*(chi_upwind + chi_current)*|dz|/|mu|          */
  const double *gamma;   /* [n_pts*n_nu] Gamma_N diagonal (Sec. 3.3), direction-free   */
  const double *P;       /* [n_dir*n_dir] angular kernel of a separable Phi = P (x) R,
                            or NULL when Psi is given                                 */
  const double *R;       /* [n_nu*n_nu] frequency kernel of a separable Phi           */
  const double *Psi;     /* [n_r*n_r] dense kernel over rays (Psi of eq. Sigma), or
                            NULL.  Sigma_p = Gamma_p Psi diag(w_dir (x) w_nu)         */
  const double *t_src;   /* [n_pts*n_nu] thermal term t = eps_t/chi, or NULL (= 0)    */
  const double *I_top;   /* [n_nu] inflow for mu < 0 at the top, or NULL (= 0)        */
  const double *I_bot;   /* [n_nu] inflow for mu > 0 at the bottom, or NULL (= 0)     */
  int32_t formal_solver; /* RT_FS_SCL, RT_FS_IE, RT_FS_QSC, or RT_FS_LC (boxes)        */
} rt_desc;

/* ---- solve options and report ----------------------------------------- */
typedef struct rt_solve_opts {
  double tol;            /* target ||b - A x||_2 / ||b||_2 per instance (e.g. 1e-12)    */
  double tol_inner;      /* RT_P_MIXED: relative reduction asked of each inner float32
                            GMRES cycle (e.g. 0.1); it stops earlier if reached        */
  int32_t restart;       /* basis length m: GMRES(m) (fp64) or the float64 flexible
                            outer basis (mixed); <= max_restart; clipped per instance to
                            what its workspace slot holds                             */
  int32_t max_outer;     /* restart cycles allowed                                      */
  int32_t use_x0;        /* 1: x holds the initial guess on entry; 0: start from x = 0  */
  int32_t inner_restart; /* RT_P_MIXED: inner float32 GMRES cycle length (0 -> the
                            length rt_autotune picked, else 20)                       */
  int32_t method;        /* RT_KRYLOV_GMRES (0) or RT_KRYLOV_BICGSTAB (1)               */
  int32_t max_iter;      /* BiCGStab: iteration cap per instance (0 -> 10000); with
                            BiCGStab, max_outer bounds the restarts from the true
                            residual (taken when the recursive residual drifted or a
                            coefficient broke down) and restart is ignored          */
} rt_solve_opts;

typedef struct rt_info {
  int32_t status;          /* RT_OK or the worst instance outcome: RT_ERR_NOCONV, RT_ERR_BREAKDOWN, RT_ERR_NONFINITE, RT_ERR_TIMEOUT */
  int32_t n_instances;     /* n_cols * n_rhs                                          */
  int32_t max_outer;       /* largest number of outer steps over the instances        */
  int32_t max_inner;       /* largest total inner (Arnoldi) iterations                */
  int64_t total_inner;     /* sum of inner iterations over the instances              */
  double max_relres;       /* largest final true relative residual                    */
  double ms;               /* device time of the solve kernel (CUDA events)           */
  double bytes;            /* algorithmic HBM bytes the solve moved: every vector read
                              or written once per operation it takes part in         */
  int32_t *inst_outer;     /* optional host arrays [n_instances] filled when non-NULL */
  int32_t *inst_inner;
  double *inst_relres;
} rt_info;

typedef struct rt_handle rt_handle;

/* Create a handle for one problem (1D column or 3D box).  Copies the
 * descriptor, precomputes the per-layer step coefficients in float64 (e^-dtau
 * via exp, 1 - e^-dtau via expm1, w1/dtau by its alternating series below
 * dtau = 0.1), factors the separable kernel, and allocates workspaces for up
 * to max_restart Krylov vectors.  precision: RT_P_FP64 or RT_P_MIXED.
 * Returns RT_ERR_ARG on an invalid descriptor, RT_ERR_OOM / RT_ERR_CUDA on
 * device failures.  Cites: Sec. 3.1-3.4. */
int rt_create(const rt_desc *desc, int32_t n_rhs, int32_t precision,
              int32_t max_restart, rt_handle **out);

/* Create a handle for a batch of independent 1D columns (each desc->dims ==
 * 1) of uneven nz, n_dir, n_nu, solved together (one persistent launch).  The
 * batch operator is block diagonal: each column is its own system A_N I = b of
 * Sec. 3.1 (eq. RT_sys_algebraic) with its own grid of Sec. 3.1 (N_s, N_Omega,
 * N_nu), and a batch vector holds the columns back to back per right-hand
 * side.  Workspace scales with the number of concurrently resident instances,
 * not with the batch.  Same errors as rt_create. */
int rt_create_batch(const rt_desc *cols, int32_t n_cols, int32_t n_rhs,
                    int32_t precision, int32_t max_restart, rt_handle **out);

/* Number of float64 values of one x / y / b argument (all columns, all rhs):
 * n_rhs * sum over columns of N = N_s N_Omega N_nu (Sec. 3.1, the size of the
 * space-based vector ordering); 0 for a NULL handle. */
int64_t rt_vector_length(const rt_handle *h);

/* Apply one operator (RT_OP_*) to all n_rhs vectors: y = op(x).  x and y must
 * not overlap.  In RT_P_MIXED handles the operator is applied in the mixed
 * precision (float32 Sigma and sweep; float64 x and y); pass fp64 = 1 to force
 * the float64 operator.  Asynchronous on `stream` (a cudaStream_t, NULL = the
 * legacy default stream) unless x or y is host memory. */
int rt_apply(rt_handle *h, int32_t op, int32_t fp64, const double *x, double *y,
             void *stream);

/* ---- launch-shape tuning ----------------------------------------------- */
typedef struct rt_tune_info {
  int32_t ray_block;     /* rays per sweep tile (threads per CTA): 64, 128 or 256        */
  int32_t ahead;         /* depth points per load chunk of a ray (two chunks in flight): 2, 4 or 8 */
  int32_t sigma_points;  /* cap on points per Sigma tile: 4, 8, or 0 (as many as fit)    */
  int32_t from_cache;    /* 1 if read from the RT_TUNE_CACHE file                       */
  double ms_best;        /* rt_apply(RT_OP_A) time of the choice                         */
  double ms_default;     /* time of the default shape; 0 if from cache                   */
  int32_t box_fb;        /* 3D boxes: frequencies per plane-sweep CTA (1, 2 or 4)        */
  int32_t box_cpt;       /* 3D boxes: cells per thread of the plane sweep (1, 2, 4, 8)   */
  int32_t solve_per_sm;  /* flags & 2: CTAs per SM of the mixed batched solve (1 or 2)   */
  int32_t solve_inner;   /* flags & 2: its inner cycle length (12, 20 or 30)             */
  double solve_ms;       /* flags & 2: solve time of the choice                          */
} rt_tune_info;

/* Pick the launch shapes of the apply kernels by timing rt_apply(RT_OP_A) on
 * this handle's own problem, and keep the fastest on the handle (every later
 * rt_apply and every solve of a 3D box uses it).  1D batches: the sweep tile
 * width and its load-ahead depth and the Sigma tile size (27 combinations).
 * 3D boxes: the plane sweep's frequencies per CTA and cells per thread (the
 * distinct feasible combinations of 1, 2, 4 and 1, 2, 4, 8).  With flags & 2,
 * on a mixed-precision 1D batch of more than one instance, also the persistent
 * solve: one 512-thread or two 256-thread CTAs per SM (the Krylov workspace is
 * re-allocated to match) and the inner cycle length used when
 * rt_solve_opts.inner_restart is 0, timed on full solves of the batch with the
 * internal right-hand side (several seconds for a large batch).  When the
 * environment variable RT_TUNE_CACHE names a file, a previous result for the
 * same problem signature is read from it (JSON lines) instead of re-timing,
 * unless flags & 1; new results are appended.  Allocates temporary vectors.
 * out may be NULL.  (Implementation choice; the paper has no counterpart.) */
int rt_autotune(rt_handle *h, int32_t flags, rt_tune_info *out, void *stream);

/* Allocation-free variant of rt_apply, for callers that cannot allocate
 * device memory at call time: a host program that gives its whole device
 * memory budget to its own pool at start-up and forbids later allocations, a
 * real-time loop that must not enter the CUDA allocator (cudaMalloc can
 * synchronise the device and take unbounded time), or a plug-in running
 * inside a program that owns the device.  (The paper has no counterpart; it
 * is a property of this library's interface.)
 * Same operators and layouts as rt_apply, on a handle created beforehand, but
 * the source-function scratch of the apply is a static 16 MiB device array in
 * the library instead of handle-owned memory, and the call allocates nothing.
 * Limits and behaviour:
 *  - x and y must be device pointers (host staging would allocate): else RT_ERR_ARG;
 *  - the scratch needed, n_rhs * E elements of the operator's precision
 *    (float64 if fp64 or an RT_P_FP64 handle, else float32; E alone for 3D
 *    boxes, whose frequencies are padded to a multiple of the sweep's
 *    frequency block), must fit in 16 MiB: else RT_ERR_ARG naming the size;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current;
 *  - on a mixed-precision handle whose Sigma runs on the tensor cores (dense
 *    kernel), ops RT_OP_A and RT_OP_SIGMA with fp64 = 0 read the kernel's
 *    device error word back and synchronise the stream before returning, as
 *    rt_apply does (RT_ERR_TIMEOUT if a bounded wait gave up); every other
 *    call is asynchronous on `stream`;
 *  - every call, from any handle, shares the one array: calls that overlap on
 *    the GPU (other streams, other threads) race and must be serialised by the
 *    caller; the array keeps the last call's contents (whatever must start at
 *    zero is cleared by the call itself). */
int rt_apply_noalloc(rt_handle *h, int32_t op, int32_t fp64, const double *x, double *y, void *stream);

/* Compressed scattering for the low-precision operator (Sec. 4, Remark
 * comput: Sigma_N is approximated at a rank r_eps with linear cost).  For
 * each column of a mixed-precision 1D handle the frequency kernel is
 * truncated in its weighted eigenbasis, W^(1/2) R W^(1/2) = U L U^T with
 * W = diag(w_nu): the eigenvalues with |l| >= tol * max|l| are kept, so the
 * frequency step of Sigma costs 2 n_nu r instead of n_nu^2 per point and
 * angular rank; its error in the W^(1/2)-weighted norm is the largest dropped
 * |l|.  Affects only the float32 operator: rt_apply with fp64 = 0 and the inner
 * cycles of rt_solve; the float64 operator, and so the solution rt_solve
 * returns, stay exact.  Columns whose rank would exceed 32, dense-Psi and
 * coherent (diagonal) kernels keep the exact kernel.  tol = 0 restores the
 * exact kernel everywhere.  max_rank (may be NULL): largest rank kept.
 * Errors: RT_ERR_ARG for a 3D box or a float64 handle, tol outside [0, 1).
 * Synchronous (host eigen-decompositions, one upload). */
int rt_set_sigma_rank(rt_handle *h, double tol, int32_t *max_rank);

/* Device time of the tensor-core Sigma kernel alone, for roofline
 * measurements (implementation property; the paper has none).  on = 1 starts a
 * timing session on this handle: every later launch of that kernel (rt_apply
 * with fp64 = 0 and op RT_OP_A or RT_OP_SIGMA on a handle with dense-Psi
 * columns) is bracketed by two CUDA events on its stream, up to 4096 launches
 * per session (later ones are not timed).  on = 0 ends the session, waits for
 * the recorded events and writes the summed device time in milliseconds to
 * *ms and the number of timed launches to *launches (either may be NULL); the
 * bf16 packing of x that precedes each launch is not included.  The events
 * are created when the session starts and destroyed when it ends.  Errors:
 * RT_ERR_ARG for a NULL handle or on = 0 without a session, RT_ERR_CUDA. */
int rt_tc_timer(rt_handle *h, int32_t on, double *ms, int64_t *launches);

/* Solve A_N x = b for all instances (eq. RT_sys_algebraic; the Krylov solvers
 * of Sec. 5, GMRES and BiCGStab, unpreconditioned).  b == NULL uses the
 * internal right-hand side Lambda t + I_in for every rhs.
 * opts->method == RT_KRYLOV_GMRES:
 *   RT_P_FP64: restarted GMRES(m) in float64 (classical Gram-Schmidt with the
 *   DGKS re-orthogonalisation test, Givens rotations).  RT_P_MIXED: flexible
 *   GMRES(m) in float64 (Arnoldi, Givens, the residual b - A x and x all
 *   float64) whose directions come from one float32 GMRES(inner_restart)
 *   cycle on the float32 operator (basis stored in binary16 for 1D batches)
 *   -- a float64 Krylov loop around low-precision inner solves.
 * opts->method == RT_KRYLOV_BICGSTAB: BiCGStab (van der Vorst) in float64
 *   with the float64 operator on either handle precision; six float64 vectors
 *   of workspace per instance (create the handle with max_restart >= 5 for
 *   RT_P_FP64, >= 3 for RT_P_MIXED batches, >= 11 for RT_P_MIXED boxes), else
 *   RT_ERR_ARG.  Converged only when the true residual b - A x meets tol.
 * Batches: one persistent launch, a CTA per (column, rhs) instance; boxes:
 * grid-wide kernels.  x0 = 0 unless opts->use_x0.  Synchronises the stream and
 * fills *info (may be NULL; for BiCGStab max_inner counts iterations and
 * max_outer restarts).  Returns RT_ERR_NOCONV if any instance missed opts->tol
 * (x still holds the last iterate). */
int rt_solve(rt_handle *h, const double *b, double *x, const rt_solve_opts *opts,
             rt_info *info, void *stream);

/* Spectral diagnostics: m steps of the Arnoldi process on A_N (float64
 * operator) for a handle holding ONE instance (a 3D box, or one 1D column with
 * n_rhs = 1), from v0 (device pointer, the instance's length; NULL: the
 * internal right-hand side Lambda t + I_in).  Classical Gram-Schmidt with the
 * DGKS second projection, grid-wide kernels.  The eigenvalues of the leading
 * m_done x m_done block of H (Ritz values) approximate the spectrum of A_N
 * whose clustering at 1 and lower bound Sec. 4 proves and Sec. 5 measures
 * (Tables mono, iso; Thm main4); computing them is the caller's (the library
 * returns H).
 *   H      : host array, (m+1) x m, column-major; zero where unused
 *   m_done : host int, steps taken (< m when the Krylov space became invariant)
 * Errors: RT_ERR_ARG for a batch handle, m < 1, a workspace holding fewer than
 * m+1 float64 vectors (create the handle with a larger max_restart), a zero or
 * non-finite v0; RT_ERR_CUDA on a CUDA failure.  Synchronises the stream. */
int rt_arnoldi(rt_handle *h, const double *v0, int32_t m, double *H, int32_t *m_done, void *stream);

/* Release every device and host resource of the handle (NULL is a no-op).
 * The handle holds the discretised operator of Sec. 3 (coefficients of
 * Lambda_N, factors of Sigma_N) and its Krylov workspaces; caller buffers
 * are never freed.  Must not be called while work of the handle is in
 * flight on any stream. */
void rt_destroy(rt_handle *h);

/* Message of the last error raised on this thread ("" if none). */
const char *rt_last_error(void);

/* Library version string. */
const char *rt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RT_GB300_H */
