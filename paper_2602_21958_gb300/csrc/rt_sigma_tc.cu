// rt_sigma_tc.cu -- Sigma with a dense kernel Psi on the 5th-generation tensor
// cores (tcgen05, sm_103a):  S_p = Gamma_p Psi W X_p  (eq. Sigma), i.e. for one
// column the GEMM  C[rows, r] = sum_q X[rows, q] PsiW[r, q]  with the rows the
// points of every right-hand side stacked, then S = gamma * C.
//
//   operands  : bf16.  X is packed to bf16 once per apply (k_to_bf16); A tiles
//               (128 rows x 64 q) arrive by 16-byte cp.async copies straight
//               into the canonical no-swizzle K-major layout; B = PsiW is
//               pre-tiled in global memory as the exact shared-memory image of
//               each (256-ray, 64-q) block and fetched with one cp.async.bulk
//               completing on an mbarrier.
//   accumulate: fp32 in tensor memory (128 lanes x 256 columns), read back
//               with tcgen05.ld and scaled by Gamma in the epilogue.
//   pipeline  : four stages; thread 0 issues tcgen05.mma (M=128, N<=256,
//               K=16, four per 64-wide chunk) and commits each chunk to an
//               mbarrier; the stage freed by chunk k-1 is refilled with chunk
//               k+3 while the MMAs of chunk k run.
// Every wait is bounded; on timeout the CTA raises an error flag, drains what
// it issued (bounded), frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "rt_async.cuh"
#include "rt_host.h"
#include "rt_internal.cuh"

namespace rt {

constexpr int kTcBM = 128;               // rows per tile (MMA M, TMEM lanes)
constexpr int kTcBN = 256;               // rays per tile (MMA N max, TMEM columns)
constexpr int kTcBK = 64;                // q per stage: four MMAs of K = 16
constexpr int kTcThreads = 256;
constexpr int kTcABytes = kTcBM * kTcBK * 2;   // 16 KB
constexpr int kTcBBytes = kTcBN * kTcBK * 2;   // 32 KB
constexpr int kTcStages = 4;
constexpr int kTcLdt = kTcBN + 4;        // row stride (floats) of the epilogue tile in shared memory
constexpr int kTcSmem = kTcStages * (kTcABytes + kTcBBytes) + 1024;

struct TcJob {
  int32_t col;  // column index
  int32_t m0;   // first stacked row (rhs * nz + point)
  int32_t n0;   // first ray
  int32_t pad;
};

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout of
// 8-row x 16-byte core matrices; lbo = byte distance of K-adjacent core
// matrices, sbo = byte distance of 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: bf16 x bf16 -> f32, both K-major.
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}

// ----------------------------------------------------------------- kernel
// X -> bf16 (same layout), the A operand of the GEMM
template <typename TX>
__global__ void k_to_bf16(const TX *__restrict__ X, uint32_t *__restrict__ Xb, int64_t n2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
    Xb[i] = pack_bf16((float)X[2 * i], (float)X[2 * i + 1]);
}

// One (rows m0.., rays n0..) tile per CTA.  A (bf16 rows of X) arrives by
// 16-byte cp.async copies straight into the core-matrix layout, B by one
// cp.async.bulk per stage; kTcStages stages in flight.
template <typename TS>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_sigma_dense_tc(const ColDev *__restrict__ cols, const TcJob *__restrict__ jobs,
                     const int64_t *__restrict__ btile_off, const uint16_t *__restrict__ btiles,
                     const float *__restrict__ gamma, int n_rhs, int64_t E, const uint16_t *__restrict__ Xb,
                     TS *__restrict__ S, int *err) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tc_smem) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bar_b[kTcStages], bar_mma[kTcStages];
  __shared__ uint32_t tmem_base;
  auto sA = [&](int st) { return base + st * kTcABytes; };
  auto sB = [&](int st) { return base + kTcStages * kTcABytes + st * kTcBBytes; };

  const TcJob job = jobs[blockIdx.x];
  const ColDev c = cols[job.col];
  const int nr = c.nr, nn = c.nn, nz = c.nz;
  const int M = n_rhs * nz;
  const int n_valid = min(kTcBN, nr - job.n0);  // multiple of 16 (nr is)
  const int nk = nr / 16;                        // MMA K-steps in total
  const int nchunk = (nr + kTcBK - 1) / kTcBK;
  const uint16_t *Bcol = btiles + btile_off[job.col] + (int64_t)(job.n0 / kTcBN) * nchunk * (kTcBN * kTcBK);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      mbar_init(&bar_b[i], 1);
      mbar_init(&bar_mma[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTcBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc_idesc(kTcBM, (n_valid + 15) / 16 * 16);

  // A chunk = 128 rows x 8 groups of 8 bf16 (16 bytes).  Thread t copies row
  // t/2, groups 2j + (t&1), j = 0..3: a lane pair reads one 32-byte sector.
  const int arow = tid >> 1, akq = tid & 1;
  const int agrow = job.m0 + arow;
  const bool arow_ok = agrow < M;
  int64_t arow_base = 0;
  if (arow_ok) {
    const int rhs = agrow / nz, p = agrow - rhs * nz;
    arow_base = rhs * E + c.x_off + (int64_t)p * nr;
  }
  const uint32_t a_dst = (uint32_t)((arow >> 3) * 128 + (arow & 7) * 16);
  int b_issued = 0;  // thread 0: B copies issued (chunks 0 .. b_issued-1)
  auto issue = [&](int kc) {  // copies of chunk kc into stage kc % kTcStages
    const int st = kc % kTcStages;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int kq = 2 * j + akq;
      const int q0 = kc * kTcBK + kq * 8;
      const bool in = arow_ok && q0 < nr;
      cp_async16(sA(st) + kq * (kTcBM / 8) * 128 + a_dst, Xb + (in ? arow_base + q0 : 0), in ? 16u : 0u);
    }
    cp_async_commit();
    if (tid == 0) {
      mbar_expect_tx(&bar_b[st], kTcBBytes);
      bulk_g2s(sB(st), Bcol + (int64_t)kc * (kTcBN * kTcBK), kTcBBytes, &bar_b[st]);
      b_issued = kc + 1;
    }
  };
  const int pre = min(kTcStages - 1, nchunk);
  for (int kc = 0; kc < pre; ++kc) issue(kc);
  // Chunk kc: wait for its copies, MMAs by thread 0, then (while those run)
  // refill the stage freed by chunk kc-1 with chunk kc+3.  A failed wait is
  // made uniform by __syncthreads_or before anyone acts on it.
  int committed = 0;  // chunks whose MMAs were committed
  bool ok = true, bad = false;
  for (int kc = 0; kc < nchunk; ++kc) {
    const int st = kc % kTcStages;
    const int later = min(nchunk - 1 - kc, kTcStages - 2);  // chunks issued after kc
    if (later >= 2) cp_async_wait<2>();
    else if (later == 1) cp_async_wait<1>();
    else cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(bad ? 1 : 0)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      if (!mbar_wait(&bar_b[st], (kc / kTcStages) & 1)) {
        bad = true;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(sA(st)), b0 = smem_u32(sB(st));
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          if (kc * 4 + ks < nk) {
            const uint64_t ad = smem_desc(a0 + ks * 2 * (kTcBM / 8) * 128, (kTcBM / 8) * 128, 128);
            const uint64_t bd = smem_desc(b0 + ks * 2 * (kTcBN / 8) * 128, (kTcBN / 8) * 128, 128);
            tc_mma(tmem, ad, bd, idesc, (kc | ks) ? 1u : 0u);
          }
        }
        tc_commit(&bar_mma[st]);
      }
    }
    if (!bad) committed = kc + 1;  // thread 0's flag decides; others follow at the next barrier
    const int nxt = kc + kTcStages - 1;
    if (!bad && nxt < nchunk) {
      // stage of chunk nxt was last read by the MMAs of chunk kc-1
      if (kc >= 1 && !mbar_wait(&bar_mma[(kc - 1) % kTcStages], ((kc - 1) / kTcStages) & 1)) bad = true;
      else issue(nxt);
    }
  }
  if (__syncthreads_or(bad ? 1 : 0)) ok = false;
  cp_async_wait<0>();
  // drain: a commit completes after every earlier MMA of the issuing thread
  bool drained = true;
  {
    __shared__ int s_committed;
    if (tid == 0) s_committed = committed;
    __syncthreads();
    const int kl = s_committed - 1;
    if (kl >= 0) drained = mbar_wait(&bar_mma[kl % kTcStages], (kl / kTcStages) & 1);
    drained = !__syncthreads_or(drained ? 0 : 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && drained) {
    // epilogue, two steps.  (1) TMEM -> shared tile ct[row][col] (the stage
    // buffers are idle now): warp w reads TMEM lanes 32*(w%4).. and columns
    // 128*(w/4)..; row stride kTcLdt floats keeps the 16-byte stores
    // conflict-free.  (2) ct -> S with Gamma, a warp per row, lanes along
    // the rays: coalesced 16-byte stores.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    float *ct = reinterpret_cast<float *>(base);
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    for (int cc = 0; cc < kTcBN / 2; cc += 16) {
      const int col0 = half * (kTcBN / 2) + cc;
      if (col0 >= n_valid) break;  // uniform across the warp
      float v[16];
      tc_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0, v);
      float4 *dst = reinterpret_cast<float4 *>(ct + row * kTcLdt + col0);
#pragma unroll
      for (int t = 0; t < 4; ++t) dst[t] = make_float4(v[4 * t], v[4 * t + 1], v[4 * t + 2], v[4 * t + 3]);
    }
    __syncthreads();
    const int nwarps = kTcThreads / 32;
    for (int r = warp; r < kTcBM; r += nwarps) {
      const int grow = job.m0 + r;
      if (grow >= M) break;  // uniform across the warp
      const int rhs = grow / nz, p = grow - rhs * nz;
      TS *srow = S + rhs * E + c.x_off + (int64_t)p * nr + job.n0;
      const float *g = gamma + c.g_off + (int64_t)p * nn;
      for (int ci = 4 * lane; ci < n_valid; ci += 128) {
        const float4 v = *reinterpret_cast<const float4 *>(ct + r * kTcLdt + ci);
        const int r0 = job.n0 + ci;
        const float a0 = g[r0 % nn] * v.x, a1 = g[(r0 + 1) % nn] * v.y;
        const float a2 = g[(r0 + 2) % nn] * v.z, a3 = g[(r0 + 3) % nn] * v.w;
        if (sizeof(TS) == 4) {
          *reinterpret_cast<float4 *>(srow + ci) = make_float4(a0, a1, a2, a3);
        } else {
          reinterpret_cast<double2 *>(srow + ci)[0] = make_double2(a0, a1);
          reinterpret_cast<double2 *>(srow + ci)[1] = make_double2(a2, a3);
        }
      }
    }
  } else {
    if (tid == 0) {
      atomicOr(err, 1);
      // B copies issued but never consumed may still be landing: wait (bounded)
      for (int kc = committed; kc < b_issued; ++kc) mbar_wait(&bar_b[kc % kTcStages], (kc / kTcStages) & 1);
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcBN) : "memory");
}

// ------------------------------------------------------------ host side
static uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);  // inf / nan
  u += 0x7FFFu + ((u >> 16) & 1u);                                    // round to nearest even
  return (uint16_t)(u >> 16);
}

// PsiW (row r, column q) = PsiwT[q][r] arranged per (256-ray tile, 64-q chunk)
// as [q/8][r/8][r%8][q%8] bf16, zero padded beyond nr.
void tc_build_tiles(const std::vector<ColDev> &cols, const std::vector<double> &psiwT,
                    std::vector<uint16_t> &tiles, std::vector<int64_t> &offs) {
  offs.assign(cols.size(), 0);
  tiles.clear();
  for (size_t ci = 0; ci < cols.size(); ++ci) {
    const ColDev &c = cols[ci];
    if (c.psi_off < 0 || c.nr % 16) continue;
    const int nr = c.nr;
    const int nt = (nr + kTcBN - 1) / kTcBN, nch = (nr + kTcBK - 1) / kTcBK;
    offs[ci] = (int64_t)tiles.size();
    tiles.resize(tiles.size() + (size_t)nt * nch * kTcBN * kTcBK, 0);
    uint16_t *dst = tiles.data() + offs[ci];
    const double *P = psiwT.data() + c.psi_off;
    for (int t = 0; t < nt; ++t)
      for (int ch = 0; ch < nch; ++ch) {
        uint16_t *blk = dst + ((size_t)t * nch + ch) * kTcBN * kTcBK;
        for (int rr = 0; rr < kTcBN; ++rr)
          for (int qq = 0; qq < kTcBK; ++qq) {
            const int r = t * kTcBN + rr, q = ch * kTcBK + qq;
            const float v = (r < nr && q < nr) ? (float)P[(size_t)q * nr + r] : 0.f;
            blk[(qq >> 3) * (kTcBN / 8) * 64 + (rr >> 3) * 64 + (rr & 7) * 8 + (qq & 7)] = bf16_bits(v);
          }
      }
  }
}

void tc_build_jobs(const std::vector<ColDev> &cols, int n_rhs, std::vector<TcJob> &jobs) {
  jobs.clear();
  for (size_t ci = 0; ci < cols.size(); ++ci) {
    const ColDev &c = cols[ci];
    if (c.psi_off < 0 || c.nr % 16) continue;
    const int M = n_rhs * c.nz;
    for (int m0 = 0; m0 < M; m0 += kTcBM)
      for (int n0 = 0; n0 < c.nr; n0 += kTcBN) jobs.push_back(TcJob{(int32_t)ci, m0, n0, 0});
  }
}

// Builds the bf16 tiles and the job list of the tensor-core Sigma (mixed
// precision handles with dense columns).  Returns a cudaError_t as int.
int tc_prepare(rt_handle *h, const std::vector<double> &psiwT) {
  std::vector<uint16_t> tiles;
  std::vector<int64_t> offs;
  std::vector<TcJob> jobs;
  tc_build_tiles(h->h_cols, psiwT, tiles, offs);
  tc_build_jobs(h->h_cols, h->n_rhs, jobs);
  // 16-byte cp.async of bf16 rows needs every row start on 8 elements
  bool aligned = h->E % 8 == 0;
  for (const ColDev &c : h->h_cols) aligned = aligned && c.x_off % 8 == 0;
  h->n_tc_jobs = aligned ? (int)jobs.size() : 0;
  if (h->n_tc_jobs == 0) return 0;
  cudaError_t ex = cudaMalloc(&h->d_tc_xb, (size_t)h->E * h->n_rhs * 2);
  if (ex != cudaSuccess) return (int)ex;
  cudaError_t e = cudaMalloc(&h->d_tc_tiles, tiles.size() * 2);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tc_tiles, tiles.data(), tiles.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_tc_off, offs.size() * 8);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tc_off, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_tc_jobs, jobs.size() * sizeof(TcJob));
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tc_jobs, jobs.data(), jobs.size() * sizeof(TcJob), cudaMemcpyHostToDevice);
  return (int)e;
}

// S is float32 scratch, or the float64 output when s_is_double (all-dense
// batches computing Sigma alone).  X is first packed to bf16 (h->d_tc_xb).
int launch_sigma_dense_tc(rt_handle *h, bool x_is_float, const void *x, void *S, bool s_is_double,
                          cudaStream_t s) {
  if (h->n_tc_jobs == 0) return 0;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_sigma_dense_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    cudaFuncSetAttribute(k_sigma_dense_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    attr_set = true;
  }
  const int64_t n2 = h->E * h->n_rhs / 2;
  const int g = (int)std::min<int64_t>((n2 + 255) / 256, 32 * 152);
  if (x_is_float) k_to_bf16<float><<<g, 256, 0, s>>>(static_cast<const float *>(x), h->d_tc_xb, n2);
  else k_to_bf16<double><<<g, 256, 0, s>>>(static_cast<const double *>(x), h->d_tc_xb, n2);
  const TcJob *jobs = static_cast<const TcJob *>(h->d_tc_jobs);
  const uint16_t *xb = reinterpret_cast<const uint16_t *>(h->d_tc_xb);
  if (s_is_double)
    k_sigma_dense_tc<double><<<h->n_tc_jobs, kTcThreads, kTcSmem, s>>>(
        h->d_cols, jobs, h->d_tc_off, h->d_tc_tiles, h->gam32, h->n_rhs, h->E, xb, static_cast<double *>(S), h->d_err);
  else
    k_sigma_dense_tc<float><<<h->n_tc_jobs, kTcThreads, kTcSmem, s>>>(
        h->d_cols, jobs, h->d_tc_off, h->d_tc_tiles, h->gam32, h->n_rhs, h->E, xb, static_cast<float *>(S), h->d_err);
  return (int)cudaGetLastError();
}

int tc_all_columns(const rt_handle *h) {
  for (const ColDev &c : h->h_cols)
    if (c.psi_off < 0 || c.nr % 16) return 0;
  return h->n_tc_jobs > 0 ? 1 : 0;
}

}  // namespace rt
