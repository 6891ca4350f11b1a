// rt_sigma_tc.cu -- Sigma with a dense kernel Psi on the 5th-generation tensor
// cores (tcgen05, sm_103a):  S_p = Gamma_p Psi W X_p  (eq. Sigma), i.e. for one
// column the GEMM  C[points, r] = sum_q X[points, q] PsiW[r, q]  per
// right-hand side, then S = gamma * C.
//
//   operands  : bf16.  X is packed to bf16 once per apply (k_to_bf16) with each
//               column's (rhs, point) rows stacked; the A tile of a 64-q chunk
//               (64 q x 128 rows, one TMA box from a 2D tensor map per column)
//               lands in the 128-byte-swizzled K-major layout (rows of 128
//               bytes, 16-byte chunks permuted within 8-row 1024-byte atoms),
//               zero-filled past the column; B = PsiW is pre-tiled in global
//               memory as the exact no-swizzle K-major shared-memory image of
//               each (256-ray, 64-q) block, one cp.async.bulk.
//   accumulate: fp32 in tensor memory, two 128 x 256 accumulators, read back
//               with tcgen05.ld and scaled by Gamma in the epilogue.
//   schedule  : persistent CTAs (one per SM) walk the tile list with
//               specialised warps -- a TMA producer, an MMA issuer and eight
//               epilogue warps -- so a tile's epilogue overlaps the next
//               tile's MMAs; stages and accumulators hand over through
//               mbarriers (full/empty, accumulator full/empty).
// Every wait is bounded: the pipeline waits by a per-launch poll limit
// (rt_handle::wait_limit), the drains of a thread's own copies and MMAs by
// kSpinLimit.  On timeout the CTA raises an error flag, lets the other roles
// stop, drains what it issued, frees its tensor memory and returns; the host
// reads the flag (RT_ERR_TIMEOUT).
#include <cuda.h>
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
constexpr int kTcABytes = kTcBM * kTcBK * 2;   // 16 KB
constexpr int kTcBBytes = kTcBN * kTcBK * 2;   // 32 KB

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout of
// 8-row x 16-byte core matrices; lbo = byte distance of K-adjacent core
// matrices, sbo = byte distance of 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// K-major operand in the 128-byte swizzled layout written by a TMA box of 64
// bf16 x rows (each row 128 bytes, 16-byte chunks permuted within 8-row
// 1024-byte atoms): stride between 8-row groups 1024 bytes, layout type
// 128B swizzle (bits 61-63 = 2); a K step of 16 inside the row advances the
// start address by 32 bytes.  The tile must start on a 1024-byte boundary.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(16u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
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

// float64 -> float32 on the integer pipe (the conversion instruction runs at
// the float64 rate on GB300); float32 passes through
__device__ __forceinline__ float to_f32(double v) { return narrow_f32(v); }
__device__ __forceinline__ float to_f32(float v) { return v; }

// ----------------------------------------------------------------- kernel
// eight consecutive values of X as float32 (16-byte vector loads)
__device__ __forceinline__ void load8(const double *p, float (&f)[8]) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
  const double2 a = q[0], b = q[1], c = q[2], d = q[3];
  f[0] = to_f32(a.x), f[1] = to_f32(a.y), f[2] = to_f32(b.x), f[3] = to_f32(b.y);
  f[4] = to_f32(c.x), f[5] = to_f32(c.y), f[6] = to_f32(d.x), f[7] = to_f32(d.y);
}
__device__ __forceinline__ void load8(const float *p, float (&f)[8]) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
  const float4 a = q[0], b = q[1];
  f[0] = a.x, f[1] = a.y, f[2] = a.z, f[3] = a.w, f[4] = b.x, f[5] = b.y, f[6] = b.z, f[7] = b.w;
}

// X -> bf16, the A operand of the GEMM.  Column c's rows of all right-hand
// sides are stacked: row m = rhs * nz + p at n_rhs * x_off + m * nr, so one 2D
// TMA map per column covers every (rhs, point) row and a 128-row tile can
// span two right-hand sides.  Block (x, col, rhs); dense tensor-core columns only.
template <typename TX>
__global__ void k_to_bf16(const ColDev *__restrict__ cols, const TX *__restrict__ X, uint32_t *__restrict__ Xb,
                          int64_t E, int n_rhs) {
  const ColDev c = cols[blockIdx.y];
  if (c.psi_off < 0 || c.nr % 16) return;
  const int rhs = blockIdx.z;
  // nz * nr is a multiple of 16 and x_off, E multiples of 8 (tc_prepare), so
  // every group of eight values starts on a 64-byte (source) and 16-byte
  // (destination) boundary
  const int64_t n8 = (int64_t)c.nz * c.nr / 8;
  const TX *src = X + rhs * E + c.x_off;
  uint4 *dst = reinterpret_cast<uint4 *>(Xb + ((int64_t)n_rhs * c.x_off + (int64_t)rhs * c.nz * c.nr) / 2);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n8; i += (int64_t)gridDim.x * blockDim.x) {
    float f[8];
    load8(src + 8 * i, f);
    dst[i] = make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), pack_bf16(f[6], f[7]));
  }
}

// Bounded mbarrier wait of the pipeline: at most `limit` polls (a launch
// parameter), and it gives up early once another role raised *abort.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t par, volatile int *abort, long long limit) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(par)
        : "memory");
    if (done) return true;
    if ((it & 1023) == 1023 && *abort) return false;
  }
  *abort = 1;
  return false;
}

// Wait for work this thread issued itself (its copies or MMAs in flight)
// before the CTA leaves: not cut short by an abort, bounded by kSpinLimit.
__device__ __forceinline__ void tc_drain(uint64_t *bar, uint32_t par) { mbar_wait(bar, par); }

// Persistent, warp-specialised tile loop.  A CTA walks tiles (column, 128
// stacked rhs/point rows, 256 rays) j = blockIdx.x, blockIdx.x + gridDim.x, ...:
//   warp 0 (one thread): per 64-q chunk, one TMA box of A (64 q x 128 rows,
//     128-byte swizzle, read by the MMA through the SWIZZLE_128B K-major
//     shared-memory descriptor; zero-filled past the column's edges) and one
//     cp.async.bulk of the pre-tiled B (no-swizzle K-major core matrices) into
//     a ring of kT2Stages stages (full / empty mbarriers);
//   warp 1 (one thread): tcgen05.mma (M=128, N<=256, K=16) into one of two
//     TMEM accumulators (2 x 256 columns), releases each stage by
//     tcgen05.commit, and the accumulator when the tile is complete;
//   warps 2-9: epilogue of the previous tile while the next one is
//     multiplied: TMEM (a warp's 32-lane quarter, half of the columns) ->
//     shared slice -> Gamma-scaled coalesced 16-byte stores, then the
//     accumulator is handed back (all eight warps arrive).
constexpr int kT2Stages = 4;
constexpr int kT2EpiWarps = 8;
constexpr int kT2Threads = 64 + 32 * kT2EpiWarps;
constexpr int kT2Ld = 16;  // floats per row of a warp's epilogue slice (16 columns, chunks rotated)
constexpr int kT2StageBytes = kTcABytes + kTcBBytes;
constexpr int kT2EpiBytes = kT2EpiWarps * 32 * kT2Ld * 4;
constexpr int kT2Smem = kT2Stages * kT2StageBytes + kT2EpiBytes + 1024;

struct TcJob2 {
  int32_t col, m0, n0, pad;  // rows m0.. of the column's stacked (rhs, point) rows, rays n0..
};

template <typename TS>
__global__ void __launch_bounds__(kT2Threads, 1)
    k_sigma_dense_tc(const CUtensorMap *__restrict__ maps, const TcJob2 *__restrict__ jobs, int n_jobs,
                     const ColDev *__restrict__ cols, const int64_t *__restrict__ btile_off,
                     const uint16_t *__restrict__ btiles, const float *__restrict__ gamma, int64_t E,
                     int n_rhs, TS *__restrict__ S, int *err, long long limit) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tc_smem) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kT2Stages], empty[kT2Stages], accf[2], acce[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  auto sA = [&](int st) { return base + st * kT2StageBytes; };
  auto sB = [&](int st) { return base + st * kT2StageBytes + kTcABytes; };
  float *epi = reinterpret_cast<float *>(base + kT2Stages * kT2StageBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int i = 0; i < kT2Stages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], kT2EpiWarps);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * kTcBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {  // ---- producer
      int64_t g = 0;
      for (int j = blockIdx.x; j < n_jobs && !abort_flag; j += gridDim.x) {
        const TcJob2 J = jobs[j];
        const ColDev c = cols[J.col];
        const int nchunk = (c.nr + kTcBK - 1) / kTcBK;
        const uint16_t *Bcol = btiles + btile_off[J.col] + (int64_t)(J.n0 / kTcBN) * nchunk * (kTcBN * kTcBK);
        const CUtensorMap *map = maps + J.col;
        for (int kc = 0; kc < nchunk; ++kc, ++g) {
          const int st = (int)(g % kT2Stages);
          if (g >= kT2Stages && !tc_wait(&empty[st], (uint32_t)((g / kT2Stages - 1) & 1), &abort_flag, limit)) break;
          mbar_expect_tx(&full[st], kT2StageBytes);
          tma_load_2d(sA(st), map, kc * kTcBK, J.m0, &full[st]);  // 64 q x 128 rows, 128-byte swizzle
          bulk_g2s(sB(st), Bcol + (int64_t)kc * (kTcBN * kTcBK), kTcBBytes, &full[st]);
        }
      }
      // drain: every issued stage must have landed before the CTA leaves
      for (int64_t q = (g > kT2Stages ? g - kT2Stages : 0); q < g; ++q)
        tc_drain(&full[q % kT2Stages], (uint32_t)((q / kT2Stages) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      int64_t g = 0;
      int t = 0;
      bool any = false;
      for (int j = blockIdx.x; j < n_jobs && !abort_flag; j += gridDim.x, ++t) {
        const TcJob2 J = jobs[j];
        const ColDev c = cols[J.col];
        const int nchunk = (c.nr + kTcBK - 1) / kTcBK, nk = c.nr / 16;
        const int n_valid = min(kTcBN, c.nr - J.n0);
        const int b = t & 1;
        if (t >= 2 && !tc_wait(&acce[b], (uint32_t)((t / 2 - 1) & 1), &abort_flag, limit)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = tc_idesc(kTcBM, (n_valid + 15) / 16 * 16);
        const uint32_t dt = tmem + (uint32_t)(b * kTcBN);
        for (int kc = 0; kc < nchunk; ++kc, ++g) {
          const int st = (int)(g % kT2Stages);
          if (!tc_wait(&full[st], (uint32_t)((g / kT2Stages) & 1), &abort_flag, limit)) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(sA(st)), b0 = smem_u32(sB(st));
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            if (kc * 4 + ks < nk) {
              const uint64_t ad = smem_desc_sw128(a0 + ks * 32);
              const uint64_t bd = smem_desc(b0 + ks * 2 * (kTcBN / 8) * 128, (kTcBN / 8) * 128, 128);
              tc_mma(dt, ad, bd, idesc, (kc | ks) ? 1u : 0u);
            }
          tc_commit(&empty[st]);
          any = true;
        }
        tc_commit(&accf[b]);
      }
      // drain: the last commit completes after every earlier MMA of this thread
      if (any && g > 0) tc_drain(&empty[(g - 1) % kT2Stages], (uint32_t)(((g - 1) / kT2Stages) & 1));
    }
  } else {  // ---- epilogue warps 2..9
    // Warp w reads the TMEM lanes of its accessible quarter (32 * (w % 4)..)
    // and the tile columns [128 * half, 128 * half + 128), half = (w - 2) / 4.
    // Per 16-column slice: TMEM -> the warp's shared slice (row = lane, the
    // four 16-byte chunks of a row rotated by (row / 2) % 4, so the
    // row-per-lane writes are free of bank conflicts) -> Gamma-scaled stores
    // in which 8 lanes write one row's 16 values: whole 128-byte lines (64
    // bytes for float32) per row, 4 rows per instruction.
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    float *tile = epi + (warp - 2) * 32 * kT2Ld;
    const int sub = lane >> 3, c2 = 2 * (lane & 7);  // store layout: row it * 4 + sub, columns c2, c2 + 1
    int t = 0;
    for (int j = blockIdx.x; j < n_jobs && !abort_flag; j += gridDim.x, ++t) {
      const TcJob2 J = jobs[j];
      const ColDev c = cols[J.col];
      const int nr = c.nr, nn = c.nn, nz = c.nz;
      const int n_valid = min(kTcBN, nr - J.n0);
      const int b = t & 1;
      // the eight rows this lane stores in every slice of the tile, resolved
      // to (right-hand side, point) once per tile: offsets of the Gamma row
      // and of the output row (below 2^31: the batch vector's length)
      int goff[8], soff[8];
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int m = J.m0 + quarter * 32 + it * 4 + sub;
        const bool ok = m < n_rhs * nz;
        const int rhs = ok ? m / nz : 0, p = ok ? m - rhs * nz : 0;
        goff[it] = ok ? (int)(c.g_off + (int64_t)p * nn) : -1;
        soff[it] = (int)(rhs * E + c.x_off + (int64_t)p * nr + J.n0);
      }
      if (!tc_wait(&accf[b], (uint32_t)((t / 2) & 1), &abort_flag, limit)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int c_hi = min(n_valid, half * 128 + 128);
      for (int cs = half * 128; cs < c_hi; cs += 16) {
        {
          float v[16];
          tc_ld16(tmem + (uint32_t)(b * kTcBN) + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cs, v);
          float4 *dst = reinterpret_cast<float4 *>(tile + lane * kT2Ld);
          const int rot = (lane >> 1) & 3;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            dst[q ^ rot] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        __syncwarp();
        // frequencies of this lane's two rays (ray = direction * nn +
        // frequency): one division per slice
        const int r0 = J.n0 + cs + c2;
        const int f0 = r0 - (r0 / nn) * nn;
        const int f1 = f0 + 1 == nn ? 0 : f0 + 1;
        float g0[8], g1[8];
#pragma unroll
        for (int it = 0; it < 8; ++it)
          if (goff[it] >= 0) {
            g0[it] = gamma[goff[it] + f0];
            g1[it] = gamma[goff[it] + f1];
          }
#pragma unroll
        for (int it = 0; it < 8; ++it)
          if (goff[it] >= 0) {
            const int row = it * 4 + sub;
            const float2 v = *reinterpret_cast<const float2 *>(
                tile + row * kT2Ld + 4 * ((c2 >> 2) ^ ((row >> 1) & 3)) + (c2 & 3));
            const float a0 = g0[it] * v.x, a1 = g1[it] * v.y;
            TS *dst = S + (int64_t)soff[it] + cs + c2;
            if (sizeof(TS) == 4)
              *reinterpret_cast<float2 *>(dst) = make_float2(a0, a1);
            else
              *reinterpret_cast<double2 *>(dst) = make_double2(widen_f64(a0), widen_f64(a1));
          }
        __syncwarp();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();  // every role has stopped: the abort flag is final
  if (tid == 0 && abort_flag) atomicOr(err, 1);
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTcBN) : "memory");
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

// Tiles of 128 stacked (rhs, point) rows x 256 rays; the tail tile of a
// column is zero-filled by TMA.
void tc_build_jobs(const std::vector<ColDev> &cols, int n_rhs, std::vector<TcJob2> &jobs) {
  jobs.clear();
  for (size_t ci = 0; ci < cols.size(); ++ci) {
    const ColDev &c = cols[ci];
    if (c.psi_off < 0 || c.nr % 16) continue;
    for (int m0 = 0; m0 < n_rhs * c.nz; m0 += kTcBM)
      for (int n0 = 0; n0 < c.nr; n0 += kTcBN) jobs.push_back(TcJob2{(int32_t)ci, m0, n0, 0});
  }
}

// TMA maps over the bf16 copy of X, one per dense column: dims (q, row) =
// (nr, n_rhs * nz), row stride nr elements, box 64 q x 128 rows with the
// 128-byte swizzle (rows and q past the column are zero-filled by the copy);
// the MMA reads the box through smem_desc_sw128.
static int tc_build_maps(rt_handle *h, std::vector<CUtensorMap> &maps) {
  using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return (int)cudaErrorNotSupported;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  maps.assign(h->h_cols.size(), CUtensorMap{});
  for (size_t ci = 0; ci < h->h_cols.size(); ++ci) {
    const ColDev &c = h->h_cols[ci];
    if (c.psi_off < 0 || c.nr % 16) continue;
    const uint16_t *base = reinterpret_cast<const uint16_t *>(h->d_tc_xb) + (int64_t)h->n_rhs * c.x_off;
    const cuuint64_t dims[2] = {(cuuint64_t)c.nr, (cuuint64_t)h->n_rhs * c.nz};
    const cuuint64_t strides[1] = {(cuuint64_t)c.nr * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcBM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(&maps[ci], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(base), dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return (int)cudaErrorInvalidValue;
  }
  return 0;
}

// Builds the bf16 B tiles, the job list and the TMA maps of the tensor-core
// Sigma (mixed precision handles with dense columns).  Returns a cudaError_t.
int tc_prepare(rt_handle *h, const std::vector<double> &psiwT) {
  std::vector<uint16_t> tiles;
  std::vector<int64_t> offs;
  std::vector<TcJob2> jobs;
  tc_build_tiles(h->h_cols, psiwT, tiles, offs);
  tc_build_jobs(h->h_cols, h->n_rhs, jobs);
  // 16-byte vector accesses of the epilogue need x_off and E multiples of 8;
  // its 32-bit row offsets need the batch vector below 2^31 values
  bool aligned = h->E % 8 == 0 && (int64_t)h->E * h->n_rhs < (int64_t(1) << 31);
  for (const ColDev &c : h->h_cols) aligned = aligned && c.x_off % 8 == 0;
  h->n_tc_jobs = aligned ? (int)jobs.size() : 0;
  if (h->n_tc_jobs == 0) return 0;
  cudaError_t ex = cudaMalloc(&h->d_tc_xb, (size_t)h->E * h->n_rhs * 2);
  if (ex != cudaSuccess) return (int)ex;
  std::vector<CUtensorMap> maps;
  if (tc_build_maps(h, maps) != 0) {
    h->n_tc_jobs = 0;  // no TMA encoder: the CUDA-core Sigma handles the dense columns
    return 0;
  }
  cudaError_t e = cudaMalloc(&h->d_tc_tiles, tiles.size() * 2);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tc_tiles, tiles.data(), tiles.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_tc_off, offs.size() * 8);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tc_off, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_tc_jobs, jobs.size() * sizeof(TcJob2));
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tc_jobs, jobs.data(), jobs.size() * sizeof(TcJob2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_tc_maps, maps.size() * sizeof(CUtensorMap));
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_tc_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
  return (int)e;
}

// S is float32 scratch, or the float64 output when s_is_double (all-dense
// batches computing Sigma alone).  X is first packed to bf16 (h->d_tc_xb).
int launch_sigma_dense_tc(rt_handle *h, bool x_is_float, const void *x, void *S, bool s_is_double,
                          cudaStream_t s) {
  if (h->n_tc_jobs == 0) return 0;
  // the shared-memory opt-in belongs to the current device's context: set it
  // on every launch (a host-side call), not once per process
  const void *kern = s_is_double ? (const void *)k_sigma_dense_tc<double> : (const void *)k_sigma_dense_tc<float>;
  cudaError_t ae = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kT2Smem);
  if (ae != cudaSuccess) return (int)ae;
  int64_t most = 1;
  for (const ColDev &c : h->h_cols) most = std::max<int64_t>(most, (int64_t)c.nz * c.nr / 8);
  const dim3 pg((unsigned)std::min<int64_t>((most + 255) / 256, 64), (unsigned)h->n_cols, (unsigned)h->n_rhs);
  if (x_is_float)
    k_to_bf16<float><<<pg, 256, 0, s>>>(h->d_cols, static_cast<const float *>(x), h->d_tc_xb, h->E, h->n_rhs);
  else
    k_to_bf16<double><<<pg, 256, 0, s>>>(h->d_cols, static_cast<const double *>(x), h->d_tc_xb, h->E, h->n_rhs);
  const TcJob2 *jobs = static_cast<const TcJob2 *>(h->d_tc_jobs);
  const CUtensorMap *maps = static_cast<const CUtensorMap *>(h->d_tc_maps);
  const int ctas = std::min(h->n_tc_jobs, h->n_sm > 0 ? h->n_sm : 152);
  // rt_tc_timer session: bracket this launch with the next event pair
  const bool timed = h->tc_ev_used + 2 <= (int)h->tc_ev.size();
  if (timed) cudaEventRecord(h->tc_ev[h->tc_ev_used], s);
  if (s_is_double)
    k_sigma_dense_tc<double><<<ctas, kT2Threads, kT2Smem, s>>>(maps, jobs, h->n_tc_jobs, h->d_cols, h->d_tc_off,
                                                               h->d_tc_tiles, h->gam32, h->E, h->n_rhs,
                                                               static_cast<double *>(S), h->d_err, h->wait_limit);
  else
    k_sigma_dense_tc<float><<<ctas, kT2Threads, kT2Smem, s>>>(maps, jobs, h->n_tc_jobs, h->d_cols, h->d_tc_off,
                                                              h->d_tc_tiles, h->gam32, h->E, h->n_rhs,
                                                              static_cast<float *>(S), h->d_err, h->wait_limit);
  if (timed) {
    cudaEventRecord(h->tc_ev[h->tc_ev_used + 1], s);
    h->tc_ev_used += 2;
  }
  return (int)cudaGetLastError();
}

int tc_all_columns(const rt_handle *h) {
  for (const ColDev &c : h->h_cols)
    if (c.psi_off < 0 || c.nr % 16) return 0;
  return h->n_tc_jobs > 0 ? 1 : 0;
}

}  // namespace rt
