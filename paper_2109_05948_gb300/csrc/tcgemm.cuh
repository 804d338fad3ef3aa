// BF16 GEMM on the 5th-generation tensor cores (tcgen05) for the offspring scorer.
//
// C[M][N] = A[M][K] . B[N][K]^T with A and B bf16, both K-major (row-major with K contiguous),
// FP32 accumulation in tensor memory (TMEM). Persistent CTAs loop over 128 x BN tiles:
//   warp 0      TMA producer: 128 x 64 and BN x 64 tiles (128-byte swizzle) into an S-stage ring
//   warp 1      allocates TMEM; one lane issues tcgen05.mma (M = 128, N = BN, K = 16 per
//               instruction, 4 per 64-wide stage) and commits each stage back to the producer
//   warps 2..9  epilogue: tcgen05.ld of their TMEM lane quarter (one output row per thread), two
//               warps per quarter, each taking half of the tile's columns, then a fused
//               epilogue functor
// Every mbarrier wait is bounded; on timeout the CTA records DLM_ETIMEOUT, stops issuing work,
// drains what it issued (again bounded), frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace dlm {
namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;            // one 128-byte swizzle atom of bf16
constexpr int kEpiWarps = 8;                // two per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bounded wait on the given phase parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// the same load without its wait: the registers are valid only after tmem_wait16 on them
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// waits for the thread's TMEM loads; the registers pass through the statement, so no use of them
// is scheduled before it
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

struct GemmShape {
  int M, N, K;          // full problem (K a multiple of 64)
  int k_chunks_per_cta; // split-K: number of 64-wide chunks per CTA along blockIdx.z
};

// Epilogue functors receive tile(z, n0) with the tile's K split and the first column of the
// half tile they drain (BN / 2 columns), then (row, col0, v[16]) for 16
// consecutive output columns of one row, then finish(row); the kernel copies the functor for
// every tile, so per-row state starts fresh.
// NA / NB = 2: the operand is given as two bf16 matrices, the hi and lo parts of an fp32 matrix
// (x = hi + lo, hi = bf16(x), lo = bf16(x - hi)); every K step then issues hi.hi, and hi.lo /
// lo.hi, into the same accumulator, so the split operand keeps about 16 mantissa bits.
//
// Persistent: CTA b takes tiles b, b + gridDim.x, ... of the (M tile, N tile, K split) grid. TMEM
// holds two accumulators, so the epilogue of one tile overlaps the loads and MMAs of the next;
// the shared-memory ring of K chunks runs across tiles without draining.
template <int BN, int STAGES, int NA, int NB, class Epi>
__global__ void __launch_bounds__(kThreads, 1) gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapA2,
                                                          const __grid_constant__ CUtensorMap mapB,
                                                          const __grid_constant__ CUtensorMap mapB2, GemmShape sh,
                                                          Epi epi, int32_t* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment for the swizzle atoms
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int A_BYTES = BM * BK * 2;
  constexpr int B_BYTES = BN * BK * 2;
  uint8_t* sA = smem;                          // [STAGES][NA][A_BYTES]
  uint8_t* sB = smem + STAGES * NA * A_BYTES;  // [STAGES][NB][B_BYTES]
  uint64_t* full = (uint64_t*)(sB + STAGES * NB * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // [2] accumulator b complete
  uint64_t* acce = accf + 2;        // [2] accumulator b drained by the epilogue
  uint32_t* tmem_slot = (uint32_t*)(acce + 2);
  int* abort_flag = (int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = (sh.M + BM - 1) / BM, nt = sh.N / BN;
  const int nchunks = sh.K / BK, kpc = sh.k_chunks_per_cta;
  const int zt = (nchunks + kpc - 1) / kpc;
  const int tiles = mt * nt * zt;
  auto tile_of = [&](int t, int& m0, int& n0, int& kc0, int& nk) {
    // N tiles fastest: the N tiles of one M tile run on consecutive CTAs, close in time, so the
    // A tile is read from DRAM once and from L2 for the others
    const int z = t / (mt * nt), r = t - z * mt * nt;
    const int mx = r / nt, ny = r - mx * nt;
    m0 = mx * BM;
    n0 = ny * BN;
    kc0 = z * kpc;
    nk = min(kc0 + kpc, nchunks) - kc0;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(accf + b, 1); mbar_init(acce + b, kEpiWarps); }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)(2 * BN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    fence_before_sync();
  }
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- producer: the K chunks of every tile, through the ring ----
    int g = 0;
    for (int t = blockIdx.x; t < tiles && !*(volatile int*)abort_flag; t += gridDim.x) {
      int m0, n0, kc0, nk;
      tile_of(t, m0, n0, kc0, nk);
      for (int i = 0; i < nk; ++i, ++g) {
        const int s = g % STAGES;
        if (g >= STAGES && !mbar_wait(empty + s, ((g / STAGES) - 1) & 1)) { *(volatile int*)abort_flag = 1; break; }
        mbar_expect_tx(full + s, NA * A_BYTES + NB * B_BYTES);
        tma_load_2d(sA + (s * NA) * A_BYTES, &mapA, (kc0 + i) * BK, m0, full + s);
        if (NA == 2) tma_load_2d(sA + (s * NA + 1) * A_BYTES, &mapA2, (kc0 + i) * BK, m0, full + s);
        tma_load_2d(sB + (s * NB) * B_BYTES, &mapB, (kc0 + i) * BK, n0, full + s);
        if (NB == 2) tma_load_2d(sB + (s * NB + 1) * B_BYTES, &mapB2, (kc0 + i) * BK, n0, full + s);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: accumulator (local tile index & 1) ----
    constexpr uint32_t idesc = idesc_bf16(BN);
    int g = 0, lt = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++lt) {
      int m0, n0, kc0, nk;
      tile_of(t, m0, n0, kc0, nk);
      if (nk <= 0) { --lt; continue; }  // no accumulator used (the epilogue writes zeros)
      if (*(volatile int*)abort_flag) break;
      const int b = lt & 1;
      if (lt >= 2 && !mbar_wait(acce + b, ((lt >> 1) - 1) & 1)) { *(volatile int*)abort_flag = 1; break; }
      fence_after_sync();
      const uint32_t acc = tmem + (uint32_t)(b * BN);
      bool ok = true;
      for (int i = 0; i < nk; ++i, ++g) {
        const int s = g % STAGES;
        if (!mbar_wait(full + s, (g / STAGES) & 1)) { ok = false; break; }
        fence_after_sync();
        const uint32_t a0 = smem_u32(sA + (s * NA) * A_BYTES), b0 = smem_u32(sB + (s * NB) * B_BYTES);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          mma_bf16(acc, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc, (i > 0 || kk > 0) ? 1u : 0u);
          if (NB == 2) mma_bf16(acc, sw128_desc(a0 + kk * 32), sw128_desc(b0 + B_BYTES + kk * 32), idesc, 1u);
          if (NA == 2) mma_bf16(acc, sw128_desc(a0 + A_BYTES + kk * 32), sw128_desc(b0 + kk * 32), idesc, 1u);
        }
        mma_commit(empty + s);
      }
      if (!ok) { *(volatile int*)abort_flag = 1; mma_commit(accf + b); break; }
      mma_commit(accf + b);  // arrives once every MMA of this tile has completed
    }
  } else if (warp >= 2) {
    // ---- epilogue: drains accumulator (local tile index & 1) ----
    const int q = warp & 3;                               // TMEM lane quarter this warp may access
    constexpr int HALF = BN / 2;
    const int c0 = ((warp - 2) / 4) * HALF;               // this warp's half of the columns
    int lt = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++lt) {
      int m0, n0, kc0, nk;
      tile_of(t, m0, n0, kc0, nk);
      const int row = m0 + q * 32 + lane;
      Epi e = epi;
      e.tile(kc0 / kpc, n0 + c0);  // the tile's K split and the first column of this half
      if (nk <= 0) {  // empty K range: the tile's contribution is zero
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
        for (int c = c0; c < c0 + HALF; c += 16) e(row, n0 + c, v);
        e.finish(row);
        --lt;  // no accumulator used
        continue;
      }
      const int b = lt & 1;
      const bool ok = mbar_wait(accf + b, (lt >> 1) & 1);
      fence_after_sync();
      if (!ok || *(volatile int*)abort_flag) {
        if (lane == 0) raise_status(status, DLM_ETIMEOUT);
        *(volatile int*)abort_flag = 1;
        break;
      }
      const uint32_t tbase = tmem + (uint32_t)(b * BN) + ((uint32_t)(q * 32) << 16);
      // the next 16 columns' TMEM load is in flight while the functor handles the current ones
      uint32_t cur[16], nxt[16];
      tmem_ld16_issue(tbase + (uint32_t)c0, cur);
      tmem_wait16(cur);
#pragma unroll 1
      for (int c = c0; c < c0 + HALF; c += 16) {
        const bool more = c + 16 < c0 + HALF;  // uniform over the warp
        if (more) tmem_ld16_issue(tbase + (uint32_t)(c + 16), nxt);
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(cur[i]);
        e(row, n0 + c, v);
        if (more) {
          tmem_wait16(nxt);
#pragma unroll
          for (int i = 0; i < 16; ++i) cur[i] = nxt[i];
        }
      }
      e.finish(row);
      fence_before_sync();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acce + b)) : "memory");
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN)));
  }
}

template <int BN, int STAGES, int NA, int NB>
constexpr size_t gemm_smem_bytes() {
  return 1024 + (size_t)STAGES * (NA * BM * BK * 2 + NB * BN * BK * 2) + (2 * STAGES + 4) * 8 + 16;
}

// host: 2-D bf16 tensor map over a row-major [rows][cols] matrix with leading dimension ld
// (elements), box = 64 columns x box_rows rows, 128-byte swizzle, zero fill out of bounds
dlm_status make_map_bf16(dlm_ctx* ctx, CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                         uint32_t box_rows);

}  // namespace tc
}  // namespace dlm
