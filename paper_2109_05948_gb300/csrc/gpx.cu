// GPX crossover (Galinier & Hao 1999, used in section "Parent matching and selection of
// crossovers"): one warp builds one child. The parents' colour classes are bucketed once
// (counting sort in shared memory), so step l only visits the members of the class it inherits;
// the largest remaining class is found with one redux.sync over packed (size, colour) keys.
#include <algorithm>

#include "common.cuh"

namespace dlm {

struct GpxWarpSmem {
  size_t A, B, child, taken, memA, memB, cntA, cntB, offA, offB, curA, curB, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline GpxWarpSmem gpx_layout(int n, int k) {
  GpxWarpSmem s;
  size_t o = 0;
  s.A = o; o += al16(n);
  s.B = o; o += al16(n);
  s.child = o; o += al16(n);
  s.taken = o; o += al16((size_t)((n + 31) / 32) * 4);
  s.memA = o; o += al16((size_t)n * 2);
  s.memB = o; o += al16((size_t)n * 2);
  s.cntA = o; o += al16((size_t)k * 4);
  s.cntB = o; o += al16((size_t)k * 4);
  s.offA = o; o += al16((size_t)k * 4);
  s.offB = o; o += al16((size_t)k * 4);
  s.curA = o; o += al16((size_t)k * 4);
  s.curB = o; o += al16((size_t)k * 4);
  s.total = o;
  return s;
}

constexpr int kGpxWarps = 8;

__device__ __forceinline__ int warp_excl_scan(int x, int lane) {
  int incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += t;
  }
  return incl - x;
}

// Builds one child in the warp's shared-memory slice; the child's labels end in `child` (u8).
__device__ void gpx_warp(int n, int k, const int16_t* gA, const int16_t* gB, uint8_t* sm, const GpxWarpSmem& L,
                         uint64_t seed, uint32_t cid, uint32_t gen, int32_t* status, int lane) {
  uint8_t* A = sm + L.A;
  uint8_t* B = sm + L.B;
  uint8_t* child = sm + L.child;
  uint32_t* taken = (uint32_t*)(sm + L.taken);
  uint16_t* memA = (uint16_t*)(sm + L.memA);
  uint16_t* memB = (uint16_t*)(sm + L.memB);
  int* cntA = (int*)(sm + L.cntA);
  int* cntB = (int*)(sm + L.cntB);
  int* offA = (int*)(sm + L.offA);
  int* offB = (int*)(sm + L.offB);
  int* curA = (int*)(sm + L.curA);
  int* curB = (int*)(sm + L.curB);
  const int nw = (n + 31) / 32;
  for (int c = lane; c < k; c += 32) { cntA[c] = 0; cntB[c] = 0; }
  for (int w = lane; w < nw; w += 32) taken[w] = 0u;
  __syncwarp();
  bool bad = false;
  for (int v = lane; v < n; v += 32) {
    int a = gA[v], b = gB[v];
    if (a < 0 || a >= k || b < 0 || b >= k) { bad = true; a = a < 0 || a >= k ? 0 : a; b = b < 0 || b >= k ? 0 : b; }
    A[v] = (uint8_t)a;
    B[v] = (uint8_t)b;
    atomicAdd(cntA + a, 1);
    atomicAdd(cntB + b, 1);
  }
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) raise_status(status, DLM_EINVAL);
  __syncwarp();
  // class offsets (exclusive prefix over colours) and bucket fill
  int runA = 0, runB = 0;
  for (int c0 = 0; c0 < k; c0 += 32) {
    const int c = c0 + lane;
    const int ca = c < k ? cntA[c] : 0, cb = c < k ? cntB[c] : 0;
    const int ea = warp_excl_scan(ca, lane), eb = warp_excl_scan(cb, lane);
    if (c < k) { offA[c] = runA + ea; curA[c] = runA + ea; offB[c] = runB + eb; curB[c] = runB + eb; }
    runA += __shfl_sync(0xFFFFFFFFu, ea + ca, 31);
    runB += __shfl_sync(0xFFFFFFFFu, eb + cb, 31);
  }
  __syncwarp();
  for (int v = lane; v < n; v += 32) {
    memA[atomicAdd(curA + A[v], 1)] = (uint16_t)v;
    memB[atomicAdd(curB + B[v], 1)] = (uint16_t)v;
  }
  __syncwarp();
  // curA/curB now hold the class ends; sizes = cur - off (class sizes in the full parents)
  for (int l = 0; l < k; ++l) {
    const bool fromA = (l & 1) == 0;
    int* cnt = fromA ? cntA : cntB;
    int* cntO = fromA ? cntB : cntA;
    const uint8_t* O = fromA ? B : A;
    const uint16_t* mem = fromA ? memA : memB;
    const int* off = fromA ? offA : offB;
    const int* end = fromA ? curA : curB;
    unsigned key = 0;
    for (int c = lane; c < k; c += 32) {
      const unsigned kk = ((unsigned)cnt[c] << 8) | (unsigned)(255 - c);
      key = kk > key ? kk : key;
    }
    key = __reduce_max_sync(0xFFFFFFFFu, key);
    if ((key >> 8) == 0) break;  // nothing left to inherit
    const int cs = 255 - (int)(key & 255);
    for (int q = off[cs] + lane; q < end[cs]; q += 32) {
      const int v = mem[q];
      if (!(taken[v >> 5] & (1u << (v & 31)))) {
        child[v] = (uint8_t)l;
        atomicOr(taken + (v >> 5), 1u << (v & 31));
        atomicSub(cntO + O[v], 1);
      }
    }
    __syncwarp();
    if (lane == 0) cnt[cs] = 0;
    __syncwarp();
  }
  for (int v = lane; v < n; v += 32)
    if (!(taken[v >> 5] & (1u << (v & 31)))) {
      const U4 r = rng(seed, (uint32_t)v, gen, cid, kTagGpx);
      child[v] = (uint8_t)below(r.x, (uint32_t)k);
    }
  __syncwarp();
}

__global__ void __launch_bounds__(32 * kGpxWarps) k_gpx(int n, int k, const int16_t* parents, int pop,
                                                         const int32_t* pairs, const uint32_t* child_id, int m,
                                                         int16_t* children, uint64_t seed, uint32_t gen,
                                                         int32_t* status) {
  extern __shared__ __align__(16) uint8_t smem[];
  const GpxWarpSmem L = gpx_layout(n, k);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* sm = smem + (size_t)warp * L.total;
  for (int t = blockIdx.x * kGpxWarps + warp; t < m; t += gridDim.x * kGpxWarps) {
    const int a = pairs[2 * t], b = pairs[2 * t + 1];
    if (a < 0 || a >= pop || b < 0 || b >= pop) {
      if (lane == 0) raise_status(status, DLM_EINVAL);
      continue;
    }
    const uint32_t cid = child_id ? child_id[t] : (uint32_t)t;
    gpx_warp(n, k, parents + (size_t)a * n, parents + (size_t)b * n, sm, L, seed, cid, gen, status, lane);
    const uint8_t* child = sm + L.child;
    for (int v = lane; v < n; v += 32) children[(size_t)t * n + v] = (int16_t)child[v];
    __syncwarp();
  }
}

}  // namespace dlm

using namespace dlm;

extern "C" dlm_status dlm_gpx_batch(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* parents, int32_t pop,
                                    const int32_t* pairs, const uint32_t* child_id, int32_t m, int16_t* children,
                                    uint64_t seed, uint32_t generation) {
  if (!ctx) return DLM_EINVAL;
  if (n < 1 || n > 2048 || k < 1 || pop < 1 || m < 0) return fail(ctx, DLM_EINVAL, "gpx_batch: bad sizes");
  if (k > 255) return fail(ctx, DLM_EUNSUPPORTED, "gpx_batch: k must be <= 255");
  if (m == 0) return DLM_OK;
  if (!parents || !pairs || !children) return fail(ctx, DLM_EINVAL, "gpx_batch: null pointer");
  const size_t smem = gpx_layout(n, k).total * kGpxWarps;
  if (smem > ctx->smem_optin) return fail(ctx, DLM_EUNSUPPORTED, "gpx_batch: shared memory");
  DLM_CUDA(ctx, cudaFuncSetAttribute(k_gpx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gpx, 32 * kGpxWarps, smem);
  const int need = (m + kGpxWarps - 1) / kGpxWarps;
  const int grid = std::min(need, std::max(1, per_sm) * ctx->num_sms);
  k_gpx<<<grid, 32 * kGpxWarps, smem, ctx->stream>>>(n, k, parents, pop, pairs, child_id, m, children, seed,
                                                      generation, ctx->d_status);
  return launch_check(ctx, "k_gpx");
}
