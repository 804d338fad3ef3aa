// Population management: approximate partition distances (section "Distance computation"),
// the distance-and-quality pool update (section "Population update") and the K-nearest-neighbour
// parent matching (section "Parent matching and selection of crossovers").
#include <algorithm>

#include "common.cuh"

namespace dlm {

// ------------------------------------------------------------------------------------------------
// Distances. One CTA holds one row X_i in shared memory; each warp owns a k x k overlap table and
// handles pairs (i, j). Per pair: count M[a][b] over the vertices (shared atomics), then the row
// and column maxima by scanning the table (lanes over rows and over columns, no atomics), then
// clear it -- O(n + k^2) per pair.
// ------------------------------------------------------------------------------------------------
constexpr int kDistWarpsMax = 8;
constexpr int kDistCols = 64;  // Y rows handled by one CTA

// overlap-table row stride in 32-bit words: ceil(k / 2) rounded up to an odd number, so that the
// lanes scanning different rows hit different banks
__host__ __device__ inline int dist_row_words(int k) {
  int r = (k + 1) / 2;
  return (r & 1) ? r : r + 1;
}

// one warp's table in words, rounded up to 16 bytes
__host__ __device__ inline int dist_table_words(int k) { return (k * dist_row_words(k) + 3) & ~3; }

__global__ void __launch_bounds__(32 * kDistWarpsMax) k_distance(int n, int k, const int16_t* X, int a, const int16_t* Y,
                                                              int b, int16_t* D, int64_t ldD, int upper,
                                                              int vec4, int32_t* status) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int i = blockIdx.y;
  const int j0 = blockIdx.x * kDistCols;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* xi = smem;  // [n]
  const size_t xoff = (n + 15) & ~15;
  // per warp: the k x k overlap table, u16 counters, rows rw words apart
  const int rw = dist_row_words(k);
  uint32_t* M32 = (uint32_t*)((uint8_t*)smem + xoff + (size_t)warp * dist_table_words(k) * 4);
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    int c = X[(size_t)i * n + v];
    if (c < 0 || c >= k) { raise_status(status, DLM_EINVAL); c = 0; }
    xi[v] = (uint8_t)c;
  }
  for (int q = lane; q < dist_table_words(k); q += 32) M32[q] = 0u;
  __syncthreads();
  const int nwarps = blockDim.x >> 5;
  for (int jj = warp; jj < kDistCols; jj += nwarps) {
    const int j = j0 + jj;
    if (j >= b) break;
    if (upper && j <= i) continue;
    const int16_t* y = Y + (size_t)j * n;
    // counts of every (class of x_i, class of y_j) pair; the partner's colours are checked by the
    // CTAs of row 0 (which see every partner) and clamped everywhere
    const bool check = blockIdx.y == 0;
    auto count1 = [&](int v, int c2) {
      if (check && (c2 < 0 || c2 >= k)) raise_status(status, DLM_EINVAL);
      c2 = (int)min((unsigned)c2, (unsigned)(k - 1));
      const int q = xi[v] * 2 * rw + c2;  // u16 index
      atomicAdd(M32 + (q >> 1), 1u << (16 * (q & 1)));
    };
    if (vec4) {  // four vertices per lane step: 8-byte colour loads (n % 4 == 0, Y 8-byte aligned)
      const uint2* y4 = reinterpret_cast<const uint2*>(y);
      for (int t = lane; t < (n >> 2); t += 32) {
        const uint2 yy = y4[t];
        const int v = 4 * t;
        count1(v, (int16_t)(yy.x & 0xFFFFu));
        count1(v + 1, (int16_t)(yy.x >> 16));
        count1(v + 2, (int16_t)(yy.y & 0xFFFFu));
        count1(v + 3, (int16_t)(yy.y >> 16));
      }
    } else {
      for (int v = lane; v < n; v += 32) count1(v, y[v]);
    }
    __syncwarp();
    // row maxima (lanes over rows, words along the row) and column maxima (lanes over column pairs)
    int sr = 0, scl = 0;
    for (int c = lane; c < k; c += 32) {
      const uint32_t* row = M32 + (size_t)c * rw;
      unsigned m = 0;
      for (int w = 0; w < rw; ++w) {
        const uint32_t x = row[w];
        m = max(m, max(x & 0xFFFFu, x >> 16));
      }
      sr += (int)m;
    }
    for (int cw = lane; cw < (k + 1) / 2; cw += 32) {
      unsigned m0 = 0, m1 = 0;
      for (int r = 0; r < k; ++r) {
        const uint32_t x = M32[(size_t)r * rw + cw];
        m0 = max(m0, x & 0xFFFFu);
        m1 = max(m1, x >> 16);
      }
      scl += (int)(m0 + m1);  // the padding column of an odd k is all zero
    }
    sr = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)sr);
    scl = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)scl);
    if (lane == 0) D[(size_t)i * ldD + j] = (int16_t)(n - (sr < scl ? sr : scl));
    __syncwarp();
    {  // clear the table, 16 bytes per store (its size is rounded up to 16 bytes)
      uint4* M4 = reinterpret_cast<uint4*>(M32);
      for (int q = lane; q < dist_table_words(k) >> 2; q += 32) M4[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------------
// Pool update: one CTA. Candidates are sorted by (f, index) with a shared-memory bitonic sort of
// 64-bit keys; then the greedy pass admits a candidate when no admitted member is within n/10
// (the check of the admitted list is split across the threads, one barrier per candidate).
// ------------------------------------------------------------------------------------------------
constexpr int kPoolThreads = 1024;

__global__ void __launch_bounds__(kPoolThreads) k_pool_update(int p, int n, const int64_t* fit, const int16_t* D,
                                                              int32_t* sel, int32_t* status) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int m = 2 * p;
  int mp = 1;
  while (mp < m) mp <<= 1;
  uint64_t* key = (uint64_t*)smem;             // [mp]
  int32_t* adm = (int32_t*)(key + mp);          // [p] admitted, in order
  uint8_t* chosen = (uint8_t*)(adm + p);        // [m]
  __shared__ int cnt;
  const int t = threadIdx.x;
  for (int q = t; q < mp; q += blockDim.x) {
    if (q < m) {
      int64_t f = fit[q];
      if (f < 0 || f >= ((int64_t)1 << 43)) { raise_status(status, DLM_EINVAL); f = 0; }
      key[q] = ((uint64_t)f << 20) | (uint64_t)q;
    } else {
      key[q] = ~0ull;
    }
  }
  for (int q = t; q < m; q += blockDim.x) chosen[q] = 0;
  if (t == 0) cnt = 0;
  __syncthreads();
  for (int size = 2; size <= mp; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = t; q < mp; q += blockDim.x) {
        const int r = q ^ stride;
        if (r > q) {
          const bool up = (q & size) == 0;
          const uint64_t x = key[q], y = key[r];
          if ((x > y) == up) { key[q] = y; key[r] = x; }
        }
      }
      __syncthreads();
    }
  const int64_t lim = n;  // admitted when 10 * D > n
  for (int s = 0; s < m; ++s) {
    const int c = cnt;  // uniform (written before the last barrier)
    if (c >= p) break;
    const int x = (int)(key[s] & 0xFFFFF);
    __syncthreads();
    int bad = 0;
    const int16_t* row = D + (size_t)x * m;
    for (int q = t; q < c; q += blockDim.x)
      if (10 * (int64_t)row[adm[q]] <= lim) bad = 1;
    bad = __syncthreads_or(bad);
    if (t == 0 && !bad) { adm[c] = x; chosen[x] = 1; cnt = c + 1; }
    __syncthreads();
  }
  // fill with the best remaining candidates when fewer than p were spaced
  if (t == 0) {
    int c = cnt;
    for (int s = 0; s < m && c < p; ++s) {
      const int x = (int)(key[s] & 0xFFFFF);
      if (!chosen[x]) { adm[c++] = x; chosen[x] = 1; }
    }
    cnt = c;
  }
  __syncthreads();
  for (int q = t; q < p; q += blockDim.x) sel[q] = adm[q];
}

// ------------------------------------------------------------------------------------------------
// K nearest neighbours: one warp per row; the row's keys (D << 16 | j) sit in shared memory and
// K rounds of redux.sync min pick them in increasing order.
// ------------------------------------------------------------------------------------------------
constexpr int kKnnWarps = 4;

__global__ void __launch_bounds__(32 * kKnnWarps) k_knn(int p, const int16_t* D, int K, int32_t* nbr) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* keys = (uint32_t*)smem + (size_t)warp * p;
  for (int i = blockIdx.x * kKnnWarps + warp; i < p; i += gridDim.x * kKnnWarps) {
    for (int j = lane; j < p; j += 32) {
      const int d = D[(size_t)i * p + j];
      keys[j] = j == i ? 0xFFFFFFFFu : (((uint32_t)(d < 0 ? 0 : d) << 16) | (uint32_t)j);
    }
    __syncwarp();
    uint32_t last = 0;
    bool first = true;
    for (int r = 0; r < K; ++r) {
      uint32_t best = 0xFFFFFFFFu;
      for (int j = lane; j < p; j += 32) {
        const uint32_t x = keys[j];
        if ((first || x > last) && x < best) best = x;
      }
      best = __reduce_min_sync(0xFFFFFFFFu, best);
      if (lane == 0) nbr[(size_t)i * K + r] = (int32_t)(best & 0xFFFF);
      last = best;
      first = false;
    }
    __syncwarp();
  }
}

}  // namespace dlm

using namespace dlm;

extern "C" dlm_status dlm_distance_batch(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* X, int32_t a,
                                         const int16_t* Y, int32_t b, int16_t* D, int64_t ldD, int32_t upper) {
  if (!ctx) return DLM_EINVAL;
  if (n < 1 || n > 2048 || k < 1 || a < 0 || b < 0 || ldD < b) return fail(ctx, DLM_EINVAL, "distance: bad sizes");
  if (k > 128) return fail(ctx, DLM_EUNSUPPORTED, "distance: k must be <= 128");
  if (a == 0 || b == 0) return DLM_OK;
  if (!X || !Y || !D) return fail(ctx, DLM_EINVAL, "distance: null pointer");
  if (a > 65535) return fail(ctx, DLM_EUNSUPPORTED, "distance: at most 65535 rows");
  // as many warps (overlap tables) as shared memory allows, up to 8
  const size_t per_warp = (size_t)dist_table_words(k) * 4;
  const size_t head = ((n + 15) & ~15) + 16;
  int warps = kDistWarpsMax;
  while (warps > 1 && head + warps * per_warp > ctx->smem_optin) --warps;
  const size_t smem = head + warps * per_warp;
  if (smem > ctx->smem_optin) return fail(ctx, DLM_EUNSUPPORTED, "distance: shared memory");
  DLM_CUDA(ctx, cudaFuncSetAttribute(k_distance, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((b + kDistCols - 1) / kDistCols, a);
  const int vec4 = (n % 4 == 0) && (((uintptr_t)Y & 7) == 0);
  k_distance<<<grid, 32 * warps, smem, ctx->stream>>>(n, k, X, a, Y, b, D, ldD, upper, vec4, ctx->d_status);
  return launch_check(ctx, "k_distance");
}

extern "C" dlm_status dlm_pool_update(dlm_ctx* ctx, int32_t p, int32_t n, const int64_t* fit, const int16_t* D,
                                      int32_t* sel) {
  if (!ctx) return DLM_EINVAL;
  if (p < 1 || n < 1) return fail(ctx, DLM_EINVAL, "pool_update: bad sizes");
  if (!fit || !D || !sel) return fail(ctx, DLM_EINVAL, "pool_update: null pointer");
  const int m = 2 * p;
  int mp = 1;
  while (mp < m) mp <<= 1;
  const size_t smem = (size_t)mp * 8 + (size_t)p * 4 + m + 16;
  if (smem > ctx->smem_optin || m > (1 << 20)) return fail(ctx, DLM_EUNSUPPORTED, "pool_update: p too large");
  DLM_CUDA(ctx, cudaFuncSetAttribute(k_pool_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_pool_update<<<1, kPoolThreads, smem, ctx->stream>>>(p, n, fit, D, sel, ctx->d_status);
  return launch_check(ctx, "k_pool_update");
}

extern "C" dlm_status dlm_knn(dlm_ctx* ctx, int32_t p, const int16_t* D, int32_t K, int32_t* nbr) {
  if (!ctx) return DLM_EINVAL;
  if (p < 2 || K < 1 || K > p - 1 || K > 64) return fail(ctx, DLM_EINVAL, "knn: need 1 <= K <= min(64, p - 1)");
  if (p > 65535) return fail(ctx, DLM_EUNSUPPORTED, "knn: p must be < 65536");
  if (!D || !nbr) return fail(ctx, DLM_EINVAL, "knn: null pointer");
  const size_t smem = (size_t)kKnnWarps * p * 4;
  if (smem > ctx->smem_optin) return fail(ctx, DLM_EUNSUPPORTED, "knn: p too large for shared memory");
  DLM_CUDA(ctx, cudaFuncSetAttribute(k_knn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::min((p + kKnnWarps - 1) / kKnnWarps, ctx->num_sms * 4);
  k_knn<<<grid, 32 * kKnnWarps, smem, ctx->stream>>>(p, D, K, nbr);
  return launch_check(ctx, "k_knn");
}
