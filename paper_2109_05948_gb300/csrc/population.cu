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
// Distances, O(n) per pair whatever k (large k, where the k^2 scan of k_distance dominates). One
// CTA of kDistTeam threads holds X_i and ONE overlap table; the whole CTA handles one pair at a
// time. Every vertex v increments M[a][b] (a = X_i(v), b = Y_j(v)); the counter's new value cnt
// is offered to the running row maximum rmax[a] and column maximum cmax[b] with atomicMax. Counts
// grow by one, so each successful raise lifts a maximum by cnt - (its previous value), and these
// raises add up to the final maximum: their sum over the CTA is sum_a max_b M[a][b] (and the
// column analogue) without a pass over the table. The vertices then clear the entries they
// touched. Two CTA barriers per pair.
// ------------------------------------------------------------------------------------------------
constexpr int kDistTeam = 128;
constexpr int kDistIncMinK = 72;  // from this k on, the automatic choice is k_distance_inc (measured crossover)

template <int VPT>
__global__ void __launch_bounds__(kDistTeam) k_distance_inc(int n, int k, const int16_t* X, int a, const int16_t* Y,
                                                           int b, int16_t* D, int64_t ldD, int upper, int vec4,
                                                           int32_t* status) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int i = blockIdx.y;
  const int j0 = blockIdx.x * kDistCols;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rw = dist_row_words(k);
  uint8_t* xi = smem;
  const size_t xoff = (n + 15) & ~15;
  uint32_t* M32 = (uint32_t*)(smem + xoff);
  uint16_t* M16 = (uint16_t*)M32;
  const int tw = dist_table_words(k);
  uint32_t* rmax = M32 + tw;
  uint32_t* cmax = rmax + k;
  int* red = (int*)(cmax + k);  // [2 parities][kDistTeam / 32 warps][2]
  for (int v = tid; v < n; v += kDistTeam) {
    int c = X[(size_t)i * n + v];
    if (c < 0 || c >= k) { raise_status(status, DLM_EINVAL); c = 0; }
    xi[v] = (uint8_t)c;
  }
  for (int q = tid; q < tw + 2 * k; q += kDistTeam) M32[q] = 0u;
  __syncthreads();
  const bool check = blockIdx.y == 0;
  int par = 0;
  for (int jj = 0; jj < kDistCols; ++jj) {
    const int j = j0 + jj;
    if (j >= b) break;
    if (upper && j <= i) continue;
    const int16_t* y = Y + (size_t)j * n;
    int qv[VPT];  // u16 index of the touched entry (a * 2 rw + b), or -1
    int rs = 0, cs = 0;
    auto touch = [&](int r, int v, int c2) {
      if (check && (c2 < 0 || c2 >= k)) raise_status(status, DLM_EINVAL);
      c2 = (int)min((unsigned)c2, (unsigned)(k - 1));
      const int av = xi[v];
      const int q = av * 2 * rw + c2;
      qv[r] = q;
      const int sh = 16 * (q & 1);
      const uint32_t old = atomicAdd(M32 + (q >> 1), 1u << sh);
      const uint32_t cnt = ((old >> sh) & 0xFFFFu) + 1u;
      const uint32_t r0 = atomicMax(rmax + av, cnt);
      if (r0 < cnt) rs += (int)(cnt - r0);
      const uint32_t c0 = atomicMax(cmax + c2, cnt);
      if (c0 < cnt) cs += (int)(cnt - c0);
    };
    if (vec4) {  // four consecutive vertices per thread and step: one 8-byte colour load
      const uint2* y4 = reinterpret_cast<const uint2*>(y);
#pragma unroll
      for (int r4 = 0; r4 < VPT / 4; ++r4) {
        const int t = tid + kDistTeam * r4;
        if (t < (n >> 2)) {
          const uint2 yy = y4[t];
          touch(4 * r4, 4 * t, (int16_t)(yy.x & 0xFFFFu));
          touch(4 * r4 + 1, 4 * t + 1, (int16_t)(yy.x >> 16));
          touch(4 * r4 + 2, 4 * t + 2, (int16_t)(yy.y & 0xFFFFu));
          touch(4 * r4 + 3, 4 * t + 3, (int16_t)(yy.y >> 16));
        } else {
          qv[4 * r4] = qv[4 * r4 + 1] = qv[4 * r4 + 2] = qv[4 * r4 + 3] = -1;
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < VPT; ++r) {
        const int v = tid + kDistTeam * r;
        if (v < n) touch(r, v, y[v]);
        else qv[r] = -1;
      }
    }
    rs = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)rs);
    cs = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)cs);
    if (lane == 0) { red[(par * (kDistTeam / 32) + warp) * 2] = rs; red[(par * (kDistTeam / 32) + warp) * 2 + 1] = cs; }
    __syncthreads();
    // clear what this pair touched (duplicates store the same zero)
#pragma unroll
    for (int r = 0; r < VPT; ++r) {
      const int q = qv[r];
      if (q >= 0) {
        M16[q] = 0;
        rmax[q / (2 * rw)] = 0u;
        cmax[q % (2 * rw)] = 0u;
      }
    }
    if (tid == 0) {
      int sr = 0, sc = 0;
      for (int w = 0; w < kDistTeam / 32; ++w) {
        sr += red[(par * (kDistTeam / 32) + w) * 2];
        sc += red[(par * (kDistTeam / 32) + w) * 2 + 1];
      }
      D[(size_t)i * ldD + j] = (int16_t)(n - (sr < sc ? sr : sc));
    }
    par ^= 1;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------
// Exact partition distance (section "Distance computation": the distance is n minus the largest
// total overlap over one-to-one matchings of the classes; the paper takes the approximation
// above, this is the exact value it approximates). One warp per pair: the k x k overlap table by
// counting, then the Hungarian algorithm (shortest augmenting paths with row and column
// potentials) on the cost -M, the lanes sharing the column loops. Costs and potentials are
// integers, so the result is exact.
// ------------------------------------------------------------------------------------------------
constexpr int kExactWarps = 4;

__host__ __device__ inline size_t exact_warp_ints(int k) { return (size_t)k * k + 6 * (size_t)(k + 1); }

__global__ void __launch_bounds__(32 * kExactWarps) k_distance_exact(int n, int k, const int16_t* X, int a,
                                                                    const int16_t* Y, int b, int16_t* D, int64_t ldD,
                                                                    int upper, int32_t* status) {
  extern __shared__ __align__(16) int esm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* M = esm + (size_t)warp * exact_warp_ints(k);  // [k][k] overlaps
  int* u = M + (size_t)k * k;                        // [k + 1] row potentials (1-based)
  int* vp = u + (k + 1);                             // [k + 1] column potentials
  int* pm = vp + (k + 1);                            // [k + 1] row matched to column j (0: none)
  int* way = pm + (k + 1);                           // [k + 1] previous column on the path
  int* minv = way + (k + 1);                         // [k + 1]
  int* used = minv + (k + 1);                        // [k + 1]
  const int64_t npairs = (int64_t)a * b;
  const int nw = blockDim.x >> 5;
  constexpr int INF = 0x3FFFFFFF;
  for (int64_t pr = (int64_t)blockIdx.x * nw + warp; pr < npairs; pr += (int64_t)gridDim.x * nw) {
    const int i = (int)(pr / b), j = (int)(pr % b);
    if (upper && j <= i) continue;
    for (int q = lane; q < k * k; q += 32) M[q] = 0;
    __syncwarp();
    const int16_t* x = X + (size_t)i * n;
    const int16_t* y = Y + (size_t)j * n;
    for (int v = lane; v < n; v += 32) {
      int c1 = x[v], c2 = y[v];
      if (c1 < 0 || c1 >= k || c2 < 0 || c2 >= k) { raise_status(status, DLM_EINVAL); c1 = 0; c2 = 0; }
      atomicAdd(M + c1 * k + c2, 1);
    }
    for (int q = lane; q <= k; q += 32) { u[q] = 0; vp[q] = 0; pm[q] = 0; way[q] = 0; }
    __syncwarp();
    for (int r = 1; r <= k; ++r) {
      if (lane == 0) pm[0] = r;
      for (int q = lane; q <= k; q += 32) { minv[q] = INF; used[q] = 0; }
      __syncwarp();
      int j0 = 0;
      for (int guard = 0; guard <= k + 1; ++guard) {
        if (lane == 0) used[j0] = 1;
        __syncwarp();
        const int i0 = pm[j0];
        // over the free columns: reduced cost of (i0, jj), the smallest minv and its column
        int best = INF, bj = k + 1;
        for (int jj = 1 + lane; jj <= k; jj += 32) {
          if (!used[jj]) {
            const int cur = -M[(i0 - 1) * k + (jj - 1)] - u[i0] - vp[jj];
            if (cur < minv[jj]) { minv[jj] = cur; way[jj] = j0; }
            if (minv[jj] < best) { best = minv[jj]; bj = jj; }
          }
        }
        const int delta = (int)__reduce_min_sync(0xFFFFFFFFu, (unsigned)(best + 0x40000000)) - 0x40000000;
        const int j1 = (int)__reduce_min_sync(0xFFFFFFFFu, best == delta ? (unsigned)bj : 0xFFFFFFFFu);
        __syncwarp();
        for (int jj = lane; jj <= k; jj += 32) {
          if (used[jj]) { u[pm[jj]] += delta; vp[jj] -= delta; }
          else minv[jj] -= delta;
        }
        __syncwarp();
        j0 = j1;
        if (j0 > k || pm[j0] == 0) break;
      }
      if (lane == 0 && j0 <= k) {  // augment along the path
        for (int guard = 0; guard <= k + 1 && j0 != 0; ++guard) {
          const int j1 = way[j0];
          pm[j0] = pm[j1];
          j0 = j1;
        }
      }
      __syncwarp();
    }
    int s = 0;
    for (int jj = 1 + lane; jj <= k; jj += 32) s += pm[jj] > 0 ? M[(pm[jj] - 1) * k + (jj - 1)] : 0;
    s = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)s);
    if (lane == 0) D[(size_t)i * ldD + j] = (int16_t)(n - s);
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------------
// Pool update. The greedy pass over the 2p candidates in (f, index) order admits a candidate when
// no member admitted before it is within n/10. A candidate's fate depends only on the candidates
// before it, so the pass runs in blocks of kPoolBlk candidates (in sorted order):
//  (1) k_pool_sort (one CTA): shared-memory bitonic sort of the 64-bit keys (f << 20 | index),
//      giving order[] and rank[] (the sorted position of every candidate);
//  (2) k_pool_scan (all SMs, one warp per candidate row of the block): one coalesced pass over
//      the candidate's row of D finds whether a member admitted in an earlier block is within
//      n/10 (pre) and which earlier candidates of the same block are within n/10 (a kPoolBlk-bit
//      row);
//  (3) k_pool_resolve (one CTA): one warp walks the block in order with those bit rows in shared
//      memory, admitting a candidate when pre is clear and no candidate admitted earlier in the
//      block is marked; it stops once p members are admitted;
//  (4) k_pool_fill (one CTA): when fewer than p were admitted, the best remaining candidates in
//      sorted order fill the population.
// The admitted members and their order are exactly those of the one-candidate-at-a-time pass.
// ------------------------------------------------------------------------------------------------
constexpr int kPoolThreads = 1024;
constexpr int kPoolBlk = 1024;            // candidates resolved per block
constexpr int kPoolWords = kPoolBlk / 32; // words of one in-block bit row
constexpr int kPoolScanWarps = 8;

struct PoolWs {
  int32_t* cnt;        // [1] members admitted so far
  int32_t* order;      // [m] candidate at each sorted position
  int32_t* rank;       // [m] sorted position of each candidate
  uint32_t* adm;       // [ceil(m / 32)] admitted-candidate bitmask
  uint8_t* pre;        // [kPoolBlk] within n/10 of a member admitted in an earlier block
  uint32_t* inblk;     // [kPoolBlk][kPoolWords] earlier candidates of the block within n/10
};

__host__ inline size_t pool_ws_layout(int m, PoolWs* w, uint8_t* base) {
  size_t o = 0;
  auto take = [&](size_t bytes) { uint8_t* q = base ? base + o : nullptr; o += (bytes + 255) & ~(size_t)255; return q; };
  uint8_t* c = take(16);
  uint8_t* ord = take((size_t)m * 4);
  uint8_t* rk = take((size_t)m * 4);
  uint8_t* ad = take((size_t)((m + 31) / 32) * 4);
  uint8_t* pr = take(kPoolBlk);
  uint8_t* ib = take((size_t)kPoolBlk * kPoolWords * 4);
  if (w) {
    w->cnt = (int32_t*)c; w->order = (int32_t*)ord; w->rank = (int32_t*)rk; w->adm = (uint32_t*)ad;
    w->pre = pr; w->inblk = (uint32_t*)ib;
  }
  return o;
}

__global__ void __launch_bounds__(kPoolThreads) k_pool_sort(int m, const int64_t* fit, PoolWs w, int32_t* status) {
  extern __shared__ __align__(16) uint8_t smem[];
  int mp = 1;
  while (mp < m) mp <<= 1;
  uint64_t* key = (uint64_t*)smem;  // [mp]
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
  for (int q = t; q < (m + 31) / 32; q += blockDim.x) w.adm[q] = 0u;
  if (t == 0) *w.cnt = 0;
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
  for (int q = t; q < m; q += blockDim.x) {
    const int x = (int)(key[q] & 0xFFFFF);
    w.order[q] = x;
    w.rank[x] = q;
  }
}

// one warp per candidate at sorted positions b0 .. b0 + kPoolBlk - 1 (D rows read 2 entries per lane step)
__global__ void __launch_bounds__(32 * kPoolScanWarps) k_pool_scan(int m, int n, int p, int b0, const int16_t* D,
                                                                   PoolWs w) {
  __shared__ uint32_t mask[kPoolScanWarps][kPoolWords];
  if (*(volatile int32_t*)w.cnt >= p) return;  // the pass has already admitted p members
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * kPoolScanWarps + warp;  // position within the block
  const int s = b0 + t;
  if (s >= m) return;
  uint32_t* mk = mask[warp];
  mk[lane] = 0u;
  __syncwarp();
  const int x = w.order[s];
  const uint32_t* row = reinterpret_cast<const uint32_t*>(D + (size_t)x * m);  // m is even: 4-byte aligned
  bool pre = false;
  for (int q = lane; q < (m >> 1); q += 32) {
    const uint32_t dd = __ldg(row + q);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int d = (int)(int16_t)(h ? (dd >> 16) : (dd & 0xFFFFu));
      if (10 * d <= n) {  // candidate y = 2q + h is within n/10 of x
        const int y = 2 * q + h;
        if ((__ldg(w.adm + (y >> 5)) >> (y & 31)) & 1u) pre = true;
        const int r = w.rank[y];
        if (r >= b0 && r < s) atomicOr(mk + ((r - b0) >> 5), 1u << ((r - b0) & 31));
      }
    }
  }
  pre = __any_sync(0xFFFFFFFFu, pre);
  __syncwarp();
  w.inblk[(size_t)t * kPoolWords + lane] = mk[lane];
  if (lane == 0) w.pre[t] = pre ? 1 : 0;
}

__global__ void __launch_bounds__(kPoolThreads) k_pool_resolve(int m, int p, int b0, PoolWs w, int32_t* sel) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int c0 = *(volatile int32_t*)w.cnt;
  if (c0 >= p) return;
  const int nb = min(kPoolBlk, m - b0);
  uint32_t* rows = (uint32_t*)smem;                 // [kPoolBlk][kPoolWords]
  uint8_t* pre = smem + (size_t)kPoolBlk * kPoolWords * 4;  // [kPoolBlk]
  {
    const uint4* src = reinterpret_cast<const uint4*>(w.inblk);
    uint4* dst = reinterpret_cast<uint4*>(rows);
    for (int q = threadIdx.x; q < nb * kPoolWords / 4; q += blockDim.x) dst[q] = src[q];
    for (int q = threadIdx.x; q < nb; q += blockDim.x) pre[q] = w.pre[q];
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  uint32_t M = 0u;  // lane l: admitted positions 32 l .. 32 l + 31 of this block
  int c = c0;
  for (int t0 = 0; t0 < nb && c < p; t0 += 4) {
    uint32_t r4[4];
    bool p4[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {  // loads of the next four rows do not depend on M
      const int t = min(t0 + u, nb - 1);
      r4[u] = rows[t * kPoolWords + lane];
      p4[u] = pre[t] != 0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + u;
      if (t >= nb || c >= p) break;
      const bool rej = p4[u] || __any_sync(0xFFFFFFFFu, (r4[u] & M) != 0u);
      if (!rej) {
        if (lane == (t >> 5)) M |= 1u << (t & 31);
        if (lane == 0) {
          const int x = w.order[b0 + t];
          sel[c] = x;
          atomicOr(w.adm + (x >> 5), 1u << (x & 31));
        }
        ++c;
      }
    }
  }
  if (lane == 0) *w.cnt = c;
}

// fewer than p admitted: the best remaining candidates (sorted order) fill sel[cnt .. p)
__global__ void __launch_bounds__(kPoolThreads) k_pool_fill(int m, int p, PoolWs w, int32_t* sel) {
  __shared__ int wsum[kPoolThreads / 32];
  const int c0 = *(volatile int32_t*)w.cnt;
  if (c0 >= p) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int per = (m + kPoolThreads - 1) / kPoolThreads;
  const int s0 = t * per, s1 = min(s0 + per, m);
  int mine = 0;
  for (int s = s0; s < s1; ++s) {
    const int x = w.order[s];
    mine += ((w.adm[x >> 5] >> (x & 31)) & 1u) ? 0 : 1;
  }
  int incl = mine;  // inclusive scan over the warp, then over the warps
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int before = 0;
  for (int q = 0; q < warp; ++q) before += wsum[q];
  int pos = c0 + before + incl - mine;
  for (int s = s0; s < s1 && pos < p; ++s) {
    const int x = w.order[s];
    if (!((w.adm[x >> 5] >> (x & 31)) & 1u)) sel[pos++] = x;
  }
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

namespace dlm {
dlm_status distance_tc(dlm_ctx* ctx, int n, int k, const int16_t* X, int a, const int16_t* Y, int b, int16_t* D,
                       int64_t ldD, int upper);
}

using namespace dlm;

extern "C" dlm_status dlm_distance_exact_batch(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* X, int32_t a,
                                               const int16_t* Y, int32_t b, int16_t* D, int64_t ldD, int32_t upper) {
  if (!ctx) return DLM_EINVAL;
  if (n < 1 || n > 2048 || k < 1 || a < 0 || b < 0 || ldD < b) return fail(ctx, DLM_EINVAL, "distance_exact: bad sizes");
  if (k > 128) return fail(ctx, DLM_EUNSUPPORTED, "distance_exact: k must be <= 128");
  if (a == 0 || b == 0) return DLM_OK;
  if (!X || !Y || !D) return fail(ctx, DLM_EINVAL, "distance_exact: null pointer");
  const size_t per_warp = exact_warp_ints(k) * 4;
  int warps = kExactWarps;
  while (warps > 1 && (size_t)warps * per_warp > ctx->smem_optin) --warps;
  const size_t smem = (size_t)warps * per_warp;
  if (smem > ctx->smem_optin) return fail(ctx, DLM_EUNSUPPORTED, "distance_exact: shared memory");
  DLM_CUDA(ctx, cudaFuncSetAttribute(k_distance_exact, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t npairs = (int64_t)a * b;
  const int grid = (int)std::min<int64_t>((npairs + warps - 1) / warps, (int64_t)ctx->num_sms * 16);
  k_distance_exact<<<grid, 32 * warps, smem, ctx->stream>>>(n, k, X, a, Y, b, D, ldD, upper, ctx->d_status);
  return launch_check(ctx, "k_distance_exact");
}

extern "C" dlm_status dlm_distance_batch_ex(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* X, int32_t a,
                                            const int16_t* Y, int32_t b, int16_t* D, int64_t ldD, int32_t upper,
                                            int32_t method) {
  if (!ctx) return DLM_EINVAL;
  if (n < 1 || n > 2048 || k < 1 || a < 0 || b < 0 || ldD < b) return fail(ctx, DLM_EINVAL, "distance: bad sizes");
  if (k > 255) return fail(ctx, DLM_EUNSUPPORTED, "distance: k must be <= 255");
  if (method < 0 || method > 3) return fail(ctx, DLM_EINVAL, "distance: method must be 0, 1, 2 or 3");
  if (a == 0 || b == 0) return DLM_OK;
  if (!X || !Y || !D) return fail(ctx, DLM_EINVAL, "distance: null pointer");
  if (a > 65535) return fail(ctx, DLM_EUNSUPPORTED, "distance: at most 65535 rows");
  if (method == 0) method = k >= kDistIncMinK ? 2 : 1;
  if (method == 3) return distance_tc(ctx, n, k, X, a, Y, b, D, ldD, upper);
  const int vec4 = (n % 4 == 0) && (((uintptr_t)Y & 7) == 0);
  dim3 grid((b + kDistCols - 1) / kDistCols, a);
  if (method == 2) {
    const size_t smem = ((n + 15) & ~15) + (size_t)dist_table_words(k) * 4 + (size_t)2 * k * 4 + 2 * (kDistTeam / 32) * 8;
    if (smem > ctx->smem_optin) return fail(ctx, DLM_EUNSUPPORTED, "distance: shared memory");
    auto kern = n <= 4 * kDistTeam ? k_distance_inc<4> : n <= 8 * kDistTeam ? k_distance_inc<8> : k_distance_inc<16>;
    DLM_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kDistTeam, smem, ctx->stream>>>(n, k, X, a, Y, b, D, ldD, upper, vec4, ctx->d_status);
    return launch_check(ctx, "k_distance_inc");
  }
  // as many warps (overlap tables) as shared memory allows, up to 8
  const size_t per_warp = (size_t)dist_table_words(k) * 4;
  const size_t head = ((n + 15) & ~15) + 16;
  int warps = kDistWarpsMax;
  while (warps > 1 && head + warps * per_warp > ctx->smem_optin) --warps;
  const size_t smem = head + warps * per_warp;
  if (smem > ctx->smem_optin) return fail(ctx, DLM_EUNSUPPORTED, "distance: shared memory");
  DLM_CUDA(ctx, cudaFuncSetAttribute(k_distance, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_distance<<<grid, 32 * warps, smem, ctx->stream>>>(n, k, X, a, Y, b, D, ldD, upper, vec4, ctx->d_status);
  return launch_check(ctx, "k_distance");
}

extern "C" dlm_status dlm_distance_batch(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* X, int32_t a,
                                         const int16_t* Y, int32_t b, int16_t* D, int64_t ldD, int32_t upper) {
  return dlm_distance_batch_ex(ctx, n, k, X, a, Y, b, D, ldD, upper, 0);
}

extern "C" dlm_status dlm_pool_update(dlm_ctx* ctx, int32_t p, int32_t n, const int64_t* fit, const int16_t* D,
                                      int32_t* sel) {
  if (!ctx) return DLM_EINVAL;
  if (p < 1 || n < 1) return fail(ctx, DLM_EINVAL, "pool_update: bad sizes");
  if (!fit || !D || !sel) return fail(ctx, DLM_EINVAL, "pool_update: null pointer");
  const int m = 2 * p;
  int mp = 1;
  while (mp < m) mp <<= 1;
  const size_t sort_smem = (size_t)mp * 8;
  if (sort_smem > ctx->smem_optin || m > (1 << 20)) return fail(ctx, DLM_EUNSUPPORTED, "pool_update: p too large");
  if (((uintptr_t)D & 3) != 0) return fail(ctx, DLM_EINVAL, "pool_update: D must be 4-byte aligned");
  uint8_t* base = nullptr;
  DLM_TRY(ctx_workspace(ctx, pool_ws_layout(m, nullptr, nullptr), (void**)&base));
  PoolWs w;
  pool_ws_layout(m, &w, base);
  DLM_CUDA(ctx, cudaFuncSetAttribute(k_pool_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem));
  k_pool_sort<<<1, kPoolThreads, sort_smem, ctx->stream>>>(m, fit, w, ctx->d_status);
  DLM_TRY(launch_check(ctx, "k_pool_sort"));
  const size_t res_smem = (size_t)kPoolBlk * kPoolWords * 4 + kPoolBlk;
  DLM_CUDA(ctx, cudaFuncSetAttribute(k_pool_resolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)res_smem));
  for (int b0 = 0; b0 < m; b0 += kPoolBlk) {
    const int nb = std::min(kPoolBlk, m - b0);
    k_pool_scan<<<(nb + kPoolScanWarps - 1) / kPoolScanWarps, 32 * kPoolScanWarps, 0, ctx->stream>>>(m, n, p, b0, D, w);
    DLM_TRY(launch_check(ctx, "k_pool_scan"));
    k_pool_resolve<<<1, kPoolThreads, res_smem, ctx->stream>>>(m, p, b0, w, sel);
    DLM_TRY(launch_check(ctx, "k_pool_resolve"));
  }
  k_pool_fill<<<1, kPoolThreads, 0, ctx->stream>>>(m, p, w, sel);
  return launch_check(ctx, "k_pool_fill");
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
