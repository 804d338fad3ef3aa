// Population-wide TabuCol for k-COL (paper: section "Adaptations of the algorithm for the vertex
// coloring problem" -- TabuCOL of Hertz & de Werra in the implementation of Galinier & Hao, run
// on every offspring; Table params-COL for alpha = 0.6 and the 128|V| depth).
//
// GB300 design (differs from the paper's one-thread-per-individual Numba kernel):
//  * one CTA of W warps per individual; its whole search state lives in shared memory:
//      gam[n][ks] u16  conflict table gamma (row stride ks u16 with ks/2 odd, so that the
//                      scattered row updates of a warp spread over the banks)
//      tab[n][ks] u16  tabu expiry relative to a base that advances by 2^14 every 2^14
//                      iterations (one sweep), so a tabu test is a single unsigned compare
//      col[n], best[n] u8 current and best colouring; cv[] u32 bitmap of conflicting vertices;
//      rowres[n] u32   (row minimum delta, tie count) of each conflicting row of the scan.
//  * scan: each warp compacts the bitmap into its own list of conflicting vertices; rows are cut
//    into segments so that every thread scans (two colours per 32-bit word, no warp collectives
//    inside a segment); the order of (row, segment) items follows the thread order.
//  * selection: per-warp minima and tie counts go through one barrier; every thread derives the
//    block minimum, the tie total and its rank range, and the warp holding the j-th tied move
//    (j drawn from the iteration's Philox block) finds its colour with ballots over the segment
//    and applies the move.
//  * update: the adjacency bit row of the moved vertex (L2 resident) is split across all threads; each neighbour costs two u16 read-modify-writes of its gamma row
//    and, when its conflict status flips, one shared atomic on the bitmap.
//  Three CTA barriers per iteration.
#include <algorithm>
#include <climits>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace dlm {

struct TabuJob {
  int32_t n, k, ks, words;
  const uint32_t* bits;  // [n][words]
  int16_t* col;          // [n] in: start, out: best
  int64_t* best_f;       // -> one int64
  int64_t* moves;        // -> one int64 or null
  int32_t* trace;        // [iters][4] or null
  int64_t* work;         // [2] or null: sum of conflicting rows scanned, sum of degrees of moved vertices
  const int32_t* off;    // CSR offsets (degrees for the work counter)
  int64_t iters;
  uint32_t ind;          // Philox stream id of this individual
};

struct TabuRule {
  uint32_t L1;           // L_max + 1
  int32_t an, ad;        // alpha = an / ad
  uint64_t seed;
  uint32_t gen;
  int32_t* status;
  size_t budget;         // shared-memory bytes of the launch
  uint16_t* slab;        // spilled rows, slab_stride u16 per CTA (null when nothing spills)
  size_t slab_stride;
  const int32_t* cancel; // device-readable flag, nonzero = stop (null: never)
};

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kNone16 = 0x7FFF;

__host__ __device__ inline int tabu_row_stride(int k) {
  int kw = (k + 1) / 2;
  if ((kw & 1) == 0) kw += 1;
  return 2 * kw;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Rows a warp's threads scan in one iteration: items [32 w C, 32 (w + 1) C) of the (row, segment)
// list, C = ceil(items / threads) <= ceil(n / threads), hence at most 32 C + 1 rows.
__host__ __device__ inline int tabu_list_cap(int n, int warps) {
  const int nt = 32 * warps;
  return 32 * ((n + nt - 1) / nt) + 1;
}

struct TabuSmem {
  size_t gam, tab, col, best, rowres, deg, cvl, cv, red, rnd, total;
  int rs;  // rows of gamma and tab held in shared memory; rows rs..n-1 live in the CTA's slab
};

// Shared-memory layout of one individual within `budget` bytes: the small arrays first, then as
// many rows of gamma and tab as fit (all n when the state fits, as for n = 500, k = 48).
__host__ __device__ inline TabuSmem tabu_smem_layout(int n, int k, int warps, size_t budget) {
  TabuSmem s;
  const int ks = tabu_row_stride(k);
  size_t o = 0;
  s.col = o; o += align16(n);
  s.best = o; o += align16(n);
  s.rowres = o; o += align16((size_t)(n > 32 * warps ? n : 32 * warps) * 4);  // items <= max(n, threads)
  s.deg = o; o += align16((size_t)n * 2);
  s.cvl = o; o += align16((size_t)warps * tabu_list_cap(n, warps) * 2);
  s.cv = o; o += 64 * 4;
  s.red = o; o += align16((size_t)warps * 8 + 64);
  s.rnd = o; o += 32 * 8;
  const size_t row = (size_t)ks * 2;
  size_t rs = budget > o + 32 ? (budget - o - 32) / (2 * row) : 0;
  if (rs > (size_t)n) rs = n;
  s.rs = (int)rs;
  s.gam = o; o += align16(rs * row);
  s.tab = o; o += align16(rs * row);
  s.total = o;
  return s;
}

// gamma and tab rows that do not fit in shared memory: per CTA, (n - rs) rows of each
__host__ __device__ inline size_t tabu_slab_elems(int n, int k, int rs) {
  return (size_t)2 * (size_t)(n - rs) * tabu_row_stride(k);
}

// position of the r-th (0-based) set bit of x (x has more than r set bits)
__device__ __forceinline__ int nth_set_bit(uint32_t x, int r) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const int c = __popc(x & ((1u << s) - 1u));
    if (r >= c) { r -= c; x >>= s; pos += s; }
  }
  return pos;
}

__device__ __forceinline__ int nth_set_bit64(uint64_t x, int r) {
  const uint32_t lo = (uint32_t)x;
  const int pl = __popc(lo);
  return r < pl ? nth_set_bit(lo, r) : 32 + nth_set_bit((uint32_t)(x >> 32), r - pl);
}

// Warp view of the conflicting-vertex bitmap: lane l owns the B = 2^lb bits of vertices
// lB .. lB + B - 1 (B the smallest power of two with 32 B >= n, so the work spreads over all
// lanes), its popcount and the exclusive prefix over lanes (= rank of its first vertex).
struct CvView {
  uint64_t w;
  int cnt, excl, total;
};

__device__ __forceinline__ CvView cv_view(const uint32_t* cv, int lb, int lane) {
  CvView c;
  const int o = lane << lb;
  if (lb == 6) {
    c.w = ((uint64_t)cv[2 * lane + 1] << 32) | cv[2 * lane];
  } else {
    const uint32_t word = cv[o >> 5];
    c.w = lb == 5 ? word : (word >> (o & 31)) & ((1u << (1 << lb)) - 1u);
  }
  c.cnt = __popcll(c.w);
  int incl = c.cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += t;
  }
  c.excl = incl - c.cnt;
  c.total = __shfl_sync(FULL, incl, 31);
  return c;
}

// Scan of words [w0, w1) of a conflicting row by one thread. The key of colour c is gamma[v][c]
// when the move (v, c) is admissible -- not tabu (relative expiry <= itrel), or tabu but
// f + delta < best_f, i.e. gamma < thr with thr = best_f - f + gamma[v][col v] -- and 0xFFFF
// otherwise; the current colour (killed here) and the padding columns carry 0xFFFF. Returns the
// segment's minimum key and how many colours reach it.
__device__ __forceinline__ void scan_seg(const uint32_t* g32, const uint32_t* t32, int w0, int w1, int killw,
                                         uint32_t killm, unsigned itrel, int thr, unsigned& kmin, int& cnt) {
  unsigned km = 0xFFFFu;
  int c = 0;
#pragma unroll 4
  for (int w = w0; w < w1; ++w) {
    uint32_t gw = g32[w];
    const uint32_t tw = t32[w];
    if (w == killw) gw |= killm;
    const unsigned ga = gw & 0xFFFFu, gb = gw >> 16;
    const unsigned k0 = ((tw & 0xFFFFu) <= itrel || (int)ga < thr) ? ga : 0xFFFFu;
    const unsigned k1 = ((tw >> 16) <= itrel || (int)gb < thr) ? gb : 0xFFFFu;
    const unsigned m = min(k0, k1);
    const int cc = (int)(k0 == m) + (int)(k1 == m);
    if (m < km) { km = m; c = cc; }
    else if (m == km) c += cc;
  }
  kmin = km;
  cnt = c;
}

// One individual, one CTA of W warps (SPILL: rows beyond the shared-memory budget live in the
// CTA's global slab).
// Per iteration: (1) every warp compacts the conflicting-vertex bitmap into its own list; the rows
// are cut into S contiguous segments (S = threads / |CV| when there are fewer rows than threads)
// and thread t scans items [tC, tC + C) of the (row, segment) list, keeping per-item (min delta,
// #ties) and its own aggregate; (2) one barrier publishes the per-warp minima and tie counts:
// every thread derives the minimum delta, the total T and its own rank range; the warp holding
// the j-th tie (j drawn from the iteration's Philox block) finds its colour with ballots over the
// tied segment and applies the move; (3) all threads update gamma on the neighbours. Three barriers per iteration. The Philox blocks of 32
// iterations are drawn at once, one per lane, by one warp every 32 iterations.
//
// Tabu list: u16 expiries relative to a base that advances by 2^14 every 2^14 iterations
// (t' = expiry - base, 0 = free); a pair is tabu when t' > it - base.
template <int W, bool SPILL>
__device__ void tabucol_individual(const TabuJob& J, const TabuRule& R, uint8_t* smem) {
  constexpr int NT = 32 * W;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = J.n, k = J.k, ks = J.ks, kw = ks / 2, nwords = J.words;
  const TabuSmem L = tabu_smem_layout(n, k, W, R.budget);
  const int rs = SPILL ? L.rs : n;
  uint16_t* gam = (uint16_t*)(smem + L.gam);
  uint16_t* tab = (uint16_t*)(smem + L.tab);
  uint16_t* gslab = SPILL ? R.slab + (size_t)blockIdx.x * R.slab_stride : nullptr;
  uint16_t* tslab = SPILL ? gslab + (size_t)(n - rs) * ks : nullptr;
  // row v of gamma / tab: shared memory for v < rs, the CTA's global slab beyond
  auto grow_of = [&](int v) -> uint16_t* {
    if (!SPILL) return gam + v * ks;
    return v < rs ? gam + (size_t)v * ks : gslab + (size_t)(v - rs) * ks;
  };
  auto trow_of = [&](int v) -> uint16_t* {
    if (!SPILL) return tab + v * ks;
    return v < rs ? tab + (size_t)v * ks : tslab + (size_t)(v - rs) * ks;
  };
  uint8_t* colS = smem + L.col;
  uint8_t* bestS = smem + L.best;
  uint32_t* rowres = (uint32_t*)(smem + L.rowres);
  uint16_t* degS = (uint16_t*)(smem + L.deg);
  uint16_t* cvl = (uint16_t*)(smem + L.cvl) + (size_t)warp * tabu_list_cap(n, W);
  uint32_t* cv = (uint32_t*)(smem + L.cv);
  int32_t* red = (int32_t*)(smem + L.red);   // [W] warp minima, [W] warp tie totals
  int32_t* sc = red + 2 * W;                 // scalars
  uint32_t* rnd = (uint32_t*)(smem + L.rnd); // Philox words (r0, r1) of the next 32 iterations
  // sc[0] moved vertex (-1 none), sc[1] old colour, sc[2] new colour, sc[3] f after,
  // sc[4] improved, sc[5] error, sc[6] bad input
  const int iters = (int)J.iters;  // at most 2^31 - 1 (checked by the host)
  auto draw32 = [&](int it0) {     // one warp: lane l draws the block of iteration it0 + l
    const U4 r = rng(R.seed, (uint32_t)(it0 + lane), R.gen, J.ind, kTagTabu);
    rnd[2 * lane] = r.x;
    rnd[2 * lane + 1] = r.y;
  };

  // ---- set-up: zero the tables (padding colours of gamma = 0xFFFF), load the start colouring --
  {
    const int nw32 = n * kw;
    for (int i = tid; i < nw32; i += NT) {
      const int v = i / kw, w = i - v * kw;
      const int c0 = 2 * w;
      ((uint32_t*)grow_of(v))[w] = (c0 >= k ? 0xFFFFu : 0u) | (c0 + 1 >= k ? 0xFFFF0000u : 0u);
      ((uint32_t*)trow_of(v))[w] = 0u;
    }
    if (tid < 16) sc[tid] = 0;
    for (int i = tid; i < 64; i += NT) cv[i] = 0u;
    if (warp == W - 1) draw32(0);
  }
  __syncthreads();
  for (int v = tid; v < n; v += NT) {
    const int c = J.col[v];
    if (c < 0 || c >= k) sc[6] = 1;
    const uint8_t cc = (uint8_t)(c < 0 ? 0 : (c >= k ? 0 : c));
    colS[v] = cc;
    bestS[v] = cc;
  }
  __syncthreads();
  if (sc[6]) {
    if (tid == 0) raise_status(R.status, DLM_EINVAL);
    return;
  }
  // gamma rows: one thread per row, neighbours from the bit rows
  for (int v = tid; v < n; v += NT) {
    const uint32_t* brow = J.bits + (size_t)v * nwords;
    uint16_t* grow = grow_of(v);
    int dv = 0;
    for (int w = 0; w < nwords; ++w) {
      uint32_t m = __ldg(brow + w);
      dv += __popc(m);
      while (m) {
        const int u = 32 * w + __ffs(m) - 1;
        m &= m - 1;
        grow[colS[u]]++;
      }
    }
    degS[v] = (uint16_t)dv;
  }
  __syncthreads();
  int f;
  {
    int part = 0;
    for (int v0 = warp * 32; v0 < n; v0 += NT) {
      const int v = v0 + lane;
      int g = 0;
      if (v < n) g = grow_of(v)[colS[v]];
      part += g;
      const unsigned b = __ballot_sync(FULL, g > 0);
      if (lane == 0) cv[v0 >> 5] = b;
    }
    part = __reduce_add_sync(FULL, part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < W; ++w) tot += red[w];
    f = tot / 2;
    __syncthreads();
  }
  int best_f = f;
  int moves = 0;
  int it = 0;
  int64_t work_rows = 0, work_deg = 0;  // kept by thread 0 only

  // per-thread slice of a bit row for the gamma update
  int per = (n + NT - 1) / NT;
  {
    int p2 = 1;
    while (p2 < per) p2 <<= 1;
    per = p2 > 32 ? 32 : p2;
  }
  const uint32_t slice_mask = per == 32 ? 0xFFFFFFFFu : ((1u << per) - 1u);
  const float fNT = (float)NT + 0.5f;
  int lb = 0;  // bitmap bits per lane = 2^lb, 32 * 2^lb >= n (n <= 2048)
  while ((32 << lb) < n) ++lb;

  for (it = 0; it < iters; ++it) {
    if (f == 0) break;
    const unsigned itrel = (unsigned)(it & 0x3FFF);
    // ---- phase 1: conflicting-vertex list of this warp, scan of this thread's items ----------
    const CvView view = cv_view(cv, lb, lane);
    const int ncv = view.total;
    if (tid == 0) {
      work_rows += ncv;
      sc[0] = -1;
      // cancellation, polled every 1024 iterations: the search stops after this iteration's
      // selection and reports its best colouring so far
      if ((it & 1023) == 0 && R.cancel && *(volatile const int32_t*)R.cancel != 0) sc[5] = 3;
    }
    // S = min(kw, floor(NT / ncv)) and Lw = ceil(kw / S) in float arithmetic: both quotients are
    // of integers below 2^16 shifted by one half, far from the next integer compared with the
    // rounding error, so the truncations are exact
    int S = 1;
    if (ncv > 0 && ncv < NT) S = min(kw, (int)(fNT / (float)ncv));
    const float rS = 1.0f / (float)S;
    const int Lw = (int)(((float)(kw + S - 1) + 0.5f) * rS);
    const int items = ncv * S;
    const int C = (items + NT - 1) / NT;
    const int i0 = tid * C;
    const int i1 = min(i0 + C, items);
    // this warp's rows [rlo, rhi] of the conflicting-vertex list, compacted from the bitmap in
    // ascending vertex order (rank = position among the conflicting vertices)
    const int wi0 = 32 * warp * C, wi1 = min(wi0 + 32 * C, items);
    const int rlo = S == 1 ? wi0 : (int)(((float)wi0 + 0.5f) * rS);
    const int rhi = wi1 <= wi0 ? rlo - 1 : (S == 1 ? wi1 - 1 : (int)(((float)(wi1 - 1) + 0.5f) * rS));
    if (view.excl <= rhi && view.excl + view.cnt > rlo) {
      uint64_t wb = view.w;
      int rank = view.excl;
      while (wb && rank <= rhi) {
        if (rank >= rlo) cvl[rank - rlo] = (uint16_t)((lane << lb) + __ffsll(wb) - 1);
        wb &= wb - 1;
        ++rank;
      }
    }
    __syncwarp();
    int tmin = INT_MAX, tcnt = 0;
    for (int i = i0; i < i1; ++i) {
      const int r = S == 1 ? i : (int)(((float)i + 0.5f) * rS), sg = i - r * S;
      const int v = cvl[r - rlo];
      const int colv = colS[v];
      const uint16_t* grow = grow_of(v);
      const int g0 = grow[colv];
      const int w0 = sg * Lw, w1 = min(w0 + Lw, kw);
      unsigned km;
      int kc;
      scan_seg((const uint32_t*)grow, (const uint32_t*)trow_of(v), w0, w1, colv >> 1,
               0xFFFFu << (16 * (colv & 1)), itrel, best_f - f + g0, km, kc);
      const int rc = km == 0xFFFFu ? 0 : kc;
      const int dm = km == 0xFFFFu ? kNone16 : (int)km - g0;
      rowres[i] = ((uint32_t)(uint16_t)dm << 16) | (uint32_t)rc;
      if (rc > 0) {
        if (dm < tmin) { tmin = dm; tcnt = rc; }
        else if (dm == tmin) tcnt += rc;
      }
    }
    {
      const int wm = __reduce_min_sync(FULL, tmin);
      const int wc = (int)__reduce_add_sync(FULL, (wm != INT_MAX && tmin == wm) ? (unsigned)tcnt : 0u);
      if (lane == 0) { red[warp] = wm; red[W + warp] = wc; }
    }
    __syncthreads();
    // ---- phase 2: minimum delta, tie ranks, move ---------------------------------------------
    int wmin[W], wcnt[W];
    if constexpr (W % 4 == 0) {
#pragma unroll
      for (int q = 0; q < W / 4; ++q) {
        const int4 a = reinterpret_cast<const int4*>(red)[q];
        const int4 b = reinterpret_cast<const int4*>(red + W)[q];
        wmin[4 * q] = a.x; wmin[4 * q + 1] = a.y; wmin[4 * q + 2] = a.z; wmin[4 * q + 3] = a.w;
        wcnt[4 * q] = b.x; wcnt[4 * q + 1] = b.y; wcnt[4 * q + 2] = b.z; wcnt[4 * q + 3] = b.w;
      }
    } else {
#pragma unroll
      for (int w = 0; w < W; ++w) { wmin[w] = red[w]; wcnt[w] = red[W + w]; }
    }
    int dstar = INT_MAX;
#pragma unroll
    for (int w = 0; w < W; ++w) dstar = min(dstar, wmin[w]);
    int T = 0, pre = 0, wtot = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const int x = (dstar != INT_MAX && wmin[w] == dstar) ? wcnt[w] : 0;
      T += x;
      pre += w < warp ? x : 0;
      wtot += w == warp ? x : 0;
    }
    const uint32_t r0 = rnd[2 * (it & 31)];
    const uint32_t j = T > 0 ? below(r0, (uint32_t)T) : 0u;
    if (T > 0 && (int)j >= pre && (int)j < pre + wtot) {  // the j-th tie is in this warp (warp-uniform)
      const int ct = (dstar != INT_MAX && tmin == dstar) ? tcnt : 0;
      int incl = ct;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
      }
      const int lo = pre + incl - ct;
      const bool hit = ct > 0 && (int)j >= lo && (int)j < lo + ct;  // this thread holds the j-th tie
      int hit_item = -1, hit_rank = 0;
      if (hit) {
        int jj = (int)j - lo;
        for (int i = i0; i < i1; ++i) {
          const uint32_t rr = rowres[i];
          const int rm = (int16_t)(rr >> 16), rcn = (int)(rr & 0xFFFF);
          if (rm != dstar || rcn == 0) continue;
          if (jj >= rcn) { jj -= rcn; continue; }
          hit_item = i;
          hit_rank = jj;
          break;
        }
      }
      // the whole warp searches the winning item's segment: lane l takes words w0 + l, w0 + 32 + l,
      // ...; ballots order the tied colours (word by word, low half first) and find the rank
      const unsigned hb = __ballot_sync(FULL, hit);
      const int hl = hb ? __ffs(hb) - 1 : 0;
      const int item = hb ? __shfl_sync(FULL, hit_item, hl) : -1;
      int jj = __shfl_sync(FULL, hit_rank, hl);
      int mv = -1, mc = -1;
      if (item >= 0) {
        const int r = S == 1 ? item : (int)(((float)item + 0.5f) * rS), sg = item - r * S;
        const int v = cvl[r - rlo];
        const int colv = colS[v];
        const uint16_t* grow = grow_of(v);
        const uint32_t* g32 = (const uint32_t*)grow;
        const uint32_t* t32 = (const uint32_t*)trow_of(v);
        const int g0 = grow[colv];
        const int w0 = sg * Lw, w1 = min(w0 + Lw, kw);
        const unsigned kmin = (unsigned)(dstar + g0);
        const int thr = best_f - f + g0;
        const int killw = colv >> 1;
        const uint32_t killm = 0xFFFFu << (16 * (colv & 1));
        const unsigned lt = (1u << lane) - 1u;
        for (int wb = w0; wb < w1 && mc < 0; wb += 32) {
          const int w = wb + lane;
          bool m0 = false, m1 = false;
          if (w < w1) {
            uint32_t gw = g32[w];
            const uint32_t tw = t32[w];
            if (w == killw) gw |= killm;
            const unsigned ga = gw & 0xFFFFu, gb = gw >> 16;
            const unsigned k0 = ((tw & 0xFFFFu) <= itrel || (int)ga < thr) ? ga : 0xFFFFu;
            const unsigned k1 = ((tw >> 16) <= itrel || (int)gb < thr) ? gb : 0xFFFFu;
            m0 = k0 == kmin;
            m1 = k1 == kmin;
          }
          const unsigned b0 = __ballot_sync(FULL, m0), b1 = __ballot_sync(FULL, m1);
          const int before = __popc(b0 & lt) + __popc(b1 & lt);
          const bool found = jj >= before && jj < before + (int)m0 + (int)m1;
          const unsigned fb = __ballot_sync(FULL, found);
          if (fb) mc = __shfl_sync(FULL, 2 * w + ((jj == before && m0) ? 0 : 1), __ffs(fb) - 1);
          else jj -= __popc(b0) + __popc(b1);
        }
        mv = v;
      }
      if (lane == 0) {
        if (mv >= 0 && mc >= 0 && mc < k) {
          const int old = colS[mv];
          colS[mv] = (uint8_t)mc;
          const int fn = f + dstar;
          // alpha f in 32-bit unsigned arithmetic: the host bounds alpha_num * |E| below 2^32
          const uint32_t tt = below(rnd[2 * (it & 31) + 1], R.L1) + ((uint32_t)R.an * (uint32_t)fn) / (uint32_t)R.ad;
          if (tt > 32766u) sc[5] = 1;
          trow_of(mv)[old] = (uint16_t)(itrel + 1u + tt);
          const uint32_t bit = 1u << (mv & 31);
          if (grow_of(mv)[mc] > 0) atomicOr(cv + (mv >> 5), bit);
          else atomicAnd(cv + (mv >> 5), ~bit);
          sc[0] = mv; sc[1] = old; sc[2] = mc; sc[3] = fn; sc[4] = fn < best_f;
          if (J.trace) reinterpret_cast<int4*>(J.trace)[it] = make_int4(mv, mc, dstar, T);
        } else {
          sc[5] = 2;  // tie counts inconsistent with the scan: refuse to move
        }
      }
    }
    if (T == 0 && tid == 0 && J.trace) reinterpret_cast<int4*>(J.trace)[it] = make_int4(-1, -1, 0, 0);
    __syncthreads();
    if (sc[5]) break;
    // ---- phase 3: gamma update over the neighbours of the moved vertex ------------------------
    const int mv = sc[0];
    if (mv >= 0) {
      const int old = sc[1], nw = sc[2];
      f = sc[3];
      ++moves;
      if (tid == 0) work_deg += degS[mv];
      const uint32_t* brow = J.bits + (size_t)mv * nwords;
      for (int b0 = tid * per; b0 < n; b0 += NT * per) {
        uint32_t m = (__ldg(brow + (b0 >> 5)) >> (b0 & 31)) & slice_mask;
        while (m) {
          const int u = b0 + __ffs(m) - 1;
          m &= m - 1;
          uint16_t* grow = grow_of(u);
          const int go = grow[old] - 1;
          grow[old] = (uint16_t)go;
          const int gn = grow[nw] + 1;
          grow[nw] = (uint16_t)gn;
          const int cu = colS[u];
          if (cu == old && go == 0) atomicAnd(cv + (u >> 5), ~(1u << (u & 31)));
          else if (cu == nw && gn == 1) atomicOr(cv + (u >> 5), 1u << (u & 31));
        }
      }
      if (sc[4]) {
        best_f = f;
        const uint32_t* s32 = (const uint32_t*)colS;
        uint32_t* d32 = (uint32_t*)bestS;
        for (int i = tid; i < (n + 3) / 4; i += NT) d32[i] = s32[i];
      }
    }
    // the Philox block of the next 32 iterations (every reader of the current one has passed
    // the barrier above)
    if (((it + 1) & 31) == 0 && warp == W - 1) draw32(it + 1);
    if (((it + 1) & 0x3FFF) == 0) {
      // the base advances by 2^14: relative expiries drop by 2^14, expired ones become 0
      for (int i = tid; i < n * kw; i += NT) {
        const int v = i / kw;
        uint32_t* t32 = (uint32_t*)trow_of(v) + (i - v * kw);
        const uint32_t w = *t32;
        const uint32_t lo = w & 0xFFFF, hi = w >> 16;
        *t32 = (lo > 0x4000u ? lo - 0x4000u : 0u) | ((hi > 0x4000u ? hi - 0x4000u : 0u) << 16);
      }
    }
    __syncthreads();
  }
  if (sc[5]) {
    if (tid == 0)
      raise_status(R.status, sc[5] == 1 ? DLM_EUNSUPPORTED : (sc[5] == 3 ? DLM_ECANCELLED : DLM_ECUDA));
  }
  __syncthreads();
  for (int v = tid; v < n; v += NT) J.col[v] = (int16_t)bestS[v];
  if (tid == 0) {
    *J.best_f = best_f;
    if (J.moves) *J.moves = moves;
    if (J.work) { J.work[0] = work_rows; J.work[1] = work_deg; }
  }
}

struct TabuBatchArgs {
  int32_t n, k, ks, words, pop;
  const uint32_t* bits;
  const int32_t* off;
  int16_t* col;
  int64_t* best_f;
  int64_t* moves;
  int32_t* trace;
  int64_t* work;
  int64_t iters;
  uint32_t ind_base;
  TabuRule rule;
};

template <int W>
__global__ void __launch_bounds__(W * 32, W >= 16 ? 1 : 2) tabucol_batch_kernel(TabuBatchArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  // one individual per CTA, or (when rows spill to a per-CTA slab) resident CTAs loop over them
  for (int i = blockIdx.x; i < a.pop; i += gridDim.x) {
    TabuJob J;
    J.n = a.n; J.k = a.k; J.ks = a.ks; J.words = a.words; J.bits = a.bits;
    J.col = a.col + (size_t)i * a.n;
    J.best_f = a.best_f + i;
    J.moves = a.moves ? a.moves + i : nullptr;
    J.trace = a.trace ? a.trace + (size_t)i * a.iters * 4 : nullptr;
    J.work = a.work ? a.work + 2 * (size_t)i : nullptr;
    J.off = a.off;
    J.iters = a.iters;
    J.ind = a.ind_base + (uint32_t)i;
    if (a.rule.slab) tabucol_individual<W, true>(J, a.rule, smem);
    else tabucol_individual<W, false>(J, a.rule, smem);
    __syncthreads();
  }
}

// ---- uneven batch: persistent CTAs pull individuals from a device queue ----------------------
struct MultiJob {
  int32_t n, k, ks, words;
  const uint32_t* bits;
  int16_t* col;
  int64_t* best_f;
  int64_t* moves;
  int64_t iters;
  uint32_t ind;
};

template <int W>
__global__ void __launch_bounds__(W * 32, W >= 16 ? 1 : 2) tabucol_multi_kernel(const MultiJob* jobs, int32_t njobs,
                                                               int32_t* queue, TabuRule rule) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int32_t next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(queue, 1);
    __syncthreads();
    const int j = next;
    __syncthreads();
    if (j >= njobs) break;
    const MultiJob& M = jobs[j];
    TabuJob J;
    J.n = M.n; J.k = M.k; J.ks = M.ks; J.words = M.words; J.bits = M.bits; J.col = M.col;
    J.best_f = M.best_f; J.moves = M.moves; J.trace = nullptr; J.work = nullptr; J.off = nullptr;
    J.iters = M.iters; J.ind = M.ind;
    if (rule.slab) tabucol_individual<W, true>(J, rule, smem);
    else tabucol_individual<W, false>(J, rule, smem);
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
template <int W>
static dlm_status launch_batch(dlm_ctx* ctx, TabuBatchArgs a, size_t smem, size_t slab_stride) {
  auto kfn = tabucol_batch_kernel<W>;
  DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int grid = a.pop;
  if (slab_stride > 0) {  // rows spill: resident CTAs only, each with its own slab
    int per_sm = 0;
    DLM_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, W * 32, smem));
    grid = std::min(a.pop, std::max(1, per_sm) * ctx->num_sms);
    uint16_t* slab = nullptr;
    DLM_TRY(ctx_workspace(ctx, (size_t)grid * slab_stride * 2, (void**)&slab));
    a.rule.slab = slab;
    a.rule.slab_stride = slab_stride;
  }
  kfn<<<grid, W * 32, smem, ctx->stream>>>(a);
  return launch_check(ctx, "tabucol_batch_kernel");
}

static int lookup_tune(const dlm_ctx* ctx, int n, int k) {
  for (int i = 0; i < ctx->n_tune; ++i)
    if (ctx->tune[i].n == n && ctx->tune[i].k == k) return ctx->tune[i].warps;
  return 0;
}

// default when not tuned: enough threads to cover a row scan and a neighbour update in few steps
static int default_warps(int n, int k) {
  (void)k;
  if (n <= 128) return 2;
  if (n <= 300) return 4;
  return 8;
}

static dlm_status tabucol_check(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int64_t iters,
                                dlm_tenure t) {
  if (!ctx || !g) return fail(ctx, DLM_EINVAL, "null context or graph");
  if (k < 2 || k > 128) return fail(ctx, DLM_EUNSUPPORTED, "tabucol: k must be in 2..128");
  if (pop < 0 || iters < 0) return fail(ctx, DLM_EINVAL, "tabucol: negative population or budget");
  if (iters > INT32_MAX) return fail(ctx, DLM_EINVAL, "tabucol: budget above 2^31");
  if (t.L_max < 0 || t.alpha_num < 0 || t.alpha_den <= 0) return fail(ctx, DLM_EINVAL, "tabucol: bad tenure");
  // the kernel forms alpha_num * f in 32-bit unsigned arithmetic (f <= |E|)
  if ((uint64_t)t.alpha_num * (uint64_t)g->m >= (1ull << 32))
    return fail(ctx, DLM_EUNSUPPORTED, "tabucol: alpha_num * |E| must be below 2^32");
  return DLM_OK;
}

static dlm_status tabucol_run(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                              int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                              uint32_t generation, uint32_t ind_base, int warps, int32_t* trace,
                              int64_t* work) {
  DLM_TRY(tabucol_check(ctx, g, k, pop, iters, tenure));
  if (pop == 0) return DLM_OK;
  if (!col || !best_f) return fail(ctx, DLM_EINVAL, "tabucol: null col or best_f");
  if (warps == 0) warps = lookup_tune(ctx, g->n, k);
  if (warps == 0) warps = default_warps(g->n, k);
  if (warps != 1 && warps != 2 && warps != 4 && warps != 8 && warps != 16)
    return fail(ctx, DLM_EINVAL, "tabucol: warps per individual must be 1, 2, 4, 8 or 16");
  const TabuSmem L = tabu_smem_layout(g->n, k, warps, ctx->smem_optin);
  if (L.rs < 1 || L.total > ctx->smem_optin)
    return fail(ctx, DLM_EUNSUPPORTED, "tabucol: the per-individual arrays exceed shared memory per block");
  const size_t slab_stride = L.rs < g->n ? tabu_slab_elems(g->n, k, L.rs) : 0;
  TabuBatchArgs a;
  a.n = g->n; a.k = k; a.ks = tabu_row_stride(k); a.words = g->words; a.pop = pop;
  a.bits = g->d_bits; a.off = g->d_off; a.col = col; a.best_f = best_f; a.moves = moves; a.trace = trace;
  a.work = work; a.iters = iters;
  a.ind_base = ind_base;
  a.rule = TabuRule{(uint32_t)tenure.L_max + 1u, tenure.alpha_num, tenure.alpha_den, seed, generation, ctx->d_status,
                    ctx->smem_optin, nullptr, 0, ctx->cancel};
  switch (warps) {
    case 1: return launch_batch<1>(ctx, a, L.total, slab_stride);
    case 2: return launch_batch<2>(ctx, a, L.total, slab_stride);
    case 4: return launch_batch<4>(ctx, a, L.total, slab_stride);
    case 8: return launch_batch<8>(ctx, a, L.total, slab_stride);
    default: return launch_batch<16>(ctx, a, L.total, slab_stride);
  }
}

}  // namespace dlm

using namespace dlm;

extern "C" dlm_status dlm_tabucol_batch(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                        int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure,
                                        uint64_t seed, uint32_t generation, uint32_t ind_base) {
  return tabucol_run(ctx, g, k, pop, col, best_f, moves, iters, tenure, seed, generation, ind_base, 0, nullptr,
                     nullptr);
}

extern "C" dlm_status dlm_tabucol_batch_ex(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                           int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure,
                                           uint64_t seed, uint32_t generation, uint32_t ind_base,
                                           int32_t warps_per_individual, int32_t* trace, int64_t* work) {
  return tabucol_run(ctx, g, k, pop, col, best_f, moves, iters, tenure, seed, generation, ind_base,
                     warps_per_individual, trace, work);
}

extern "C" dlm_status dlm_tabucol_autotune(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int64_t iters,
                                           int32_t* best) {
  if (!ctx || !g || pop <= 0 || iters <= 0) return fail(ctx, DLM_EINVAL, "autotune: bad arguments");
  // the trial colourings get their own allocation: the launches below take the context workspace
  // for their spilled rows, so colourings kept there would be overwritten (or freed on growth)
  const size_t col_bytes = align16((size_t)pop * g->n * sizeof(int16_t));
  uint8_t* buf = nullptr;
  if (cudaMalloc(&buf, col_bytes + (size_t)pop * sizeof(int64_t)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DLM_ENOMEM, "autotune: trial buffer allocation failed");
  }
  int16_t* col = (int16_t*)buf;
  int64_t* bf = (int64_t*)(buf + col_bytes);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  int best_w = default_warps(g->n, k);
  const int cand[5] = {1, 2, 4, 8, 16};
  dlm_status st = DLM_OK;
  for (int c = 0; c < 5 && st == DLM_OK; ++c) {
    const TabuSmem L = tabu_smem_layout(g->n, k, cand[c], ctx->smem_optin);
    if (L.total > ctx->smem_optin) continue;
    float ms_sum = 0.f;
    for (int rep = 0; rep < 2 && st == DLM_OK; ++rep) {
      st = dlm_init_colors(ctx, g->n, k, pop, 0x7u, 0u, col);
      if (st != DLM_OK) break;
      cudaEventRecord(e0, ctx->stream);
      st = tabucol_run(ctx, g, k, pop, col, bf, nullptr, iters, dlm_tenure{9, 6, 10}, 1u, 0u, 0u, cand[c], nullptr,
                       nullptr);
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep == 1) ms_sum += ms;  // first repetition warms up
    }
    if (st == DLM_OK && ms_sum < best_ms) { best_ms = ms_sum; best_w = cand[c]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(buf);
  if (st != DLM_OK) return st;
  int slot = -1;
  for (int i = 0; i < ctx->n_tune; ++i)
    if (ctx->tune[i].n == g->n && ctx->tune[i].k == k) slot = i;
  if (slot < 0 && ctx->n_tune < 64) slot = ctx->n_tune++;
  if (slot >= 0) ctx->tune[slot] = dlm_ctx::TuneEntry{g->n, k, best_w};
  if (best) *best = best_w;
  return DLM_OK;
}

extern "C" dlm_status dlm_tabucol_multi(dlm_ctx* ctx, int32_t n_graphs, const dlm_graph* const* graphs,
                                        const int32_t* k, const int32_t* pop, int16_t* const* col,
                                        int64_t* const* best_f, int64_t* const* moves, const int64_t* iters,
                                        dlm_tenure tenure, uint64_t seed, uint32_t generation, uint32_t ind_base) {
  if (!ctx || n_graphs <= 0 || !graphs || !k || !pop || !col || !best_f || !iters)
    return fail(ctx, DLM_EINVAL, "tabucol_multi: bad arguments");
  // one launch: the block size is the largest tuned/default warp count, shared memory the largest
  // per-individual state; individuals sorted by decreasing work (n * k * iters) go to a queue
  int warps = 1;
  size_t smem = 0;
  size_t njobs = 0;
  for (int gi = 0; gi < n_graphs; ++gi) {
    DLM_TRY(tabucol_check(ctx, graphs[gi], k[gi], pop[gi], iters[gi], tenure));
    if (pop[gi] > 0 && (!col[gi] || !best_f[gi])) return fail(ctx, DLM_EINVAL, "tabucol_multi: null output");
    int w = lookup_tune(ctx, graphs[gi]->n, k[gi]);
    if (w == 0) w = default_warps(graphs[gi]->n, k[gi]);
    warps = w > warps ? w : warps;
    njobs += (size_t)pop[gi];
  }
  size_t slab_stride = 0;  // graphs whose state exceeds shared memory keep their last rows in a slab
  for (int gi = 0; gi < n_graphs; ++gi) {
    const TabuSmem L = tabu_smem_layout(graphs[gi]->n, k[gi], warps, ctx->smem_optin);
    if (L.rs < 1 || L.total > ctx->smem_optin)
      return fail(ctx, DLM_EUNSUPPORTED, "tabucol_multi: a graph's arrays exceed shared memory");
    smem = L.total > smem ? L.total : smem;
    if (L.rs < graphs[gi]->n) slab_stride = std::max(slab_stride, tabu_slab_elems(graphs[gi]->n, k[gi], L.rs));
  }
  if (njobs == 0) return DLM_OK;
  std::vector<MultiJob> jobs;
  jobs.reserve(njobs);
  uint32_t id = ind_base;
  for (int gi = 0; gi < n_graphs; ++gi) {
    const dlm_graph* g = graphs[gi];
    for (int j = 0; j < pop[gi]; ++j) {
      MultiJob M;
      M.n = g->n; M.k = k[gi]; M.ks = tabu_row_stride(k[gi]); M.words = g->words; M.bits = g->d_bits;
      M.col = col[gi] + (size_t)j * g->n; M.best_f = best_f[gi] + j; M.moves = moves && moves[gi] ? moves[gi] + j : nullptr;
      M.iters = iters[gi]; M.ind = id++;
      jobs.push_back(M);
    }
  }
  std::stable_sort(jobs.begin(), jobs.end(), [](const MultiJob& a, const MultiJob& b) {
    return (double)a.n * a.k * a.iters > (double)b.n * b.k * b.iters;
  });
  const size_t job_bytes = align16(jobs.size() * sizeof(MultiJob));
  TabuRule rule{(uint32_t)tenure.L_max + 1u, tenure.alpha_num, tenure.alpha_den, seed, generation, ctx->d_status,
                ctx->smem_optin, nullptr, slab_stride, ctx->cancel};
  int per_sm = 0;
  dlm_status st = DLM_OK;
  auto go = [&](auto kfn) -> dlm_status {
    DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    DLM_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, warps * 32, smem));
    if (per_sm < 1) per_sm = 1;
    const int grid = (int)std::min<size_t>((size_t)per_sm * ctx->num_sms, jobs.size());
    uint8_t* ws = nullptr;
    DLM_TRY(ctx_workspace(ctx, job_bytes + 16 + (size_t)grid * slab_stride * 2, (void**)&ws));
    MultiJob* d_jobs = (MultiJob*)ws;
    int32_t* d_queue = (int32_t*)(ws + job_bytes);
    if (slab_stride) rule.slab = (uint16_t*)(ws + job_bytes + 16);
    DLM_CUDA(ctx, cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(MultiJob), cudaMemcpyHostToDevice,
                                  ctx->stream));
    DLM_CUDA(ctx, cudaMemsetAsync(d_queue, 0, sizeof(int32_t), ctx->stream));
    kfn<<<grid, warps * 32, smem, ctx->stream>>>(d_jobs, (int32_t)jobs.size(), d_queue, rule);
    return launch_check(ctx, "tabucol_multi_kernel");
  };
  switch (warps) {
    case 1: st = go(tabucol_multi_kernel<1>); break;
    case 2: st = go(tabucol_multi_kernel<2>); break;
    case 4: st = go(tabucol_multi_kernel<4>); break;
    case 8: st = go(tabucol_multi_kernel<8>); break;
    default: st = go(tabucol_multi_kernel<16>); break;
  }
  return st;
}

// ------------------------------------------------------------------------------------------------
// Allocation-free variant of the uneven-batch launch. Its scratch (the job list and the queue
// counter of the persistent kernel) lives in a file-scope device array instead of the context's
// workspace, so the call never allocates device memory.
// ------------------------------------------------------------------------------------------------
namespace dlm {

constexpr int kNoAllocMaxJobs = 16384;
constexpr size_t kNoAllocJobBytes = (size_t)kNoAllocMaxJobs * sizeof(MultiJob);
constexpr size_t kNoAllocScratchBytes = kNoAllocJobBytes + 256;  // job list, then the queue counter

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once with that device current (in
// host code the symbol itself is only a host-side stand-in, not a device address).
static void* g_noalloc_addr[128];
static std::mutex g_noalloc_mu;

static dlm_status noalloc_scratch(dlm_ctx* ctx, uint8_t** out) {
  if (ctx->device < 0 || ctx->device >= 128) return fail(ctx, DLM_EUNSUPPORTED, "tabucol_multi_noalloc: device index");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[ctx->device]) {
    int cur = -1;
    DLM_CUDA(ctx, cudaGetDevice(&cur));
    if (cur != ctx->device) DLM_CUDA(ctx, cudaSetDevice(ctx->device));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != ctx->device) cudaSetDevice(cur);
    if (e != cudaSuccess || !p) return cuda_check(ctx, e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
    g_noalloc_addr[ctx->device] = p;
  }
  *out = (uint8_t*)g_noalloc_addr[ctx->device];
  return DLM_OK;
}

}  // namespace dlm

extern "C" dlm_status dlm_tabucol_multi_noalloc(dlm_ctx* ctx, int32_t n_graphs, const dlm_graph* const* graphs,
                                                const int32_t* k, const int32_t* pop, int16_t* const* col,
                                                int64_t* const* best_f, int64_t* const* moves, const int64_t* iters,
                                                dlm_tenure tenure, uint64_t seed, uint32_t generation,
                                                uint32_t ind_base) {
  if (!ctx || n_graphs <= 0 || !graphs || !k || !pop || !col || !best_f || !iters)
    return fail(ctx, DLM_EINVAL, "tabucol_multi_noalloc: bad arguments");
  int warps = 1;
  size_t smem = 0;
  size_t njobs = 0;
  for (int gi = 0; gi < n_graphs; ++gi) {
    DLM_TRY(tabucol_check(ctx, graphs[gi], k[gi], pop[gi], iters[gi], tenure));
    if (pop[gi] > 0 && (!col[gi] || !best_f[gi])) return fail(ctx, DLM_EINVAL, "tabucol_multi_noalloc: null output");
    int w = lookup_tune(ctx, graphs[gi]->n, k[gi]);
    if (w == 0) w = default_warps(graphs[gi]->n, k[gi]);
    warps = w > warps ? w : warps;
    njobs += (size_t)pop[gi];
  }
  if (njobs > (size_t)kNoAllocMaxJobs)
    return fail(ctx, DLM_EUNSUPPORTED, "tabucol_multi_noalloc: at most " + std::to_string(kNoAllocMaxJobs) +
                                           " individuals per call (the static scratch array holds that many jobs)");
  for (int gi = 0; gi < n_graphs; ++gi) {
    const TabuSmem L = tabu_smem_layout(graphs[gi]->n, k[gi], warps, ctx->smem_optin);
    smem = L.total > smem ? L.total : smem;
    if (L.rs < graphs[gi]->n)  // a slab for the spilled rows would have to be allocated
      return fail(ctx, DLM_EUNSUPPORTED, "tabucol_multi_noalloc: a graph's state exceeds shared memory");
  }
  if (njobs == 0) return DLM_OK;
  std::vector<MultiJob> jobs;
  jobs.reserve(njobs);
  uint32_t id = ind_base;
  for (int gi = 0; gi < n_graphs; ++gi) {
    const dlm_graph* g = graphs[gi];
    for (int j = 0; j < pop[gi]; ++j) {
      MultiJob M;
      M.n = g->n; M.k = k[gi]; M.ks = tabu_row_stride(k[gi]); M.words = g->words; M.bits = g->d_bits;
      M.col = col[gi] + (size_t)j * g->n; M.best_f = best_f[gi] + j; M.moves = moves && moves[gi] ? moves[gi] + j : nullptr;
      M.iters = iters[gi]; M.ind = id++;
      jobs.push_back(M);
    }
  }
  std::stable_sort(jobs.begin(), jobs.end(), [](const MultiJob& a, const MultiJob& b) {
    return (double)a.n * a.k * a.iters > (double)b.n * b.k * b.iters;
  });
  uint8_t* scratch = nullptr;
  DLM_TRY(noalloc_scratch(ctx, &scratch));
  MultiJob* d_jobs = (MultiJob*)scratch;
  int32_t* d_queue = (int32_t*)(scratch + kNoAllocJobBytes);
  DLM_CUDA(ctx, cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(MultiJob), cudaMemcpyHostToDevice, ctx->stream));
  DLM_CUDA(ctx, cudaMemsetAsync(d_queue, 0, sizeof(int32_t), ctx->stream));  // the queue starts at zero
  const TabuRule rule{(uint32_t)tenure.L_max + 1u, tenure.alpha_num, tenure.alpha_den, seed, generation, ctx->d_status,
                      ctx->smem_optin, nullptr, 0, ctx->cancel};
  auto go = [&](auto kfn) -> dlm_status {
    int per_sm = 0;
    DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    DLM_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, warps * 32, smem));
    if (per_sm < 1) per_sm = 1;
    const int grid = (int)std::min<size_t>((size_t)per_sm * ctx->num_sms, jobs.size());
    kfn<<<grid, warps * 32, smem, ctx->stream>>>(d_jobs, (int32_t)jobs.size(), d_queue, rule);
    return launch_check(ctx, "tabucol_multi_kernel");
  };
  switch (warps) {
    case 1: return go(tabucol_multi_kernel<1>);
    case 2: return go(tabucol_multi_kernel<2>);
    case 4: return go(tabucol_multi_kernel<4>);
    case 8: return go(tabucol_multi_kernel<8>);
    default: return go(tabucol_multi_kernel<16>);
  }
}

// ------------------------------------------------------------------------------------------------
// Uneven batch as a reusable plan: the job list, the queue and the slab are uploaded once into
// plan-owned memory, and the launch (queue reset + persistent kernel) is captured once into a CUDA
// graph; every dlm_tabucol_multi_plan_launch replays that graph on the context's stream.
// ------------------------------------------------------------------------------------------------
struct dlm_multi_plan {
  uint8_t* mem = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int warps = 0, grid = 0;
  size_t njobs = 0;
};

extern "C" void dlm_tabucol_multi_plan_destroy(dlm_multi_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  cudaFree(p->mem);
  delete p;
}

extern "C" dlm_status dlm_tabucol_multi_plan_create(dlm_ctx* ctx, int32_t n_graphs, const dlm_graph* const* graphs,
                                                    const int32_t* k, const int32_t* pop, int16_t* const* col,
                                                    int64_t* const* best_f, int64_t* const* moves,
                                                    const int64_t* iters, dlm_tenure tenure, uint64_t seed,
                                                    uint32_t generation, uint32_t ind_base, dlm_multi_plan** out) {
  if (!ctx || !out || n_graphs <= 0 || !graphs || !k || !pop || !col || !best_f || !iters)
    return fail(ctx, DLM_EINVAL, "tabucol_multi_plan: bad arguments");
  *out = nullptr;
  int warps = 1;
  size_t smem = 0, slab_stride = 0, njobs = 0;
  for (int gi = 0; gi < n_graphs; ++gi) {
    DLM_TRY(tabucol_check(ctx, graphs[gi], k[gi], pop[gi], iters[gi], tenure));
    if (pop[gi] > 0 && (!col[gi] || !best_f[gi])) return fail(ctx, DLM_EINVAL, "tabucol_multi_plan: null output");
    int w = lookup_tune(ctx, graphs[gi]->n, k[gi]);
    if (w == 0) w = default_warps(graphs[gi]->n, k[gi]);
    warps = std::max(warps, w);
    njobs += (size_t)pop[gi];
  }
  for (int gi = 0; gi < n_graphs; ++gi) {
    const TabuSmem L = tabu_smem_layout(graphs[gi]->n, k[gi], warps, ctx->smem_optin);
    if (L.rs < 1 || L.total > ctx->smem_optin)
      return fail(ctx, DLM_EUNSUPPORTED, "tabucol_multi_plan: a graph's arrays exceed shared memory");
    smem = std::max(smem, L.total);
    if (L.rs < graphs[gi]->n) slab_stride = std::max(slab_stride, tabu_slab_elems(graphs[gi]->n, k[gi], L.rs));
  }
  if (njobs == 0) return fail(ctx, DLM_EINVAL, "tabucol_multi_plan: empty batch");
  std::vector<MultiJob> jobs;
  jobs.reserve(njobs);
  uint32_t id = ind_base;
  for (int gi = 0; gi < n_graphs; ++gi) {
    const dlm_graph* g = graphs[gi];
    for (int j = 0; j < pop[gi]; ++j) {
      MultiJob M;
      M.n = g->n; M.k = k[gi]; M.ks = tabu_row_stride(k[gi]); M.words = g->words; M.bits = g->d_bits;
      M.col = col[gi] + (size_t)j * g->n; M.best_f = best_f[gi] + j; M.moves = moves && moves[gi] ? moves[gi] + j : nullptr;
      M.iters = iters[gi]; M.ind = id++;
      jobs.push_back(M);
    }
  }
  std::stable_sort(jobs.begin(), jobs.end(), [](const MultiJob& a, const MultiJob& b) {
    return (double)a.n * a.k * a.iters > (double)b.n * b.k * b.iters;
  });
  dlm_multi_plan* p = new dlm_multi_plan();
  p->warps = warps;
  p->njobs = jobs.size();
  auto cleanup = [&](dlm_status s, const std::string& m) { dlm_tabucol_multi_plan_destroy(p); return fail(ctx, s, m); };
  void* kfn = nullptr;
  switch (warps) {
    case 1: kfn = (void*)tabucol_multi_kernel<1>; break;
    case 2: kfn = (void*)tabucol_multi_kernel<2>; break;
    case 4: kfn = (void*)tabucol_multi_kernel<4>; break;
    case 8: kfn = (void*)tabucol_multi_kernel<8>; break;
    default: kfn = (void*)tabucol_multi_kernel<16>; break;
  }
  int per_sm = 0;
  if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, warps * 32, smem) != cudaSuccess)
    return cleanup(DLM_ECUDA, "tabucol_multi_plan: kernel attributes");
  p->grid = (int)std::min<size_t>((size_t)std::max(1, per_sm) * ctx->num_sms, jobs.size());
  const size_t job_bytes = align16(jobs.size() * sizeof(MultiJob));
  if (cudaMalloc(&p->mem, job_bytes + 16 + (size_t)p->grid * slab_stride * 2) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(DLM_ENOMEM, "tabucol_multi_plan: allocation failed");
  }
  MultiJob* d_jobs = (MultiJob*)p->mem;
  int32_t* d_queue = (int32_t*)(p->mem + job_bytes);
  if (cudaMemcpy(d_jobs, jobs.data(), jobs.size() * sizeof(MultiJob), cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(DLM_ECUDA, "tabucol_multi_plan: upload");
  TabuRule rule{(uint32_t)tenure.L_max + 1u, tenure.alpha_num, tenure.alpha_den, seed, generation, ctx->d_status,
                ctx->smem_optin, slab_stride ? (uint16_t*)(p->mem + job_bytes + 16) : nullptr, slab_stride,
                ctx->cancel};
  int32_t njobs32 = (int32_t)jobs.size();
  void* params[] = {&d_jobs, &njobs32, &d_queue, &rule};
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return cleanup(DLM_ECUDA, "stream");
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_queue, 0, sizeof(int32_t), cs);
  if (e == cudaSuccess) e = cudaLaunchKernel(kfn, dim3(p->grid), dim3(warps * 32), params, smem, cs);
  const cudaError_t e2 = cudaStreamEndCapture(cs, &p->graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess || e2 != cudaSuccess) { cudaGetLastError(); return cleanup(DLM_ECUDA, "tabucol_multi_plan: capture"); }
  if (cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(DLM_ECUDA, "tabucol_multi_plan: instantiate");
  }
  *out = p;
  return DLM_OK;
}

extern "C" dlm_status dlm_tabucol_multi_plan_launch(dlm_ctx* ctx, dlm_multi_plan* p) {
  if (!ctx || !p) return fail(ctx, DLM_EINVAL, "tabucol_multi_plan_launch: null argument");
  DLM_CUDA(ctx, cudaGraphLaunch(p->exec, ctx->stream));
  return DLM_OK;
}
