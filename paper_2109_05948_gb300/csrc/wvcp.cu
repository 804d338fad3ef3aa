// Weighted vertex colouring (WVCP): randomised greedy initialisation (section "Initialization with
// a greedy random algorithm") and the feasible/infeasible tabu search on the penalised objective
// g = f + phi * c (section "Parallel iterated feasible and infeasible Tabu Search", Eq.
// AFISA_score, Eq. score_WVCP), run on every individual of a population.
//
// GB300 design of the tabu search (one CTA per individual, persistent over the population):
//  * every one-move (v, c) of every vertex is a candidate each iteration (n * k pairs, ~145 000
//    at n = 1000): delta = rem(v) + max(0, w_v - max1[c]) + phi (gamma[v][c] - gamma[v][col v]),
//    rem(v) the drop of v's class maximum when v leaves it. Each row v keeps a summary of its
//    colour keys max(0, w_v - max1[c]) + phi gamma[v][c] over c != col v (their minimum and how
//    many reach it); the selection reads one summary per row. A move from colour a to b changes
//    only the keys of colours a and b (gamma of the neighbours, the two class maxima), which
//    update the summaries in O(1) per row; a row whose only minimum key rose, and the moved
//    vertex's row, are scanned again;
//  * gamma is stored transposed, gT[c][v], so that the lanes of a warp, each on its own rows,
//    read neighbouring addresses of one colour. With u8 entries the whole table stays in shared
//    memory (n * k bytes: 144 KB at n = 1000, k = 144); gamma[v][c] never exceeds the size of class
//    c, so u8 is exact while every class holds at most 255 vertices: the u8 search of an individual
//    gives up (at set-up, or before the move that would grow a class past 255) and a u16 pass
//    searches the individuals it gave up from their start colourings, with the same draws, hence
//    the same result. With u16 entries the first Cs colours live in shared memory and the rest in
//    an L2-resident slab of global memory owned by the CTA;
//  * class maxima are kept exactly by per-class counts per weight level plus a level bitmask, so
//    max1, its multiplicity and the second largest weight come from two bit scans after a move;
//  * ties: the j-th admissible minimum in (v ascending, c ascending) order. Thread t owns the rows
//    of slice t, so warps hold consecutive row ranges; each warp publishes its minimum and how many
//    moves reach it, every warp finds the global minimum and the warp holding tie j from those 16
//    pairs, and that warp alone ranks its lanes, finds the row and then the colour (a ballot over
//    32 colours at a time);
//  * an iteration has two block barriers: after the move, and after the neighbour updates, which
//    end with the next iteration's per-row selection (the owner of a row updates and selects it);
//    rows whose summary must be scanned again are scanned by the owner's whole warp, and the moved
//    vertex's adjacency row is loaded during the colour search.
#include <algorithm>
#include <climits>
#include <vector>

#include "common.cuh"

namespace dlm {

constexpr int kWThreads = 512;
constexpr int kWWarps = kWThreads / 32;
constexpr uint32_t kWClass8 = 255;  // largest class the u8 conflict table holds exactly

struct WvcpLayout {
  size_t col, best, w, fz, lvl, lmask, info, max1, csz, mvrow, rmin, rcnt, skey, scnt, red, gT, total;
  int npad, lw, cs;  // vertices padded to 8, mask words per class, colours held in shared memory
};

__host__ __device__ inline size_t wal16(size_t x) { return (x + 15) & ~(size_t)15; }

// as many colours in shared memory as `budget` allows (the rest go to the CTA's global slab);
// eb = bytes per conflict-table entry (1 or 2)
__host__ __device__ inline WvcpLayout wvcp_layout(int n, int k, int wmax, size_t budget, int eb) {
  WvcpLayout L;
  L.npad = (n + 7) & ~7;
  L.lw = (wmax + 32) / 32;  // levels 0..wmax
  size_t o = 0;
  L.col = o; o += wal16(n);
  L.best = o; o += wal16(n);
  L.w = o; o += wal16(n);
  L.fz = o; o += wal16((size_t)n * 2);
  L.lvl = o; o += wal16((size_t)k * (wmax + 1) * 2);
  L.lmask = o; o += wal16((size_t)k * L.lw * 4);
  L.info = o; o += wal16((size_t)k * 4);
  L.max1 = o; o += wal16((size_t)k);
  L.csz = o; o += wal16((size_t)k * 4);
  L.mvrow = o; o += wal16((size_t)((n + 31) / 32) * 4);
  L.rmin = o; o += wal16((size_t)n * 4);
  L.rcnt = o; o += wal16((size_t)n * 2);
  L.skey = o; o += wal16((size_t)n * 4);
  L.scnt = o; o += wal16((size_t)n * 2);
  L.red = o; o += 1024;  // 2 kWWarps + 8 ints, then 8 + 2 kWWarps long longs; 2 ints at byte 896
  L.gT = o;
  const size_t per_col = (size_t)L.npad * eb;
  size_t cs = budget > o ? (budget - o) / per_col : 0;
  if (cs > (size_t)k) cs = k;
  L.cs = (int)cs;
  o += cs * per_col;
  L.total = o;
  return L;
}

struct WvcpArgs {
  int32_t n, k, words, pop, wmax;
  const uint32_t* bits;
  const int32_t* weight;
  int16_t* col;
  int64_t* best_g;
  int64_t* best_fc;
  int64_t* moves;
  int32_t* trace;
  void* slab;      // per CTA: (k - cs) * npad entries
  int32_t* redo;   // [pop]: individuals the u8 search gave up
  int32_t redo_mode;  // 0: every individual; 1: u8 search, flags what it gives up; 2: flagged only
  int64_t iters;
  int64_t phi;             // penalty (g = fscale f + phi c), or per individual from phi_arr
  const int64_t* phi_arr;  // [pop] or null
  int32_t fscale;
  uint32_t L1, ttbase;
  uint64_t seed;
  uint32_t gen, ind_base;
  int32_t* status;
  size_t smem_budget;
};

// class c: max1 (largest weight present, 0 if empty), cnt1 (its multiplicity), max2 (next level)
__device__ __forceinline__ uint32_t class_info(const uint16_t* lvl, const uint32_t* lmask, int lw, int wmax, int c) {
  const uint32_t* m = lmask + (size_t)c * lw;
  int m1 = 0, m2 = 0;
  int w = lw - 1;
  for (; w >= 0; --w)
    if (m[w]) { m1 = 32 * w + 31 - __clz(m[w]); break; }
  if (m1 > 0) {
    uint32_t rest = m[w] & ~(1u << (m1 & 31));
    if (rest) m2 = 32 * w + 31 - __clz(rest);
    else
      for (int q = w - 1; q >= 0; --q)
        if (m[q]) { m2 = 32 * q + 31 - __clz(m[q]); break; }
  }
  const uint32_t c1 = m1 > 0 ? lvl[(size_t)c * (wmax + 1) + m1] : 0u;
  return (uint32_t)m1 | ((uint32_t)m2 << 8) | (c1 << 16);
}

__device__ __forceinline__ void class_add(uint16_t* lvl, uint32_t* lmask, int lw, int wmax, int c, int w, int d) {
  uint16_t* p = lvl + (size_t)c * (wmax + 1) + w;
  const int nv = (int)*p + d;
  *p = (uint16_t)nv;
  uint32_t* m = lmask + (size_t)c * lw + (w >> 5);
  if (nv > 0) *m |= 1u << (w & 31);
  else *m &= ~(1u << (w & 31));
}

// key of colour c for row v: the weight term of joining class c plus phi times gamma[v][c]
__device__ __forceinline__ int wvcp_key(int fs, int wv, int m1c, int phi, int gc) {
  return fs * (wv > m1c ? wv - m1c : 0) + phi * gc;
}

// a key of a row changed from kold to knew: update the row's (minimum, count); false when the
// key was the row's only minimum and rose (the row must be scanned again)
__device__ __forceinline__ bool wvcp_summ_apply(int& km, int& kc, int kold, int knew) {
  if (knew == kold) return true;
  if (knew < kold) {
    if (knew < km) { km = knew; kc = 1; }
    else if (knew == km) ++kc;
    return true;
  }
  if (kold == km) {
    if (kc > 1) { --kc; return true; }
    return false;
  }
  return true;
}

// minimum key of row v over the colours c != o and how many colours reach it (in colour order:
// the shared-memory colours, then the slab colours sixteen loads at a time)
template <typename G>
__device__ __forceinline__ void wvcp_row_summary(int v, int o, int wv, const uint8_t* max1s, const G* gS,
                                                 const G* gG, int npad, int cs, int k, int fs, int phi,
                                                 int& km, int& kc) {
  km = INT_MAX;
  kc = 0;
  auto take = [&](int c, int gc) {
    if (c == o) return;
    const int key = wvcp_key(fs, wv, max1s[c], phi, gc);
    if (key < km) { km = key; kc = 1; }
    else if (key == km) ++kc;
  };
  for (int c = 0; c < cs; ++c) take(c, gS[(size_t)c * npad + v]);
  int c = cs;
  for (; c + 16 <= k; c += 16) {
    int q16[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) q16[q] = gG[(size_t)(c + q - cs) * npad + v];
#pragma unroll
    for (int q = 0; q < 16; ++q) take(c + q, q16[q]);
  }
  for (; c < k; ++c) take(c, gG[(size_t)(c - cs) * npad + v]);
}

// the same summary computed by a warp: lane l takes the colours l, l + 32, ...; the minimum and
// its count do not depend on the order the colours are taken in
template <typename G>
__device__ __forceinline__ void wvcp_row_summary_warp(int v, int o, int wv, const uint8_t* max1s, const G* gS,
                                                      const G* gG, int npad, int cs, int k, int fs, int phi, int lane,
                                                      int& km, int& kc) {
  int lm = INT_MAX, lc = 0;
  for (int c = lane; c < k; c += 32) {
    if (c == o) continue;
    const int gc = c < cs ? gS[(size_t)c * npad + v] : gG[(size_t)(c - cs) * npad + v];
    const int key = wvcp_key(fs, wv, max1s[c], phi, gc);
    if (key < lm) { lm = key; lc = 1; }
    else if (key == lm) ++lc;
  }
  km = __reduce_min_sync(0xFFFFFFFFu, lm);
  kc = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)(lm == km ? lc : 0));
}

template <typename G>
__global__ void __launch_bounds__(kWThreads, 1) k_wvcp_tabu(WvcpArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int n = a.n, k = a.k, wmax = a.wmax, nwords = a.words;
  const WvcpLayout L = wvcp_layout(n, k, wmax, a.smem_budget, (int)sizeof(G));
  const int npad = L.npad, lw = L.lw, cs = L.cs;
  uint8_t* colS = smem + L.col;
  uint8_t* bestS = smem + L.best;
  uint8_t* wS = smem + L.w;
  uint16_t* fz = (uint16_t*)(smem + L.fz);
  uint16_t* lvl = (uint16_t*)(smem + L.lvl);
  uint32_t* lmask = (uint32_t*)(smem + L.lmask);
  uint32_t* info = (uint32_t*)(smem + L.info);
  uint8_t* max1s = smem + L.max1;
  uint32_t* csz = (uint32_t*)(smem + L.csz);  // class sizes
  int32_t* rmin = (int32_t*)(smem + L.rmin);
  uint16_t* rcnt = (uint16_t*)(smem + L.rcnt);
  int32_t* skey = (int32_t*)(smem + L.skey);   // per row: minimum key over the colours c != col v
  uint16_t* scnt = (uint16_t*)(smem + L.scnt); // per row: colours reaching it
  int32_t* sx = (int32_t*)(smem + L.red + 896); // class maxima of the move's two colours before it
  int32_t* mvslot = (int32_t*)(smem + L.red + 904);  // moved vertex of even / odd iterations (-1: none)
  uint32_t* mvrow = (uint32_t*)(smem + L.mvrow);     // its adjacency row
  int32_t* red = (int32_t*)(smem + L.red);  // [kWWarps] warp minima, [kWWarps] warp tie totals
  int32_t* sc = red + 2 * kWWarps;          // -, old, new, improved, error, bad input, r0, r1
  // g, conf, best g, best f, best conf; from 8: per-warp conflict and score partial sums
  long long* sc64 = (long long*)(red + 2 * kWWarps + 8);
  G* gS = (G*)(smem + L.gT);
  G* gG = (G*)a.slab + (size_t)blockIdx.x * (size_t)(k - cs) * npad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int fs = a.fscale;
  int per = (n + kWThreads - 1) / kWThreads;
  {
    int p2 = 1;
    while (p2 < per) p2 <<= 1;
    per = p2 > 32 ? 32 : p2;
  }
  const uint32_t slice_mask = per == 32 ? 0xFFFFFFFFu : ((1u << per) - 1u);

  for (int ind = blockIdx.x; ind < a.pop; ind += gridDim.x) {
    if (a.redo_mode == 2 && a.redo[ind] == 0) continue;
    int16_t* gcol = a.col + (size_t)ind * n;
    const int64_t phi = a.phi_arr ? a.phi_arr[ind] : a.phi;
    // ---- set-up ---------------------------------------------------------------------------
    {
      uint32_t* l32 = (uint32_t*)lvl;
      for (int i = tid; i < (k * (wmax + 1) + 1) / 2; i += kWThreads) l32[i] = 0u;
      for (int i = tid; i < k * npad; i += kWThreads) {
        const int c = i / npad, v = i - c * npad;
        if (c < cs) gS[(size_t)c * npad + v] = 0;
        else gG[(size_t)(c - cs) * npad + v] = 0;
      }
      for (int c = tid; c < k; c += kWThreads) csz[c] = 0u;
      if (tid < 8) sc[tid] = 0;
    }
    __syncthreads();
    for (int v = tid; v < n; v += kWThreads) {
      int c = gcol[v];
      if (c < 0 || c >= k) { sc[5] = 1; c = 0; }
      colS[v] = (uint8_t)c;
      bestS[v] = (uint8_t)c;
      const int w = a.weight[v];
      wS[v] = (uint8_t)w;
      fz[v] = 0;
      const int q = c * (wmax + 1) + w;
      atomicAdd((uint32_t*)lvl + (q >> 1), 1u << (16 * (q & 1)));
      atomicAdd(csz + c, 1u);
    }
    __syncthreads();
    if (sc[5]) {
      if (tid == 0) raise_status(a.status, DLM_EINVAL);
      __syncthreads();
      continue;
    }
    if (a.redo_mode == 1) {  // a start class too large for u8 entries: left to the u16 pass
      bool big = false;
      for (int c = tid; c < k; c += kWThreads) big |= csz[c] > kWClass8;
      if (__syncthreads_or(big)) {
        if (tid == 0) a.redo[ind] = 1;
        continue;
      }
    }
    for (int i = tid; i < k * lw; i += kWThreads) {
      const int c = i / lw, wd = i - c * lw;
      uint32_t m = 0;
      for (int b = 0; b < 32; ++b) {
        const int lev = 32 * wd + b;
        if (lev <= wmax && lvl[(size_t)c * (wmax + 1) + lev] > 0) m |= 1u << b;
      }
      lmask[i] = m;
    }
    // transposed conflict table: the thread of vertex v is the only writer of position v
    long long cpart = 0;
    for (int v = tid; v < n; v += kWThreads) {
      const uint32_t* brow = a.bits + (size_t)v * nwords;
      for (int wd = 0; wd < nwords; ++wd) {
        uint32_t m = __ldg(brow + wd);
        while (m) {
          const int u = 32 * wd + __ffs(m) - 1;
          m &= m - 1;
          const int c = colS[u];
          if (c < cs) gS[(size_t)c * npad + v]++;
          else gG[(size_t)(c - cs) * npad + v]++;
          if (c == colS[v]) ++cpart;
        }
      }
    }
    __syncthreads();
    long long fpart = 0;
    for (int c = tid; c < k; c += kWThreads) {
      const uint32_t ic = class_info(lvl, lmask, lw, wmax, c);
      info[c] = ic;
      max1s[c] = (uint8_t)(ic & 0xFF);
      fpart += ic & 0xFF;
    }
    for (int d = 16; d >= 1; d >>= 1) {
      cpart += __shfl_down_sync(0xFFFFFFFFu, cpart, d);
      fpart += __shfl_down_sync(0xFFFFFFFFu, fpart, d);
    }
    if (lane == 0) { sc64[8 + warp] = cpart; sc64[8 + kWWarps + warp] = fpart; }
    __syncthreads();
    if (tid == 0) {
      long long ct = 0, ft = 0;
      for (int w = 0; w < kWWarps; ++w) { ct += sc64[8 + w]; ft += sc64[8 + kWWarps + w]; }
      const long long conf = ct / 2;
      sc64[0] = fs * ft + phi * conf;
      sc64[1] = conf;
      sc64[2] = fs * ft + phi * conf;
      sc64[3] = ft;
      sc64[4] = conf;
    }
    __syncthreads();
    long long g = sc64[0], conf = sc64[1], best_g = sc64[2];
    for (int v = tid; v < n; v += kWThreads) {  // every row's key summary at the start colouring
      int km, kc;
      wvcp_row_summary(v, colS[v], wS[v], max1s, gS, gG, npad, cs, k, fs, (int)phi, km, kc);
      skey[v] = km;
      scnt[v] = (uint16_t)kc;
    }
    __syncthreads();
    int64_t moves = 0;
    int32_t* trace = a.trace ? a.trace + (size_t)ind * a.iters * 4 : nullptr;
    // thread t owns rows [b0, b1) (slice t of per rows): warps hold consecutive row ranges, so the
    // tie order (v ascending) is warp, lane, row
    const int b0 = tid * per, b1 = min(b0 + per, n);
    // the best one-move of every row of this thread from its key summary: d = rem(v) fs -
    // phi gamma[v][col v] + key; a frozen vertex's moves count only when they reach below the
    // aspiration threshold (all its tied moves have the same d). Per warp: the minimum and the
    // number of moves that reach it
    auto select_rows = [&](unsigned itn, long long g_now, long long best_now) {
      const long long thr64 = best_now - g_now;
      const int thr = thr64 < (long long)INT_MIN + 1 ? INT_MIN + 1 : (int)thr64;
      int tmin = INT_MAX, tcnt = 0;
      for (int v = b0; v < b1; ++v) {
        const int o = colS[v], wv = wS[v];
        const uint32_t io = info[o];
        const int rem = (wv == (int)(io & 0xFF) && (io >> 16) == 1) ? (int)((io >> 8) & 0xFF) - (int)(io & 0xFF) : 0;
        const int g0 = o < cs ? gS[(size_t)o * npad + v] : gG[(size_t)(o - cs) * npad + v];
        const int d = fs * rem - (int)phi * g0 + skey[v];
        const bool ok = !(fz[v] > itn) || d < thr;
        const int dv = ok ? d : INT_MAX, cv = ok ? (int)scnt[v] : 0;
        rmin[v] = dv;
        rcnt[v] = (uint16_t)cv;
        if (dv < tmin) { tmin = dv; tcnt = cv; }
        else if (dv == tmin) tcnt += cv;
      }
      const int wm = __reduce_min_sync(0xFFFFFFFFu, tmin);
      const int wc = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)(tmin == wm ? tcnt : 0));
      if (lane == 0) { red[warp] = wm; red[kWWarps + warp] = wc; }
    };
    select_rows(0u, g, best_g);
    if (tid == 0) {
      const U4 r = rng(a.seed, 0u, a.gen, a.ind_base + (uint32_t)ind, kTagTabu);
      sc[6] = (int32_t)r.x;
      sc[7] = (int32_t)r.y;
      mvslot[0] = -1;
      mvslot[1] = -1;
    }
    __syncthreads();
    for (int64_t it = 0; it < a.iters; ++it) {
      const unsigned itrel = (unsigned)(it & 0x3FFF);
      const long long thr64 = best_g - g;
      const int thr = thr64 < (long long)INT_MIN + 1 ? INT_MIN + 1 : (int)thr64;
      // ---- phase 2: minimum over the warps, the tie j (Philox r0), its warp, lane and row; the
      // warp then finds the colour, 32 colours at a time in colour order (a ballot of the colours
      // that reach dstar, the jj-th set bit), and one lane makes the move ------------------------
      const int wmin = lane < kWWarps ? red[lane] : INT_MAX;
      const int dstar = __reduce_min_sync(0xFFFFFFFFu, wmin);
      const int wcnt = (lane < kWWarps && dstar != INT_MAX && wmin == dstar) ? red[kWWarps + lane] : 0;
      int winc = wcnt;
#pragma unroll
      for (int d = 1; d < kWWarps; d <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, winc, d);
        if (lane >= d) winc += t;
      }
      const int T = __shfl_sync(0xFFFFFFFFu, winc, kWWarps - 1);
      const int wpre = __shfl_sync(0xFFFFFFFFu, winc - wcnt, warp);
      const int wown = __shfl_sync(0xFFFFFFFFu, wcnt, warp);
      const int j = T > 0 ? (int)below((uint32_t)sc[6], (uint32_t)T) : 0;
      if (T > 0 && j >= wpre && j < wpre + wown) {
        int ct = 0;
        for (int v = b0; v < b1; ++v) ct += rmin[v] == dstar ? rcnt[v] : 0;
        int incl = ct;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
          if (lane >= d) incl += t;
        }
        const int lo = wpre + incl - ct;
        const bool win = ct > 0 && j >= lo && j < lo + ct;
        const unsigned wb = __ballot_sync(0xFFFFFFFFu, win);
        const int src = wb ? __ffs(wb) - 1 : 0;
        int mv = -1, jj = j - lo;
        if (win)
          for (int v = b0; v < b1; ++v) {
            if (rmin[v] != dstar) continue;
            if (jj >= rcnt[v]) { jj -= rcnt[v]; continue; }
            mv = v;
            break;
          }
        mv = __shfl_sync(0xFFFFFFFFu, mv, src);
        jj = __shfl_sync(0xFFFFFFFFu, jj, src);
        int mc = -1;
        uint32_t rw0 = 0u, rw1 = 0u;  // the moved vertex's adjacency row, loaded during the search
        if (mv >= 0) {
          const uint32_t* brow = a.bits + (size_t)mv * nwords;
          if (lane < nwords) rw0 = __ldg(brow + lane);
          if (lane + 32 < nwords) rw1 = __ldg(brow + lane + 32);
          const int o = colS[mv], wv = wS[mv];
          const uint32_t io = info[o];
          const int m1o = io & 0xFF, m2o = (io >> 8) & 0xFF, c1o = io >> 16;
          const int rem = (wv == m1o && c1o == 1) ? m2o - m1o : 0;
          const int g0 = o < cs ? gS[(size_t)o * npad + mv] : gG[(size_t)(o - cs) * npad + mv];
          const bool frozen = fz[mv] > itrel;
          const int base = fs * rem - (int)phi * g0;
          for (int c0 = 0; c0 < k && mc < 0; c0 += 32) {
            const int c = c0 + lane;
            bool hit = false;
            if (c < k && c != o) {
              const int gc = c < cs ? gS[(size_t)c * npad + mv] : gG[(size_t)(c - cs) * npad + mv];
              const int d = base + wvcp_key(fs, wv, max1s[c], (int)phi, gc);
              hit = d == dstar && (!frozen || d < thr);
            }
            const unsigned hb = __ballot_sync(0xFFFFFFFFu, hit);
            const int pc = __popc(hb);
            if (jj < pc) {
              unsigned x = hb;
              for (int q = 0; q < jj; ++q) x &= x - 1;
              mc = c0 + __ffs(x) - 1;
            } else {
              jj -= pc;
            }
          }
        }
        if (lane == src) {
          if (mv >= 0 && mc >= 0 && a.redo_mode == 1 && csz[mc] >= kWClass8) {
            sc[4] = 3;  // class mc would outgrow u8 entries: give the individual up
          } else if (mv >= 0 && mc >= 0) {
            const int o = colS[mv], wv = wS[mv];
            --csz[o];
            ++csz[mc];
            const int go = o < cs ? gS[(size_t)o * npad + mv] : gG[(size_t)(o - cs) * npad + mv];
            const int gn = mc < cs ? gS[(size_t)mc * npad + mv] : gG[(size_t)(mc - cs) * npad + mv];
            sx[0] = max1s[o];
            sx[1] = max1s[mc];
            class_add(lvl, lmask, lw, wmax, o, wv, -1);
            class_add(lvl, lmask, lw, wmax, mc, wv, +1);
            info[o] = class_info(lvl, lmask, lw, wmax, o);
            info[mc] = class_info(lvl, lmask, lw, wmax, mc);
            max1s[o] = (uint8_t)(info[o] & 0xFF);
            max1s[mc] = (uint8_t)(info[mc] & 0xFF);
            colS[mv] = (uint8_t)mc;
            const long long gn64 = g + dstar, cn64 = conf + (gn - go);
            fz[mv] = (uint16_t)(itrel + 1 + below((uint32_t)sc[7], a.L1) + a.ttbase);
            mvslot[it & 1] = mv;
            sc[1] = o; sc[2] = mc; sc[3] = gn64 < best_g;
            sc64[0] = gn64;
            sc64[1] = cn64;
            if (gn64 < best_g) { sc64[2] = gn64; sc64[3] = (gn64 - phi * cn64) / fs; sc64[4] = cn64; }
            if (trace) reinterpret_cast<int4*>(trace)[it] = make_int4(mv, mc, dstar, T);
          } else {
            sc[4] = 2;
          }
        }
        if (lane < nwords) mvrow[lane] = rw0;
        if (lane + 32 < nwords) mvrow[lane + 32] = rw1;
      }
      if (T == 0 && tid == 0 && trace) reinterpret_cast<int4*>(trace)[it] = make_int4(-1, -1, 0, 0);
      __syncthreads();
      if (sc[4]) break;
      // ---- phase 3: conflict-table update on the neighbours of the moved vertex, then the next
      // iteration's row selection ----------------------------------------------------------------
      const int mv = mvslot[it & 1];
      if (mv >= 0) {
        g = sc64[0];
        conf = sc64[1];
        ++moves;
        const int old = sc[1], nw = sc[2];
        const bool improved = sc[3] != 0;
        if (improved) best_g = sc64[2];
        G* po = old < cs ? gS + (size_t)old * npad : gG + (size_t)(old - cs) * npad;
        G* pn = nw < cs ? gS + (size_t)nw * npad : gG + (size_t)(nw - cs) * npad;
        const int m1a_old = sx[0], m1b_old = sx[1], m1a = max1s[old], m1b = max1s[nw], ph = (int)phi;
        uint32_t need = 0;  // rows of this thread whose only minimum rose (and the moved vertex's)
        if (b0 < n) {
          const uint32_t nb = (mvrow[b0 >> 5] >> (b0 & 31)) & slice_mask;
          uint32_t m = nb;
          while (m) {
            const int u = b0 + __ffs(m) - 1;
            m &= m - 1;
            po[u]--;
            pn[u]++;
          }
          // the key summaries of this thread's rows: colours old and nw changed (gamma of the
          // neighbours, both class maxima)
          for (int u = b0; u < b1; ++u) {
            const int cu = colS[u], wu = wS[u];
            int km = skey[u], kc = scnt[u];
            bool ok = u != mv;
            const int adj = (int)((nb >> (u - b0)) & 1u);
            if (ok && old != cu) {
              const int gnew = po[u];
              ok = wvcp_summ_apply(km, kc, wvcp_key(fs, wu, m1a_old, ph, gnew + adj), wvcp_key(fs, wu, m1a, ph, gnew));
            }
            if (ok && nw != cu) {
              const int gnew = pn[u];
              ok = wvcp_summ_apply(km, kc, wvcp_key(fs, wu, m1b_old, ph, gnew - adj), wvcp_key(fs, wu, m1b, ph, gnew));
            }
            if (ok) {
              skey[u] = km;
              scnt[u] = (uint16_t)kc;
            } else {
              need |= 1u << (u - b0);
            }
          }
        }
        // the flagged rows are scanned again by the owner's whole warp
        __syncwarp();
        unsigned lanes = __ballot_sync(0xFFFFFFFFu, need != 0);
        while (lanes) {
          const int src = __ffs(lanes) - 1;
          lanes &= lanes - 1;
          uint32_t rows = __shfl_sync(0xFFFFFFFFu, need, src);
          const int bs = src * per + warp * 32 * per;
          while (rows) {
            const int u = bs + __ffs(rows) - 1;
            rows &= rows - 1;
            int km, kc;
            wvcp_row_summary_warp(u, colS[u], wS[u], max1s, gS, gG, npad, cs, k, fs, ph, lane, km, kc);
            if (lane == 0) {
              skey[u] = km;
              scnt[u] = (uint16_t)kc;
            }
          }
        }
        if (improved) {
          const uint32_t* s32 = (const uint32_t*)colS;
          uint32_t* d32 = (uint32_t*)bestS;
          for (int i = tid; i < (n + 3) / 4; i += kWThreads) d32[i] = s32[i];
        }
      }
      if (((it + 1) & 0x3FFF) == 0)
        for (int v = b0; v < b1; ++v) fz[v] = fz[v] > 0x4000 ? (uint16_t)(fz[v] - 0x4000) : 0;
      __syncwarp();
      select_rows((unsigned)((it + 1) & 0x3FFF), g, best_g);
      if (tid == 0) {
        const U4 r = rng(a.seed, (uint32_t)(it + 1), a.gen, a.ind_base + (uint32_t)ind, kTagTabu);
        sc[6] = (int32_t)r.x;
        sc[7] = (int32_t)r.y;
        mvslot[(it + 1) & 1] = -1;
      }
      __syncthreads();
    }
    if (sc[4] == 3) {  // given up: the u16 pass searches it from its start colouring
      if (tid == 0) a.redo[ind] = 1;
      __syncthreads();
      continue;
    }
    if (sc[4] && tid == 0) raise_status(a.status, DLM_ECUDA);
    for (int v = tid; v < n; v += kWThreads) gcol[v] = (int16_t)bestS[v];
    if (tid == 0) {
      a.best_g[ind] = sc64[2];
      if (a.best_fc) { a.best_fc[2 * ind] = sc64[3]; a.best_fc[2 * ind + 1] = sc64[4]; }
      if (a.moves) a.moves[ind] = moves;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------
// Randomised greedy initialisation: one warp per individual. Vertex order (decreasing weight, then
// decreasing degree, then increasing index) is shared; vertex pos takes a colour drawn uniformly
// (Philox(a = pos, b = 0, c = individual, tag = WINIT)) among the opened colours that no coloured
// neighbour uses, or opens a new colour. The lanes OR their neighbours' colour bits into a 256-bit
// mask reduced with redux.sync.
// ------------------------------------------------------------------------------------------------
constexpr int kGWarps = 4;

__global__ void __launch_bounds__(32 * kGWarps) k_wvcp_greedy(int n, const int32_t* order, const int32_t* off,
                                                              const uint16_t* idx, int pop, uint64_t seed,
                                                              uint32_t ind_base, int16_t* col, int32_t* used_out,
                                                              int32_t* status) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* cw = smem + (size_t)warp * ((n + 15) & ~15);
  for (int i = blockIdx.x * kGWarps + warp; i < pop; i += gridDim.x * kGWarps) {
    for (int v = lane; v < n; v += 32) cw[v] = 0xFF;
    __syncwarp();
    int used = 0;
    bool overflow = false;
    for (int pos = 0; pos < n && !overflow; ++pos) {
      const int v = order[pos];
      uint32_t bm[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int e = off[v] + lane; e < off[v + 1]; e += 32) {
        const int c = cw[idx[e]];
        if (c != 0xFF) bm[c >> 5] |= 1u << (c & 31);
      }
      int cnt = 0;
      uint32_t legal[8];
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const uint32_t b = __reduce_or_sync(0xFFFFFFFFu, bm[w]);
        const int lo = 32 * w;
        const uint32_t usedm = used >= lo + 32 ? 0xFFFFFFFFu : (used <= lo ? 0u : ((1u << (used - lo)) - 1u));
        legal[w] = ~b & usedm;
        cnt += __popc(legal[w]);
      }
      int c;
      if (cnt == 0) {
        c = used++;
        if (c > 254) overflow = true;
      } else {
        const U4 r = rng(seed, (uint32_t)pos, 0u, ind_base + (uint32_t)i, kTagWInit);
        int j = (int)below(r.x, (uint32_t)cnt);
        c = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
          const int pc = __popc(legal[w]);
          if (j >= 0 && j < pc) {
            uint32_t x = legal[w];
            for (int q = 0; q < j; ++q) x &= x - 1;
            c = 32 * w + __ffs(x) - 1;
          }
          j -= pc;
        }
      }
      if (lane == 0) cw[v] = (uint8_t)c;
      __syncwarp();
    }
    if (overflow) {
      if (lane == 0) raise_status(status, DLM_EUNSUPPORTED);
      continue;
    }
    for (int v = lane; v < n; v += 32) col[(size_t)i * n + v] = (int16_t)cw[v];
    if (lane == 0 && used_out) used_out[i] = used;
    __syncwarp();
  }
}

}  // namespace dlm

using namespace dlm;

extern "C" dlm_status dlm_wvcp_greedy(dlm_ctx* ctx, const dlm_graph* g, int32_t pop, uint64_t seed, uint32_t ind_base,
                                      int16_t* col, int32_t* used) {
  if (!ctx || !g) return fail(ctx, DLM_EINVAL, "wvcp_greedy: null argument");
  if (!g->d_weight) return fail(ctx, DLM_EINVAL, "wvcp_greedy: the graph has no vertex weights");
  if (pop < 0 || (pop > 0 && !col)) return fail(ctx, DLM_EINVAL, "wvcp_greedy: bad arguments");
  if (pop == 0) return DLM_OK;
  const int n = g->n;
  // vertex order on the host: decreasing weight, decreasing degree, increasing index
  std::vector<int32_t> w(n), off(n + 1), order(n);
  DLM_CUDA(ctx, cudaMemcpyAsync(w.data(), g->d_weight, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(off.data(), g->d_off, (size_t)(n + 1) * 4, cudaMemcpyDeviceToHost, ctx->stream));
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int v = 0; v < n; ++v) order[v] = v;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (w[a] != w[b]) return w[a] > w[b];
    return off[a + 1] - off[a] > off[b + 1] - off[b];
  });
  int32_t* d_order = nullptr;
  DLM_TRY(ctx_workspace(ctx, (size_t)n * 4, (void**)&d_order));
  DLM_CUDA(ctx, cudaMemcpyAsync(d_order, order.data(), (size_t)n * 4, cudaMemcpyHostToDevice, ctx->stream));
  const size_t smem = (size_t)kGWarps * ((n + 15) & ~15);
  const int grid = std::min((pop + kGWarps - 1) / kGWarps, ctx->num_sms * 8);
  k_wvcp_greedy<<<grid, 32 * kGWarps, smem, ctx->stream>>>(n, d_order, g->d_off, g->d_idx, pop, seed, ind_base, col, used,
                                                           ctx->d_status);
  DLM_TRY(launch_check(ctx, "k_wvcp_greedy"));
  // the order array lives in the workspace: keep it alive until the kernel has read it
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return DLM_OK;
}

// entry size of the conflict table: u8 when only u8 entries keep the whole table in shared memory
// (entry_bits 0), or as the caller forces it (8 or 16); 0 when the state does not fit at all
static int wvcp_entry_bits(const dlm_ctx* ctx, int n, int k, int wmax, int entry_bits) {
  const WvcpLayout L16 = wvcp_layout(n, k, wmax, ctx->smem_optin, 2);
  const WvcpLayout L8 = wvcp_layout(n, k, wmax, ctx->smem_optin, 1);
  if (entry_bits == 16) return L16.gT <= ctx->smem_optin ? 16 : 0;
  if (entry_bits == 8) return L8.cs == k ? 8 : 0;
  if (L16.cs < k && L8.cs == k) return 8;
  return L16.gT <= ctx->smem_optin ? 16 : 0;
}

template <typename G>
static dlm_status wvcp_launch(dlm_ctx* ctx, const WvcpArgs& a, size_t smem, int grid) {
  DLM_CUDA(ctx, cudaFuncSetAttribute(k_wvcp_tabu<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_wvcp_tabu<G><<<grid, kWThreads, smem, ctx->stream>>>(a);
  return launch_check(ctx, "k_wvcp_tabu");
}

static dlm_status wvcp_run(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col, int64_t* best_g,
                           int64_t* best_fc, int64_t* moves, int64_t iters, dlm_tenure tenure, int64_t phi, uint64_t seed,
                           uint32_t generation, uint32_t ind_base, int32_t* trace, const int64_t* phi_arr = nullptr,
                           int32_t fscale = 1, int32_t entry_bits = 0) {
  if (!ctx || !g) return fail(ctx, DLM_EINVAL, "wvcp_tabu: null argument");
  if (!g->d_weight) return fail(ctx, DLM_EINVAL, "wvcp_tabu: the graph has no vertex weights");
  if (k < 2 || k > 255) return fail(ctx, DLM_EUNSUPPORTED, "wvcp_tabu: k must be in 2..255");
  if (g->max_weight > 255) return fail(ctx, DLM_EUNSUPPORTED, "wvcp_tabu: vertex weights must be <= 255");
  if (pop < 0 || iters < 0 || iters > INT32_MAX) return fail(ctx, DLM_EINVAL, "wvcp_tabu: bad population or budget");
  if (entry_bits != 0 && entry_bits != 8 && entry_bits != 16)
    return fail(ctx, DLM_EINVAL, "wvcp_tabu: entry_bits must be 0, 8 or 16");
  // keys are 32-bit: fscale (max w) + phi (max degree + 1) must stay below 2^30 (phi: the largest
  // per-individual value the caller can pass, checked by the caller for phi_arr)
  if (phi < 0 || fscale < 1 ||
      (int64_t)fscale * g->max_weight + phi * (int64_t)(g->max_degree + 1) >= ((int64_t)1 << 30))
    return fail(ctx, DLM_EUNSUPPORTED, "wvcp_tabu: fscale * max w + phi * (max degree + 1) must stay below 2^30");
  if (tenure.L_max < 0 || tenure.alpha_num < 0 || tenure.alpha_den <= 0) return fail(ctx, DLM_EINVAL, "wvcp_tabu: bad tenure");
  const int64_t ttbase = ((int64_t)tenure.alpha_num * g->n) / tenure.alpha_den;
  if (ttbase + tenure.L_max + 1 >= 0x4000) return fail(ctx, DLM_EUNSUPPORTED, "wvcp_tabu: tenure must stay below 2^14");
  if (pop == 0) return DLM_OK;
  if (!col || !best_g) return fail(ctx, DLM_EINVAL, "wvcp_tabu: null col or best_g");
  const int eb = wvcp_entry_bits(ctx, g->n, k, g->max_weight, entry_bits);
  if (eb == 0)
    return fail(ctx, DLM_EUNSUPPORTED, entry_bits == 8 ? "wvcp_tabu: the u8 conflict table does not fit shared memory"
                                                       : "wvcp_tabu: per-individual state exceeds shared memory");
  const WvcpLayout L16 = wvcp_layout(g->n, k, g->max_weight, ctx->smem_optin, 2);
  const WvcpLayout L8 = wvcp_layout(g->n, k, g->max_weight, ctx->smem_optin, 1);
  const int grid = std::min(pop, ctx->num_sms);
  // a u8 search can give an individual up only when a class can exceed 255 vertices; the u16 pass
  // (its slab, the flags) then follows
  const bool redo = eb == 8 && g->n > (int)kWClass8;
  const size_t slab_bytes = eb == 16 || redo ? (size_t)grid * (size_t)(k - L16.cs) * L16.npad * 2 : 0;
  const size_t redo_off = wal16(std::max<size_t>(16, slab_bytes));
  uint8_t* ws = nullptr;
  DLM_TRY(ctx_workspace(ctx, redo_off + (redo ? (size_t)pop * 4 : 0), (void**)&ws));
  WvcpArgs a;
  a.n = g->n; a.k = k; a.words = g->words; a.pop = pop; a.wmax = g->max_weight;
  a.bits = g->d_bits; a.weight = g->d_weight; a.col = col; a.best_g = best_g; a.best_fc = best_fc; a.moves = moves;
  a.trace = trace; a.slab = ws; a.iters = iters; a.phi = phi; a.phi_arr = phi_arr; a.fscale = fscale;
  a.L1 = (uint32_t)tenure.L_max + 1u;
  a.ttbase = (uint32_t)ttbase; a.seed = seed; a.gen = generation; a.ind_base = ind_base; a.status = ctx->d_status;
  a.smem_budget = ctx->smem_optin;
  a.redo = redo ? (int32_t*)(ws + redo_off) : nullptr;
  a.redo_mode = 0;
  if (eb == 16) return wvcp_launch<uint16_t>(ctx, a, L16.total, grid);
  if (redo) {
    DLM_CUDA(ctx, cudaMemsetAsync(a.redo, 0, (size_t)pop * 4, ctx->stream));
    a.redo_mode = 1;
  }
  DLM_TRY(wvcp_launch<uint8_t>(ctx, a, L8.total, grid));
  if (!redo) return DLM_OK;
  a.redo_mode = 2;
  return wvcp_launch<uint16_t>(ctx, a, L16.total, grid);
}

extern "C" dlm_status dlm_wvcp_tabu_batch(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                          int64_t* best_g, int64_t* best_fc, int64_t* moves, int64_t iters,
                                          dlm_tenure tenure, int64_t phi, uint64_t seed, uint32_t generation,
                                          uint32_t ind_base) {
  return wvcp_run(ctx, g, k, pop, col, best_g, best_fc, moves, iters, tenure, phi, seed, generation, ind_base, nullptr);
}

extern "C" dlm_status dlm_wvcp_tabu_batch_ex(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                             int64_t* best_g, int64_t* best_fc, int64_t* moves, int64_t iters,
                                             dlm_tenure tenure, int64_t phi, uint64_t seed, uint32_t generation,
                                             uint32_t ind_base, int32_t* trace, int32_t entry_bits) {
  return wvcp_run(ctx, g, k, pop, col, best_g, best_fc, moves, iters, tenure, phi, seed, generation, ind_base, trace,
                  nullptr, 1, entry_bits);
}

extern "C" dlm_status dlm_wvcp_entry_bits(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t* bits) {
  if (!ctx || !g || !bits) return fail(ctx, DLM_EINVAL, "wvcp_entry_bits: null argument");
  if (k < 2 || k > 255 || !g->d_weight) return fail(ctx, DLM_EINVAL, "wvcp_entry_bits: bad k or no weights");
  *bits = wvcp_entry_bits(ctx, g->n, k, g->max_weight, 0);
  return DLM_OK;
}

// ---- Algorithm 2: iterated feasible/infeasible tabu search with the adaptive penalty -----------
namespace dlm {

__global__ void k_ls_init(int pop, int64_t phi0, int64_t* phi, int64_t* best_f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < pop) { phi[i] = phi0; best_f[i] = -1; }
}

// after search t: keep the best legal colouring, then adapt phi (halve after a legal result,
// double otherwise; the last search uses phi_last); one block per individual
__global__ void k_ls_update(int pop, int n, const int16_t* col, const int64_t* fc, int64_t* phi, int64_t* best_f,
                            int16_t* best_col, int t, int max_ls, int64_t phi_last) {
  const int i = blockIdx.x;
  if (i >= pop) return;
  const int64_t f = fc[2 * i], c = fc[2 * i + 1];
  const bool take = c == 0 && (best_f[i] < 0 || f < best_f[i]);
  if (take)
    for (int v = threadIdx.x; v < n; v += blockDim.x) best_col[(size_t)i * n + v] = col[(size_t)i * n + v];
  __syncthreads();
  if (threadIdx.x == 0) {
    if (take) best_f[i] = f;
    if (t + 1 < max_ls - 1) phi[i] = c == 0 ? (phi[i] / 2 > 1 ? phi[i] / 2 : 1) : 2 * phi[i];
    else phi[i] = phi_last;
  }
}

// individuals that never reached a legal colouring report the last search's best
__global__ void k_ls_finish(int pop, int n, const int16_t* col, const int64_t* best_f, int16_t* best_col) {
  const int i = blockIdx.x;
  if (i >= pop || best_f[i] >= 0) return;
  for (int v = threadIdx.x; v < n; v += blockDim.x) best_col[(size_t)i * n + v] = col[(size_t)i * n + v];
}

}  // namespace dlm

extern "C" dlm_status dlm_wvcp_iterated(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                        int16_t* best_col, int64_t* best_f, int64_t iters, int32_t max_ls,
                                        dlm_tenure tenure, int32_t fscale, int64_t phi0, int64_t phi_last,
                                        uint64_t seed, uint32_t generation, uint32_t ind_base) {
  if (!ctx || !g) return fail(ctx, DLM_EINVAL, "wvcp_iterated: null argument");
  if (max_ls < 1 || max_ls > 16 || fscale < 1 || phi0 < 1 || phi_last < 1)
    return fail(ctx, DLM_EINVAL, "wvcp_iterated: need 1 <= max_ls <= 16, fscale >= 1, phi0 >= 1, phi_last >= 1");
  if (pop == 0) return DLM_OK;
  if (!col || !best_col || !best_f || pop < 0) return fail(ctx, DLM_EINVAL, "wvcp_iterated: null output");
  // the largest penalty any search can use: phi0 doubled before every search but the last, or phi_last
  int64_t phi_max = phi0;
  for (int t = 0; t + 2 < max_ls && phi_max < ((int64_t)1 << 40); ++t) phi_max *= 2;
  phi_max = phi_max > phi_last ? phi_max : phi_last;
  if ((int64_t)fscale * g->max_weight + phi_max * (int64_t)(g->max_degree + 1) >= ((int64_t)1 << 30))
    return fail(ctx, DLM_EUNSUPPORTED, "wvcp_iterated: the penalty schedule would overflow 32-bit move keys");
  // per-individual phi, (f, c) and best g of each search: their own allocation (the searches use the
  // context workspace for their slabs)
  uint8_t* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)pop * 32) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DLM_ENOMEM, "wvcp_iterated: scratch allocation failed");
  }
  int64_t* phi = (int64_t*)buf;
  int64_t* fc = phi + pop;
  int64_t* bg = fc + 2 * (size_t)pop;
  dlm_status st = DLM_OK;
  k_ls_init<<<(pop + 255) / 256, 256, 0, ctx->stream>>>(pop, phi0, phi, best_f);
  st = launch_check(ctx, "k_ls_init");
  for (int t = 0; t < max_ls && st == DLM_OK; ++t) {
    if (t == max_ls - 1 && max_ls == 1) {
      k_ls_init<<<(pop + 255) / 256, 256, 0, ctx->stream>>>(pop, phi_last, phi, best_f);
      st = launch_check(ctx, "k_ls_init");
      if (st != DLM_OK) break;
    }
    st = wvcp_run(ctx, g, k, pop, col, bg, fc, nullptr, iters, tenure, phi_max, seed, generation * 16u + (uint32_t)t,
                  ind_base, nullptr, phi, fscale);
    if (st != DLM_OK) break;
    k_ls_update<<<pop, 128, 0, ctx->stream>>>(pop, g->n, col, fc, phi, best_f, best_col, t, max_ls, phi_last);
    st = launch_check(ctx, "k_ls_update");
  }
  if (st == DLM_OK) {
    k_ls_finish<<<pop, 128, 0, ctx->stream>>>(pop, g->n, col, best_f, best_col);
    st = launch_check(ctx, "k_ls_finish");
  }
  cudaStreamSynchronize(ctx->stream);
  cudaFree(buf);
  return st;
}
