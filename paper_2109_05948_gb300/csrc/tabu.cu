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
//      col[n], best[n] u8 current and best colouring
//      summ[n]         per row: the smallest gamma among its non-tabu colours and among its tabu
//                      colours with their multiplicities, and its earliest tabu expiry
//  * selection reads one summary per conflicting vertex (thread t owns vertices t per ..
//    t per + per - 1, so thread order is vertex order) instead of scanning k colours per row;
//    aspiration (f + delta < best f) is decided from the tabu minimum;
//  * the warp holding the j-th tied move (j drawn from the iteration's Philox block) finds its
//    colour with ballots over that one row and applies the move;
//  * update: each thread changes gamma on its vertices adjacent to the moved vertex (bit row of
//    the graph, L1/L2 resident) and adjusts their summaries in O(1); rows whose class minimum may
//    have risen, the moved vertex and rows with an expiring tabu colour are summarised again by
//    the owner's warp (lanes over colours); the next iteration's selection follows in the same
//    phase. Two CTA barriers per iteration.
#include <algorithm>
#include <climits>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "tabu_group.cuh"

namespace dlm {

struct TabuJob {
  int32_t n, k, ks, words;
  const uint32_t* bits;  // [n][words]
  int16_t* col;          // [n] in: start, out: best
  int64_t* best_f;       // -> one int64
  int64_t* moves;        // -> one int64 or null
  int32_t* trace;        // [iters][4] or null
  int64_t* work;         // [3] or null: sums of conflicting rows evaluated, of degrees of moved vertices, of rows summarised again
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

__host__ __device__ inline int tabu_row_stride(int k) {
  int kw = (k + 1) / 2;
  if ((kw & 1) == 0) kw += 1;
  return 2 * kw;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Per-row summary of the admissible-move structure of a row v (colours c != col v, c < k), valid
// for one iteration's selection: the smallest gamma over the colours whose move is not tabu and
// how many reach it, the same over the tabu colours, and the earliest relative expiry among the
// tabu colours (0xFFFF: none). Keys are raw gamma values, so a change of gamma[v][col v] leaves
// the summary valid.
struct Summ {
  uint16_t ntmin, tmin;
  uint8_t ntcnt, tcnt;
  uint16_t nexp;
};
static_assert(sizeof(Summ) == 8, "a row summary is 8 bytes");
constexpr unsigned kNoKey = 0xFFFFu;

struct TabuSmem {
  size_t gam, tab, col, best, summ, vres, deg, red, rnd, brow, total;
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
  s.summ = o; o += align16((size_t)n * sizeof(Summ));
  s.vres = o; o += align16((size_t)n * 4);
  s.deg = o; o += align16((size_t)n * 2);
  s.red = o; o += align16((size_t)warps * 12 + 64);
  s.rnd = o; o += 32 * 8;
  s.brow = o; o += 64 * 4;  // the moved vertex's adjacency bit row (n <= 2048)
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

// Summary of row u by one warp (lanes over the 32-bit words, two colours each): classes at
// relative iteration itn (tabu when the expiry exceeds itn); the current colour and the padding
// columns (gamma 0xFFFF) are skipped.
__device__ __forceinline__ Summ summarise_row(const uint32_t* g32, const uint32_t* t32, int kw, int colu,
                                              unsigned itn, int lane) {
  unsigned ntm = kNoKey, tm = kNoKey, nex = kNoKey;
  unsigned ntc = 0, tc = 0;
  const int killw = colu >> 1;
  const uint32_t killm = 0xFFFFu << (16 * (colu & 1));
  for (int w = lane; w < kw; w += 32) {
    uint32_t gw = g32[w];
    const uint32_t tw = t32[w];
    if (w == killw) gw |= killm;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned g = (gw >> (16 * h)) & 0xFFFFu, t = (tw >> (16 * h)) & 0xFFFFu;
      if (g == kNoKey) continue;
      if (t > itn) {
        if (g < tm) { tm = g; tc = 1; } else if (g == tm) ++tc;
        nex = min(nex, t);
      } else {
        if (g < ntm) { ntm = g; ntc = 1; } else if (g == ntm) ++ntc;
      }
    }
  }
  Summ s;
  const unsigned NTM = __reduce_min_sync(0xFFFFFFFFu, ntm), TM = __reduce_min_sync(0xFFFFFFFFu, tm);
  s.ntmin = (uint16_t)NTM;
  s.tmin = (uint16_t)TM;
  s.ntcnt = (uint8_t)__reduce_add_sync(0xFFFFFFFFu, ntm == NTM ? ntc : 0u);
  s.tcnt = (uint8_t)__reduce_add_sync(0xFFFFFFFFu, tm == TM ? tc : 0u);
  s.nexp = (uint16_t)__reduce_min_sync(0xFFFFFFFFu, nex);
  return s;
}

// The key of one colour dropped to g: it may become its class minimum.
__device__ __forceinline__ void summ_lower(Summ& s, bool tabu, unsigned g) {
  if (tabu) {
    if (g < s.tmin) { s.tmin = (uint16_t)g; s.tcnt = 1; } else if (g == s.tmin) ++s.tcnt;
  } else {
    if (g < s.ntmin) { s.ntmin = (uint16_t)g; s.ntcnt = 1; } else if (g == s.ntmin) ++s.ntcnt;
  }
}

// The key of one colour rose from g: false when it was its class's only minimum (the row must be
// summarised again).
__device__ __forceinline__ bool summ_raise(Summ& s, bool tabu, unsigned g) {
  if (tabu) {
    if (g == s.tmin) { if (s.tcnt > 1) --s.tcnt; else return false; }
  } else {
    if (g == s.ntmin) { if (s.ntcnt > 1) --s.ntcnt; else return false; }
  }
  return true;
}

// One individual, one CTA of W warps (SPILL: rows beyond the shared-memory budget live in the
// CTA's global slab). Thread t owns the vertices [t per, (t + 1) per), per = ceil(n / threads), so
// thread order is vertex order. Every row carries a summary of its admissible-move structure
// (Summ); a row's neighbourhood is evaluated from its summary in O(1) instead of a scan of its k
// colours. Per iteration:
//  (A) selection: each thread evaluates its conflicting vertices from their summaries (minimum
//      delta and number of admissible colours reaching it), warps reduce; it runs at the end of
//      phase (C) of the previous iteration (its inputs come from the thread's own warp), and one
//      barrier follows;
//  (B) every warp derives (warp collectives) the minimum delta, the tie total T and its rank range; the warp
//      holding the j-th tie (j drawn from the iteration's Philox block) finds the vertex and,
//      with ballots over that row, the colour, and applies the move; one barrier;
//  (C) each thread updates gamma on its vertices adjacent to the moved vertex and adjusts their
//      summaries in O(1); a row whose class minimum may have risen, the moved vertex's row and
//      rows whose earliest tabu expiry falls at the next iteration are flagged by their owner
//      thread, and the owner's warp summarises them again (lanes over colours), then (A) of the
//      next iteration.
// The Philox blocks of 32 iterations are drawn at once, one per lane, every 32 iterations.
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
  Summ* summ = (Summ*)(smem + L.summ);
  uint32_t* vres = (uint32_t*)(smem + L.vres);  // per vertex of the selection: (delta + 2^15) << 16 | count
  uint16_t* degS = (uint16_t*)(smem + L.deg);
  int32_t* red = (int32_t*)(smem + L.red);   // [W] warp minima, [W] tie totals, [W] conflicting rows
  int32_t* sc = red + 3 * W;                 // scalars
  uint32_t* rnd = (uint32_t*)(smem + L.rnd); // Philox words (r0, r1) of the next 32 iterations
  uint32_t* browS = (uint32_t*)(smem + L.brow);  // adjacency bit row of this iteration's moved vertex
  // sc[0] moved vertex (-1 none), sc[1] old colour, sc[2] new colour, sc[3] f after,
  // sc[4] improved, sc[5] error, sc[6] bad input, sc[7] summarise every row
  const int iters = (int)J.iters;  // at most 2^31 - 1 (checked by the host)
  const int per = (n + NT - 1) / NT;
  const int v0 = tid * per, v1 = min(v0 + per, n);
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
  for (int u = warp; u < n; u += W) {  // every row's summary at iteration 0, one row per warp
    const Summ su = summarise_row((const uint32_t*)grow_of(u), (const uint32_t*)trow_of(u), kw, colS[u], 0u, lane);
    if (lane == 0) summ[u] = su;
  }
  int f;
  {
    int part = 0;
    for (int v = tid; v < n; v += NT) part += grow_of(v)[colS[v]];
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
  int64_t work_rows = 0, work_deg = 0, work_resum = 0;  // kept by thread 0 only

  // ---- (A) selection from the summaries of this thread's conflicting vertices: per-vertex
  // (delta, count) in vres, the thread's minimum and tie count, the warp's in red. Every input was
  // written by this thread's own warp or before the last barrier, so the next iteration's
  // selection runs straight after the update, without a barrier of its own.
  int tmin = INT_MAX, tcnt = 0;
  auto select = [&]() {
    int nconf = 0;
    tmin = INT_MAX;
    tcnt = 0;
    const int thrb = best_f - f;  // a tabu move is aspirated when gamma < thrb + gamma[v][col v]
    for (int v = v0; v < v1; ++v) {
      const int g0 = grow_of(v)[colS[v]];
      uint32_t res = 0u;
      if (g0 > 0) {
        ++nconf;
        const Summ s = summ[v];
        const unsigned nt = s.ntcnt ? s.ntmin : kNoKey;
        const unsigned ta = (s.tcnt && (int)s.tmin < thrb + g0) ? s.tmin : kNoKey;
        const unsigned adm = min(nt, ta);
        if (adm != kNoKey) {
          const int c = (nt == adm ? s.ntcnt : 0) + (ta == adm ? s.tcnt : 0);
          const int d = (int)adm - g0;
          res = ((uint32_t)(d + 32768) << 16) | (uint32_t)c;
          if (d < tmin) { tmin = d; tcnt = c; }
          else if (d == tmin) tcnt += c;
        }
      }
      vres[v] = res;
    }
    const int wm = __reduce_min_sync(FULL, tmin);
    const int wc = (int)__reduce_add_sync(FULL, (wm != INT_MAX && tmin == wm) ? (unsigned)tcnt : 0u);
    const int wn = (int)__reduce_add_sync(FULL, (unsigned)nconf);
    if (lane == 0) { red[warp] = wm; red[W + warp] = wc; red[2 * W + warp] = wn; }
  };
  select();
  for (it = 0; it < iters; ++it) {
    if (f == 0) break;
    const unsigned itrel = (unsigned)(it & 0x3FFF);
    __syncthreads();
    // ---- (B) minimum delta, tie ranks, move -------------------------------------------------
    if (tid == 0) {
      int nc = 0;
      for (int w = 0; w < W; ++w) nc += red[2 * W + w];
      work_rows += nc;
      // cancellation, polled every 1024 iterations: the search stops after this iteration's
      // selection and reports its best colouring so far
      if ((it & 1023) == 0 && R.cancel && *(volatile const int32_t*)R.cancel != 0) sc[5] = 3;
    }
    // lanes 0..W-1 hold the warps' minima and tie totals
    const int lw = lane < W ? red[lane] : INT_MAX;
    const int lc = lane < W ? red[W + lane] : 0;
    const int dstar = __reduce_min_sync(FULL, lw);
    const int xl = (dstar != INT_MAX && lw == dstar) ? lc : 0;
    const int T = (int)__reduce_add_sync(FULL, (unsigned)xl);
    const int pre = (int)__reduce_add_sync(FULL, lane < warp ? (unsigned)xl : 0u);
    const int wtot = __shfl_sync(FULL, xl, warp);
    const uint32_t j = T > 0 ? below(rnd[2 * (it & 31)], (uint32_t)T) : 0u;
    if (T > 0 && (int)j >= pre && (int)j < pre + wtot) {  // the j-th tie is in this warp (warp-uniform)
      const int ct = tmin == dstar ? tcnt : 0;
      int incl = ct;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
      }
      const int lo = pre + incl - ct;
      const bool hit = ct > 0 && (int)j >= lo && (int)j < lo + ct;  // this thread holds the j-th tie
      int hit_v = -1, hit_rank = 0;
      if (hit) {
        int jj = (int)j - lo;
        for (int v = v0; v < v1; ++v) {
          const uint32_t rr = vres[v];
          const int rcn = (int)(rr & 0xFFFFu);
          if (rcn == 0 || (int)(rr >> 16) - 32768 != dstar) continue;
          if (jj >= rcn) { jj -= rcn; continue; }
          hit_v = v;
          hit_rank = jj;
          break;
        }
      }
      // the whole warp searches the winning row: lane l takes words l, l + 32, ...; ballots order
      // the tied colours (word by word, low half first) and find the rank
      const unsigned hb = __ballot_sync(FULL, hit);
      const int hl = hb ? __ffs(hb) - 1 : 0;
      const int v = hb ? __shfl_sync(FULL, hit_v, hl) : -1;
      int jj = __shfl_sync(FULL, hit_rank, hl);
      int mc = -1, colv = 0;
      // the moved vertex's bit row, loaded now and stored to shared memory after the colour search
      // so that the load latency overlaps it
      uint32_t bw0 = 0u, bw1 = 0u;
      if (v >= 0) {
        const uint32_t* bsrc = J.bits + (size_t)v * nwords;
        if (lane < nwords) bw0 = __ldg(bsrc + lane);
        if (lane + 32 < nwords) bw1 = __ldg(bsrc + lane + 32);
        colv = colS[v];
        const uint16_t* grow = grow_of(v);
        const uint32_t* g32 = (const uint32_t*)grow;
        const uint32_t* t32 = (const uint32_t*)trow_of(v);
        const int g0 = grow[colv];
        const unsigned kmin = (unsigned)(dstar + g0);
        const int thr = best_f - f + g0;
        const int killw = colv >> 1;
        const uint32_t killm = 0xFFFFu << (16 * (colv & 1));
        const unsigned lt = (1u << lane) - 1u;
        for (int wb = 0; wb < kw && mc < 0; wb += 32) {
          const int w = wb + lane;
          bool m0 = false, m1 = false;
          if (w < kw) {
            uint32_t gw = g32[w];
            const uint32_t tw = t32[w];
            if (w == killw) gw |= killm;
            const unsigned ga = gw & 0xFFFFu, gb = gw >> 16;
            const unsigned k0 = ((tw & 0xFFFFu) <= itrel || (int)ga < thr) ? ga : kNoKey;
            const unsigned k1 = ((tw >> 16) <= itrel || (int)gb < thr) ? gb : kNoKey;
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
      }
      if (lane < nwords) browS[lane] = bw0;
      if (lane + 32 < nwords) browS[lane + 32] = bw1;
      if (lane == 0) {
        if (v >= 0 && mc >= 0 && mc < k) {
          colS[v] = (uint8_t)mc;
          const int fn = f + dstar;
          // alpha f in 32-bit unsigned arithmetic: the host bounds alpha_num * |E| below 2^32
          const uint32_t tt = below(rnd[2 * (it & 31) + 1], R.L1) + ((uint32_t)R.an * (uint32_t)fn) / (uint32_t)R.ad;
          if (tt > 32766u) sc[5] = 1;
          trow_of(v)[colv] = (uint16_t)(itrel + 1u + tt);
          sc[0] = v; sc[1] = colv; sc[2] = mc; sc[3] = fn; sc[4] = fn < best_f;
          if (J.trace) reinterpret_cast<int4*>(J.trace)[it] = make_int4(v, mc, dstar, T);
        } else {
          sc[5] = 2;  // tie counts inconsistent with the row: refuse to move
        }
      }
    }
    if (T == 0 && tid == 0) {
      sc[0] = -1;  // no admissible move: the iteration counts, nothing changes
      if (J.trace) reinterpret_cast<int4*>(J.trace)[it] = make_int4(-1, -1, 0, 0);
    }
    __syncthreads();
    if (sc[5]) break;
    // ---- (C) gamma and summaries of the moved vertex's neighbours ------------------------------
    const int mv = sc[0];
    const bool sweep = ((it + 1) & 0x3FFF) == 0;
    const unsigned itn = sweep ? 0u : itrel + 1u;  // relative iteration of the next selection
    uint64_t flags = 0;  // owned rows to summarise again: bit q = vertex v0 + q
    if (mv >= 0) {
      const int old = sc[1], nw = sc[2];
      f = sc[3];
      ++moves;
      if (tid == 0) work_deg += degS[mv];
      for (int u = v0; u < v1; ++u) {
        Summ s = summ[u];
        // its colour changed and its old colour became tabu, or one of its tabu colours expires
        bool again = u == mv || s.nexp <= itn;
        if ((browS[u >> 5] >> (u & 31)) & 1u) {
          uint16_t* grow = grow_of(u);
          const uint16_t* trow = trow_of(u);
          const unsigned go = grow[old], gn = grow[nw];
          const unsigned to = trow[old], tn = trow[nw];
          const int cu = colS[u];
          grow[old] = (uint16_t)(go - 1u);
          grow[nw] = (uint16_t)(gn + 1u);
          if (old != cu) summ_lower(s, to > itrel, go - 1u);
          if (nw != cu && !summ_raise(s, tn > itrel, gn)) again = true;
          summ[u] = s;
        }
        if (again) flags |= 1ull << (u - v0);
      }
      if (sc[4]) {
        best_f = f;
        const uint32_t* s32 = (const uint32_t*)colS;
        uint32_t* d32 = (uint32_t*)bestS;
        for (int i = tid; i < (n + 3) / 4; i += NT) d32[i] = s32[i];
      }
    } else {
      for (int u = v0; u < v1; ++u)
        if (summ[u].nexp <= itn) flags |= 1ull << (u - v0);
    }
    // the Philox block of the next 32 iterations (every reader of the current one has passed
    // the barrier above)
    if (((it + 1) & 31) == 0 && warp == W - 1) draw32(it + 1);
    if (sweep) {
      // the base advances by 2^14: relative expiries drop by 2^14, expired ones become 0; each
      // thread rebases its own rows, and every row is summarised again
      for (int u = v0; u < v1; ++u) {
        uint32_t* t32 = (uint32_t*)trow_of(u);
        for (int w = 0; w < kw; ++w) {
          const uint32_t x = t32[w];
          const uint32_t lo = x & 0xFFFF, hi = x >> 16;
          t32[w] = (lo > 0x4000u ? lo - 0x4000u : 0u) | ((hi > 0x4000u ? hi - 0x4000u : 0u) << 16);
        }
      }
      flags = v1 > v0 ? (~0ull >> (64 - (v1 - v0))) : 0ull;
    }
    // the warp summarises its lanes' flagged rows (lanes over colours); a row is written only by
    // its owner thread, so no other warp touches it
    __syncwarp();
    for (unsigned pend = __ballot_sync(FULL, flags != 0); pend; pend &= pend - 1) {
      const int l = __ffs(pend) - 1;
      uint64_t fl = __shfl_sync(FULL, flags, l);
      const int base = __shfl_sync(FULL, v0, l);
      for (; fl; fl &= fl - 1) {
        const int u = base + __ffsll(fl) - 1;
        const Summ su = summarise_row((const uint32_t*)grow_of(u), (const uint32_t*)trow_of(u), kw, colS[u], itn, lane);
        if (lane == 0) {
          summ[u] = su;
          ++work_resum;
        }
      }
    }
    __syncwarp();
    select();  // the next iteration's selection
  }
  {  // rows summarised again, summed over the warps
    if (lane == 0) red[warp] = (int32_t)work_resum;
    __syncthreads();
    if (tid == 0) {
      work_resum = 0;
      for (int w = 0; w < W; ++w) work_resum += red[w];
    }
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
    if (J.work) { J.work[0] = work_rows; J.work[1] = work_deg; J.work[2] = work_resum; }
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
  const int32_t* only;  // [pop] or null: search only the individuals flagged here
};

// Two CTAs per SM up to 16 warps (64 registers a thread); a 32-warp CTA takes the SM's registers alone.
template <int W>
__global__ void __launch_bounds__(W * 32, W >= 32 ? 1 : 2) tabucol_batch_kernel(TabuBatchArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  // one individual per CTA, or (when rows spill to a per-CTA slab) resident CTAs loop over them
  for (int i = blockIdx.x; i < a.pop; i += gridDim.x) {
    if (a.only && a.only[i] == 0) continue;  // the same for every thread of the CTA
    TabuJob J;
    J.n = a.n; J.k = a.k; J.ks = a.ks; J.words = a.words; J.bits = a.bits;
    J.col = a.col + (size_t)i * a.n;
    J.best_f = a.best_f + i;
    J.moves = a.moves ? a.moves + i : nullptr;
    J.trace = a.trace ? a.trace + (size_t)i * a.iters * 4 : nullptr;
    J.work = a.work ? a.work + 3 * (size_t)i : nullptr;
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
__global__ void __launch_bounds__(W * 32, W >= 32 ? 1 : 2) tabucol_multi_kernel(const MultiJob* jobs, int32_t njobs,
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
static dlm_status launch_batch(dlm_ctx* ctx, TabuBatchArgs a, size_t smem, size_t slab_stride,
                               uint16_t* slab_mem = nullptr) {
  auto kfn = tabucol_batch_kernel<W>;
  DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int grid = a.pop;
  if (slab_stride > 0) {  // rows spill: resident CTAs only, each with its own slab
    int per_sm = 0;
    DLM_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, W * 32, smem));
    grid = std::min(a.pop, std::max(1, per_sm) * ctx->num_sms);
    uint16_t* slab = slab_mem;
    if (!slab) DLM_TRY(ctx_workspace(ctx, (size_t)grid * slab_stride * 2, (void**)&slab));
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
  return 16;  // each thread owns at most ceil(n / 512) vertices: short phases between the barriers
}

// default of the one-graph launch: a state that leaves room for only one 16-warp CTA per SM
// (n = 1000, k = 48 takes 217 KB) gets 32 warps, all of the SM's registers, so each thread owns
// at most ceil(n / 1024) vertices (about 10 % faster at n = 700..1000 than 16 warps, same result)
static int default_warps_batch(dlm_ctx* ctx, int n, int k) {
  const int w = default_warps(n, k);
  if (w != 16) return w;
  const TabuSmem L = tabu_smem_layout(n, k, 16, ctx->smem_optin);
  int per_sm = 0;
  if (cudaFuncSetAttribute(tabucol_batch_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<16>, 16 * 32, L.total) !=
          cudaSuccess) {
    cudaGetLastError();
    return 16;
  }
  return per_sm == 1 ? 32 : 16;
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

// default warps per individual of the grouped kernel: the fewest (at least 2) that give each
// thread at most 4 vertices
static int default_group_warps(int n) {
  int w = 2;
  while (w < 16 && 32 * w * 4 < n) w *= 2;
  return w;
}

// the one-individual-per-CTA launch of a batch (rows beyond shared memory in per-CTA slabs);
// only: search just the individuals flagged there (null: all); slab_mem: the slabs, or null for the
// context's workspace
static dlm_status legacy_launch(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                                uint32_t generation, uint32_t ind_base, int warps, int32_t* trace, int64_t* work,
                                const int32_t* only, uint16_t* slab_mem) {
  const TabuSmem L = tabu_smem_layout(g->n, k, warps, ctx->smem_optin);
  if (L.rs < 1 || L.total > ctx->smem_optin)
    return fail(ctx, DLM_EUNSUPPORTED, "tabucol: the per-individual arrays exceed shared memory per block");
  const size_t slab_stride = L.rs < g->n ? tabu_slab_elems(g->n, k, L.rs) : 0;
  TabuBatchArgs a;
  a.n = g->n; a.k = k; a.ks = tabu_row_stride(k); a.words = g->words; a.pop = pop;
  a.bits = g->d_bits; a.off = g->d_off; a.col = col; a.best_f = best_f; a.moves = moves; a.trace = trace;
  a.work = work; a.iters = iters;
  a.ind_base = ind_base;
  a.only = only;
  a.rule = TabuRule{(uint32_t)tenure.L_max + 1u, tenure.alpha_num, tenure.alpha_den, seed, generation, ctx->d_status,
                    ctx->smem_optin, nullptr, 0, ctx->cancel};
  switch (warps) {
    case 1: return launch_batch<1>(ctx, a, L.total, slab_stride, slab_mem);
    case 2: return launch_batch<2>(ctx, a, L.total, slab_stride, slab_mem);
    case 4: return launch_batch<4>(ctx, a, L.total, slab_stride, slab_mem);
    case 8: return launch_batch<8>(ctx, a, L.total, slab_stride, slab_mem);
    case 16: return launch_batch<16>(ctx, a, L.total, slab_stride, slab_mem);
    default: return launch_batch<32>(ctx, a, L.total, slab_stride, slab_mem);
  }
}

// bytes of the slabs legacy_launch uses for pop individuals (0 when every row fits)
static size_t legacy_slab_bytes(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int warps) {
  const TabuSmem L = tabu_smem_layout(g->n, k, warps, ctx->smem_optin);
  if (L.rs < 1 || L.rs >= g->n) return 0;
  int per_sm = 0;
  switch (warps) {
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<1>, 32, L.total); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<2>, 64, L.total); break;
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<4>, 128, L.total); break;
    case 8: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<8>, 256, L.total); break;
    case 16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<16>, 512, L.total); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<32>, 1024, L.total); break;
  }
  cudaGetLastError();
  const size_t grid = (size_t)std::min(pop, std::max(1, per_sm) * ctx->num_sms);
  return grid * tabu_slab_elems(g->n, k, L.rs) * 2;
}

// u8 entries where the u16 state exceeds one SM: the grouped u8 launch, then the one-individual-
// per-CTA kernel over the individuals it gave up (a class grew beyond 126 vertices); both use one
// workspace, so the flags survive between them
static dlm_status tabucol_u8_then_legacy(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                         int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure,
                                         uint64_t seed, uint32_t generation, uint32_t ind_base, const GroupPlan& P,
                                         int warps, int32_t* trace, int64_t* work) {
  const int wl = warps ? warps : default_warps_batch(ctx, g->n, k);
  const size_t gbytes = align16(group_far_bytes(ctx, g, k, pop, iters, tenure, P));
  const size_t sbytes = legacy_slab_bytes(ctx, g, k, pop, wl);
  uint8_t* ws = nullptr;
  DLM_TRY(ctx_workspace(ctx, gbytes + sbytes + 16, (void**)&ws));
  int32_t* redo = nullptr;
  DLM_TRY(tabucol_group_launch(ctx, g, k, pop, col, best_f, moves, iters, tenure, seed, generation, ind_base, P, trace,
                               work, ws, &redo));
  return legacy_launch(ctx, g, k, pop, col, best_f, moves, iters, tenure, seed, generation, ind_base, wl, trace, work,
                       redo, sbytes ? (uint16_t*)(ws + gbytes) : nullptr);
}

// the grouped kernel's plan for a problem: u16 gamma entries, or u8 entries when they fit more
// individuals on an SM (eb = 0: that choice; 8 or 16: forced, u8 only where u16 also fits, for
// the fallback)
// legacy_fb (or null): u8 entries may also be taken where no u16 grouped plan exists; then
// *legacy_fb is set and the caller searches the individuals the u8 launch gives up with the
// one-individual-per-CTA kernel
static bool choose_group_plan(dlm_ctx* ctx, const dlm_graph* g, int k, int pop, int W, int ring, int eb,
                              GroupPlan* out, bool* legacy_fb = nullptr) {
  GroupPlan P16, P8;
  if (legacy_fb) *legacy_fb = false;
  if (!group_plan(g->n, k, g->words, W, ctx->smem_optin, pop, ctx->num_sms, ring, 16, &P16)) {
    if (!legacy_fb || eb == 16 || ring || k > 128 ||
        !group_plan(g->n, k, g->words, W, ctx->smem_optin, pop, ctx->num_sms, 0, 8, &P8))
      return false;
    *legacy_fb = true;
    *out = P8;
    return true;
  }
  if (eb == 16) { *out = P16; return true; }
  const bool ok8 = k <= 128 && group_plan(g->n, k, g->words, W, ctx->smem_optin, pop, ctx->num_sms, ring, 8, &P8);
  if (eb == 8) {
    if (!ok8) return false;
    *out = P8;
    return true;
  }
  *out = (ok8 && P8.G * group_ctas_per_sm(P8) > P16.G * group_ctas_per_sm(P16)) ? P8 : P16;
  return true;
}

static dlm_status tabucol_run(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                              int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                              uint32_t generation, uint32_t ind_base, int warps, int32_t* trace,
                              int64_t* work, int ring = 0, int legacy = 0, int eb = 0) {
  DLM_TRY(tabucol_check(ctx, g, k, pop, iters, tenure));
  if (pop == 0) return DLM_OK;
  if (!col || !best_f) return fail(ctx, DLM_EINVAL, "tabucol: null col or best_f");
  if (warps == 0) warps = lookup_tune(ctx, g->n, k);
  if (warps != 0 && warps != 1 && warps != 2 && warps != 4 && warps != 8 && warps != 16 && warps != 32)
    return fail(ctx, DLM_EINVAL, "tabucol: warps per individual must be 1, 2, 4, 8, 16 or 32");
  if (ring != 0 && (ring < 64 || ring > 8192 || (ring & (ring - 1)) != 0))
    return fail(ctx, DLM_EINVAL, "tabucol: the tabu ring size must be a power of two in 64..8192");
  if (eb != 0 && eb != 8 && eb != 16) return fail(ctx, DLM_EINVAL, "tabucol: entry bits must be 0, 8 or 16");
  if (!legacy) {
    // several individuals per CTA, tabu flags inside gamma: whenever one individual's state fits
    const int wg = warps ? warps : default_group_warps(g->n);
    GroupPlan P;
    bool legacy_fb = false;
    if (choose_group_plan(ctx, g, k, pop, wg, ring, eb, &P, &legacy_fb)) {
      const uint64_t tt_max =
          (uint64_t)tenure.L_max + ((uint64_t)tenure.alpha_num * (uint64_t)g->m) / (uint64_t)tenure.alpha_den;
      if ((uint64_t)iters + tt_max + 2 >= (1ull << 32))
        return fail(ctx, DLM_EUNSUPPORTED, "tabucol: budget plus the longest tenure must stay below 2^32");
      if (!legacy_fb)
        return tabucol_group_launch(ctx, g, k, pop, col, best_f, moves, iters, tenure, seed, generation, ind_base, P,
                                    trace, work);
      return tabucol_u8_then_legacy(ctx, g, k, pop, col, best_f, moves, iters, tenure, seed, generation, ind_base, P,
                                    warps, trace, work);
    }
    if (ring) return fail(ctx, DLM_EINVAL, "tabucol: the requested tabu ring does not fit in shared memory");
    if (eb) return fail(ctx, DLM_EINVAL, "tabucol: the requested gamma entries do not fit in shared memory");
  }
  if (warps == 0) warps = default_warps_batch(ctx, g->n, k);
  return legacy_launch(ctx, g, k, pop, col, best_f, moves, iters, tenure, seed, generation, ind_base, warps, trace,
                       work, nullptr, nullptr);
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

extern "C" dlm_status dlm_tabucol_launch_info(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop,
                                              int32_t warps, int32_t* info) {
  if (!ctx || !g || !info || pop <= 0 || k < 2 || k > 128) return fail(ctx, DLM_EINVAL, "launch_info: bad arguments");
  if (warps == 0) warps = lookup_tune(ctx, g->n, k);
  GroupPlan P;
  bool legacy_fb = false;
  if (choose_group_plan(ctx, g, k, pop, warps ? warps : default_group_warps(g->n), 0, 0, &P, &legacy_fb)) {
    const int grid = group_grid(ctx, P, pop);
    const int32_t v[8] = {P.eb == 8 ? 2 : 1, P.W, P.G, P.R, P.per, P.bsm ? 1 : 0, grid, grid * P.G};
    for (int i = 0; i < 8; ++i) info[i] = v[i];
    return DLM_OK;
  }
  if (warps == 0) warps = default_warps_batch(ctx, g->n, k);
  const TabuSmem L = tabu_smem_layout(g->n, k, warps, ctx->smem_optin);
  int grid = pop;
  if (L.rs < g->n) {
    int per_sm = 1;
    switch (warps) {
      case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<1>, 32, L.total); break;
      case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<2>, 64, L.total); break;
      case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<4>, 128, L.total); break;
      case 8: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<8>, 256, L.total); break;
      case 16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<16>, 512, L.total); break;
      default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_batch_kernel<32>, 1024, L.total); break;
    }
    cudaGetLastError();
    grid = std::min(pop, std::max(1, per_sm) * ctx->num_sms);
  }
  const int32_t v[8] = {0, warps, 1, 0, (g->n + 32 * warps - 1) / (32 * warps), 0, grid, grid};
  for (int i = 0; i < 8; ++i) info[i] = v[i];
  return DLM_OK;
}

extern "C" dlm_status dlm_tabucol_batch_opts(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                             int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure,
                                             uint64_t seed, uint32_t generation, uint32_t ind_base,
                                             const dlm_tabu_opts* opts, int32_t* trace, int64_t* work) {
  const dlm_tabu_opts o = opts ? *opts : dlm_tabu_opts{0, 0, 0, 0};
  return tabucol_run(ctx, g, k, pop, col, best_f, moves, iters, tenure, seed, generation, ind_base,
                     o.warps_per_individual, trace, work, o.ring, o.legacy, o.entry_bits);
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

// ---- the uneven batch on the grouped kernel: one launch per graph, side by side on the context's
// stream pool, the graphs with the most work per individual first; individual j of graph gi draws
// the Philox id ind_base + (individuals of the graphs before gi) + j, as in the one-launch path ----
struct MultiGroupPlan {
  std::vector<int> order;       // graphs with individuals, by decreasing n k iters
  std::vector<GroupPlan> plans;
  std::vector<size_t> far_off;  // byte offset of each graph's far lists
  std::vector<uint32_t> ind0;   // Philox id of each graph's first individual
  size_t far_total = 0;
};

static bool multi_group_plan(dlm_ctx* ctx, int n_graphs, const dlm_graph* const* graphs, const int32_t* k,
                             const int32_t* pop, const int64_t* iters, dlm_tenure tenure, uint32_t ind_base,
                             MultiGroupPlan* out) {
  MultiGroupPlan M;
  M.plans.resize(n_graphs);
  M.far_off.assign(n_graphs, 0);
  M.ind0.resize(n_graphs);
  uint32_t id = ind_base;
  for (int gi = 0; gi < n_graphs; ++gi) {
    M.ind0[gi] = id;
    id += (uint32_t)pop[gi];
    if (pop[gi] == 0) continue;
    const dlm_graph* g = graphs[gi];
    if (!choose_group_plan(ctx, g, k[gi], pop[gi], default_group_warps(g->n), 0, 0, &M.plans[gi])) return false;
    const uint64_t tt_max =
        (uint64_t)tenure.L_max + ((uint64_t)tenure.alpha_num * (uint64_t)g->m) / (uint64_t)tenure.alpha_den;
    if ((uint64_t)iters[gi] + tt_max + 2 >= (1ull << 32)) return false;
    M.far_off[gi] = M.far_total;
    M.far_total += align16(group_far_bytes(ctx, g, k[gi], pop[gi], iters[gi], tenure, M.plans[gi]));
    M.order.push_back(gi);
  }
  std::stable_sort(M.order.begin(), M.order.end(), [&](int a, int b) {
    return (double)graphs[a]->n * k[a] * iters[a] > (double)graphs[b]->n * k[b] * iters[b];
  });
  *out = std::move(M);
  return true;
}

static dlm_status ensure_pool(dlm_ctx* ctx) {
  for (int i = 0; i < dlm_ctx::kPool; ++i)
    if (!ctx->pool[i]) DLM_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->pool[i], cudaStreamNonBlocking));
  for (int i = 0; i <= dlm_ctx::kPool; ++i)
    if (!ctx->pool_ev[i]) DLM_CUDA(ctx, cudaEventCreateWithFlags(&ctx->pool_ev[i], cudaEventDisableTiming));
  return DLM_OK;
}

// forks from `base` to the pool, launches every graph, joins back into `base`; far: device memory
// of M.far_total bytes
static dlm_status multi_group_launch(dlm_ctx* ctx, cudaStream_t base, const MultiGroupPlan& M,
                                     const dlm_graph* const* graphs, const int32_t* k, const int32_t* pop,
                                     int16_t* const* col, int64_t* const* best_f, int64_t* const* moves,
                                     const int64_t* iters, dlm_tenure tenure, uint64_t seed, uint32_t generation,
                                     uint8_t* far) {
  if (M.order.empty()) return DLM_OK;
  DLM_TRY(ensure_pool(ctx));
  const int ns = std::min<int>(dlm_ctx::kPool, (int)M.order.size());
  DLM_CUDA(ctx, cudaEventRecord(ctx->pool_ev[dlm_ctx::kPool], base));
  for (int i = 0; i < ns; ++i) DLM_CUDA(ctx, cudaStreamWaitEvent(ctx->pool[i], ctx->pool_ev[dlm_ctx::kPool], 0));
  const cudaStream_t saved = ctx->stream;
  dlm_status st = DLM_OK;
  for (size_t t = 0; t < M.order.size() && st == DLM_OK; ++t) {
    const int gi = M.order[t];
    ctx->stream = ctx->pool[t % ns];
    st = tabucol_group_launch(ctx, graphs[gi], k[gi], pop[gi], col[gi], best_f[gi], moves ? moves[gi] : nullptr,
                              iters[gi], tenure, seed, generation, M.ind0[gi], M.plans[gi], nullptr, nullptr,
                              far ? far + M.far_off[gi] : nullptr);
  }
  ctx->stream = saved;
  for (int i = 0; i < ns; ++i) {  // join, also after an error, so that no pool stream stays forked
    DLM_CUDA(ctx, cudaEventRecord(ctx->pool_ev[i], ctx->pool[i]));
    DLM_CUDA(ctx, cudaStreamWaitEvent(base, ctx->pool_ev[i], 0));
  }
  return st;
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
  if (njobs == 0) return DLM_OK;
  {  // every graph's state fits the grouped kernel: one launch per graph, side by side
    MultiGroupPlan M;
    if (multi_group_plan(ctx, n_graphs, graphs, k, pop, iters, tenure, ind_base, &M)) {
      uint8_t* far = nullptr;
      if (M.far_total) DLM_TRY(ctx_workspace(ctx, M.far_total, (void**)&far));
      return multi_group_launch(ctx, ctx->stream, M, graphs, k, pop, col, best_f, moves, iters, tenure, seed,
                                generation, far);
    }
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
  bool grouped = false;  // one grouped launch per graph (branches of the captured graph)
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
  {  // the grouped kernel when every graph fits it: the per-graph launches captured as branches
    MultiGroupPlan M;
    if (multi_group_plan(ctx, n_graphs, graphs, k, pop, iters, tenure, ind_base, &M)) {
      dlm_multi_plan* p = new dlm_multi_plan();
      p->grouped = true;
      p->njobs = njobs;
      auto bail = [&](dlm_status s, const std::string& m) { dlm_tabucol_multi_plan_destroy(p); return fail(ctx, s, m); };
      if (M.far_total && cudaMalloc(&p->mem, M.far_total) != cudaSuccess) {
        cudaGetLastError();
        return bail(DLM_ENOMEM, "tabucol_multi_plan: allocation failed");
      }
      DLM_TRY(ensure_pool(ctx));
      cudaStream_t cs = nullptr;
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return bail(DLM_ECUDA, "stream");
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      dlm_status ls = DLM_OK;
      if (e == cudaSuccess)
        ls = multi_group_launch(ctx, cs, M, graphs, k, pop, col, best_f, moves, iters, tenure, seed, generation, p->mem);
      const cudaError_t e2 = cudaStreamEndCapture(cs, &p->graph);
      cudaStreamDestroy(cs);
      if (e != cudaSuccess || e2 != cudaSuccess || ls != DLM_OK) {
        cudaGetLastError();
        return bail(ls != DLM_OK ? ls : DLM_ECUDA, "tabucol_multi_plan: capture");
      }
      if (cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return bail(DLM_ECUDA, "tabucol_multi_plan: instantiate");
      }
      *out = p;
      return DLM_OK;
    }
  }
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
