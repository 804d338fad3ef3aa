// Population-wide TabuCol for k-COL with several individuals per CTA (paper: section "Adaptations
// of the algorithm for the vertex coloring problem" -- TabuCOL of Hertz & de Werra in the
// implementation of Galinier & Hao, run on every offspring; Table params-COL for alpha = 0.6).
//
// One TabuCol iteration is a short dependent chain (evaluate the conflicting vertices, pick the
// j-th tied minimum, apply the move, update the moved vertex's neighbours), so the kernel is bound
// by the latency of that chain and by the instructions issued per iteration, not by bandwidth.
// The design keeps both small and puts as many independent individuals on an SM as its shared
// memory allows:
//  * state of one individual (shared memory):
//      gam[n][ks] u16   conflict table gamma; bit 15 of each entry is the tabu flag of (v, c), so
//                       one load gives a colour's key and whether its move is tabu (no n x k
//                       expiry table: 60 KB per individual at n = 500, k = 48 instead of 100 KB)
//      rec[v]  8 B      per row and per class (non-tabu / tabu colours c != col v): the smallest
//                       gamma, how many colours reach it and how many reach it + 1 (or unknown)
//      g0[v]  u16       gamma[v][col v]; col, best u8; dirty u8 (row to summarise again)
//      ring[R] 8 B      tabu entries (v, c, expiry) in insertion order; entries whose tenure does
//                       not fit the ring go to a per-slot list in global memory (the far list)
//  * a group of W warps per individual, thread t owning vertices [t per, t per + per) so that
//    thread order is vertex order; G groups per CTA share the graph's bit rows in shared memory
//    and synchronise on their own named barrier;
//  * per iteration: (D) after a barrier every warp reduces the warps' minima and tie counts, the
//    warp holding the j-th tie finds the vertex and, with ballots over its row, the colour; warp
//    W-1 meanwhile maintains the ring (inserts the previous move's entry, lists the entries that
//    expire before the next selection); (U) after a second barrier the owner of the moved vertex
//    updates its row, each warp clears the flags of its expiring entries and updates gamma on its
//    neighbours of the moved vertex (compacted across lanes), adjusting the row summaries in O(1)
//    (two count levels make a raised or removed unique minimum exact in most cases), summarises
//    the rows it could not adjust again, and evaluates its conflicting vertices for the next
//    selection.
#include <algorithm>
#include <climits>
#include <cstring>

#include "common.cuh"
#include "tabu_group.cuh"

namespace dlm {
namespace tg {

constexpr unsigned FULL = 0xFFFFFFFFu;
// gamma entries of EB bits: the top bit is the tabu flag, the rest the count; the largest value
// (NONE) marks an absent colour. u8 entries hold counts up to 126, which the kernel guarantees by
// keeping every colour class at most 126 vertices (gamma[v][c] <= |V_c|); an individual whose
// search would grow a class beyond that gives up and is searched again with u16 entries.
template <int EB>
struct Ent {
  using T = typename std::conditional<EB == 8, uint8_t, uint16_t>::type;
  static constexpr unsigned NONE = EB == 8 ? 0x7Fu : 0x7FFFu;
  static constexpr unsigned FLAG = EB == 8 ? 0x80u : 0x8000u;
  static constexpr int EPW = 32 / EB;  // entries per 32-bit word
};
constexpr int kMaxClass8 = 126;
constexpr int kDueCap = 32;          // expiring ring entries listed per iteration (more: window scan)

// sc[] slots of a group (shared memory); 0..3, 4..7 and 8..11 are each read as one int4
enum { SC_MV = 0, SC_OLD, SC_NEW, SC_F,          // the iteration's move and f after it
       SC_DUE, SC_LO, SC_NINS, SC_FARN,          // expiring entries (count | far flag << 30), ring window, far list size
       SC_STOP, SC_ERR, SC_BAD, SC_FARMIN,
       SC_REQ = 12,                              // two int4 (by iteration parity): the move's tabu entry
                                                 // (v, c, tenure, was tabu) for the ring, v < 0: none
       SC_ABORT = 20,                            // u8 entries: a class would exceed kMaxClass8
       SC_N = 32 };

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline GroupLayout group_layout(int n, int k, int W, int per, int R, int eb) {
  GroupLayout L;
  const size_t nv = (size_t)32 * W * per;  // rows: every thread's per slots (n rounded up)
  const int ks = eb == 8 ? group_row_stride8(k) : group_row_stride(k);
  (void)n;
  size_t o = 0;
  L.gam = o; o += a16(nv * ks * (eb / 8));
  L.csz = o; o += eb == 8 ? a16((size_t)k * 4) : 0;  // class sizes (u8 entries only)
  L.col = o; o += a16(nv);
  L.best = o; o += a16(nv);
  L.ring = o; o += a16((size_t)R * 8);
  L.due = o; o += a16((size_t)kDueCap * 4);
  L.red = o; o += a16((size_t)W * 32);  // per warp: selection (int4), at the end 3 work counters (int64)
  L.sc = o; o += SC_N * 4;
  L.total = a16(o);
  return L;
}

// ---- class summaries ---------------------------------------------------------------------------
// A row keeps one 32-bit word per class (its non-tabu colours, its tabu colours; the current colour
// belongs to neither): bits 0-11 the smallest key (kEmpty: no colour), 12-19 how many colours reach
// it, bit 20 set when the count at the minimum + 1 is unknown, 24-31 that count. One colour's key
// can enter the class (ins), leave it (rem), drop by one (dec) or rise by one (inc); the common
// cases are one addition to the word. rem and inc report false when the new minimum cannot be
// derived (the row is then summarised again from its gamma entries). When the count at the
// minimum + 1 is unknown its byte may wrap; the byte is the word's top, so nothing else changes.
constexpr uint32_t kEmpty = 0xFFFu, kC1 = 1u << 12, kUnkBit = 1u << 20, kC2 = 1u << 24;

__device__ __forceinline__ uint32_t cw_make(uint32_t mn, uint32_t c1, uint32_t c2, bool unk) {
  return mn | (c1 << 12) | (unk ? kUnkBit : (c2 << 24));
}
__device__ __forceinline__ uint32_t cw_mn(uint32_t w) { return w & 0xFFFu; }
__device__ __forceinline__ uint32_t cw_c1(uint32_t w) { return (w >> 12) & 0xFFu; }
__device__ __forceinline__ bool cw_unk(uint32_t w) { return (w & kUnkBit) != 0; }
__device__ __forceinline__ uint32_t cw_c2(uint32_t w) { return w >> 24; }

__device__ __forceinline__ uint32_t cw_ins(uint32_t w, uint32_t g) {
  const uint32_t mn = cw_mn(w);
  if (g + 1u < mn) return cw_make(g, 1u, 0u, false);
  if (g + 1u == mn) return cw_make(g, 1u, cw_c1(w), false);
  return w + (g == mn ? kC1 : (g == mn + 1u ? kC2 : 0u));
}
__device__ __forceinline__ uint32_t cw_rem(uint32_t w, uint32_t g, bool& ok) {
  const uint32_t mn = cw_mn(w), c1 = cw_c1(w);
  if (g == mn && c1 == 1u) {
    ok = !cw_unk(w) && cw_c2(w) > 0u;
    return cw_make(mn + 1u, cw_c2(w), 0u, true);
  }
  ok = true;
  return w - (g == mn ? kC1 : (g == mn + 1u ? kC2 : 0u));
}
__device__ __forceinline__ uint32_t cw_dec(uint32_t w, uint32_t g) {  // g -> g - 1, g >= minimum
  const uint32_t mn = cw_mn(w);
  if (g == mn) return cw_make(g - 1u, 1u, cw_c1(w) - 1u, false);
  return w + (g == mn + 1u ? kC1 - kC2 : (g == mn + 2u ? kC2 : 0u));
}
__device__ __forceinline__ uint32_t cw_inc(uint32_t w, uint32_t g, bool& ok) {  // g -> g + 1
  const uint32_t mn = cw_mn(w), c1 = cw_c1(w);
  ok = true;
  if (g == mn && c1 == 1u) {
    ok = !cw_unk(w);
    return cw_make(mn + 1u, cw_c2(w) + 1u, 0u, true);
  }
  return w + (g == mn ? kC2 - kC1 : (g == mn + 1u ? 0u - kC2 : 0u));
}

// Summary of row u by one warp (lanes over its 32-bit words, two colours each, at most 3 words a
// lane for k <= 128): the current colour cu and the padding colours (key NONE) are skipped.
// Returns (non-tabu class word, tabu class word), the same in every lane.
template <int NWL, int EB>
__device__ __forceinline__ uint2 summarise_n(const uint32_t* row32, int kw, int cu, int lane) {
  constexpr unsigned NONE = Ent<EB>::NONE;
  constexpr int EPW = Ent<EB>::EPW;
  uint32_t x[NWL];
  unsigned nm = NONE, tm = NONE;
#pragma unroll
  for (int t = 0; t < NWL; ++t) {
    const int w = lane + 32 * t;
    uint32_t v = 0xFFFFFFFFu;
    if (w < kw) {
      v = row32[w];
      if (w == cu / EPW) v |= NONE << (EB * (cu % EPW));
    }
    x[t] = v;
#pragma unroll
    for (int h = 0; h < EPW; ++h) {
      const unsigned key = (v >> (EB * h)) & NONE;
      const bool fl = (v >> (EB * h + EB - 1)) & 1u;
      tm = fl ? min(tm, key) : tm;
      nm = fl ? nm : min(nm, key);
    }
  }
  const unsigned NM = __reduce_min_sync(FULL, nm), TM = __reduce_min_sync(FULL, tm);
  unsigned cn = 0, ct = 0;  // count at the minimum | count at the minimum + 1 << 16
#pragma unroll
  for (int t = 0; t < NWL; ++t) {
#pragma unroll
    for (int h = 0; h < EPW; ++h) {
      const unsigned key = (x[t] >> (EB * h)) & NONE;
      const bool fl = (x[t] >> (EB * h + EB - 1)) & 1u;
      const unsigned ref = fl ? TM : NM;
      const unsigned add = key == NONE ? 0u : ((key == ref ? 1u : 0u) + (key == ref + 1u ? 0x10000u : 0u));
      ct += fl ? add : 0u;
      cn += fl ? 0u : add;
    }
  }
  const unsigned CN = __reduce_add_sync(FULL, cn), CT = __reduce_add_sync(FULL, ct);
  return make_uint2(cw_make(NM == NONE ? kEmpty : NM, CN & 0xFFFFu, CN >> 16, false),
                    cw_make(TM == NONE ? kEmpty : TM, CT & 0xFFFFu, CT >> 16, false));
}
template <int EB>
__device__ __forceinline__ uint2 summarise(const uint32_t* row32, int kw, int cu, int lane) {
  if (kw <= 32) return summarise_n<1, EB>(row32, kw, cu, lane);
  if (kw <= 64) return summarise_n<2, EB>(row32, kw, cu, lane);
  return summarise_n<3, EB>(row32, kw, cu, lane);
}

// Best admissible move of a conflicting row from its class words (N, T): (delta, number of
// colours reaching it); count 0 when every colour is tabu and none is aspirated. A tabu colour is
// aspirated when f + gamma - g0 < best f, i.e. gamma < thrb + g0 with thrb = best f - f.
__device__ __forceinline__ void eval_row(const uint2 r, int gv, int thrb, int& d, int& c) {
  const unsigned nt = cw_mn(r.x);
  const unsigned tmn = cw_mn(r.y);
  const unsigned ta = (int)tmn < thrb + gv ? tmn : kEmpty;
  const unsigned adm = min(nt, ta);
  c = adm == kEmpty ? 0 : (int)((nt == adm ? cw_c1(r.x) : 0u) + (ta == adm ? cw_c1(r.y) : 0u));
  d = adm == kEmpty ? INT_MAX : (int)adm - gv;
}

__device__ __forceinline__ int incl_scan(int x, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x += t;
  }
  return x;
}

__device__ __forceinline__ void group_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ring entry: x = v | c << 16 | state << 24 (0 retired, 1 live, 2 expires before the next
// selection), y = iteration from which the pair is no longer tabu
__device__ __forceinline__ unsigned ent_v(uint32_t x) { return x & 0xFFFFu; }
__device__ __forceinline__ unsigned ent_c(uint32_t x) { return (x >> 16) & 0xFFu; }
__device__ __forceinline__ unsigned ent_st(uint32_t x) { return x >> 24; }

// threads of a CTA (all its groups): 768 (85 registers a thread) with 2 vertices a thread and with
// 4 vertices and u8 entries, 512 (128 registers) otherwise
__host__ __device__ constexpr int max_threads_for(int per, int eb) {
  return per <= 2 ? 768 : (eb == 8 && per == 4 ? 768 : 512);
}

// One individual by the W warps of one group (W at run time, PER vertices a thread at compile
// time). Thread t owns the vertices v0 = t PER .. v0 + PER - 1 and keeps their colours, their
// gamma[v][col v] and their two class words in registers; the gamma row of vertex v is q NT + t
// (slot q of its owner thread t), so that the threads of a warp touching their slot q address
// consecutive rows (distinct banks).
template <int PER, bool BSM, int EB>
__device__ void run_individual(const GroupArgs& a, const int W, int ind, uint8_t* gs, const uint32_t* bits,
                               int bar_id, uint2* far) {
  using ET = typename Ent<EB>::T;
  constexpr unsigned NONE = Ent<EB>::NONE, FLAG = Ent<EB>::FLAG;
  constexpr int EPW = Ent<EB>::EPW;
  const int NT = 32 * W;
  const int tid = threadIdx.x % NT, lane = tid & 31, warp = tid >> 5;
  // u16 pass after a u8 launch: only the individuals the u8 launch gave up (a uniform branch)
  if (a.redo_mode == 2 && a.redo[ind] == 0) return;
  const int n = a.n, k = a.k, ks = a.ks, kw = ks / EPW, words = a.words, R = a.R;
  const GroupLayout L = group_layout(n, k, W, PER, R, EB);
  ET* gam = (ET*)(gs + L.gam);
  uint32_t* csz = (uint32_t*)(gs + L.csz);
  uint8_t* colS = gs + L.col;
  uint8_t* bestS = gs + L.best;
  uint2* ring = (uint2*)(gs + L.ring);
  uint32_t* due = (uint32_t*)(gs + L.due);
  int4* red = (int4*)(gs + L.red);
  int32_t* sc = (int32_t*)(gs + L.sc);
  const int v0 = tid * PER;
  const uint32_t ind_id = a.ind_base + (uint32_t)ind;
  int16_t* gcol = a.col + (size_t)ind * n;
  const unsigned lt = (1u << lane) - 1u;
  auto bar = [&]() { group_bar(bar_id, NT); };
  auto rowof = [&](int v) -> ET* { return gam + ((v % PER) * NT + v / PER) * ks; };
  auto myrow = [&](int q) -> ET* { return gam + (q * NT + tid) * ks; };

  int colq[PER], g0q[PER];
  uint2 recq[PER];

  // ---- set-up: tables, start colouring, gamma, summaries, f ------------------------------------
  int bad = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    uint32_t* r32 = (uint32_t*)myrow(q);
    for (int w = 0; w < kw; ++w) {
      uint32_t x = 0u;
#pragma unroll
      for (int e = 0; e < EPW; ++e) x |= (EPW * w + e >= k) ? NONE << (EB * e) : 0u;
      r32[w] = x;
    }
    const int v = v0 + q;
    int c = 0;
    if (v < n) {
      const int cc = gcol[v];
      if (cc < 0 || cc >= k) bad = 1;
      else c = cc;
    }
    colq[q] = c;
    colS[v] = (uint8_t)c;
    bestS[v] = (uint8_t)c;
  }
  if (tid < SC_N) sc[tid] = 0;
  if (EB == 8)
    for (int c = tid; c < k; c += NT) csz[c] = 0u;
  bar();
  if (bad) sc[SC_BAD] = 1;
  if (EB == 8 && !bad) {  // class sizes of the start colouring
#pragma unroll
    for (int q = 0; q < PER; ++q)
      if (v0 + q < n) atomicAdd(csz + colq[q], 1u);
  }
  if (tid == 0) {
    sc[SC_REQ] = -1;
    sc[SC_REQ + 4] = -1;
    sc[SC_FARMIN] = -1;
  }
  bar();
  if (sc[SC_BAD]) {
    if (tid == 0) raise_status(a.status, DLM_EINVAL);
    bar();  // every thread has read the flag before the next individual clears it
    return;
  }
  if (EB == 8) {  // a start class above the u8 bound: the u16 pass searches this individual
    bool big = false;
    for (int c = lane; c < k; c += 32) big |= csz[c] > (uint32_t)kMaxClass8;
    if (__any_sync(FULL, big)) {
      bar();
      if (tid == 0 && a.redo_mode == 1) a.redo[ind] = 1;
      bar();
      return;
    }
  }
  int part = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int v = v0 + q;
    g0q[q] = 0;
    if (v < n) {
      const uint32_t* br = bits + v * words;
      ET* gr = myrow(q);
      for (int w = 0; w < words; ++w) {
        uint32_t m = br[w];
        while (m) {
          const int u = 32 * w + __ffs(m) - 1;
          m &= m - 1;
          gr[colS[u]]++;
        }
      }
      g0q[q] = gr[colq[q]];
      part += g0q[q];
    }
  }
  __syncwarp();
  // every row's summary, the warp's lanes in turn (the result of the reductions is in every lane)
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    for (int l = 0; l < 32; ++l) {
      const int cu = __shfl_sync(FULL, colq[q], l);
      const uint2 r = summarise<EB>((const uint32_t*)(gam + (q * NT + warp * 32 + l) * ks), kw, cu, lane);
      if (lane == l) recq[q] = r;
    }
  }
  part = __reduce_add_sync(FULL, part);
  if (lane == 0) red[warp].x = part;
  bar();
  int f = 0;
  for (int w = 0; w < W; ++w) f += red[w].x;
  f /= 2;
  bar();

  int best_f = f, moves = 0;
  int64_t w_rows = 0, w_deg = 0, w_resum = 0;
  // Philox blocks: lane l holds (r0, r1) of iteration (it & ~31) + l
  U4 rr = rng(a.seed, (uint32_t)lane, a.gen, ind_id, kTagTabu);
  uint32_t r0l = rr.x, r1l = rr.y;
  // the warp's vertex range, for the scanner's expiry lists (bit w: warp w has an expiring entry)
  const int wpv = 32 * PER;

  // selection from the class words in registers: per slot (delta, number of tied colours), the
  // thread's minimum and tie count (kept for the deciding warp), the warp's in red[warp]
  int dq[PER], cq[PER];
  int tmin = INT_MAX, tcnt = 0;
  auto select = [&]() {
    int nconf = 0;
    const int thrb = best_f - f;
    tmin = INT_MAX;
    tcnt = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      eval_row(recq[q], g0q[q], thrb, dq[q], cq[q]);
      cq[q] = g0q[q] > 0 ? cq[q] : 0;
      dq[q] = cq[q] > 0 ? dq[q] : INT_MAX;
      nconf += g0q[q] > 0 ? 1 : 0;
      const bool lo2 = dq[q] < tmin;
      tcnt = lo2 ? cq[q] : (dq[q] == tmin ? tcnt + cq[q] : tcnt);
      tmin = lo2 ? dq[q] : tmin;
    }
    const int wm = __reduce_min_sync(FULL, tmin);
    const int wc = (int)__reduce_add_sync(FULL, (wm != INT_MAX && tmin == wm) ? (unsigned)tcnt : 0u);
    const int wn = (int)__reduce_add_sync(FULL, (unsigned)nconf);
    if (lane == 0) red[warp] = make_int4(wm, wc, wn, 0);
  };

  select();
  int it = 0;
  const int iters = (int)a.iters;  // at most 2^31 - 1 (checked by the host)
  for (it = 0; it < iters; ++it) {
    if (f == 0) break;
    bar();
    uint32_t dmask = 0;  // own rows to summarise again
    // ---- (D) minimum delta, tie rank, move; ring maintenance ----------------------------------
    if ((it & 31) == 0 && it > 0) {
      rr = rng(a.seed, (uint32_t)(it + lane), a.gen, ind_id, kTagTabu);
      r0l = rr.x;
      r1l = rr.y;
    }
    const uint32_t r0 = __shfl_sync(FULL, r0l, it & 31), r1 = __shfl_sync(FULL, r1l, it & 31);
    // lanes 0..W-1 hold the warps' results: the minimum, the tie total, the warp holding the j-th
    // tie and the ties before it
    const int4 rw = lane < W ? red[lane] : make_int4(INT_MAX, 0, 0, 0);
    const int dstar = __reduce_min_sync(FULL, rw.x);
    const int xl = (dstar != INT_MAX && rw.x == dstar) ? rw.y : 0;
    int xincl = xl;
    for (int d = 1; d < W; d <<= 1) {  // inclusive scan over lanes 0..W-1 (W <= 16, a power of two)
      const int t = __shfl_up_sync(FULL, xincl, d);
      if (lane >= d) xincl += t;
    }
    const int T = __shfl_sync(FULL, xincl, W - 1);
    const uint32_t j = T > 0 ? below(r0, (uint32_t)T) : 0u;
    const unsigned dball = __ballot_sync(FULL, lane < W && xincl > (int)j);
    const int wdec = T > 0 ? __ffs(dball) - 1 : -1;
    const int wscan = wdec < 0 ? 0 : (wdec + 1 == W ? 0 : wdec + 1);
    if (warp == 0) {
      const int nc = (int)__reduce_add_sync(FULL, (unsigned)(lane < W ? rw.z : 0));
      if (lane == 0) w_rows += nc;
    }
    if (warp == wdec) {
      const int pre = __shfl_sync(FULL, xincl - xl, wdec);
      const int ct = tmin == dstar ? tcnt : 0;
      const unsigned hbal = __ballot_sync(FULL, ct > 0);
      int hl, lo_h;
      if ((hbal & (hbal - 1)) == 0) {  // one lane holds every tie of this warp
        hl = hbal ? __ffs(hbal) - 1 : 0;
        lo_h = pre;
      } else {
        const int incl = incl_scan(ct, lane);
        const int lo_l = pre + incl - ct;
        const unsigned hb = __ballot_sync(FULL, ct > 0 && (int)j >= lo_l && (int)j < lo_l + ct);
        hl = __ffs(hb) - 1;
        lo_h = __shfl_sync(FULL, lo_l, hl);
      }
      // the tied slot of lane hl, its rank among the row's tied colours, its colour and g0
      int hv = -1, hr = 0, hc = 0, hg = 0;
      {
        int jj = (int)j - lo_h;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          const bool tie = hv < 0 && dq[q] == dstar && cq[q] > 0;
          const bool take = tie && jj < cq[q];
          hv = take ? v0 + q : hv;
          hr = take ? jj : hr;
          hc = take ? colq[q] : hc;
          hg = take ? g0q[q] : hg;
          jj = (tie && !take) ? jj - cq[q] : jj;
        }
      }
      const int v = __shfl_sync(FULL, hv, hl);
      const int jj = __shfl_sync(FULL, hr, hl);
      const int colv = __shfl_sync(FULL, hc, hl);
      const int gv = __shfl_sync(FULL, hg, hl);
      int mc = -1;
      if (v >= 0) {
        const unsigned kmin = (unsigned)(dstar + gv);
        const int thr = best_f - f + gv;
        const uint32_t* row32 = (const uint32_t*)rowof(v);
        int rem = jj;
        for (int wb = 0; wb < kw && mc < 0; wb += 32) {
          const int w = wb + lane;
          bool mh[EPW];
          uint32_t x = 0u;
          if (w < kw) {
            x = row32[w];
            if (w == colv / EPW) x |= NONE << (EB * (colv % EPW));
          }
          int mine = 0;
#pragma unroll
          for (int h = 0; h < EPW; ++h) {
            const unsigned kh = (x >> (EB * h)) & NONE;
            mh[h] = w < kw && kh == kmin && (!((x >> (EB * h + EB - 1)) & 1u) || (int)kh < thr);
            mine += mh[h] ? 1 : 0;
          }
          // colours EPW w + h in colour order: the lane whose word holds the rem-th
          unsigned bh[EPW];
          int before = 0, total = 0;
#pragma unroll
          for (int h = 0; h < EPW; ++h) {
            bh[h] = __ballot_sync(FULL, mh[h]);
            before += __popc(bh[h] & lt);
            total += __popc(bh[h]);
          }
          const unsigned fb = __ballot_sync(FULL, rem >= before && rem < before + mine);
          if (fb) {
            const int wl = __ffs(fb) - 1;
            const unsigned lw = (1u << wl) - 1u;
            int r = rem;
#pragma unroll
            for (int h = 0; h < EPW; ++h) r -= __popc(bh[h] & lw);
            int pick = EPW - 1;
#pragma unroll
            for (int h = EPW - 1; h >= 0; --h) {  // the r-th set colour of word wl, in colour order
              int before_h = 0;
#pragma unroll
              for (int g = 0; g < h; ++g) before_h += (bh[g] >> wl) & 1u;
              if (((bh[h] >> wl) & 1u) && before_h == r) pick = h;
            }
            mc = EPW * (wb + wl) + pick;
          } else {
            rem -= total;
          }
        }
      }
      // u8 entries: a move that would grow a class beyond kMaxClass8 ends this search (the u16
      // pass repeats the individual from its start)
      const bool full = EB == 8 && v >= 0 && mc >= 0 && mc < k && csz[mc] >= (uint32_t)kMaxClass8;
      const bool good = v >= 0 && mc >= 0 && mc < k && !full;
      if (lane == 0) {
        if (good) {
          *(int4*)(sc + SC_MV) = make_int4(v, colv, mc, f + dstar);
          if (a.trace) reinterpret_cast<int4*>(a.trace)[(size_t)ind * iters + it] = make_int4(v, mc, dstar, T);
        } else if (full) {
          sc[SC_ABORT] = 1;
        } else {
          sc[SC_ERR] = 2;  // tie counts inconsistent with the row: refuse to move
        }
      }
      if (good && lane == hl) {  // the deciding lane owns the moved vertex: it updates the row now
        const int qs = v - v0;
        uint2 rc = recq[0];
#pragma unroll
        for (int q = 1; q < PER; ++q) rc = q == qs ? recq[q] : rc;
        ET* gr = rowof(v);
        const unsigned go = gr[colv], gn = gr[mc];
        const bool was = (go & FLAG) != 0;
        // alpha f (f after the move): 32-bit unsigned (the host bounds alpha_num * |E| below
        // 2^32), divided by alpha_den through its precomputed 64-bit reciprocal
        const uint32_t af = (uint32_t)a.an * (uint32_t)(f + dstar);
        const uint32_t tt = below(r1, a.L1) + (a.ad == 1 ? af : (uint32_t)__umul64hi((uint64_t)af, a.ad_recip));
        const bool tabu = tt > 0;
        gr[colv] = (ET)((go & NONE) | (tabu ? FLAG : 0u));
        if (EB == 8) {
          csz[colv] -= 1u;
          csz[mc] += 1u;
        }
        // the new colour leaves its class, the old one joins the tabu (or the free) class
        bool ok;
        if (gn & FLAG) rc.y = cw_rem(rc.y, gn & NONE, ok);
        else rc.x = cw_rem(rc.x, gn & NONE, ok);
        if (tabu) rc.y = cw_ins(rc.y, go & NONE);
        else rc.x = cw_ins(rc.x, go & NONE);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          if (q == qs) {
            recq[q] = rc;
            colq[q] = mc;
            g0q[q] = (int)(gn & NONE);
          }
        }
        dmask |= ok ? 0u : (1u << qs);
        *(int4*)(sc + SC_REQ + 4 * (it & 1)) =
            (tabu || was) ? make_int4(v, colv, (int32_t)tt, was ? 1 : 0) : make_int4(-1, 0, 0, 0);
      }
    }
    if (tid == 0) {
      if (T == 0 && a.trace) reinterpret_cast<int4*>(a.trace)[(size_t)ind * iters + it] = make_int4(-1, -1, 0, 0);
      // cancellation, polled every 1024 iterations: the search stops before this iteration's move
      if ((it & 1023) == 0 && a.cancel && *(volatile const int32_t*)a.cancel != 0) sc[SC_STOP] = 1;
    }
    if (warp == wscan) {
      int lo = sc[SC_LO], nins = sc[SC_NINS], far_n = sc[SC_FARN];
      uint32_t far_min = (uint32_t)sc[SC_FARMIN];
      // (a) retired entries at the front of the ring; far entries that expired at iteration it
      while (lo < nins) {
        const int s = lo + lane;
        const unsigned st = s < nins ? ent_st(ring[s & (R - 1)].x) : 1u;
        const unsigned live = __ballot_sync(FULL, st != 0);
        if (live) { lo += __ffs(live) - 1; break; }
        lo = min(lo + 32, nins);
      }
      if (far_n > 0 && far_min <= (uint32_t)it) {
        int keep = 0;
        uint32_t mn = 0xFFFFFFFFu;
        for (int b = 0; b < far_n; b += 32) {
          const int s = b + lane;
          uint2 e = make_uint2(0, 0);
          bool k2 = false;
          if (s < far_n) { e = far[s]; k2 = e.y > (uint32_t)it; }
          const unsigned kb = __ballot_sync(FULL, k2);
          __syncwarp();
          if (k2) { far[keep + __popc(kb & lt)] = e; mn = min(mn, e.y); }
          keep += __popc(kb);
          __syncwarp();
        }
        far_n = keep;
        far_min = __reduce_min_sync(FULL, mn);
      }
      // (b) the previous iteration's move: drop the pair's older entry when it was still tabu,
      // then insert the new one (tabu until it + tt)
      int32_t* req = sc + SC_REQ + 4 * ((it + 1) & 1);  // written by the previous iteration's decider
      const int rv = req[0];
      if (rv >= 0) {
        const int rc = req[1];
        const uint32_t rtt = (uint32_t)req[2];
        const uint32_t key = (uint32_t)rv | ((uint32_t)rc << 16);
        if (req[3]) {
          bool done = false;
          for (int b = lo; b < nins && !done; b += 32) {
            const int s = b + lane;
            const bool m = s < nins && (ring[s & (R - 1)].x & 0xFFFFFFu) == key && ent_st(ring[s & (R - 1)].x) == 1;
            const unsigned mb = __ballot_sync(FULL, m);
            if (m) ring[s & (R - 1)].x = key;  // state 0: retired
            done = mb != 0;
          }
          if (!done) {
            for (int b = 0; b < far_n && !done; b += 32) {
              const int s = b + lane;
              const bool m = s < far_n && far[s].x == key;
              const unsigned mb = __ballot_sync(FULL, m);
              if (mb) {
                const int sl = b + __ffs(mb) - 1;
                __syncwarp();
                if (lane == 0) { far[sl] = far[far_n - 1]; }
                __syncwarp();
                --far_n;
                done = true;
                uint32_t mn = 0xFFFFFFFFu;
                for (int b2 = lane; b2 < far_n; b2 += 32) mn = min(mn, far[b2].y);
                far_min = __reduce_min_sync(FULL, mn);
              }
            }
          }
        }
        if (rtt > 0) {
          const uint32_t e = (uint32_t)it + rtt;
          if (rtt < (uint32_t)R && nins - lo < R) {
            if (lane == 0) ring[nins & (R - 1)] = make_uint2(key | (1u << 24), e);
            ++nins;
          } else if (far_n < a.far_cap) {
            if (lane == 0) far[far_n] = make_uint2(key, e);
            ++far_n;
            far_min = min(far_min, e);
          } else if (lane == 0) {
            sc[SC_ERR] = 1;  // more long tenures than the far list holds
          }
        }
        __syncwarp();
        if (lane == 0) req[0] = -1;
      }
      // (c) entries that expire before the next selection (no longer tabu at it + 1), and which
      // warps own their rows
      int dcnt = 0;
      unsigned dwarps = 0;
      for (int b = lo; b < nins; b += 32) {
        const int s = b + lane;
        bool d = false;
        uint32_t x = 0;
        if (s < nins) {
          const uint2 e = ring[s & (R - 1)];
          x = e.x;
          d = ent_st(x) == 1 && e.y == (uint32_t)(it + 1);
        }
        const unsigned db = __ballot_sync(FULL, d);
        if (d) {
          const int pos = dcnt + __popc(db & lt);
          if (pos < kDueCap) due[pos] = (uint32_t)(s & (R - 1));
          ring[s & (R - 1)].x = (x & 0xFFFFFFu) | (2u << 24);
        }
        dwarps |= __reduce_or_sync(FULL, d ? 1u << (ent_v(x) / wpv) : 0u);
        dcnt += __popc(db);
      }
      const bool fdue = far_n > 0 && far_min == (uint32_t)(it + 1);
      __syncwarp();
      if (lane == 0) {
        *(int4*)(sc + SC_DUE) = make_int4(min(dcnt, 0x3FFF) | (fdue ? 1 << 14 : 0) | (int)(dwarps << 16), lo, nins, far_n);
        sc[SC_FARMIN] = (int32_t)far_min;
      }
    }
    bar();
    // ---- (U) the move, expiries, neighbours, summaries, next selection ------------------------
    const int4 A = *(const int4*)(sc + SC_MV);
    const int4 B = *(const int4*)(sc + SC_DUE);
    const int4 C = *(const int4*)(sc + SC_STOP);
    if (C.x | C.y) break;
    if (EB == 8 && sc[SC_ABORT]) break;
    int mv = -1, old = -1, nw = -1;
    bool improved = false;
    if (T > 0) {
      mv = A.x;
      old = A.y;
      nw = A.z;
      f = A.w;
      ++moves;
      improved = f < best_f;
      best_f = improved ? f : best_f;
    }
    // expiring entries of this thread's rows, in list order (several may touch one row)
    auto expire = [&](int v, int c) {
      if (v == mv && c == old) return;
      const int qs = v - v0;
      ET* ge = myrow(qs) + c;
      const unsigned g = *ge;
      if (!(g & FLAG)) return;
      *ge = (ET)(g & NONE);
      int cu = colq[0];
      uint2 rc = recq[0];
#pragma unroll
      for (int q = 1; q < PER; ++q) {
        cu = q == qs ? colq[q] : cu;
        rc = q == qs ? recq[q] : rc;
      }
      if (c == cu) return;
      bool ok;
      rc.y = cw_rem(rc.y, g & NONE, ok);
      rc.x = cw_ins(rc.x, g & NONE);
#pragma unroll
      for (int q = 0; q < PER; ++q) recq[q] = q == qs ? rc : recq[q];
      dmask |= ok ? 0u : (1u << qs);
    };
    if ((B.x >> (16 + warp)) & 1) {
      const int dcnt = B.x & 0x3FFF;
      if (dcnt < kDueCap) {
        for (int i = 0; i < dcnt; ++i) {
          const int s = (int)due[i];
          const uint32_t x = ring[s].x;
          const int ev = (int)ent_v(x);
          if (ev >= v0 && ev < v0 + PER) {
            expire(ev, (int)ent_c(x));
            ring[s].x = x & 0xFFFFFFu;
          }
        }
      } else {
        for (int s = B.y; s < B.z; ++s) {
          const uint32_t x = ring[s & (R - 1)].x;
          const int ev = (int)ent_v(x);
          if (ent_st(x) == 2 && ev >= v0 && ev < v0 + PER) {
            expire(ev, (int)ent_c(x));
            ring[s & (R - 1)].x = x & 0xFFFFFFu;
          }
        }
      }
    }
    if ((B.x >> 14) & 1) {  // far entries expire too
      for (int s = 0; s < B.w; ++s) {
        const uint2 e = far[s];
        const int ev = (int)ent_v(e.x);
        if (e.y == (uint32_t)(it + 1) && ev >= v0 && ev < v0 + PER) expire(ev, (int)ent_c(e.x));
      }
    }
    // gamma of this thread's neighbours of the moved vertex: every load first, then the updates
    if (mv >= 0) {
      uint32_t m = 0;
      if (v0 < n) {
        const uint32_t* br = bits + mv * words;
        const int w0 = v0 >> 5, sh = v0 & 31;
        const uint32_t lw = br[w0];
        const uint32_t hw = (sh + PER > 32 && w0 + 1 < words) ? br[w0 + 1] : 0u;
        constexpr uint32_t kPerMask = PER >= 32 ? 0xFFFFFFFFu : ((1u << (PER & 31)) - 1u);
        m = __funnelshift_r(lw, hw, sh) & kPerMask;
      }
      w_deg += __popc(m);
      // branch-free over the thread's slots, so that their chains overlap: every slot loads and
      // stores its two entries (a non-neighbour stores them back unchanged; rows belong to their
      // owner thread, and old != nw) and its class words take the adjusted value only when the
      // vertex is a neighbour
      unsigned go[PER], gn[PER];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const ET* gr = myrow(q);
        go[q] = gr[old];
        gn[q] = gr[nw];
      }
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const unsigned nb = (m >> q) & 1u;
        ET* gr = myrow(q);
        gr[old] = (ET)(go[q] - nb);
        gr[nw] = (ET)(gn[q] + nb);
        const bool fo = (go[q] & FLAG) != 0, fn = (gn[q] & FLAG) != 0;
        const bool is_old = colq[q] == old, is_new = colq[q] == nw;
        // the old colour's key drops by one, the new colour's rises by one (when neither is the
        // vertex's own colour, whose gamma is g0)
        const uint32_t wo = cw_dec(fo ? recq[q].y : recq[q].x, go[q] & NONE);
        const bool ao = nb && !is_old;
        recq[q].y = (ao && fo) ? wo : recq[q].y;
        recq[q].x = (ao && !fo) ? wo : recq[q].x;
        bool ok = true;
        const uint32_t wn = cw_inc(fn ? recq[q].y : recq[q].x, gn[q] & NONE, ok);
        const bool an = nb && !is_new;
        recq[q].y = (an && fn) ? wn : recq[q].y;
        recq[q].x = (an && !fn) ? wn : recq[q].x;
        const int g0n = is_old ? (int)(go[q] & NONE) - 1 : (is_new ? (int)(gn[q] & NONE) + 1 : g0q[q]);
        g0q[q] = nb ? g0n : g0q[q];
        dmask |= (!nb || ok || is_new) ? 0u : (1u << q);
      }
    }
    // rows whose summary could not be adjusted, summarised again by the warp (lanes over colours)
    if (__any_sync(FULL, dmask != 0)) {
      __syncwarp();
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        for (unsigned pend = __ballot_sync(FULL, (dmask >> q) & 1u); pend; pend &= pend - 1) {
          const int l = __ffs(pend) - 1;
          const int cu = __shfl_sync(FULL, colq[q], l);
          const uint2 r = summarise<EB>((const uint32_t*)(gam + (q * NT + warp * 32 + l) * ks), kw, cu, lane);
          if (lane == l) recq[q] = r;
          if (lane == 0) ++w_resum;
        }
      }
    }
    if (improved) {
#pragma unroll
      for (int q = 0; q < PER; ++q) bestS[v0 + q] = (uint8_t)colq[q];
    }
    select();  // the next iteration's selection
  }
  // ---- results ---------------------------------------------------------------------------------
  const int err = sc[SC_ERR], stop = sc[SC_STOP];
  const int gave_up = EB == 8 ? sc[SC_ABORT] : 0;
  long long* wk = (long long*)(gs + L.red);
  bar();  // every warp has left the loop: red[] is free
  if (gave_up) {  // no result: the u16 pass searches this individual from its start colouring
    if (tid == 0 && a.redo_mode == 1) a.redo[ind] = 1;
    bar();
    return;
  }
  {
    long long d = w_deg;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(FULL, d, o);
    if (lane == 0) {
      wk[4 * warp + 0] = w_rows;
      wk[4 * warp + 1] = d;
      wk[4 * warp + 2] = w_resum;
    }
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int v = v0 + q;
    if (v < n) gcol[v] = (int16_t)bestS[v];
  }
  bar();
  if (tid == 0) {
    if (err) raise_status(a.status, err == 1 ? DLM_EUNSUPPORTED : DLM_ECUDA);
    if (stop) raise_status(a.status, DLM_ECANCELLED);
    a.best_f[ind] = best_f;
    if (a.moves) a.moves[ind] = moves;
    if (a.work) {
      long long s0 = 0, s1 = 0, s2 = 0;
      for (int w = 0; w < W; ++w) { s0 += wk[4 * w]; s1 += wk[4 * w + 1]; s2 += wk[4 * w + 2]; }
      a.work[3 * (size_t)ind + 0] = s0;
      a.work[3 * (size_t)ind + 1] = s1;
      a.work[3 * (size_t)ind + 2] = s2;
    }
  }
  bar();  // shared memory is reused by the next individual
}

template <int PER, bool BSM, int EB>
__global__ void __launch_bounds__(max_threads_for(PER, EB)) tabucol_group_kernel(GroupArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int G = a.G, W = a.W;
  const int grp = threadIdx.x / (32 * W);
  const uint32_t* bits = a.bits;
  if (BSM) {  // the graph's bit rows, shared by the CTA's individuals
    uint32_t* bs = (uint32_t*)smem;
    const int nw = a.n * a.words;
    const uint4* src = (const uint4*)a.bits;
    uint4* dst = (uint4*)bs;
    const int n4 = nw / 4;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = src[i];
    for (int i = 4 * n4 + threadIdx.x; i < nw; i += blockDim.x) bs[i] = a.bits[i];
    if (threadIdx.x == 0) bs[nw] = 0u;
    __syncthreads();
    bits = bs;
  }
  uint8_t* gs = smem + a.bits_bytes + (size_t)grp * a.group_bytes;
  // slots group-major: a last, partial round of individuals spreads over every CTA (fewer groups
  // per SM run each faster) instead of filling the first CTAs
  const int slot = grp * gridDim.x + blockIdx.x;
  uint2* far = a.far ? a.far + (size_t)slot * (size_t)a.far_cap : nullptr;
  for (int i = slot; i < a.pop; i += gridDim.x * G) run_individual<PER, BSM, EB>(a, W, i, gs, bits, 1 + grp, far);
}

template <int PER, bool BSM, int EB>
static dlm_status launch_one(dlm_ctx* ctx, GroupArgs a, int grid, size_t smem) {
  auto kfn = tabucol_group_kernel<PER, BSM, EB>;
  DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  kfn<<<grid, 32 * a.W * a.G, smem, ctx->stream>>>(a);
  return launch_check(ctx, "tabucol_group_kernel");
}

template <int PER, bool BSM, int EB>
static int occupancy_one(int threads, size_t smem) {
  int per_sm = 0;
  cudaError_t e = cudaFuncSetAttribute(tabucol_group_kernel<PER, BSM, EB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_group_kernel<PER, BSM, EB>, threads, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return per_sm < 1 ? 1 : per_sm;
}

}  // namespace tg

using namespace tg;

bool group_plan(int n, int k, int words, int W, size_t optin, int pop, int num_sms, int ring_force, int eb,
                GroupPlan* out) {
  if (W != 1 && W != 2 && W != 4 && W != 8 && W != 16) return false;
  if (eb != 8 && eb != 16) return false;
  const int NT = 32 * W;
  int per = 2;
  while (per < 8 && per * NT < n) per *= 2;  // a power of two up to 8: each value is its own kernel
  if (per * NT < n) return false;
  if (eb == 8 && per > 4) return false;  // u8 entries: kernels for 2 and 4 vertices a thread
  const size_t bits_bytes = a16(((size_t)n * words + 1) * 4);
  const int gmax_pop = std::max(1, (pop + num_sms - 1) / std::max(1, num_sms));
  const int gmax = std::min(std::min(max_threads_for(per, eb) / NT, 8), gmax_pop);
  auto ring_for = [&](int G, bool bsm, int* R) -> bool {
    for (int r = ring_force > 0 ? ring_force : 8192; r >= 64; r >>= 1) {
      const size_t tot = (size_t)G * group_layout(n, k, W, per, r, eb).total + (bsm ? bits_bytes : 0);
      if (tot <= optin) { *R = r; return true; }
      if (ring_force > 0) return false;
    }
    return false;
  };
  for (int G = gmax; G >= 1; --G) {
    for (int b = 0; b < 2; ++b) {
      const bool bsm = b == 0;
      int R = 0;
      if (ring_for(G, bsm, &R) && (R >= 512 || ring_force > 0 || (G == 1 && !bsm))) {
        out->W = W; out->G = G; out->R = R; out->per = per; out->bsm = bsm; out->eb = eb;
        out->group_bytes = group_layout(n, k, W, per, R, eb).total;
        out->bits_bytes = bsm ? bits_bytes : 0;
        out->smem = (size_t)G * out->group_bytes + out->bits_bytes;
        return true;
      }
    }
  }
  return false;
}

int group_ctas_per_sm(const GroupPlan& P) {
  const int threads = 32 * P.W * P.G;
  if (P.eb == 8) {
    if (P.per == 2) return P.bsm ? occupancy_one<2, true, 8>(threads, P.smem) : occupancy_one<2, false, 8>(threads, P.smem);
    return P.bsm ? occupancy_one<4, true, 8>(threads, P.smem) : occupancy_one<4, false, 8>(threads, P.smem);
  }
  switch (P.per) {
    case 2: return P.bsm ? occupancy_one<2, true, 16>(threads, P.smem) : occupancy_one<2, false, 16>(threads, P.smem);
    case 4: return P.bsm ? occupancy_one<4, true, 16>(threads, P.smem) : occupancy_one<4, false, 16>(threads, P.smem);
    default: return P.bsm ? occupancy_one<8, true, 16>(threads, P.smem) : occupancy_one<8, false, 16>(threads, P.smem);
  }
}

int group_grid(dlm_ctx* ctx, const GroupPlan& P, int pop) {
  const int blocks = (pop + P.G - 1) / P.G;
  return std::max(1, std::min(blocks, group_ctas_per_sm(P) * ctx->num_sms));
}

template <int PER, int EB>
static dlm_status launch_per(dlm_ctx* ctx, const GroupArgs& a, const GroupPlan& P, uint2* far_mem) {
  const int grid = group_grid(ctx, P, a.pop);
  GroupArgs b = a;
  b.far = b.far_cap > 0 ? far_mem : nullptr;
  return P.bsm ? launch_one<PER, true, EB>(ctx, b, grid, P.smem) : launch_one<PER, false, EB>(ctx, b, grid, P.smem);
}

// far list: tabu entries whose tenure does not fit the ring. A pair holds at most one live entry,
// at most one entry is made per iteration and a tenure never exceeds L_max + alpha |E|, so
// n (k - 1) + 1 entries, the budget + 1 and L_max + alpha |E| + 1 each bound what one search
// keeps there at once; 0 when every tenure fits the ring
int64_t group_far_cap(const dlm_graph* g, int32_t k, int64_t iters, dlm_tenure tenure, const GroupPlan& P) {
  const uint64_t tt_max = (uint64_t)tenure.L_max + ((uint64_t)tenure.alpha_num * (uint64_t)g->m) / tenure.alpha_den;
  if (tt_max < (uint64_t)P.R) return 0;
  int64_t far_cap = std::min<int64_t>((int64_t)g->n * (k - 1) + 1, iters + 1);
  return std::min<int64_t>(far_cap, (int64_t)tt_max + 1);
}

static size_t far_bytes_of(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int64_t iters, dlm_tenure tenure,
                           const GroupPlan& P) {
  return (size_t)group_grid(ctx, P, pop) * P.G * (size_t)group_far_cap(g, k, iters, tenure, P) * sizeof(uint2);
}

// the u16 plan that repeats the individuals a u8 launch gives up
static bool fallback_plan(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, const GroupPlan& P, GroupPlan* F) {
  return group_plan(g->n, k, g->words, P.W, ctx->smem_optin, pop, ctx->num_sms, 0, 16, F);
}

size_t group_far_bytes(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int64_t iters, dlm_tenure tenure,
                       const GroupPlan& P) {
  size_t far = far_bytes_of(ctx, g, k, pop, iters, tenure, P);
  if (P.eb == 8) {
    GroupPlan F;
    if (fallback_plan(ctx, g, k, pop, P, &F)) far = std::max(far, far_bytes_of(ctx, g, k, pop, iters, tenure, F));
    far = a16(far) + a16((size_t)pop * 4);  // then the flags of the individuals to search again
  }
  return far;
}

dlm_status tabucol_group_launch(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                                uint32_t generation, uint32_t ind_base, const GroupPlan& P, int32_t* trace,
                                int64_t* work, void* far_mem, int32_t** redo_out) {
  GroupArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = g->n; a.k = k; a.ks = P.eb == 8 ? group_row_stride8(k) : group_row_stride(k); a.words = g->words; a.pop = pop;
  a.G = P.G; a.R = P.R;
  a.W = P.W; a.per = P.per;
  a.bits = g->d_bits; a.col = col; a.best_f = best_f; a.moves = moves; a.trace = trace; a.work = work;
  a.iters = iters; a.ind_base = ind_base;
  a.L1 = (uint32_t)tenure.L_max + 1u; a.an = tenure.alpha_num; a.ad = tenure.alpha_den;
  a.seed = seed; a.gen = generation; a.status = ctx->d_status; a.cancel = ctx->cancel;
  a.group_bytes = P.group_bytes; a.bits_bytes = P.bits_bytes;
  // floor(x / alpha_den) for x < 2^32 as the high word of x * ceil(2^64 / alpha_den) (division by
  // an invariant integer through a multiplication, Granlund and Montgomery 1994)
  a.ad_recip = tenure.alpha_den >= 2 ? ~0ull / (uint64_t)tenure.alpha_den + 1ull : 0ull;
  a.far_cap = (int32_t)group_far_cap(g, k, iters, tenure, P);
  uint8_t* scratch = (uint8_t*)far_mem;
  const size_t need = group_far_bytes(ctx, g, k, pop, iters, tenure, P);
  if (!scratch && need) DLM_TRY(ctx_workspace(ctx, need, (void**)&scratch));
  if (P.eb == 16) {
    switch (P.per) {
      case 2: return launch_per<2, 16>(ctx, a, P, (uint2*)scratch);
      case 4: return launch_per<4, 16>(ctx, a, P, (uint2*)scratch);
      default: return launch_per<8, 16>(ctx, a, P, (uint2*)scratch);
    }
  }
  // u8 entries, then a u16 pass over the individuals the u8 launch gave up (their start colourings
  // are untouched; the same random streams give the same searches)
  GroupPlan F;
  const bool have_f = fallback_plan(ctx, g, k, pop, P, &F);
  if (!have_f && !redo_out) return fail(ctx, DLM_EUNSUPPORTED, "tabucol: no u16 plan for the fallback");
  if (!have_f) F = P;  // the caller searches the flagged individuals (one-individual-per-CTA kernel)
  const size_t far16 = std::max(far_bytes_of(ctx, g, k, pop, iters, tenure, P), far_bytes_of(ctx, g, k, pop, iters, tenure, F));
  int32_t* redo = (int32_t*)(scratch + a16(far16));
  DLM_CUDA(ctx, cudaMemsetAsync(redo, 0, (size_t)pop * 4, ctx->stream));
  a.redo = redo;
  a.redo_mode = 1;
  if (P.per == 2) DLM_TRY((launch_per<2, 8>(ctx, a, P, (uint2*)scratch)));
  else DLM_TRY((launch_per<4, 8>(ctx, a, P, (uint2*)scratch)));
  if (!have_f) {
    *redo_out = redo;
    return DLM_OK;
  }
  GroupArgs b = a;
  b.ks = group_row_stride(k);
  b.G = F.G; b.R = F.R; b.W = F.W; b.per = F.per;
  b.group_bytes = F.group_bytes; b.bits_bytes = F.bits_bytes;
  b.far_cap = (int32_t)group_far_cap(g, k, iters, tenure, F);
  b.redo_mode = 2;
  switch (F.per) {
    case 2: return launch_per<2, 16>(ctx, b, F, (uint2*)scratch);
    case 4: return launch_per<4, 16>(ctx, b, F, (uint2*)scratch);
    default: return launch_per<8, 16>(ctx, b, F, (uint2*)scratch);
  }
}

}  // namespace dlm
