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
constexpr unsigned kNone = 0x7FFFu;  // key of an absent colour, minimum of an empty class
constexpr unsigned kFlag = 0x8000u;  // tabu flag of a gamma entry
constexpr uint8_t kUnk = 0xFF;       // count at minimum + 1 not known
constexpr int kDueCap = 32;          // expiring ring entries listed per iteration (more: window scan)

// sc[] slots of a group (shared memory)
enum { SC_MV = 0, SC_OLD, SC_NEW, SC_F, SC_STOP, SC_ERR, SC_LO, SC_NINS, SC_DUE, SC_FARDUE, SC_FARN,
       SC_REQV, SC_REQC, SC_REQTT, SC_REQWAS, SC_BAD, SC_N = 32 };

struct Rec {
  uint16_t nmin, tmin;   // smallest key among the non-tabu / tabu colours (kNone: class empty)
  uint8_t ncnt, ncnt2;   // colours at nmin, at nmin + 1 (kUnk: unknown)
  uint8_t tcnt, tcnt2;
};
static_assert(sizeof(Rec) == 8, "a row summary is 8 bytes");

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline GroupLayout group_layout(int n, int k, int W, int per, int R) {
  GroupLayout L;
  const size_t nv = (size_t)32 * W * per;
  const int ks = group_row_stride(k);
  size_t o = 0;
  L.gam = o; o += a16((size_t)n * ks * 2);
  L.rec = o; o += a16(nv * 8);
  L.g0 = o; o += a16(nv * 2);
  L.col = o; o += a16(nv);
  L.best = o; o += a16(nv);
  L.dirty = o; o += a16(nv);
  L.nb = o; o += a16(nv * 2);
  L.ring = o; o += a16((size_t)R * 8);
  L.due = o; o += a16((size_t)kDueCap * 4);
  L.red = o; o += a16((size_t)W * 32);  // per warp: selection (int4), at the end 3 work counters (int64)
  L.sc = o; o += SC_N * 4;
  L.total = a16(o);
  return L;
}

// ---- class summaries: insert / remove / decrement / increment one colour's key ---------------
// A class (the non-tabu or the tabu colours of a row) keeps its minimum key mn, the number of
// colours at mn (c1) and at mn + 1 (c2, or kUnk). Each operation returns false when the new
// minimum cannot be derived (the row is then summarised again from its gamma entries).
__device__ __forceinline__ void cls_ins(uint16_t& mn, uint8_t& c1, uint8_t& c2, unsigned g) {
  if (g + 1u < mn) { mn = (uint16_t)g; c1 = 1; c2 = 0; }
  else if (g + 1u == mn) { c2 = c1; mn = (uint16_t)g; c1 = 1; }
  else if (g == mn) { ++c1; }
  else if (g == mn + 1u) { if (c2 != kUnk) ++c2; }
}
__device__ __forceinline__ bool cls_rem(uint16_t& mn, uint8_t& c1, uint8_t& c2, unsigned g) {
  if (g == mn) {
    if (c1 > 1) { --c1; return true; }
    if (c2 != kUnk && c2 > 0) { mn = (uint16_t)(mn + 1u); c1 = c2; c2 = kUnk; return true; }
    return false;
  }
  if (g == mn + 1u && c2 != kUnk) --c2;
  return true;
}
__device__ __forceinline__ void cls_dec(uint16_t& mn, uint8_t& c1, uint8_t& c2, unsigned g) {  // g -> g - 1
  if (g == mn) { c2 = (uint8_t)(c1 - 1); mn = (uint16_t)(g - 1u); c1 = 1; }
  else if (g == mn + 1u) { ++c1; if (c2 != kUnk) --c2; }
  else if (g == mn + 2u) { if (c2 != kUnk) ++c2; }
}
__device__ __forceinline__ bool cls_inc(uint16_t& mn, uint8_t& c1, uint8_t& c2, unsigned g) {  // g -> g + 1
  if (g == mn) {
    if (c1 > 1) { --c1; if (c2 != kUnk) ++c2; return true; }
    if (c2 == kUnk) return false;
    mn = (uint16_t)(mn + 1u); c1 = (uint8_t)(c2 + 1); c2 = kUnk;
    return true;
  }
  if (g == mn + 1u && c2 != kUnk) --c2;
  return true;
}

// Summary of row u by one warp (lanes over its 32-bit words, two colours each, at most 3 words a
// lane for k <= 128): the current colour cu and the padding colours (key kNone) are skipped.
__device__ __forceinline__ Rec summarise(const uint32_t* row32, int kw, int cu, int lane) {
  uint32_t x[3];
  unsigned nm = kNone, tm = kNone;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int w = lane + 32 * t;
    uint32_t v = 0xFFFFFFFFu;
    if (w < kw) {
      v = row32[w];
      if (w == (cu >> 1)) v |= (cu & 1) ? (kNone << 16) : kNone;
    }
    x[t] = v;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned key = (v >> (16 * h)) & kNone, fl = (v >> (16 * h + 15)) & 1u;
      if (key != kNone) {
        if (fl) tm = min(tm, key); else nm = min(nm, key);
      }
    }
  }
  const unsigned NM = __reduce_min_sync(FULL, nm), TM = __reduce_min_sync(FULL, tm);
  unsigned cn = 0, ct = 0;  // count at the minimum | count at the minimum + 1 << 16
#pragma unroll
  for (int t = 0; t < 3; ++t) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned key = (x[t] >> (16 * h)) & kNone, fl = (x[t] >> (16 * h + 15)) & 1u;
      if (key != kNone) {
        if (fl) ct += (key == TM ? 1u : 0u) + (key == TM + 1u ? 0x10000u : 0u);
        else cn += (key == NM ? 1u : 0u) + (key == NM + 1u ? 0x10000u : 0u);
      }
    }
  }
  const unsigned CN = __reduce_add_sync(FULL, cn), CT = __reduce_add_sync(FULL, ct);
  Rec r;
  r.nmin = (uint16_t)NM; r.tmin = (uint16_t)TM;
  r.ncnt = (uint8_t)(CN & 0xFFFFu); r.ncnt2 = (uint8_t)(CN >> 16);
  r.tcnt = (uint8_t)(CT & 0xFFFFu); r.tcnt2 = (uint8_t)(CT >> 16);
  return r;
}

// Best admissible move of a conflicting row from its summary: (delta, number of colours reaching
// it); count 0 when every colour is tabu and none is aspirated. A tabu colour is aspirated when
// f + gamma - g0 < best f, i.e. gamma < thrb + g0 with thrb = best f - f.
__device__ __forceinline__ void eval_row(const Rec r, int gv, int thrb, int& d, int& c) {
  const unsigned nt = r.ncnt ? (unsigned)r.nmin : kNone;
  const unsigned ta = (r.tcnt && (int)r.tmin < thrb + gv) ? (unsigned)r.tmin : kNone;
  const unsigned adm = min(nt, ta);
  if (adm == kNone) { c = 0; d = INT_MAX; return; }
  c = (nt == adm ? r.ncnt : 0) + (ta == adm ? r.tcnt : 0);
  d = (int)adm - gv;
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

template <int W>
struct GroupMax { static constexpr int value = W >= 16 ? 1 : (W == 8 ? 2 : (W == 4 ? 4 : 8)); };

template <int W, bool BSM>
__device__ void run_individual(const GroupArgs& a, int ind, uint8_t* gs, const uint32_t* bits, int bar_id,
                               uint2* far) {
  constexpr int NT = 32 * W;
  const int tid = threadIdx.x % NT, lane = tid & 31, warp = tid >> 5;
  const int n = a.n, k = a.k, ks = a.ks, kw = ks >> 1, words = a.words, per = a.per, R = a.R;
  const GroupLayout L = group_layout(n, k, W, per, R);
  uint16_t* gam = (uint16_t*)(gs + L.gam);
  Rec* rec = (Rec*)(gs + L.rec);
  uint16_t* g0 = (uint16_t*)(gs + L.g0);
  uint8_t* colS = gs + L.col;
  uint8_t* bestS = gs + L.best;
  uint8_t* dirty = gs + L.dirty;
  uint16_t* nbw = (uint16_t*)(gs + L.nb) + (size_t)warp * 32 * per;  // this warp's neighbour list
  uint2* ring = (uint2*)(gs + L.ring);
  uint32_t* due = (uint32_t*)(gs + L.due);
  int4* red = (int4*)(gs + L.red);
  int32_t* sc = (int32_t*)(gs + L.sc);
  const int v0 = tid * per;                           // this thread's vertices [v0, v0 + per)
  const int wv0 = warp * 32 * per, wv1 = wv0 + 32 * per;  // this warp's
  const uint32_t ind_id = a.ind_base + (uint32_t)ind;
  int16_t* gcol = a.col + (size_t)ind * n;
  const unsigned lt = (1u << lane) - 1u;
  auto bar = [&]() { group_bar(bar_id, NT); };

  // ---- set-up: tables, start colouring, gamma, summaries, f ------------------------------------
  for (int i = tid; i < n * kw; i += NT) {
    const int v = i / kw, w = i - v * kw, c0 = 2 * w;
    ((uint32_t*)gam)[i] = (c0 >= k ? kNone : 0u) | (c0 + 1 >= k ? (kNone << 16) : 0u);
  }
  if (tid < SC_N) sc[tid] = 0;
  int bad = 0;
  for (int q = 0; q < per; ++q) {
    const int v = v0 + q;
    uint8_t c = 0;
    if (v < n) {
      const int cc = gcol[v];
      if (cc < 0 || cc >= k) bad = 1;
      else c = (uint8_t)cc;
    }
    colS[v] = c;
    bestS[v] = c;
    dirty[v] = 0;
    g0[v] = 0;
  }
  bar();
  if (bad) sc[SC_BAD] = 1;
  if (tid == 0) sc[SC_REQV] = -1;
  bar();
  if (sc[SC_BAD]) {
    if (tid == 0) raise_status(a.status, DLM_EINVAL);
    bar();  // every thread has read the flag before the next individual clears it
    return;
  }
  for (int v = tid; v < n; v += NT) {
    const uint32_t* br = bits + (size_t)v * words;
    uint16_t* gr = gam + (size_t)v * ks;
    for (int w = 0; w < words; ++w) {
      uint32_t m = br[w];
      while (m) {
        const int u = 32 * w + __ffs(m) - 1;
        m &= m - 1;
        gr[colS[u]]++;
      }
    }
  }
  bar();
  {
    int part = 0;
    for (int q = 0; q < per; ++q) {
      const int v = v0 + q;
      if (v < n) {
        const int g = gam[(size_t)v * ks + colS[v]];
        g0[v] = (uint16_t)g;
        part += g;
      }
    }
    part = __reduce_add_sync(FULL, part);
    if (lane == 0) red[warp].x = part;
  }
  for (int u = warp; u < n; u += W) {
    const Rec r = summarise((const uint32_t*)(gam + (size_t)u * ks), kw, colS[u], lane);
    if (lane == 0) rec[u] = r;
  }
  bar();
  int f = 0;
  for (int w = 0; w < W; ++w) f += red[w].x;
  f /= 2;
  bar();

  int best_f = f, moves = 0;
  int64_t w_rows = 0, w_deg = 0, w_resum = 0;
  // ring maintenance state (used by warp W - 1 only; identical in its lanes)
  int lo = 0, nins = 0, far_n = 0;
  uint32_t far_min = 0xFFFFFFFFu;
  // Philox blocks: lane l holds (r0, r1) of iteration (it & ~31) + l
  U4 rr = rng(a.seed, (uint32_t)lane, a.gen, ind_id, kTagTabu);
  uint32_t r0l = rr.x, r1l = rr.y;

  // selection from the summaries of this thread's conflicting vertices; the thread's minimum and
  // tie count stay in registers (the deciding warp needs them), the warp's go to red[warp]
  int tmin = INT_MAX, tcnt = 0;
  auto select = [&]() {
    int nconf = 0;
    tmin = INT_MAX;
    tcnt = 0;
    const int thrb = best_f - f;
    for (int q = 0; q < per; q += 2) {
      const uint32_t gg = *(const uint32_t*)(g0 + v0 + q);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gv = (int)((gg >> (16 * h)) & 0xFFFFu);
        if (gv > 0) {
          ++nconf;
          int d, c;
          eval_row(rec[v0 + q + h], gv, thrb, d, c);
          if (c) {
            if (d < tmin) { tmin = d; tcnt = c; }
            else if (d == tmin) tcnt += c;
          }
        }
      }
    }
    const int wm = __reduce_min_sync(FULL, tmin);
    const int wc = (int)__reduce_add_sync(FULL, (wm != INT_MAX && tmin == wm) ? (unsigned)tcnt : 0u);
    const int wn = (int)__reduce_add_sync(FULL, (unsigned)nconf);
    if (lane == 0) red[warp] = make_int4(wm, wc, wn, 0);
  };

  // expiry of the tabu entry (v, c) before the next selection, unless this iteration's move has
  // just made the same pair tabu again; called by one lane at a time of the warp owning v
  auto expire = [&](int v, int c, int mv, int old) {
    if (v == mv && c == old) return;
    uint16_t* ge = gam + (size_t)v * ks + c;
    const unsigned g = *ge;
    if (!(g & kFlag)) return;
    *ge = (uint16_t)(g & kNone);
    if (c != colS[v]) {
      Rec r = rec[v];
      const bool ok = cls_rem(r.tmin, r.tcnt, r.tcnt2, g & kNone);
      cls_ins(r.nmin, r.ncnt, r.ncnt2, g & kNone);
      rec[v] = r;
      if (!ok) dirty[v] = 1;
    }
  };

  select();
  int it = 0;
  const int iters = (int)a.iters;  // at most 2^31 - 1 (checked by the host)
  for (it = 0; it < iters; ++it) {
    if (f == 0) break;
    bar();
    // ---- (D) minimum delta, tie rank, move; ring maintenance ----------------------------------
    if ((it & 31) == 0 && it > 0) {
      rr = rng(a.seed, (uint32_t)(it + lane), a.gen, ind_id, kTagTabu);
      r0l = rr.x;
      r1l = rr.y;
    }
    const uint32_t r0 = __shfl_sync(FULL, r0l, it & 31), r1 = __shfl_sync(FULL, r1l, it & 31);
    const int4 rw = lane < W ? red[lane] : make_int4(INT_MAX, 0, 0, 0);
    const int dstar = __reduce_min_sync(FULL, rw.x);
    const int xl = (lane < W && dstar != INT_MAX && rw.x == dstar) ? rw.y : 0;
    const int T = (int)__reduce_add_sync(FULL, (unsigned)xl);
    const int pre = (int)__reduce_add_sync(FULL, lane < warp ? (unsigned)xl : 0u);
    const int wtot = __shfl_sync(FULL, xl, warp);
    if (warp == 0) {
      const int nc = (int)__reduce_add_sync(FULL, lane < W ? (unsigned)rw.z : 0u);
      if (lane == 0) w_rows += nc;
    }
    const uint32_t j = T > 0 ? below(r0, (uint32_t)T) : 0u;
    if (T > 0 && (int)j >= pre && (int)j < pre + wtot) {  // this warp holds the j-th tie
      const int ct = tmin == dstar ? tcnt : 0;
      const int incl = incl_scan(ct, lane);
      const int lo_l = pre + incl - ct;
      const bool hit = ct > 0 && (int)j >= lo_l && (int)j < lo_l + ct;
      int hit_v = -1, hit_rank = 0;
      if (hit) {
        int jj = (int)j - lo_l;
        const int thrb = best_f - f;
        for (int q = 0; q < per; ++q) {
          const int v = v0 + q;
          const int gv = g0[v];
          if (v >= n || gv == 0) continue;
          int d, c;
          eval_row(rec[v], gv, thrb, d, c);
          if (c == 0 || d != dstar) continue;
          if (jj >= c) { jj -= c; continue; }
          hit_v = v;
          hit_rank = jj;
          break;
        }
      }
      const unsigned hb = __ballot_sync(FULL, hit);
      const int hl = hb ? __ffs(hb) - 1 : 0;
      const int v = hb ? __shfl_sync(FULL, hit_v, hl) : -1;
      int jj = __shfl_sync(FULL, hit_rank, hl);
      int mc = -1, colv = 0;
      if (v >= 0) {
        colv = colS[v];
        const int gv = g0[v];
        const unsigned kmin = (unsigned)(dstar + gv);
        const int thr = best_f - f + gv;
        const uint32_t* row32 = (const uint32_t*)(gam + (size_t)v * ks);
        for (int wb = 0; wb < kw && mc < 0; wb += 32) {
          const int w = wb + lane;
          bool m0 = false, m1 = false;
          if (w < kw) {
            uint32_t x = row32[w];
            if (w == (colv >> 1)) x |= (colv & 1) ? (kNone << 16) : kNone;
            const unsigned ka = x & kNone, kb = (x >> 16) & kNone;
            m0 = ka == kmin && (!(x & kFlag) || (int)ka < thr);
            m1 = kb == kmin && (!((x >> 16) & kFlag) || (int)kb < thr);
          }
          const unsigned b0 = __ballot_sync(FULL, m0), b1 = __ballot_sync(FULL, m1);
          const int before = __popc(b0 & lt) + __popc(b1 & lt);
          const bool found = jj >= before && jj < before + (int)m0 + (int)m1;
          const unsigned fb = __ballot_sync(FULL, found);
          if (fb) mc = __shfl_sync(FULL, 2 * w + ((jj == before && m0) ? 0 : 1), __ffs(fb) - 1);
          else jj -= __popc(b0) + __popc(b1);
        }
      }
      if (lane == 0) {
        if (v >= 0 && mc >= 0 && mc < k) {
          sc[SC_MV] = v;
          sc[SC_OLD] = colv;
          sc[SC_NEW] = mc;
          sc[SC_F] = f + dstar;
          if (a.trace) reinterpret_cast<int4*>(a.trace)[(size_t)ind * iters + it] = make_int4(v, mc, dstar, T);
        } else {
          sc[SC_ERR] = 2;  // tie counts inconsistent with the row: refuse to move
        }
      }
    }
    if (tid == 0) {
      if (T == 0 && a.trace) reinterpret_cast<int4*>(a.trace)[(size_t)ind * iters + it] = make_int4(-1, -1, 0, 0);
      // cancellation, polled every 1024 iterations: the search stops before this iteration's move
      if ((it & 1023) == 0 && a.cancel && *(volatile const int32_t*)a.cancel != 0) sc[SC_STOP] = 1;
    }
    if (warp == W - 1) {
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
      const int rv = sc[SC_REQV];
      if (rv >= 0) {
        const int rc = sc[SC_REQC];
        const uint32_t rtt = (uint32_t)sc[SC_REQTT];
        const uint32_t key = (uint32_t)rv | ((uint32_t)rc << 16);
        if (sc[SC_REQWAS]) {
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
        if (lane == 0) sc[SC_REQV] = -1;
      }
      // (c) entries that expire before the next selection (no longer tabu at it + 1)
      int dcnt = 0;
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
        dcnt += __popc(db);
      }
      if (lane == 0) {
        sc[SC_LO] = lo;
        sc[SC_NINS] = nins;
        sc[SC_DUE] = dcnt;
        sc[SC_FARDUE] = far_n > 0 && far_min == (uint32_t)(it + 1);
        sc[SC_FARN] = far_n;
      }
    }
    bar();
    if (sc[SC_STOP] | sc[SC_ERR]) break;
    // ---- (U) the move, expiries, neighbours, summaries, next selection ------------------------
    const int mv = T > 0 ? sc[SC_MV] : -1;
    int old = -1, nw = -1;
    bool improved = false;
    if (mv >= 0) {
      old = sc[SC_OLD];
      nw = sc[SC_NEW];
      f = sc[SC_F];
      ++moves;
      improved = f < best_f;
      if (improved) best_f = f;
      if (mv >= v0 && mv < v0 + per) {  // the owner of the moved vertex updates its row
        uint16_t* gr = gam + (size_t)mv * ks;
        const unsigned go = gr[old], gn = gr[nw];
        const bool was = (go & kFlag) != 0;
        // alpha f in 32-bit unsigned arithmetic: the host bounds alpha_num * |E| below 2^32
        const uint32_t tt = below(r1, a.L1) + ((uint32_t)a.an * (uint32_t)f) / (uint32_t)a.ad;
        const bool tabu = tt > 0;
        gr[old] = (uint16_t)((go & kNone) | (tabu ? kFlag : 0u));
        colS[mv] = (uint8_t)nw;
        g0[mv] = (uint16_t)(gn & kNone);
        Rec r = rec[mv];
        bool ok;  // the new colour leaves its class, the old one joins the tabu (or free) class
        if (gn & kFlag) ok = cls_rem(r.tmin, r.tcnt, r.tcnt2, gn & kNone);
        else ok = cls_rem(r.nmin, r.ncnt, r.ncnt2, gn & kNone);
        if (tabu) cls_ins(r.tmin, r.tcnt, r.tcnt2, go & kNone);
        else cls_ins(r.nmin, r.ncnt, r.ncnt2, go & kNone);
        rec[mv] = r;
        if (!ok) dirty[mv] = 1;
        if (tabu || was) {
          sc[SC_REQC] = old;
          sc[SC_REQTT] = (int32_t)tt;
          sc[SC_REQWAS] = was ? 1 : 0;
          sc[SC_REQV] = mv;
        }
      }
    }
    __syncwarp();
    // expiring entries of this warp's rows, one at a time (several may touch one row)
    {
      const int dcnt = sc[SC_DUE];
      if (dcnt > 0 && dcnt <= kDueCap) {
        int s = -1, ev = 0, ec = 0;
        if (lane < dcnt) {
          s = (int)due[lane];
          const uint32_t x = ring[s].x;
          ev = (int)ent_v(x);
          ec = (int)ent_c(x);
        }
        const bool mine = s >= 0 && ev >= wv0 && ev < wv1;
        for (unsigned b = __ballot_sync(FULL, mine); b; b &= b - 1) {
          if (lane == __ffs(b) - 1) {
            expire(ev, ec, mv, old);
            ring[s].x &= 0xFFFFFFu;
          }
          __syncwarp();
        }
      } else if (dcnt > kDueCap) {
        const int slo = sc[SC_LO], snins = sc[SC_NINS];
        for (int bb = slo; bb < snins; bb += 32) {
          const int s = bb + lane;
          bool mine = false;
          int ev = 0, ec = 0;
          if (s < snins) {
            const uint32_t x = ring[s & (R - 1)].x;
            ev = (int)ent_v(x);
            ec = (int)ent_c(x);
            mine = ent_st(x) == 2 && ev >= wv0 && ev < wv1;
          }
          for (unsigned b = __ballot_sync(FULL, mine); b; b &= b - 1) {
            if (lane == __ffs(b) - 1) {
              expire(ev, ec, mv, old);
              ring[s & (R - 1)].x &= 0xFFFFFFu;
            }
            __syncwarp();
          }
        }
      }
      if (sc[SC_FARDUE]) {
        const int fn = sc[SC_FARN];
        for (int bb = 0; bb < fn; bb += 32) {
          const int s = bb + lane;
          bool mine = false;
          int ev = 0, ec = 0;
          if (s < fn) {
            const uint2 e = far[s];
            ev = (int)ent_v(e.x);
            ec = (int)ent_c(e.x);
            mine = e.y == (uint32_t)(it + 1) && ev >= wv0 && ev < wv1;
          }
          for (unsigned b = __ballot_sync(FULL, mine); b; b &= b - 1) {
            if (lane == __ffs(b) - 1) expire(ev, ec, mv, old);
            __syncwarp();
          }
        }
      }
    }
    __syncwarp();
    // gamma of this warp's neighbours of the moved vertex, listed across the lanes
    if (mv >= 0) {
      uint32_t m = 0;
      if (v0 < n) {
        const uint32_t* br = bits + (size_t)mv * words;
        const int w0 = v0 >> 5, sh = v0 & 31;
        const uint32_t lw = br[w0];
        const uint32_t hw = (sh + per > 32 && w0 + 1 < words) ? br[w0 + 1] : 0u;
        m = __funnelshift_r(lw, hw, sh);
        if (per < 32) m &= (1u << per) - 1u;
      }
      const int cnt = __popc(m);
      const int incl = incl_scan(cnt, lane);
      const int total = __shfl_sync(FULL, incl, 31);
      int o = incl - cnt;
      while (m) {
        nbw[o++] = (uint16_t)(v0 + __ffs(m) - 1);
        m &= m - 1;
      }
      __syncwarp();
      if (lane == 0) w_deg += total;
      for (int r = lane; r < total; r += 32) {
        const int u = nbw[r];
        const int cu = colS[u];
        uint16_t* gr = gam + (size_t)u * ks;
        const unsigned go = gr[old], gn = gr[nw];
        gr[old] = (uint16_t)(go - 1u);
        gr[nw] = (uint16_t)(gn + 1u);
        Rec rc = rec[u];
        bool ok = true;
        if (old != cu) {
          if (go & kFlag) cls_dec(rc.tmin, rc.tcnt, rc.tcnt2, go & kNone);
          else cls_dec(rc.nmin, rc.ncnt, rc.ncnt2, go & kNone);
        } else {
          g0[u] = (uint16_t)((go & kNone) - 1u);
        }
        if (nw != cu) {
          if (gn & kFlag) ok = cls_inc(rc.tmin, rc.tcnt, rc.tcnt2, gn & kNone);
          else ok = cls_inc(rc.nmin, rc.ncnt, rc.ncnt2, gn & kNone);
        } else {
          g0[u] = (uint16_t)((gn & kNone) + 1u);
        }
        rec[u] = rc;
        if (!ok) dirty[u] = 1;
      }
      __syncwarp();
    }
    // rows whose summary could not be adjusted, summarised again by the warp (lanes over colours)
    {
      uint32_t dm = 0;
      for (int q = 0; q < per; q += 2) {
        const uint32_t x = *(const uint16_t*)(dirty + v0 + q);
        if (x & 0xFFu) dm |= 1u << q;
        if (x >> 8) dm |= 2u << q;
      }
      for (unsigned pend = __ballot_sync(FULL, dm != 0); pend; pend &= pend - 1) {
        const int l = __ffs(pend) - 1;
        uint32_t fl = __shfl_sync(FULL, dm, l);
        const int base = (warp * 32 + l) * per;
        for (; fl; fl &= fl - 1) {
          const int u = base + __ffs(fl) - 1;
          const Rec r = summarise((const uint32_t*)(gam + (size_t)u * ks), kw, colS[u], lane);
          if (lane == 0) {
            rec[u] = r;
            dirty[u] = 0;
            ++w_resum;
          }
        }
      }
      if (improved)
        for (int q = 0; q < per; q += 2) *(uint16_t*)(bestS + v0 + q) = *(const uint16_t*)(colS + v0 + q);
      __syncwarp();
    }
    select();  // the next iteration's selection
  }
  // ---- results ---------------------------------------------------------------------------------
  const int err = sc[SC_ERR], stop = sc[SC_STOP];
  long long* wk = (long long*)(gs + L.red);
  bar();  // every warp has left the loop: red[] is free
  if (lane == 0) {
    wk[4 * warp + 0] = w_rows;
    wk[4 * warp + 1] = w_deg;
    wk[4 * warp + 2] = w_resum;
  }
  for (int q = 0; q < per; ++q) {
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

template <int W, bool BSM>
__global__ void __launch_bounds__(32 * W * GroupMax<W>::value) tabucol_group_kernel(GroupArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int G = a.G;
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
  const int slot = blockIdx.x * G + grp;
  uint2* far = a.far ? a.far + (size_t)slot * (size_t)a.far_cap : nullptr;
  for (int i = slot; i < a.pop; i += gridDim.x * G) run_individual<W, BSM>(a, i, gs, bits, 1 + grp, far);
}

template <int W, bool BSM>
static dlm_status launch_one(dlm_ctx* ctx, GroupArgs a, int grid, size_t smem) {
  auto kfn = tabucol_group_kernel<W, BSM>;
  DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  kfn<<<grid, 32 * W * a.G, smem, ctx->stream>>>(a);
  return launch_check(ctx, "tabucol_group_kernel");
}

template <int W>
static int occupancy(int G, size_t smem, bool bsm) {
  int per_sm = 0;
  cudaError_t e;
  if (bsm) {
    e = cudaFuncSetAttribute(tabucol_group_kernel<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_group_kernel<W, true>, 32 * W * G, smem);
  } else {
    e = cudaFuncSetAttribute(tabucol_group_kernel<W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tabucol_group_kernel<W, false>, 32 * W * G, smem);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return per_sm < 1 ? 1 : per_sm;
}

}  // namespace tg

using namespace tg;

static int group_max_for(int W) {
  switch (W) {
    case 1: return GroupMax<1>::value;
    case 2: return GroupMax<2>::value;
    case 4: return GroupMax<4>::value;
    case 8: return GroupMax<8>::value;
    case 16: return GroupMax<16>::value;
    default: return GroupMax<32>::value;
  }
}

bool group_plan(int n, int k, int words, int W, size_t optin, int pop, int num_sms, int ring_force,
                GroupPlan* out) {
  if (W != 1 && W != 2 && W != 4 && W != 8 && W != 16 && W != 32) return false;
  const int NT = 32 * W;
  int per = (n + NT - 1) / NT;
  per = (per + 1) & ~1;  // even: vertices are read in pairs
  if (per < 2) per = 2;
  if (per > 32) return false;
  const size_t bits_bytes = a16(((size_t)n * words + 1) * 4);
  const int gmax_pop = std::max(1, (pop + num_sms - 1) / std::max(1, num_sms));
  const int gmax = std::min(group_max_for(W), gmax_pop);
  auto ring_for = [&](int G, bool bsm, int* R) -> bool {
    for (int r = ring_force > 0 ? ring_force : 8192; r >= 64; r >>= 1) {
      const size_t tot = (size_t)G * group_layout(n, k, W, per, r).total + (bsm ? bits_bytes : 0);
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
        out->W = W; out->G = G; out->R = R; out->per = per; out->bsm = bsm;
        out->group_bytes = group_layout(n, k, W, per, R).total;
        out->bits_bytes = bsm ? bits_bytes : 0;
        out->smem = (size_t)G * out->group_bytes + out->bits_bytes;
        return true;
      }
    }
  }
  return false;
}

dlm_status tabucol_group_launch(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                                uint32_t generation, uint32_t ind_base, const GroupPlan& P, int32_t* trace,
                                int64_t* work) {
  GroupArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = g->n; a.k = k; a.ks = group_row_stride(k); a.words = g->words; a.pop = pop; a.G = P.G; a.R = P.R;
  a.per = P.per;
  a.bits = g->d_bits; a.col = col; a.best_f = best_f; a.moves = moves; a.trace = trace; a.work = work;
  a.iters = iters; a.ind_base = ind_base;
  a.L1 = (uint32_t)tenure.L_max + 1u; a.an = tenure.alpha_num; a.ad = tenure.alpha_den;
  a.seed = seed; a.gen = generation; a.status = ctx->d_status; a.cancel = ctx->cancel;
  a.group_bytes = P.group_bytes; a.bits_bytes = P.bits_bytes;
  int per_sm = 1;
  switch (P.W) {
    case 1: per_sm = occupancy<1>(P.G, P.smem, P.bsm); break;
    case 2: per_sm = occupancy<2>(P.G, P.smem, P.bsm); break;
    case 4: per_sm = occupancy<4>(P.G, P.smem, P.bsm); break;
    case 8: per_sm = occupancy<8>(P.G, P.smem, P.bsm); break;
    case 16: per_sm = occupancy<16>(P.G, P.smem, P.bsm); break;
    default: per_sm = occupancy<32>(P.G, P.smem, P.bsm); break;
  }
  const int blocks = (pop + P.G - 1) / P.G;
  const int grid = std::max(1, std::min(blocks, per_sm * ctx->num_sms));
  // far list: tabu entries whose tenure does not fit the ring. A pair holds at most one live
  // entry, at most one entry is made per iteration and a tenure never exceeds L_max + alpha |E|,
  // so n (k - 1) + 1 entries, the budget + 1 and L_max + alpha |E| + 1 each bound what one search
  // keeps there at once.
  const uint64_t tt_max = (uint64_t)tenure.L_max + ((uint64_t)tenure.alpha_num * (uint64_t)g->m) / tenure.alpha_den;
  int64_t far_cap = 0;
  if (tt_max >= (uint64_t)P.R) {
    far_cap = std::min<int64_t>((int64_t)g->n * (k - 1) + 1, iters + 1);
    far_cap = std::min<int64_t>(far_cap, (int64_t)tt_max + 1);
  }
  a.far_cap = (int32_t)far_cap;
  if (far_cap > 0) {
    void* ws = nullptr;
    DLM_TRY(ctx_workspace(ctx, (size_t)grid * P.G * (size_t)far_cap * sizeof(uint2), &ws));
    a.far = (uint2*)ws;
  }
  switch (P.W) {
    case 1: return P.bsm ? launch_one<1, true>(ctx, a, grid, P.smem) : launch_one<1, false>(ctx, a, grid, P.smem);
    case 2: return P.bsm ? launch_one<2, true>(ctx, a, grid, P.smem) : launch_one<2, false>(ctx, a, grid, P.smem);
    case 4: return P.bsm ? launch_one<4, true>(ctx, a, grid, P.smem) : launch_one<4, false>(ctx, a, grid, P.smem);
    case 8: return P.bsm ? launch_one<8, true>(ctx, a, grid, P.smem) : launch_one<8, false>(ctx, a, grid, P.smem);
    case 16: return P.bsm ? launch_one<16, true>(ctx, a, grid, P.smem) : launch_one<16, false>(ctx, a, grid, P.smem);
    default: return P.bsm ? launch_one<32, true>(ctx, a, grid, P.smem) : launch_one<32, false>(ctx, a, grid, P.smem);
  }
}

}  // namespace dlm
