// DLMCOL oracle: a plain, slow, single-threaded CPU statement of what the GPU hot path computes.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and its Python binding)
// may link, load or call this file; only the tests, the smoke check and the bench's CPU-baseline
// leg use it. It shares no source with the CUDA path: the one thing both sides agree on is the
// published definition of the Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), written here from that definition.
//
// Paper: Goudet, Grelier, Hao, "A deep learning guided memetic framework for graph coloring
// problems" (arXiv 2109.05948). Each function cites the section or equation it follows.
//
// Pins (what fixes each function independently of itself) live in tests/test_oracle_*.py:
//   philox           - published known-answer vectors (Random123 kat_vectors).
//   init / gamma / f - the definition of f (Eq. f, section "Adaptations ... vertex coloring")
//                      recounted from the edge list; uniformity.
//   tabucol          - brute-force chromatic numbers (n <= 10), K_n closed form, odd/even cycles,
//                      bipartite and planted graphs reaching f = 0, gamma and f recomputed from
//                      scratch after every move (check mode), admissibility/min of every traced move.
//   gpx              - the defining properties of GPX (largest remaining class, alternating parents).
//   distance         - D(S, sigma S) = 0; lower bound of, and equal when injective to, the exact
//                      partition distance computed by an assignment solver.
//   pool / knn       - spacing invariant and greedy characterisation; library sort.
//   scorer           - central finite differences, colour-permutation invariance, closed forms.
//   adam             - closed form of the first step.
//   wvcp             - f recount from the class maxima (Eq. score_WVCP), w = 1 reduces to #classes.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

// ----------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al. 2011): 10 rounds of the Philox S-box on a 4x32-bit counter with a
// 2x32-bit key; the key is bumped by the Weyl constants between rounds.
// ----------------------------------------------------------------------------------------------
const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void philox_block(const uint32_t in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t x0 = in[0], x1 = in[1], x2 = in[2], x3 = in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += PHILOX_W0; k1 += PHILOX_W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// Stream convention of this project: key = (seed low word, seed high word); counter =
// (a, b, c, tag), the tag separating the uses of randomness in the method.
enum Tag : uint32_t { TAG_INIT = 1, TAG_TABU = 2, TAG_GPX = 3, TAG_SELECT = 4, TAG_NNINIT = 7,
                      TAG_BATCH = 8, TAG_WINIT = 9 };

void draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t tag, uint32_t out[4]) {
  uint32_t ctr[4] = {a, b, c, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  philox_block(ctr, key, out);
}

// Uniform integer in [0, m): the high word of the 64-bit product r * m.
inline uint32_t below(uint32_t r, uint32_t m) { return (uint32_t)(((uint64_t)r * m) >> 32); }

std::vector<std::vector<int>> neighbour_lists(int n, const uint8_t* adj) {
  std::vector<std::vector<int>> nb(n);
  for (int v = 0; v < n; ++v)
    for (int u = 0; u < n; ++u)
      if (u != v && adj[(size_t)v * n + u]) nb[v].push_back(u);
  return nb;
}

// gamma[v][c] = number of neighbours of v coloured c; f = number of edges with equal colours.
int64_t build_gamma(int n, int k, const std::vector<std::vector<int>>& nb, const int16_t* col,
                    std::vector<int32_t>& gamma) {
  gamma.assign((size_t)n * k, 0);
  for (int v = 0; v < n; ++v)
    for (int u : nb[v]) gamma[(size_t)v * k + col[u]]++;
  int64_t twice = 0;
  for (int v = 0; v < n; ++v) twice += gamma[(size_t)v * k + col[v]];
  return twice / 2;
}

int64_t count_conflicts(int n, const std::vector<std::vector<int>>& nb, const int16_t* col) {
  int64_t f = 0;
  for (int v = 0; v < n; ++v)
    for (int u : nb[v])
      if (u > v && col[u] == col[v]) ++f;
  return f;
}

// ----------------------------------------------------------------------------------------------
// Invariant deep-set scorer (section "Deep neural network training"): layer 0 pools the rows of
// the embedding E over each colour class (V_i Lambda_0, the rho Gamma_0 term being a constant for
// a partition and folded into beta_0), then nl layers phi(S)_i = LeakyReLU_0.2(beta + H_i Lambda
// + rho(H) Gamma), then a linear head averaged over the k classes.
// Flat parameter layout (shared by every consumer of a parameter vector):
//   E[n][d0], b0[d0], then for l = 1..nl: Lam[din][d], Gam[din][d], b[d]; then wh[d], bh[1].
// ----------------------------------------------------------------------------------------------
struct Dims {
  int n, d0, d, nl;
  size_t off_E() const { return 0; }
  size_t off_b0() const { return (size_t)n * d0; }
  int din(int l) const { return l == 1 ? d0 : d; }
  size_t off_layer(int l) const {  // l in 1..nl
    size_t o = off_b0() + d0;
    for (int j = 1; j < l; ++j) o += (size_t)2 * din(j) * d + d;
    return o;
  }
  size_t off_lam(int l) const { return off_layer(l); }
  size_t off_gam(int l) const { return off_layer(l) + (size_t)din(l) * d; }
  size_t off_b(int l) const { return off_layer(l) + (size_t)2 * din(l) * d; }
  size_t off_wh() const { return off_layer(nl + 1); }
  size_t off_bh() const { return off_wh() + d; }
  size_t total() const { return off_bh() + 1; }
};

inline double lrelu(double x) { return x > 0.0 ? x : 0.2 * x; }
inline double lrelu_grad(double x) { return x > 0.0 ? 1.0 : 0.2; }

struct Cache {
  std::vector<std::vector<double>> Z;  // Z[l] : k x width(l), l = 0..nl (pre-activations)
  std::vector<std::vector<double>> H;  // H[l] : k x width(l)
  std::vector<std::vector<double>> M;  // M[l] : mean over classes of H[l]
};

double scorer_forward(const Dims& dm, int k, const double* th, const int16_t* col, Cache* cache) {
  const int d0 = dm.d0, d = dm.d, nl = dm.nl;
  std::vector<std::vector<double>> Z(nl + 1), H(nl + 1), M(nl + 1);
  Z[0].assign((size_t)k * d0, 0.0);
  for (int c = 0; c < k; ++c)
    for (int f = 0; f < d0; ++f) Z[0][(size_t)c * d0 + f] = th[dm.off_b0() + f];
  for (int v = 0; v < dm.n; ++v)
    for (int f = 0; f < d0; ++f) Z[0][(size_t)col[v] * d0 + f] += th[dm.off_E() + (size_t)v * d0 + f];
  for (int l = 0; l <= nl; ++l) {
    const int w = l == 0 ? d0 : d;
    if (l > 0) {
      const int din = dm.din(l);
      const double* lam = th + dm.off_lam(l);
      const double* gam = th + dm.off_gam(l);
      const double* b = th + dm.off_b(l);
      Z[l].assign((size_t)k * d, 0.0);
      std::vector<double> mg(d, 0.0);  // rho(H) Gamma
      for (int o = 0; o < d; ++o)
        for (int f = 0; f < din; ++f) mg[o] += M[l - 1][f] * gam[(size_t)f * d + o];
      for (int c = 0; c < k; ++c)
        for (int o = 0; o < d; ++o) {
          double z = b[o] + mg[o];
          for (int f = 0; f < din; ++f) z += H[l - 1][(size_t)c * din + f] * lam[(size_t)f * d + o];
          Z[l][(size_t)c * d + o] = z;
        }
    }
    H[l].resize(Z[l].size());
    for (size_t i = 0; i < Z[l].size(); ++i) H[l][i] = lrelu(Z[l][i]);
    M[l].assign(w, 0.0);
    for (int c = 0; c < k; ++c)
      for (int f = 0; f < w; ++f) M[l][f] += H[l][(size_t)c * w + f];
    for (int f = 0; f < w; ++f) M[l][f] /= k;
  }
  double out = th[dm.off_bh()];
  for (int o = 0; o < d; ++o) out += M[nl][o] * th[dm.off_wh() + o];
  if (cache) { cache->Z = std::move(Z); cache->H = std::move(H); cache->M = std::move(M); }
  return out;
}

// Reverse mode of scorer_forward for one sample; g = dLoss/dout; adds into grad.
void scorer_backward(const Dims& dm, int k, const double* th, const int16_t* col, const Cache& ca,
                     double g, double* grad) {
  const int d0 = dm.d0, d = dm.d, nl = dm.nl;
  // head: out = bh + mean_c(H[nl][c]) . wh
  grad[dm.off_bh()] += g;
  for (int o = 0; o < d; ++o) grad[dm.off_wh() + o] += g * ca.M[nl][o];
  std::vector<double> dH((size_t)k * d);
  for (int c = 0; c < k; ++c)
    for (int o = 0; o < d; ++o) dH[(size_t)c * d + o] = g * th[dm.off_wh() + o] / k;
  for (int l = nl; l >= 1; --l) {
    const int din = dm.din(l);
    const double* lam = th + dm.off_lam(l);
    const double* gam = th + dm.off_gam(l);
    std::vector<double> dZ((size_t)k * d), s(d, 0.0);
    for (size_t i = 0; i < dZ.size(); ++i) dZ[i] = dH[i] * lrelu_grad(ca.Z[l][i]);
    for (int c = 0; c < k; ++c)
      for (int o = 0; o < d; ++o) s[o] += dZ[(size_t)c * d + o];
    for (int o = 0; o < d; ++o) grad[dm.off_b(l) + o] += s[o];
    for (int c = 0; c < k; ++c)
      for (int f = 0; f < din; ++f) {
        const double h = ca.H[l - 1][(size_t)c * din + f];
        for (int o = 0; o < d; ++o) grad[dm.off_lam(l) + (size_t)f * d + o] += h * dZ[(size_t)c * d + o];
      }
    for (int f = 0; f < din; ++f)
      for (int o = 0; o < d; ++o) grad[dm.off_gam(l) + (size_t)f * d + o] += ca.M[l - 1][f] * s[o];
    std::vector<double> dHp((size_t)k * din, 0.0), dm_((size_t)din, 0.0);
    for (int f = 0; f < din; ++f)
      for (int o = 0; o < d; ++o) dm_[f] += s[o] * gam[(size_t)f * d + o];
    for (int c = 0; c < k; ++c)
      for (int f = 0; f < din; ++f) {
        double acc = dm_[f] / k;
        for (int o = 0; o < d; ++o) acc += dZ[(size_t)c * d + o] * lam[(size_t)f * d + o];
        dHp[(size_t)c * din + f] = acc;
      }
    dH.swap(dHp);
  }
  // layer 0: Z0[c] = b0 + sum_{v in V_c} E[v]
  std::vector<double> dZ0((size_t)k * d0);
  for (size_t i = 0; i < dZ0.size(); ++i) dZ0[i] = dH[i] * lrelu_grad(ca.Z[0][i]);
  for (int c = 0; c < k; ++c)
    for (int f = 0; f < d0; ++f) grad[dm.off_b0() + f] += dZ0[(size_t)c * d0 + f];
  for (int v = 0; v < dm.n; ++v)
    for (int f = 0; f < d0; ++f) grad[dm.off_E() + (size_t)v * d0 + f] += dZ0[(size_t)col[v] * d0 + f];
}

// PyTorch-form Adam step (Kingma & Ba) with betas (0.9, 0.999), eps 1e-8.
void adam_apply(size_t P, double* th, double* m, double* v, const double* g, int64_t t, double lr) {
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  const double bc1 = 1.0 - std::pow(b1, (double)t), bc2 = 1.0 - std::pow(b2, (double)t);
  for (size_t i = 0; i < P; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    const double denom = std::sqrt(v[i]) / std::sqrt(bc2) + eps;
    th[i] -= (lr / bc1) * m[i] / denom;
  }
}

}  // namespace

extern "C" {

// Philox4x32-10 block function (Salmon et al. 2011), exported for the known-answer pin.
void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox_block(ctr, key, out);
}

void oracle_draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t tag, uint32_t* out) {
  draw(seed, a, b, c, tag, out);
}

// Graph storage used by the hot path (setup step): CSR (ascending neighbour ids) and bit-packed
// adjacency rows, from the dense 0/1 matrix. The graph lives in global memory shared by all
// searches (section "Parallel iterated feasible and infeasible Tabu Search").
void oracle_graph_csr(int32_t n, const uint8_t* adj, int32_t* off, int32_t* idx, uint32_t* bits) {
  const int words = (n + 31) / 32;
  int32_t e = 0;
  for (int v = 0; v < n; ++v) {
    off[v] = e;
    for (int w = 0; w < words; ++w) bits[(size_t)v * words + w] = 0;
    for (int u = 0; u < n; ++u)
      if (u != v && adj[(size_t)v * n + u]) {
        idx[e++] = u;
        bits[(size_t)v * words + u / 32] |= 1u << (u % 32);
      }
  }
  off[n] = e;
}

// Random initialisation for k-COL (section "Adaptations ... vertex coloring"): every vertex of
// every individual receives a uniform colour in {0..k-1} (the paper's 1..k shifted to 0-based).
void oracle_init_colors(int32_t n, int32_t k, int32_t pop, uint64_t seed, uint32_t ind_base, int16_t* col) {
  for (int i = 0; i < pop; ++i)
    for (int v = 0; v < n; ++v) {
      uint32_t r[4];
      draw(seed, (uint32_t)v, 0u, ind_base + (uint32_t)i, TAG_INIT, r);
      col[(size_t)i * n + v] = (int16_t)below(r[0], (uint32_t)k);
    }
}

// Conflict table gamma (the data structure of the "efficient implementation" of TabuCol) and
// the k-COL objective f (Eq. f): number of edges whose end points share a colour.
int64_t oracle_gamma(int32_t n, const uint8_t* adj, int32_t k, const int16_t* col, int32_t* gamma_out) {
  auto nb = neighbour_lists(n, adj);
  std::vector<int32_t> g;
  int64_t f = build_gamma(n, k, nb, col, g);
  if (gamma_out) std::copy(g.begin(), g.end(), gamma_out);
  return f;
}

// TabuCol for k-COL (section "Adaptations ... vertex coloring"; Table params-COL: tenure
// parameter alpha = 0.6, depth 128|V|). Per iteration: among the one-moves (v, c) of conflicting
// vertices v to colours c != col(v), take the one with the smallest change
// delta = gamma[v][c] - gamma[v][col v] that is not tabu, or is tabu but leads below the best f
// seen (aspiration). Ties: the j-th admissible minimum in (v asc, c asc) order, j drawn uniformly
// from the iteration's Philox block. After moving v from colour `old`, (v, old) is tabu for
// tt = U{0..L_max} + floor(alpha * f) iterations. The search stops when f reaches 0.
// trace (optional, 4 ints per iteration): v, c, delta, number of tied admissible moves.
// check != 0: after every move gamma and f are recomputed from scratch and compared.
// Returns 0, -1 on a colour outside 0..k-1, -2 on a failed check.
int32_t oracle_tabucol(int32_t n, const uint8_t* adj, int32_t k, const int16_t* col_in, int64_t iters,
                       int32_t L_max, int32_t alpha_num, int32_t alpha_den, uint64_t seed, uint32_t ind,
                       uint32_t gen, int16_t* best_col, int64_t* best_f_out, int64_t* moves_out,
                       int64_t* iters_out, int32_t* trace, int32_t check) {
  auto nb = neighbour_lists(n, adj);
  std::vector<int16_t> col(col_in, col_in + n);
  for (int v = 0; v < n; ++v)
    if (col[v] < 0 || col[v] >= k) return -1;
  std::vector<int32_t> gamma;
  int64_t f = build_gamma(n, k, nb, col.data(), gamma);
  std::vector<int64_t> tabu_until((size_t)n * k, 0);
  int64_t best_f = f, moves = 0, it = 0;
  std::copy(col.begin(), col.end(), best_col);
  for (it = 0; it < iters; ++it) {
    if (f == 0) break;
    uint32_t r[4];
    draw(seed, (uint32_t)it, gen, ind, TAG_TABU, r);
    int64_t dmin = INT64_MAX, ties = 0;
    for (int v = 0; v < n; ++v) {
      const int32_t gv = gamma[(size_t)v * k + col[v]];
      if (gv == 0) continue;
      for (int c = 0; c < k; ++c) {
        if (c == col[v]) continue;
        const int64_t delta = gamma[(size_t)v * k + c] - gv;
        const bool admissible = tabu_until[(size_t)v * k + c] <= it || f + delta < best_f;
        if (!admissible) continue;
        if (delta < dmin) { dmin = delta; ties = 1; }
        else if (delta == dmin) ++ties;
      }
    }
    if (ties == 0) {  // every move tabu and none aspirated: the iteration passes without a move
      if (trace) { trace[4 * it] = -1; trace[4 * it + 1] = -1; trace[4 * it + 2] = 0; trace[4 * it + 3] = 0; }
      continue;
    }
    const int64_t pick = below(r[0], (uint32_t)ties);
    int mv = -1, mc = -1;
    int64_t seen = 0;
    for (int v = 0; v < n && mv < 0; ++v) {
      const int32_t gv = gamma[(size_t)v * k + col[v]];
      if (gv == 0) continue;
      for (int c = 0; c < k; ++c) {
        if (c == col[v]) continue;
        const int64_t delta = gamma[(size_t)v * k + c] - gv;
        const bool admissible = tabu_until[(size_t)v * k + c] <= it || f + delta < best_f;
        if (!admissible || delta != dmin) continue;
        if (seen == pick) { mv = v; mc = c; break; }
        ++seen;
      }
    }
    const int old = col[mv];
    col[mv] = (int16_t)mc;
    for (int u : nb[mv]) {
      gamma[(size_t)u * k + old]--;
      gamma[(size_t)u * k + mc]++;
    }
    const int64_t f_before = f;
    f += dmin;
    const int64_t tt = (int64_t)below(r[1], (uint32_t)(L_max + 1)) + ((int64_t)alpha_num * f) / alpha_den;
    tabu_until[(size_t)mv * k + old] = it + 1 + tt;
    ++moves;
    if (f < best_f) { best_f = f; std::copy(col.begin(), col.end(), best_col); }
    if (trace) { trace[4 * it] = mv; trace[4 * it + 1] = mc; trace[4 * it + 2] = (int32_t)dmin; trace[4 * it + 3] = (int32_t)ties; }
    if (check) {
      std::vector<int32_t> g2;
      const int64_t f2 = build_gamma(n, k, nb, col.data(), g2);
      if (g2 != gamma || f2 != f || count_conflicts(n, nb, col.data()) != f) return -2;
      if (f - f_before != dmin) return -2;
    }
  }
  *best_f_out = best_f;
  if (moves_out) *moves_out = moves;
  if (iters_out) *iters_out = it;
  return 0;
}

// GPX crossover (Galinier & Hao 1999; section "Parent matching and selection of crossovers"):
// for step l = 0..k-1 the child takes, with label l, the largest class still unassigned in parent
// A (even l) or parent B (odd l), smallest colour on ties; those vertices leave both parents.
// Vertices never inherited receive a uniform random label from the child's own Philox stream.
void oracle_gpx(int32_t n, int32_t k, const int16_t* A, const int16_t* B, uint64_t seed,
                uint32_t child_id, uint32_t gen, int16_t* child) {
  std::vector<char> taken(n, 0);
  std::vector<int32_t> cnt(k);
  for (int l = 0; l < k; ++l) {
    const int16_t* P = (l % 2 == 0) ? A : B;
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int v = 0; v < n; ++v)
      if (!taken[v]) cnt[P[v]]++;
    int best = 0;
    for (int c = 1; c < k; ++c)
      if (cnt[c] > cnt[best]) best = c;
    if (cnt[best] == 0) continue;
    for (int v = 0; v < n; ++v)
      if (!taken[v] && P[v] == best) { child[v] = (int16_t)l; taken[v] = 1; }
  }
  for (int v = 0; v < n; ++v)
    if (!taken[v]) {
      uint32_t r[4];
      draw(seed, (uint32_t)v, gen, child_id, TAG_GPX, r);
      child[v] = (int16_t)below(r[0], (uint32_t)k);
    }
}

// Approximate set-theoretic partition distance (section "Distance computation"): with the
// overlap matrix M[c][c'] = |A_c intersect B_c'|, each class is matched to its best-overlapping
// class of the other partition without requiring a bijection; D = n - min(sum_c max_c' M,
// sum_c' max_c M). It never exceeds the exact (Hungarian) distance and equals it when the
// best-match map is injective; taking the smaller similarity makes it symmetric.
int32_t oracle_distance(int32_t n, int32_t k, const int16_t* A, const int16_t* B) {
  std::vector<int32_t> M((size_t)k * k, 0);
  for (int v = 0; v < n; ++v) M[(size_t)A[v] * k + B[v]]++;
  int64_t srow = 0, scol = 0;
  for (int c = 0; c < k; ++c) {
    int32_t mr = 0, mc = 0;
    for (int c2 = 0; c2 < k; ++c2) {
      mr = std::max(mr, M[(size_t)c * k + c2]);
      mc = std::max(mc, M[(size_t)c2 * k + c]);
    }
    srow += mr; scol += mc;
  }
  return (int32_t)(n - std::min(srow, scol));
}

// All distances between the rows of X (a x n) and Y (b x n); out is a x b.
void oracle_distance_matrix(int32_t n, int32_t k, const int16_t* X, int32_t a, const int16_t* Y,
                            int32_t b, int16_t* out) {
  for (int i = 0; i < a; ++i)
    for (int j = 0; j < b; ++j)
      out[(size_t)i * b + j] = (int16_t)oracle_distance(n, k, X + (size_t)i * n, Y + (size_t)j * n);
}

// Distance-and-quality pool update (section "Population update"): the 2p candidates (the current
// population first, then the improved individuals) are visited by increasing f, ties by lower
// index; a candidate joins the next population when its distance to every member already chosen
// exceeds n/10. When fewer than p pass, the best remaining candidates by the same order fill it.
// sel receives the p chosen candidate indices in the order they were chosen.
void oracle_pool_update(int32_t p, int32_t n, const int64_t* fit, const int16_t* D, int32_t* sel) {
  const int m = 2 * p;
  std::vector<int32_t> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return fit[a] < fit[b]; });
  std::vector<char> chosen(m, 0);
  int cnt = 0;
  for (int t = 0; t < m && cnt < p; ++t) {
    const int x = order[t];
    bool ok = true;
    for (int s = 0; s < cnt && ok; ++s)
      if (10 * (int64_t)D[(size_t)x * m + sel[s]] <= (int64_t)n) ok = false;
    if (ok) { sel[cnt++] = x; chosen[x] = 1; }
  }
  for (int t = 0; t < m && cnt < p; ++t)
    if (!chosen[order[t]]) { sel[cnt++] = order[t]; chosen[order[t]] = 1; }
}

// Parent matching (section "Parent matching and selection of crossovers"): the K nearest
// individuals of each i by the distance matrix, j != i, ties by lower index, nearest first.
void oracle_knn(int32_t p, const int16_t* D, int32_t K, int32_t* nbr) {
  for (int i = 0; i < p; ++i) {
    std::vector<int32_t> js;
    for (int j = 0; j < p; ++j)
      if (j != i) js.push_back(j);
    std::stable_sort(js.begin(), js.end(), [&](int a, int b) {
      return D[(size_t)i * p + a] < D[(size_t)i * p + b];
    });
    for (int t = 0; t < K; ++t) nbr[(size_t)i * K + t] = js[t];
  }
}

size_t oracle_scorer_nparams(int32_t n, int32_t d0, int32_t d, int32_t nl) {
  Dims dm{n, d0, d, nl};
  return dm.total();
}

// Parameter initialisation: uniform in +-1/sqrt(fan_in) from the NNINIT Philox stream, one
// draw per parameter index (fan_in of E and b0 is n, the one-hot input width of layer 0).
void oracle_scorer_init(int32_t n, int32_t d0, int32_t d, int32_t nl, uint64_t seed, double* th) {
  Dims dm{n, d0, d, nl};
  auto fill = [&](size_t off, size_t cnt, int fan_in) {
    const double bound = 1.0 / std::sqrt((double)fan_in);
    for (size_t i = 0; i < cnt; ++i) {
      uint32_t r[4];
      draw(seed, (uint32_t)(off + i), 0u, 0u, TAG_NNINIT, r);
      const double u = (double)(r[0] >> 8) * (1.0 / 16777216.0);
      th[off + i] = (2.0 * u - 1.0) * bound;
    }
  };
  fill(dm.off_E(), (size_t)n * d0, n);
  fill(dm.off_b0(), d0, n);
  for (int l = 1; l <= nl; ++l) {
    fill(dm.off_lam(l), (size_t)dm.din(l) * d, dm.din(l));
    fill(dm.off_gam(l), (size_t)dm.din(l) * d, dm.din(l));
    fill(dm.off_b(l), d, dm.din(l));
  }
  fill(dm.off_wh(), d, d);
  fill(dm.off_bh(), 1, d);
}

// f_theta(S) for c colourings (c x n) with k classes.
void oracle_scorer_forward(int32_t n, int32_t d0, int32_t d, int32_t nl, int32_t k, const double* th,
                           const int16_t* cols, int32_t c, double* out) {
  Dims dm{n, d0, d, nl};
  for (int i = 0; i < c; ++i) out[i] = scorer_forward(dm, k, th, cols + (size_t)i * n, nullptr);
}

// Mean squared error over a batch of B samples and its gradient (grad is overwritten).
double oracle_scorer_loss_grad(int32_t n, int32_t d0, int32_t d, int32_t nl, int32_t k, const double* th,
                               const int16_t* cols, const double* y, int32_t B, double* grad, double* out) {
  Dims dm{n, d0, d, nl};
  std::fill(grad, grad + dm.total(), 0.0);
  double loss = 0.0;
  for (int i = 0; i < B; ++i) {
    Cache ca;
    const double o = scorer_forward(dm, k, th, cols + (size_t)i * n, &ca);
    if (out) out[i] = o;
    const double e = o - y[i];
    loss += e * e / B;
    scorer_backward(dm, k, th, cols + (size_t)i * n, ca, 2.0 * e / B, grad);
  }
  return loss;
}

void oracle_adam_step(int64_t P, double* th, double* m, double* v, const double* g, int64_t t, double lr) {
  adam_apply((size_t)P, th, m, v, g, t, lr);
}

// Online training (section "Deep neural network training"): targets f(S'_i) standardised by the
// generation's mean and standard deviation; N epochs over the p samples in batches of b, each
// epoch visiting the samples in the order of their BATCH-stream keys (ties by index); one Adam
// step per batch. adam_t is the running step counter. Returns the last batch's loss.
double oracle_scorer_train(int32_t n, int32_t d0, int32_t d, int32_t nl, int32_t k, double* th, double* am,
                           double* av, int64_t* adam_t, int32_t p, const int16_t* cols, const int64_t* fvals,
                           int32_t epochs, int32_t b, double lr, uint64_t seed, uint32_t gen) {
  Dims dm{n, d0, d, nl};
  double mean = 0.0, var = 0.0;
  for (int i = 0; i < p; ++i) mean += (double)fvals[i];
  mean /= p;
  for (int i = 0; i < p; ++i) var += ((double)fvals[i] - mean) * ((double)fvals[i] - mean);
  var /= p;
  double sd = std::sqrt(var);
  if (!(sd > 1e-12)) sd = 1.0;
  std::vector<double> y(p);
  for (int i = 0; i < p; ++i) y[i] = ((double)fvals[i] - mean) / sd;
  std::vector<double> grad(dm.total());
  double loss = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    std::vector<uint64_t> key(p);
    for (int i = 0; i < p; ++i) {
      uint32_t r[4];
      draw(seed, (uint32_t)i, (uint32_t)ep, gen, TAG_BATCH, r);
      key[i] = ((uint64_t)r[0] << 32) | (uint32_t)i;
    }
    std::vector<int32_t> order(p);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int bb) { return key[a] < key[bb]; });
    for (int s = 0; s < p; s += b) {
      const int B = std::min(b, p - s);
      std::vector<int16_t> bc((size_t)B * n);
      std::vector<double> by(B);
      for (int t = 0; t < B; ++t) {
        std::copy(cols + (size_t)order[s + t] * n, cols + (size_t)order[s + t] * n + n, bc.begin() + (size_t)t * n);
        by[t] = y[order[s + t]];
      }
      loss = oracle_scorer_loss_grad(n, d0, d, nl, k, th, bc.data(), by.data(), B, grad.data(), nullptr);
      *adam_t += 1;
      adam_apply(dm.total(), th, am, av, grad.data(), *adam_t, lr);
    }
  }
  return loss;
}

}  // extern "C"

namespace {
// Algorithm 1 after the local search of the offspring (Sp, fSp): best so far, training,
// distances over P u P', pool update, K nearest neighbours and the offspring of the next
// generation. Shared by the k-COL and the WVCP generations; the population arrays are updated in
// place.
int32_t memetic_after_search(int32_t n, int32_t k, int32_t p, int32_t K, int16_t* P, int64_t* fP, int16_t* DP,
                             int16_t* SO, std::vector<int16_t>& Sp, std::vector<int64_t>& fSp, int32_t use_scorer,
                             int32_t d0, int32_t d, int32_t nl, double* th, double* am, double* av, int64_t* adam_t,
                             int32_t epochs, int32_t batch, double lr, const float* ext_scores, uint64_t seed,
                             uint32_t gen, int16_t* best_col, int64_t* best_f, int64_t* diag_fprime,
                             int32_t* diag_pick) {
  if (diag_fprime) std::copy(fSp.begin(), fSp.end(), diag_fprime);
  // 2. best so far
  int ib = 0;
  for (int i = 1; i < p; ++i)
    if (fSp[i] < fSp[ib]) ib = i;
  if (fSp[ib] < *best_f) {
    *best_f = fSp[ib];
    std::copy(Sp.begin() + (size_t)ib * n, Sp.begin() + (size_t)(ib + 1) * n, best_col);
  }
  // 3. training
  if (use_scorer)
    oracle_scorer_train(n, d0, d, nl, k, th, am, av, adam_t, p, SO, fSp.data(), epochs, batch, lr, seed, gen);
  // 4. distances over P u P'
  const int m = 2 * p;
  std::vector<int16_t> Dall((size_t)m * m, 0);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) Dall[(size_t)i * m + j] = DP[(size_t)i * p + j];
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) {
      const int16_t dij = (int16_t)oracle_distance(n, k, P + (size_t)i * n, Sp.data() + (size_t)j * n);
      Dall[(size_t)i * m + p + j] = dij;
      Dall[(size_t)(p + j) * m + i] = dij;
    }
  for (int i = 0; i < p; ++i)
    for (int j = i + 1; j < p; ++j) {
      const int16_t dij = (int16_t)oracle_distance(n, k, Sp.data() + (size_t)i * n, Sp.data() + (size_t)j * n);
      Dall[(size_t)(p + i) * m + p + j] = dij;
      Dall[(size_t)(p + j) * m + p + i] = dij;
    }
  // 5. pool update
  std::vector<int64_t> fall(m);
  for (int i = 0; i < p; ++i) { fall[i] = fP[i]; fall[p + i] = fSp[i]; }
  std::vector<int32_t> sel(p);
  oracle_pool_update(p, n, fall.data(), Dall.data(), sel.data());
  std::vector<int16_t> Pn((size_t)p * n);
  for (int s = 0; s < p; ++s) {
    const int x = sel[s];
    const int16_t* src = x < p ? P + (size_t)x * n : Sp.data() + (size_t)(x - p) * n;
    std::copy(src, src + n, Pn.begin() + (size_t)s * n);
    fP[s] = fall[x];
  }
  std::copy(Pn.begin(), Pn.end(), P);
  for (int s = 0; s < p; ++s)
    for (int t = 0; t < p; ++t) DP[(size_t)s * p + t] = Dall[(size_t)sel[s] * m + sel[t]];
  // 6. parent matching
  std::vector<int32_t> nbr((size_t)p * K);
  oracle_knn(p, DP, K, nbr.data());
  // 7. offspring
  std::vector<int16_t> child(n);
  for (int i = 0; i < p; ++i) {
    int pick;
    if (use_scorer) {
      double bestv = 0.0;
      pick = -1;
      std::vector<int16_t> kids((size_t)K * n);
      for (int j = 0; j < K; ++j)
        oracle_gpx(n, k, P + (size_t)i * n, P + (size_t)nbr[(size_t)i * K + j] * n, seed,
                   (uint32_t)(i * K + j), gen, kids.data() + (size_t)j * n);
      for (int j = 0; j < K; ++j) {
        double sc;
        if (ext_scores) sc = (double)ext_scores[(size_t)i * K + j];
        else oracle_scorer_forward(n, d0, d, nl, k, th, kids.data() + (size_t)j * n, 1, &sc);
        if (pick < 0 || sc < bestv) { bestv = sc; pick = j; }
      }
      std::copy(kids.begin() + (size_t)pick * n, kids.begin() + (size_t)(pick + 1) * n, SO + (size_t)i * n);
    } else {
      uint32_t r[4];
      draw(seed, (uint32_t)i, gen, 0u, TAG_SELECT, r);
      pick = (int)below(r[0], (uint32_t)K);
      oracle_gpx(n, k, P + (size_t)i * n, P + (size_t)nbr[(size_t)i * K + pick] * n, seed,
                 (uint32_t)(i * K + pick), gen, SO + (size_t)i * n);
    }
    if (diag_pick) diag_pick[i] = pick;
  }
  return 0;
}
}  // namespace

extern "C" {

// One generation of the deep-learning-guided memetic framework (Algorithm 1, one pass of its
// loop) for k-COL: tabu search of every offspring S^O_i -> S'_i; best-so-far update; training of
// f_theta on {(S^O_i, f(S'_i))} (when use_scorer); distances between P and P' and within P';
// pool update; K nearest neighbours; offspring selection. With use_scorer the offspring of i is
// the argmin of the scores of its K GPX children (ext_scores, when given, replaces the oracle's
// own scores); without it the second parent is drawn uniformly among the K nearest (the
// ablation of section "Benefits of the neural network based crossover selection").
// State arrays are updated in place. diag_fprime (p) receives f(S'_i); diag_pick (p) the chosen j.
int32_t oracle_memetic_generation(int32_t n, const uint8_t* adj, int32_t k, int32_t p, int32_t K,
                                  int16_t* P, int64_t* fP, int16_t* DP, int16_t* SO, int64_t iters,
                                  int32_t L_max, int32_t a_num, int32_t a_den, int32_t use_scorer,
                                  int32_t d0, int32_t d, int32_t nl, double* th, double* am, double* av,
                                  int64_t* adam_t, int32_t epochs, int32_t batch, double lr,
                                  const float* ext_scores, uint64_t seed, uint32_t gen, int16_t* best_col,
                                  int64_t* best_f, int64_t* diag_fprime, int32_t* diag_pick) {
  if (K > p - 1 || K < 1) return -1;
  // 1. parallel local search
  std::vector<int16_t> Sp((size_t)p * n);
  std::vector<int64_t> fSp(p);
  for (int i = 0; i < p; ++i) {
    int64_t mv, itd;
    int32_t rc = oracle_tabucol(n, adj, k, SO + (size_t)i * n, iters, L_max, a_num, a_den, seed, (uint32_t)i,
                                gen, Sp.data() + (size_t)i * n, &fSp[i], &mv, &itd, nullptr, 0);
    if (rc) return rc;
  }
  return memetic_after_search(n, k, p, K, P, fP, DP, SO, Sp, fSp, use_scorer, d0, d, nl, th, am, av, adam_t, epochs,
                              batch, lr, ext_scores, seed, gen, best_col, best_f, diag_fprime, diag_pick);
}

// ----------------------------------------------------------------------------------------------
// Weighted vertex colouring (WVCP).
// ----------------------------------------------------------------------------------------------

// WVCP score f (Eq. score_WVCP): sum over colour classes of the largest vertex weight in the
// class (an empty class contributes 0); conflicts_out receives c(S), the number of edges whose
// end points share a colour (the penalty term of Eq. AFISA_score).
int64_t oracle_wvcp_score(int32_t n, const uint8_t* adj, const int32_t* w, int32_t k, const int16_t* col,
                          int64_t* conflicts_out) {
  std::vector<int64_t> mx(k, 0);
  for (int v = 0; v < n; ++v) mx[col[v]] = std::max<int64_t>(mx[col[v]], w[v]);
  int64_t f = 0;
  for (int c = 0; c < k; ++c) f += mx[c];
  if (conflicts_out) {
    auto nb = neighbour_lists(n, adj);
    *conflicts_out = count_conflicts(n, nb, col);
  }
  return f;
}

// Randomised greedy initialisation for the WVCP (section "Initialization with a greedy random
// algorithm"): vertices by decreasing weight, then decreasing degree (then increasing index);
// each takes a colour drawn uniformly among the already-opened colours that no neighbour uses,
// or opens a new colour when there is none. Returns the number of colours opened.
int32_t oracle_wvcp_greedy(int32_t n, const uint8_t* adj, const int32_t* w, uint64_t seed, uint32_t ind,
                           int16_t* col) {
  auto nb = neighbour_lists(n, adj);
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (w[a] != w[b]) return w[a] > w[b];
    return nb[a].size() > nb[b].size();
  });
  std::vector<int16_t> c(n, -1);
  int used = 0;
  for (int pos = 0; pos < n; ++pos) {
    const int v = order[pos];
    std::vector<char> blocked(used, 0);
    for (int u : nb[v])
      if (c[u] >= 0) blocked[c[u]] = 1;
    std::vector<int> legal;
    for (int q = 0; q < used; ++q)
      if (!blocked[q]) legal.push_back(q);
    if (legal.empty()) {
      c[v] = (int16_t)used++;
    } else {
      uint32_t r[4];
      draw(seed, (uint32_t)pos, 0u, ind, TAG_WINIT, r);
      c[v] = (int16_t)legal[below(r[0], (uint32_t)legal.size())];
    }
  }
  std::copy(c.begin(), c.end(), col);
  return used;
}

// Feasible and infeasible tabu search for the WVCP with a fixed penalty phi (section "Parallel
// iterated feasible and infeasible Tabu Search"; Algorithm 2 with the last-run setting
// phi = 2 max w). The search minimises g(S) = f(S) + phi c(S) (Eq. AFISA_score) over all
// one-moves (v, c), c != col(v), of all vertices. A vertex that has just moved is frozen for
// tt = U{0..L_max} + floor(alpha |V|) iterations (alpha = 0.2 in Table params-WVCP); a move of a
// frozen vertex is admissible only when it leads below the best g of the run (aspiration).
// Ties: the j-th admissible minimum in (v asc, c asc) order, j uniform from the iteration's
// Philox block. The run keeps the best g visited; best_fc receives (f, c) of that colouring.
// Generalised objective g = fscale f + phi c (fscale = 1 is Eq. AFISA_score with an integer
// phi; fscale > 1 holds phi in fixed point with resolution 1 / fscale).
int32_t oracle_wvcp_tabu_scaled(int32_t n, const uint8_t* adj, const int32_t* w, int32_t k, const int16_t* col_in,
                                int64_t iters, int32_t L_max, int32_t alpha_num, int32_t alpha_den, int64_t fscale,
                                int64_t phi, uint64_t seed, uint32_t ind, uint32_t gen, int16_t* best_col,
                                int64_t* best_g_out, int64_t* best_fc, int64_t* moves_out, int32_t* trace, int32_t check) {
  auto nb = neighbour_lists(n, adj);
  std::vector<int16_t> col(col_in, col_in + n);
  for (int v = 0; v < n; ++v)
    if (col[v] < 0 || col[v] >= k) return -1;
  std::vector<int32_t> gamma;
  int64_t conf = build_gamma(n, k, nb, col.data(), gamma);
  int64_t f = oracle_wvcp_score(n, adj, w, k, col.data(), nullptr);
  int64_t g = fscale * f + phi * conf;
  std::vector<int64_t> frozen(n, 0);
  int64_t best_g = g, best_f = f, best_c = conf, moves = 0;
  std::copy(col.begin(), col.end(), best_col);
  const int64_t tt_base = ((int64_t)alpha_num * n) / alpha_den;
  std::vector<int64_t> max1(k), max2(k), cnt1(k);
  for (int64_t it = 0; it < iters; ++it) {
    // class maxima: largest weight, how many vertices carry it, and the next smaller weight
    std::fill(max1.begin(), max1.end(), 0);
    std::fill(max2.begin(), max2.end(), 0);
    std::fill(cnt1.begin(), cnt1.end(), 0);
    for (int v = 0; v < n; ++v) {
      const int c = col[v];
      if (w[v] > max1[c]) { max2[c] = max1[c]; max1[c] = w[v]; cnt1[c] = 1; }
      else if (w[v] == max1[c]) cnt1[c]++;
      else if (w[v] > max2[c]) max2[c] = w[v];
    }
    uint32_t r[4];
    draw(seed, (uint32_t)it, gen, ind, TAG_TABU, r);
    int64_t dmin = INT64_MAX, ties = 0;
    // change of f when v moves to c: its old class may lose its maximum, the new one may gain
    auto df_of = [&](int v, int c) -> int64_t {
      const int o = col[v];
      const int64_t old_after = (w[v] == max1[o] && cnt1[o] == 1) ? max2[o] : max1[o];
      return (old_after - max1[o]) + (std::max<int64_t>(max1[c], w[v]) - max1[c]);
    };
    auto delta_of = [&](int v, int c) -> int64_t {
      const int o = col[v];
      return fscale * df_of(v, c) + phi * (int64_t)(gamma[(size_t)v * k + c] - gamma[(size_t)v * k + o]);
    };
    for (int v = 0; v < n; ++v)
      for (int c = 0; c < k; ++c) {
        if (c == col[v]) continue;
        const int64_t delta = delta_of(v, c);
        if (!(frozen[v] <= it || g + delta < best_g)) continue;
        if (delta < dmin) { dmin = delta; ties = 1; }
        else if (delta == dmin) ++ties;
      }
    if (ties == 0) {
      if (trace) { trace[4 * it] = -1; trace[4 * it + 1] = -1; trace[4 * it + 2] = 0; trace[4 * it + 3] = 0; }
      continue;
    }
    const int64_t pick = below(r[0], (uint32_t)ties);
    int mv = -1, mc = -1;
    int64_t seen = 0;
    for (int v = 0; v < n && mv < 0; ++v)
      for (int c = 0; c < k; ++c) {
        if (c == col[v]) continue;
        const int64_t delta = delta_of(v, c);
        if (!(frozen[v] <= it || g + delta < best_g) || delta != dmin) continue;
        if (seen == pick) { mv = v; mc = c; break; }
        ++seen;
      }
    const int old = col[mv];
    const int64_t dfm = df_of(mv, mc);
    conf += gamma[(size_t)mv * k + mc] - gamma[(size_t)mv * k + old];
    col[mv] = (int16_t)mc;
    for (int u : nb[mv]) {
      gamma[(size_t)u * k + old]--;
      gamma[(size_t)u * k + mc]++;
    }
    const int64_t g_before = g;
    g += dmin;
    f += dfm;
    frozen[mv] = it + 1 + (int64_t)below(r[1], (uint32_t)(L_max + 1)) + tt_base;
    ++moves;
    if (g < best_g) { best_g = g; best_f = f; best_c = conf; std::copy(col.begin(), col.end(), best_col); }
    if (trace) { trace[4 * it] = mv; trace[4 * it + 1] = mc; trace[4 * it + 2] = (int32_t)dmin; trace[4 * it + 3] = (int32_t)ties; }
    if (check) {
      std::vector<int32_t> g2;
      const int64_t c2 = build_gamma(n, k, nb, col.data(), g2);
      const int64_t f2 = oracle_wvcp_score(n, adj, w, k, col.data(), nullptr);
      if (g2 != gamma || c2 != conf || f2 != f || fscale * f2 + phi * c2 != g || g - g_before != dmin) return -2;
    }
  }
  *best_g_out = best_g;
  best_fc[0] = best_f;
  best_fc[1] = best_c;
  if (moves_out) *moves_out = moves;
  return 0;
}

int32_t oracle_wvcp_tabu(int32_t n, const uint8_t* adj, const int32_t* w, int32_t k, const int16_t* col_in,
                         int64_t iters, int32_t L_max, int32_t alpha_num, int32_t alpha_den, int64_t phi,
                         uint64_t seed, uint32_t ind, uint32_t gen, int16_t* best_col, int64_t* best_g_out,
                         int64_t* best_fc, int64_t* moves_out, int32_t* trace, int32_t check) {
  return oracle_wvcp_tabu_scaled(n, adj, w, k, col_in, iters, L_max, alpha_num, alpha_den, 1, phi, seed, ind, gen,
                                 best_col, best_g_out, best_fc, moves_out, trace, check);
}

// Parallel iterated feasible and infeasible tabu search (Algorithm 2), one individual. max_ls
// successive searches of `iters` iterations each, from the previous search's best colouring
// (by g). phi is held in fixed point with resolution 1 / fscale and starts at phi0. After search
// t, when t + 1 < max_ls - 1, phi is halved (floor, at least 1) if that search's best colouring
// is legal and doubled otherwise; the last search (t = max_ls - 1) uses phi_last (the paper's
// 2 max w, times fscale). Search t draws from generation gen * 16 + t (max_ls <= 16). The best
// legal colouring over the searches (smallest f) is S'; best_f = -1 when no search ended legal
// (best_col then receives the last search's best colouring). phi_trace (max_ls, or null)
// receives the phi each search used; fc_trace (2 max_ls, or null) each search's (f, c).
int32_t oracle_wvcp_iterated(int32_t n, const uint8_t* adj, const int32_t* w, int32_t k, const int16_t* col_in,
                             int64_t iters, int32_t max_ls, int32_t L_max, int32_t alpha_num, int32_t alpha_den,
                             int64_t fscale, int64_t phi0, int64_t phi_last, uint64_t seed, uint32_t ind, uint32_t gen,
                             int16_t* best_col, int64_t* best_f, int64_t* phi_trace, int64_t* fc_trace) {
  if (max_ls < 1 || max_ls > 16 || fscale < 1 || phi0 < 1 || phi_last < 1) return -1;
  std::vector<int16_t> s(col_in, col_in + n), sb(n);
  int64_t phi = phi0, bf = -1;
  for (int t = 0; t < max_ls; ++t) {
    if (t == max_ls - 1) phi = phi_last;
    if (phi_trace) phi_trace[t] = phi;
    int64_t bg, fc[2], mv;
    const int32_t rc = oracle_wvcp_tabu_scaled(n, adj, w, k, s.data(), iters, L_max, alpha_num, alpha_den, fscale, phi,
                                               seed, ind, gen * 16u + (uint32_t)t, sb.data(), &bg, fc, &mv, nullptr, 0);
    if (rc != 0) return rc;
    s = sb;
    if (fc_trace) { fc_trace[2 * t] = fc[0]; fc_trace[2 * t + 1] = fc[1]; }
    if (fc[1] == 0 && (bf < 0 || fc[0] < bf)) {
      bf = fc[0];
      std::copy(s.begin(), s.end(), best_col);
    }
    if (t + 1 < max_ls - 1) phi = fc[1] == 0 ? std::max<int64_t>(1, phi / 2) : phi * 2;
  }
  if (bf < 0) std::copy(s.begin(), s.end(), best_col);
  *best_f = bf;
  return 0;
}

// One generation of Algorithm 1 for the WVCP: as oracle_memetic_generation, with the iterated
// feasible and infeasible tabu search (Algorithm 2, oracle_wvcp_iterated) as the local search of
// every offspring; the fitness of S'_i is the WVCP score f of its best legal colouring, or
// sum(w) + 1 (worse than every legal colouring) when none of its searches ended legal.
int32_t oracle_wvcp_memetic_generation(int32_t n, const uint8_t* adj, const int32_t* w, int32_t k, int32_t p,
                                       int32_t K, int16_t* P, int64_t* fP, int16_t* DP, int16_t* SO, int64_t iters,
                                       int32_t max_ls, int32_t L_max, int32_t a_num, int32_t a_den, int64_t fscale,
                                       int64_t phi0, int64_t phi_last, int32_t use_scorer, int32_t d0, int32_t d,
                                       int32_t nl, double* th, double* am, double* av, int64_t* adam_t,
                                       int32_t epochs, int32_t batch, double lr, const float* ext_scores,
                                       uint64_t seed, uint32_t gen, int16_t* best_col, int64_t* best_f,
                                       int64_t* diag_fprime, int32_t* diag_pick) {
  if (K > p - 1 || K < 1) return -1;
  int64_t wsum = 0;
  for (int v = 0; v < n; ++v) wsum += w[v];
  std::vector<int16_t> Sp((size_t)p * n);
  std::vector<int64_t> fSp(p);
  for (int i = 0; i < p; ++i) {
    int64_t bf = -1;
    const int32_t rc = oracle_wvcp_iterated(n, adj, w, k, SO + (size_t)i * n, iters, max_ls, L_max, a_num, a_den,
                                            fscale, phi0, phi_last, seed, (uint32_t)i, gen, Sp.data() + (size_t)i * n,
                                            &bf, nullptr, nullptr);
    if (rc) return rc;
    fSp[i] = bf >= 0 ? bf : wsum + 1;
  }
  return memetic_after_search(n, k, p, K, P, fP, DP, SO, Sp, fSp, use_scorer, d0, d, nl, th, am, av, adam_t, epochs,
                              batch, lr, ext_scores, seed, gen, best_col, best_f, diag_fprime, diag_pick);
}

}  // extern "C"

