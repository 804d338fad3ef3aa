// One generation of the deep-learning-guided memetic framework (Algorithm 1), stream-ordered on
// the GPU: TabuCol of every offspring -> best-so-far -> scorer training (learned selection) ->
// distances P x P' and P' x P' -> pool update -> gather of the new population and its distance
// matrix -> K nearest neighbours -> GPX offspring (best-scored of K, or one random neighbour).
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "common.cuh"

struct dlm_memetic {
  const dlm_graph* g = nullptr;
  dlm_memetic_params prm{};
  int n = 0;
  uint32_t gen = 0;
  // population state
  int16_t *P = nullptr, *Pn = nullptr, *SO = nullptr, *Sp = nullptr, *best_col = nullptr, *kids = nullptr;
  int64_t *fP = nullptr, *fPn = nullptr, *fSp = nullptr, *fall = nullptr, *best_f = nullptr, *moves = nullptr;
  int16_t *DP = nullptr, *Dall = nullptr;
  int32_t *sel = nullptr, *nbr = nullptr, *pairs = nullptr, *pick = nullptr;
  uint32_t* cid = nullptr;
  float* scores = nullptr;
  // per-generation diagnostics: the predicted score of each selected offspring (learned
  // selection), the standardisation of the last training targets, and the statistics of the last
  // generation (k_gen_stats)
  float* pred = nullptr;
  double* dstat = nullptr;  // [16] device: accumulators and results
  double* h_stat = nullptr;  // [16] pinned
  uint64_t fingerprint = 0;  // of the graph's bit rows and of every search / training parameter
  // WVCP (problem 1): the total weight (fitness of an offspring that never became legal) and the
  // fixed-point penalty schedule of the iterated search
  int64_t wsum = 0, phi0 = 0, phi_last = 0;
  int64_t* h_best = nullptr;  // pinned
  dlm_scorer* scorer = nullptr;
  dlm_deepnet* deep = nullptr;  // use_scorer = 2: the paper-size network
  // the scorer trains on a side stream while the distances and the pool update run
  cudaStream_t side = nullptr;
  cudaEvent_t ev_ready = nullptr, ev_trained = nullptr;
  // the start of the last generation and the end of its best-so-far update (dlm_memetic_found_ms)
  cudaEvent_t ev_gen = nullptr, ev_found = nullptr;
  // optional stage timing (dlm_memetic_profile): events at the stage boundaries of the main
  // stream (tabu, best-so-far, distances, pool update, matching, offspring) and around training
  bool prof = false;
  // (pev[7], pev[8]: the offspring stage's GPX end and, with the scorer, the end of its wait for
  // the training)
  cudaEvent_t pev[9] = {}, tev[2] = {};
  double stage_ms[10] = {};
  int64_t prof_gens = 0;
};

namespace dlm {

__global__ void k_best_of(int p, int n, const int64_t* fSp, const int16_t* Sp, int64_t* best_f, int16_t* best_col) {
  __shared__ unsigned long long s[32];
  __shared__ int win;
  unsigned long long key = ~0ull;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const unsigned long long kk = ((unsigned long long)fSp[i] << 20) | (unsigned)i;
    key = kk < key ? kk : key;
  }
  for (int d = 16; d >= 1; d >>= 1) {
    const unsigned long long o = __shfl_down_sync(0xFFFFFFFFu, key, d);
    key = o < key ? o : key;
  }
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = key;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = ~0ull;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = s[w] < b ? s[w] : b;
    const int ib = (int)(b & 0xFFFFF);
    win = -1;
    if (fSp[ib] < *best_f) { *best_f = fSp[ib]; win = ib; }
  }
  __syncthreads();
  if (win >= 0)
    for (int v = threadIdx.x; v < n; v += blockDim.x) best_col[v] = Sp[(size_t)win * n + v];
}

// Dall (2p x 2p): top-left <- DP, mirror of the cross block, mirror + zero diagonal of the P'P' block
__global__ void k_dall_assemble(int p, const int16_t* DP, int16_t* Dall) {
  const int m = 2 * p;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * m) return;
  const int r = (int)(t / m), c = (int)(t % m);
  int16_t v;
  if (r < p && c < p) v = DP[(size_t)r * p + c];
  else if (r >= p && c < p) v = Dall[(size_t)c * m + r];        // cross block computed as rows < p
  else if (r >= p && c >= p) v = r == c ? 0 : (c > r ? Dall[(size_t)r * m + c] : Dall[(size_t)c * m + r]);
  else return;  // r < p, c >= p: computed in place
  Dall[(size_t)r * m + c] = v;
}

__global__ void k_fit_all(int p, const int64_t* fP, const int64_t* fSp, int64_t* fall) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < p) { fall[t] = fP[t]; fall[p + t] = fSp[t]; }
}

__global__ void k_gather_pop(int p, int n, const int32_t* sel, const int16_t* P, const int16_t* Sp, const int64_t* fall,
                             int16_t* Pn, int64_t* fPn) {
  const int s = blockIdx.x;
  const int x = sel[s];
  const int16_t* src = x < p ? P + (size_t)x * n : Sp + (size_t)(x - p) * n;
  for (int v = threadIdx.x; v < n; v += blockDim.x) Pn[(size_t)s * n + v] = src[v];
  if (threadIdx.x == 0) fPn[s] = fall[x];
}

__global__ void k_gather_dist(int p, const int32_t* sel, const int16_t* Dall, int16_t* DP) {
  const int s = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p) return;
  DP[(size_t)s * p + t] = Dall[(size_t)sel[s] * (2 * p) + sel[t]];
}

// random GPX: one neighbour per individual, drawn from the SELECT stream
__global__ void k_pairs_random(int p, int K, const int32_t* nbr, uint64_t seed, uint32_t gen, int32_t* pairs,
                               uint32_t* cid, int32_t* pick) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p) return;
  const U4 r = rng(seed, (uint32_t)i, gen, 0u, kTagSelect);
  const int j = (int)below(r.x, (uint32_t)K);
  pairs[2 * i] = i;
  pairs[2 * i + 1] = nbr[(size_t)i * K + j];
  cid[i] = (uint32_t)(i * K + j);
  pick[i] = j;
}

// learned selection: all K neighbours
__global__ void k_pairs_all(int p, int K, const int32_t* nbr, int32_t* pairs, uint32_t* cid) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p * K) return;
  pairs[2 * t] = t / K;
  pairs[2 * t + 1] = nbr[t];
  cid[t] = (uint32_t)t;
}

// argmin over the K scores of individual i, visiting j in order: the first candidate is taken and
// only a strictly smaller score replaces it (ties: lowest j); copies that child into S^O_i
__global__ void k_select_best(int p, int K, int n, const float* scores, const int16_t* kids, int16_t* SO, int32_t* pick,
                              float* pred) {
  const int i = blockIdx.x;
  __shared__ int best;
  if (threadIdx.x == 0) {
    int bj = 0;
    float bv = scores[(size_t)i * K];
    for (int j = 1; j < K; ++j) {
      const float sc = scores[(size_t)i * K + j];
      if (sc < bv) { bv = sc; bj = j; }
    }
    best = bj;
    pick[i] = bj;
    pred[i] = bv;
  }
  __syncthreads();
  const int16_t* src = kids + ((size_t)i * K + best) * n;
  for (int v = threadIdx.x; v < n; v += blockDim.x) SO[(size_t)i * n + v] = src[v];
}

// Per-generation diagnostics (section "Analysis of the contributions of deep learning": the
// predicted against the actual fitness of the selected offspring, and the spread of the
// population). dstat layout: [0..7] results of the last generation (generation, Pearson of
// prediction and actual f(S'), mean relative error of the de-standardised prediction, mean f(S'),
// min f(S'), mean / min / max distance between distinct members of P), [8..9] mean and std of the
// f(S') the scorer was last trained on, [10..12] distance accumulators (sum, min, max).
__global__ void k_dist_stats(int p, const int16_t* D, double* dstat) {
  double sum = 0.0;
  int mn = INT_MAX, mx = INT_MIN;
  const int64_t tot = (int64_t)p * p;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / p), c = (int)(t - (int64_t)r * p);
    if (r == c) continue;
    const int v = D[t];
    sum += v;
    mn = min(mn, v);
    mx = max(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(dstat + 10, sum);
    atomicMin((unsigned long long*)(dstat + 11), (unsigned long long)(int64_t)mn);  // non-negative ints
    atomicMax((unsigned long long*)(dstat + 12), (unsigned long long)(int64_t)mx);
  }
}

// one block: prediction quality over the p offspring just searched (pred from the previous
// selection, learned = 1 when there was one), then the distance results; trained = 1 records the
// standardisation of f(S') the scorer is trained on now
__global__ void __launch_bounds__(1024) k_gen_stats(int p, uint32_t gen, int learned, int trained, const float* pred,
                                                    const int64_t* fSp, double* dstat) {
  __shared__ double red[6][32];
  double sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0, are = 0;
  int64_t mnf = INT64_MAX;
  const double mu = dstat[8], sd = dstat[9];
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const double y = (double)fSp[i];
    mnf = min(mnf, (int64_t)fSp[i]);
    sy += y; syy += y * y;
    if (learned) {
      const double x = pred[i];
      sx += x; sxx += x * x; sxy += x * y;
      const double yhat = mu + sd * x;
      are += fabs(yhat - y) / fmax(y, 1.0);
    }
  }
  double v[6] = {sx, sy, sxx, syy, sxy, are};
  for (int q = 0; q < 6; ++q) {
    double a = v[q];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = a;
  }
  __shared__ long long smn[32];
  long long m2 = mnf;
  for (int o = 16; o > 0; o >>= 1) m2 = min(m2, __shfl_xor_sync(0xFFFFFFFFu, m2, o));
  if ((threadIdx.x & 31) == 0) smn[threadIdx.x >> 5] = m2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[6] = {0, 0, 0, 0, 0, 0};
    long long mm = LLONG_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      for (int q = 0; q < 6; ++q) t[q] += red[q][w];
      mm = min(mm, smn[w]);
    }
    const double np = p;
    dstat[0] = gen;
    if (learned) {
      const double cxy = t[4] - t[0] * t[1] / np, cxx = t[2] - t[0] * t[0] / np, cyy = t[3] - t[1] * t[1] / np;
      dstat[1] = (cxx > 0 && cyy > 0) ? cxy / sqrt(cxx * cyy) : 0.0;
      dstat[2] = t[5] / np;
    } else {
      dstat[1] = nan("");
      dstat[2] = nan("");
    }
    dstat[3] = t[1] / np;
    dstat[4] = (double)mm;
    if (trained) {  // the mean and (population) std of f(S') the scorer is being trained on
      dstat[8] = t[1] / np;
      const double var = t[3] / np - dstat[8] * dstat[8];
      dstat[9] = var > 0 ? sqrt(var) : 1.0;
    }
  }
}

__global__ void k_dist_stats_init(double* dstat) {
  dstat[10] = 0.0;
  *(unsigned long long*)(dstat + 11) = (unsigned long long)INT64_MAX;
  *(unsigned long long*)(dstat + 12) = 0ull;
}

__global__ void k_dist_stats_done(int p, double* dstat) {
  const double pairs = (double)p * (p - 1);
  dstat[5] = pairs > 0 ? dstat[10] / pairs : 0.0;
  dstat[6] = (double)(int64_t)*(unsigned long long*)(dstat + 11);
  dstat[7] = (double)(int64_t)*(unsigned long long*)(dstat + 12);
}

// WVCP score f(S) = sum over colour classes of the largest weight in the class (section "Weighted
// vertex coloring problem"), one block per colouring; k <= 256
__global__ void __launch_bounds__(256) k_wvcp_fitness(int n, int k, const int16_t* col, const int32_t* w, int64_t* f) {
  __shared__ int mx[256];
  for (int c = threadIdx.x; c < k; c += blockDim.x) mx[c] = 0;
  __syncthreads();
  const int16_t* s = col + (size_t)blockIdx.x * n;
  for (int v = threadIdx.x; v < n; v += blockDim.x) atomicMax(&mx[s[v]], w[v]);
  __syncthreads();
  if (threadIdx.x < 32) {
    long long t = 0;
    for (int c = threadIdx.x; c < k; c += 32) t += mx[c];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if (threadIdx.x == 0) f[blockIdx.x] = t;
  }
}

// an offspring none of whose searches ended legal (best f = -1) gets sum(w) + 1, above every legal
// colouring's score
__global__ void k_wvcp_fix(int p, int64_t wsum, int64_t* f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < p && f[i] < 0) f[i] = wsum + 1;
}

template <typename T>
static dlm_status alloc(dlm_ctx* ctx, T** p, size_t count) {
  if (cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DLM_ENOMEM, "memetic: device allocation failed");
  }
  return DLM_OK;
}

}  // namespace dlm

using namespace dlm;

extern "C" void dlm_memetic_destroy(dlm_memetic* mm) {
  if (!mm) return;
  cudaFree(mm->P); cudaFree(mm->Pn); cudaFree(mm->SO); cudaFree(mm->Sp); cudaFree(mm->best_col); cudaFree(mm->kids);
  cudaFree(mm->fP); cudaFree(mm->fPn); cudaFree(mm->fSp); cudaFree(mm->fall); cudaFree(mm->best_f); cudaFree(mm->moves);
  cudaFree(mm->DP); cudaFree(mm->Dall); cudaFree(mm->sel); cudaFree(mm->nbr); cudaFree(mm->pairs); cudaFree(mm->pick);
  cudaFree(mm->cid); cudaFree(mm->scores); cudaFree(mm->pred); cudaFree(mm->dstat);
  if (mm->h_best) cudaFreeHost(mm->h_best);
  if (mm->h_stat) cudaFreeHost(mm->h_stat);
  if (mm->scorer) dlm_scorer_destroy(mm->scorer);
  if (mm->deep) dlm_deepnet_destroy(mm->deep);
  for (auto e : mm->pev) if (e) cudaEventDestroy(e);
  for (auto e : mm->tev) if (e) cudaEventDestroy(e);
  if (mm->ev_ready) cudaEventDestroy(mm->ev_ready);
  if (mm->ev_trained) cudaEventDestroy(mm->ev_trained);
  if (mm->ev_gen) cudaEventDestroy(mm->ev_gen);
  if (mm->ev_found) cudaEventDestroy(mm->ev_found);
  if (mm->side) cudaStreamDestroy(mm->side);
  delete mm;
}

extern "C" dlm_status dlm_memetic_create(dlm_ctx* ctx, const dlm_graph* g, const dlm_memetic_params* prm,
                                         dlm_memetic** out) {
  if (!ctx || !g || !prm || !out) return fail(ctx, DLM_EINVAL, "memetic_create: null argument");
  *out = nullptr;
  const int p = prm->p, K = prm->K, n = g->n, k = prm->k;
  const bool wvcp = prm->problem == 1;
  if (prm->problem != 0 && prm->problem != 1) return fail(ctx, DLM_EINVAL, "memetic_create: problem must be 0 or 1");
  if (p < 2 || K < 1 || K > p - 1 || K > 64 || k < 2 || k > (wvcp ? 255 : 128) || prm->iters < 0)
    return fail(ctx, DLM_EINVAL, "memetic_create: need p >= 2, 1 <= K <= min(64, p-1), 2 <= k <= 128 (255 for WVCP)");
  if (p > 8192) return fail(ctx, DLM_EUNSUPPORTED, "memetic_create: p must be <= 8192");
  if (wvcp && !g->d_weight) return fail(ctx, DLM_EINVAL, "memetic_create: WVCP needs a graph with vertex weights");
  if (wvcp && (prm->max_ls < 1 || prm->max_ls > 16)) return fail(ctx, DLM_EINVAL, "memetic_create: max_ls must be in 1..16");
  if (prm->use_scorer < 0 || prm->use_scorer > 2) return fail(ctx, DLM_EINVAL, "memetic_create: use_scorer must be 0, 1 or 2");
  if (prm->use_scorer && (prm->epochs < 0 || prm->batch < 1)) return fail(ctx, DLM_EINVAL, "memetic_create: bad training parameters");
  dlm_memetic* mm = new dlm_memetic();
  mm->g = g;
  mm->prm = *prm;
  mm->n = n;
  const size_t pn = (size_t)p * n;
  const int nk = prm->use_scorer ? K : 1;
  dlm_status st = DLM_OK;
  auto A = [&](auto** ptr, size_t cnt) { if (st == DLM_OK) st = alloc(ctx, ptr, cnt); };
  A(&mm->P, pn); A(&mm->Pn, pn); A(&mm->SO, pn); A(&mm->Sp, pn); A(&mm->best_col, (size_t)n);
  A(&mm->kids, pn * nk);
  A(&mm->fP, (size_t)p); A(&mm->fPn, (size_t)p); A(&mm->fSp, (size_t)p); A(&mm->fall, (size_t)2 * p);
  A(&mm->best_f, 1); A(&mm->moves, (size_t)p);
  A(&mm->DP, (size_t)p * p); A(&mm->Dall, (size_t)4 * p * p);
  A(&mm->sel, (size_t)p); A(&mm->nbr, (size_t)p * K); A(&mm->pairs, (size_t)2 * p * nk); A(&mm->pick, (size_t)p);
  A(&mm->cid, (size_t)p * nk); A(&mm->scores, (size_t)p * K); A(&mm->pred, (size_t)p); A(&mm->dstat, 16);
  if (st == DLM_OK && cudaMallocHost(&mm->h_best, sizeof(int64_t)) != cudaSuccess) st = fail(ctx, DLM_ENOMEM, "pinned");
  if (st == DLM_OK && cudaMallocHost(&mm->h_stat, 16 * sizeof(double)) != cudaSuccess) st = fail(ctx, DLM_ENOMEM, "pinned");
  if (st == DLM_OK) st = cuda_check(ctx, cudaMemsetAsync(mm->dstat, 0, 16 * sizeof(double), ctx->stream), "memset");
  if (st == DLM_OK && prm->use_scorer == 1) st = dlm_scorer_create(ctx, n, k, prm->seed, &mm->scorer);
  // the selection takes the best-scored of each individual's K children: bf16 activations (two
  // MMA passes) keep every group's best equal to the FP64 one's in the parity tests, at a third
  // of the split-activation scoring time
  if (st == DLM_OK && prm->use_scorer == 1) st = dlm_scorer_set_scoring_precision(ctx, mm->scorer, 0);
  if (st == DLM_OK && prm->use_scorer == 2) {  // hidden widths of section "Implementation and parameter setting"
    std::vector<int32_t> w = wvcp ? std::vector<int32_t>{5 * n, 2 * n, n, std::max(1, n / 2)}
                                  : std::vector<int32_t>{10 * n, 5 * n, 2 * n, 2 * n, 2 * n, 2 * n, 2 * n, n,
                                                         std::max(1, n / 2)};
    st = dlm_deepnet_create(ctx, n, k, (int32_t)w.size(), w.data(), prm->seed, &mm->deep);
  }
  int prio_least = 0, prio_greatest = 0;  // the training's short kernels take SMs as the distance blocks drain
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (st == DLM_OK && prm->use_scorer &&
      (cudaStreamCreateWithPriority(&mm->side, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
       cudaEventCreateWithFlags(&mm->ev_ready, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&mm->ev_trained, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    st = fail(ctx, DLM_ECUDA, "memetic_create: side stream");
  }
  if (st == DLM_OK && (cudaEventCreate(&mm->ev_gen) != cudaSuccess || cudaEventCreate(&mm->ev_found) != cudaSuccess)) {
    cudaGetLastError();
    st = fail(ctx, DLM_ECUDA, "memetic_create: events");
  }
  if (st != DLM_OK) { dlm_memetic_destroy(mm); return st; }
  // fingerprint (FNV-1a, 64 bits) of the graph's bit rows and of the parameters: a checkpoint
  // only loads into a run of the same problem
  if (st == DLM_OK) {
    std::vector<uint32_t> hb((size_t)g->n * g->words);
    st = cuda_check(ctx, cudaMemcpy(hb.data(), g->d_bits, hb.size() * 4, cudaMemcpyDeviceToHost), "copy");
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* d, size_t len) {
      const uint8_t* b = (const uint8_t*)d;
      for (size_t i = 0; i < len; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    };
    mix(hb.data(), hb.size() * 4);
    mix(&g->n, sizeof(g->n));
    mix(&prm->k, sizeof(prm->k)); mix(&prm->p, sizeof(prm->p)); mix(&prm->K, sizeof(prm->K));
    mix(&prm->iters, sizeof(prm->iters)); mix(&prm->tenure, sizeof(prm->tenure));
    mix(&prm->use_scorer, sizeof(prm->use_scorer)); mix(&prm->epochs, sizeof(prm->epochs));
    mix(&prm->batch, sizeof(prm->batch)); mix(&prm->lr, sizeof(prm->lr)); mix(&prm->seed, sizeof(prm->seed));
    mix(&prm->problem, sizeof(prm->problem));
    if (wvcp && st == DLM_OK) {
      std::vector<int32_t> hw((size_t)n);
      st = cuda_check(ctx, cudaMemcpy(hw.data(), g->d_weight, (size_t)n * 4, cudaMemcpyDeviceToHost), "copy");
      mix(hw.data(), hw.size() * 4);
      mix(&prm->max_ls, sizeof(prm->max_ls));
      for (int32_t x : hw) mm->wsum += x;
      // phi0 = k max w / (2 |V|) and phi_last = 2 max w (Algorithm 2), in fixed point of 1/256
      const int64_t wmax = g->max_weight;
      mm->phi0 = std::max<int64_t>(1, (256 * (int64_t)k * wmax + n) / (2 * (int64_t)n));
      mm->phi_last = std::max<int64_t>(1, 256 * 2 * wmax);
    }
    mm->fingerprint = h;
  }
  if (st != DLM_OK) { dlm_memetic_destroy(mm); return st; }
  // initial population: random colourings (k-COL) or the randomised greedy initialisation (WVCP),
  // their fitness and their distance matrix
  const int64_t big = INT64_MAX;
  if (wvcp) {
    st = dlm_wvcp_greedy(ctx, g, p, prm->seed, 0u, mm->P, mm->sel);
    if (st == DLM_OK) {
      std::vector<int32_t> used((size_t)p);
      st = cuda_check(ctx, cudaMemcpy(used.data(), mm->sel, (size_t)p * 4, cudaMemcpyDeviceToHost), "copy");
      if (st == DLM_OK && *std::max_element(used.begin(), used.end()) > k)
        st = fail(ctx, DLM_EINVAL, "memetic_create: the greedy initialisation opens more than k colours");
    }
    if (st == DLM_OK) {
      k_wvcp_fitness<<<p, 256, 0, ctx->stream>>>(n, k, mm->P, g->d_weight, mm->fP);
      st = launch_check(ctx, "k_wvcp_fitness");
    }
  } else {
    st = dlm_init_colors(ctx, n, k, p, prm->seed, 0u, mm->P);
    if (st == DLM_OK) st = dlm_gamma(ctx, g, k, p, mm->P, nullptr, mm->fP);
  }
  if (st == DLM_OK) st = dlm_distance_batch(ctx, n, k, mm->P, p, mm->P, p, mm->DP, p, 0);
  if (st == DLM_OK) st = cuda_check(ctx, cudaMemcpyAsync(mm->SO, mm->P, pn * 2, cudaMemcpyDeviceToDevice, ctx->stream), "copy");
  if (st == DLM_OK) st = cuda_check(ctx, cudaMemcpyAsync(mm->best_f, &big, 8, cudaMemcpyHostToDevice, ctx->stream), "copy");
  if (st == DLM_OK) st = cuda_check(ctx, cudaMemsetAsync(mm->Dall, 0, (size_t)4 * p * p * 2, ctx->stream), "memset");
  if (st == DLM_OK) st = cuda_check(ctx, cudaMemsetAsync(mm->best_col, 0, (size_t)n * 2, ctx->stream), "memset");
  if (st == DLM_OK) st = dlm_sync(ctx);
  if (st != DLM_OK) { dlm_memetic_destroy(mm); return st; }
  *out = mm;
  return DLM_OK;
}

extern "C" dlm_status dlm_memetic_step(dlm_ctx* ctx, dlm_memetic* mm, int64_t* best_f_host) {
  if (!ctx || !mm) return fail(ctx, DLM_EINVAL, "memetic_step: null argument");
  const dlm_memetic_params& q = mm->prm;
  const int p = q.p, K = q.K, n = mm->n, k = q.k, m = 2 * p;
  const size_t pn = (size_t)p * n;
  cudaStream_t s = ctx->stream;
  auto mark = [&](int i) { if (mm->prof) cudaEventRecord(mm->pev[i], s); };
  DLM_CUDA(ctx, cudaEventRecord(mm->ev_gen, s));
  mark(0);
  // 1. local search of every offspring: S'_i <- TabuCol(S^O_i) (k-COL), or the iterated feasible
  //    and infeasible tabu search from S^O_i (WVCP; Pn, free until the gather, holds its running
  //    colourings)
  if (q.problem == 1) {
    DLM_CUDA(ctx, cudaMemcpyAsync(mm->Pn, mm->SO, pn * 2, cudaMemcpyDeviceToDevice, s));
    DLM_TRY(dlm_wvcp_iterated(ctx, mm->g, k, p, mm->Pn, mm->Sp, mm->fSp, q.iters, q.max_ls, q.tenure, 256, mm->phi0,
                              mm->phi_last, q.seed, mm->gen, 0u));
    k_wvcp_fix<<<(p + 255) / 256, 256, 0, s>>>(p, mm->wsum, mm->fSp);
    DLM_TRY(launch_check(ctx, "k_wvcp_fix"));
  } else {
    DLM_CUDA(ctx, cudaMemcpyAsync(mm->Sp, mm->SO, pn * 2, cudaMemcpyDeviceToDevice, s));
    DLM_TRY(dlm_tabucol_batch(ctx, mm->g, k, p, mm->Sp, mm->fSp, mm->moves, q.iters, q.tenure, q.seed, mm->gen, 0u));
  }
  mark(1);
  // 2. best so far
  k_best_of<<<1, 1024, 0, s>>>(p, n, mm->fSp, mm->Sp, mm->best_f, mm->best_col);
  DLM_TRY(launch_check(ctx, "k_best_of"));
  DLM_CUDA(ctx, cudaEventRecord(mm->ev_found, s));
  // diagnostics: the last selection's predictions against the conflicts its offspring reached
  k_gen_stats<<<1, 1024, 0, s>>>(p, mm->gen, (q.use_scorer && mm->gen > 0) ? 1 : 0, q.use_scorer ? 1 : 0, mm->pred,
                                 mm->fSp, mm->dstat);
  DLM_TRY(launch_check(ctx, "k_gen_stats"));
  mark(2);
  // 3. training on {(S^O_i, f(S'_i))}, on the side stream: it only reads S^O and f(S'), which
  //    nothing below writes before the scoring, and the scoring waits for it
  if (q.use_scorer) {
    DLM_CUDA(ctx, cudaEventRecord(mm->ev_ready, s));
    DLM_CUDA(ctx, cudaStreamWaitEvent(mm->side, mm->ev_ready, 0));
    ctx->stream = mm->side;
    if (mm->prof) cudaEventRecord(mm->tev[0], mm->side);
    const dlm_status ts = mm->deep ? dlm_deepnet_train(ctx, mm->deep, mm->SO, mm->fSp, p, q.epochs, q.batch, q.lr,
                                                       q.seed, mm->gen)
                                   : dlm_scorer_train(ctx, mm->scorer, mm->SO, mm->fSp, p, q.epochs, q.batch, q.lr,
                                                      q.seed, mm->gen);
    if (mm->prof) cudaEventRecord(mm->tev[1], mm->side);
    ctx->stream = s;
    DLM_TRY(ts);
    DLM_CUDA(ctx, cudaEventRecord(mm->ev_trained, mm->side));
  }
  // 4. distances: P x P' (rows < p, columns >= p) and P' x P' (upper triangle), then assemble
  DLM_TRY(dlm_distance_batch(ctx, n, k, mm->P, p, mm->Sp, p, mm->Dall + p, m, 0));
  DLM_TRY(dlm_distance_batch(ctx, n, k, mm->Sp, p, mm->Sp, p, mm->Dall + (size_t)p * m + p, m, 1));
  {
    const int64_t tot = (int64_t)m * m;
    k_dall_assemble<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(p, mm->DP, mm->Dall);
    DLM_TRY(launch_check(ctx, "k_dall_assemble"));
  }
  mark(3);
  // 5. pool update over P u P'
  k_fit_all<<<(p + 255) / 256, 256, 0, s>>>(p, mm->fP, mm->fSp, mm->fall);
  DLM_TRY(launch_check(ctx, "k_fit_all"));
  DLM_TRY(dlm_pool_update(ctx, p, n, mm->fall, mm->Dall, mm->sel));
  k_gather_pop<<<p, 128, 0, s>>>(p, n, mm->sel, mm->P, mm->Sp, mm->fall, mm->Pn, mm->fPn);
  DLM_TRY(launch_check(ctx, "k_gather_pop"));
  k_gather_dist<<<dim3((p + 255) / 256, p), 256, 0, s>>>(p, mm->sel, mm->Dall, mm->DP);
  DLM_TRY(launch_check(ctx, "k_gather_dist"));
  std::swap(mm->P, mm->Pn);
  std::swap(mm->fP, mm->fPn);
  mark(4);
  // 6. parent matching
  DLM_TRY(dlm_knn(ctx, p, mm->DP, K, mm->nbr));
  // diagnostics: the spread of the new population
  k_dist_stats_init<<<1, 1, 0, s>>>(mm->dstat);
  k_dist_stats<<<ctx->num_sms * 2, 256, 0, s>>>(p, mm->DP, mm->dstat);
  k_dist_stats_done<<<1, 1, 0, s>>>(p, mm->dstat);
  DLM_TRY(launch_check(ctx, "k_dist_stats"));
  mark(5);
  // 7. offspring
  if (q.use_scorer) {
    k_pairs_all<<<(p * K + 255) / 256, 256, 0, s>>>(p, K, mm->nbr, mm->pairs, mm->cid);
    DLM_TRY(launch_check(ctx, "k_pairs_all"));
    DLM_TRY(dlm_gpx_batch(ctx, n, k, mm->P, p, mm->pairs, mm->cid, p * K, mm->kids, q.seed, mm->gen));
    mark(7);
    DLM_CUDA(ctx, cudaStreamWaitEvent(s, mm->ev_trained, 0));
    mark(8);
    if (mm->deep) DLM_TRY(dlm_deepnet_forward(ctx, mm->deep, mm->kids, p * K, 0, mm->scores));
    else DLM_TRY(dlm_score_offspring(ctx, mm->scorer, mm->kids, p * K, mm->scores));
    k_select_best<<<p, 128, 0, s>>>(p, K, n, mm->scores, mm->kids, mm->SO, mm->pick, mm->pred);
    DLM_TRY(launch_check(ctx, "k_select_best"));
  } else {
    k_pairs_random<<<(p + 255) / 256, 256, 0, s>>>(p, K, mm->nbr, q.seed, mm->gen, mm->pairs, mm->cid, mm->pick);
    DLM_TRY(launch_check(ctx, "k_pairs_random"));
    DLM_TRY(dlm_gpx_batch(ctx, n, k, mm->P, p, mm->pairs, mm->cid, p, mm->SO, q.seed, mm->gen));
  }
  mark(6);
  if (mm->prof) {
    DLM_CUDA(ctx, cudaEventSynchronize(mm->pev[6]));
    for (int i = 0; i < 6; ++i) {
      float e = 0.f;
      if (cudaEventElapsedTime(&e, mm->pev[i], mm->pev[i + 1]) == cudaSuccess) mm->stage_ms[i] += e;
    }
    float e = 0.f;
    if (q.use_scorer && cudaEventElapsedTime(&e, mm->tev[0], mm->tev[1]) == cudaSuccess) mm->stage_ms[6] += e;
    if (q.use_scorer) {  // the offspring stage in three parts: GPX, the wait for training, scoring and selection
      if (cudaEventElapsedTime(&e, mm->pev[5], mm->pev[7]) == cudaSuccess) mm->stage_ms[7] += e;
      if (cudaEventElapsedTime(&e, mm->pev[7], mm->pev[8]) == cudaSuccess) mm->stage_ms[8] += e;
      if (cudaEventElapsedTime(&e, mm->pev[8], mm->pev[6]) == cudaSuccess) mm->stage_ms[9] += e;
    }
    ++mm->prof_gens;
  }
  mm->gen++;
  if (best_f_host) {
    DLM_CUDA(ctx, cudaMemcpyAsync(mm->h_best, mm->best_f, 8, cudaMemcpyDeviceToHost, s));
    DLM_TRY(dlm_sync(ctx));
    *best_f_host = *mm->h_best;
  }
  return DLM_OK;
}

extern "C" dlm_status dlm_memetic_stats(dlm_ctx* ctx, dlm_memetic* mm, double* out) {
  if (!ctx || !mm || !out) return fail(ctx, DLM_EINVAL, "memetic_stats: null argument");
  DLM_CUDA(ctx, cudaMemcpyAsync(mm->h_stat, mm->dstat, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  DLM_TRY(dlm_sync(ctx));
  for (int i = 0; i < 8; ++i) out[i] = mm->h_stat[i];
  return DLM_OK;
}

extern "C" dlm_status dlm_memetic_get(dlm_ctx* ctx, dlm_memetic* mm, int32_t which, void* dst) {
  if (!ctx || !mm || !dst) return fail(ctx, DLM_EINVAL, "memetic_get: null argument");
  const int p = mm->prm.p, n = mm->n, K = mm->prm.K;
  const void* src = nullptr;
  size_t bytes = 0;
  switch (which) {
    case 0: src = mm->P; bytes = (size_t)p * n * 2; break;
    case 1: src = mm->fP; bytes = (size_t)p * 8; break;
    case 2: src = mm->DP; bytes = (size_t)p * p * 2; break;
    case 3: src = mm->SO; bytes = (size_t)p * n * 2; break;
    case 4: src = mm->best_col; bytes = (size_t)n * 2; break;
    case 5: src = mm->fSp; bytes = (size_t)p * 8; break;
    case 6: src = mm->pick; bytes = (size_t)p * 4; break;
    case 7: if (!mm->prm.use_scorer) return fail(ctx, DLM_EINVAL, "memetic_get: no scores without the scorer");
            src = mm->scores; bytes = (size_t)p * K * 4; break;
    case 8: if (mm->deep) return dlm_deepnet_get(ctx, mm->deep, 0, (float*)dst);
            if (!mm->scorer) return fail(ctx, DLM_EINVAL, "memetic_get: no scorer");
            return dlm_scorer_get_params(ctx, mm->scorer, (float*)dst);
    case 9: if (!mm->deep) return fail(ctx, DLM_EINVAL, "memetic_get: no paper-size network");
            return dlm_deepnet_get(ctx, mm->deep, 1, (float*)dst);
    default: return fail(ctx, DLM_EINVAL, "memetic_get: unknown array");
  }
  DLM_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return DLM_OK;
}

extern "C" dlm_status dlm_memetic_set(dlm_ctx* ctx, dlm_memetic* mm, int32_t which, const void* src) {
  if (!ctx || !mm || !src) return fail(ctx, DLM_EINVAL, "memetic_set: null argument");
  const int p = mm->prm.p, n = mm->n;
  void* dst = nullptr;
  size_t bytes = 0;
  switch (which) {
    case 0: dst = mm->P; bytes = (size_t)p * n * 2; break;
    case 1: dst = mm->fP; bytes = (size_t)p * 8; break;
    case 2: dst = mm->DP; bytes = (size_t)p * p * 2; break;
    case 3: dst = mm->SO; bytes = (size_t)p * n * 2; break;
    default: return fail(ctx, DLM_EINVAL, "memetic_set: unknown array");
  }
  DLM_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return DLM_OK;
}

// ---- checkpoint: the state carried from one generation to the next ------------------------------
namespace {
struct CkptHeader {
  char magic[8];
  int32_t n, k, p, K, use_scorer, reserved;
  uint32_t gen, reserved2;
  int64_t scorer_bytes;
  int64_t total;
  uint64_t fingerprint;  // graph and parameters of the run that wrote it
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");
constexpr char kMagic[8] = {'D', 'L', 'M', 'M', 'E', 'M', '0', '2'};

inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

struct CkptLayout {
  size_t P, fP, DP, SO, best_f, best_col, scorer, total;
};

CkptLayout ckpt_layout(const dlm_memetic* mm) {
  const size_t p = (size_t)mm->prm.p, n = (size_t)mm->n;
  CkptLayout L;
  size_t o = sizeof(CkptHeader);
  L.P = o; o += a16(p * n * 2);
  L.fP = o; o += a16(p * 8);
  L.DP = o; o += a16(p * p * 2);
  L.SO = o; o += a16(p * n * 2);
  L.best_f = o; o += 16;
  L.best_col = o; o += a16(n * 2);
  L.scorer = o;
  o += a16(mm->scorer ? (size_t)dlm_scorer_state_bytes(mm->scorer)
                      : (mm->deep ? (size_t)dlm_deepnet_state_bytes(mm->deep) : 0));
  L.total = o;
  return L;
}
}  // namespace

extern "C" int64_t dlm_memetic_state_bytes(const dlm_memetic* mm) {
  return mm ? (int64_t)ckpt_layout(mm).total : 0;
}

extern "C" dlm_status dlm_memetic_save(dlm_ctx* ctx, dlm_memetic* mm, void* host) {
  if (!ctx || !mm || !host) return fail(ctx, DLM_EINVAL, "memetic_save: null argument");
  const CkptLayout L = ckpt_layout(mm);
  uint8_t* h = (uint8_t*)host;
  const size_t p = (size_t)mm->prm.p, n = (size_t)mm->n;
  CkptHeader H{};
  memcpy(H.magic, kMagic, 8);
  H.n = mm->n; H.k = mm->prm.k; H.p = mm->prm.p; H.K = mm->prm.K; H.use_scorer = mm->prm.use_scorer;
  H.gen = mm->gen;
  H.scorer_bytes = mm->scorer ? dlm_scorer_state_bytes(mm->scorer) : (mm->deep ? dlm_deepnet_state_bytes(mm->deep) : 0);
  H.total = (int64_t)L.total;
  H.fingerprint = mm->fingerprint;
  cudaStream_t s = ctx->stream;
  DLM_CUDA(ctx, cudaMemcpyAsync(h + L.P, mm->P, p * n * 2, cudaMemcpyDeviceToHost, s));
  DLM_CUDA(ctx, cudaMemcpyAsync(h + L.fP, mm->fP, p * 8, cudaMemcpyDeviceToHost, s));
  DLM_CUDA(ctx, cudaMemcpyAsync(h + L.DP, mm->DP, p * p * 2, cudaMemcpyDeviceToHost, s));
  DLM_CUDA(ctx, cudaMemcpyAsync(h + L.SO, mm->SO, p * n * 2, cudaMemcpyDeviceToHost, s));
  DLM_CUDA(ctx, cudaMemcpyAsync(h + L.best_f, mm->best_f, 8, cudaMemcpyDeviceToHost, s));
  DLM_CUDA(ctx, cudaMemcpyAsync(h + L.best_col, mm->best_col, n * 2, cudaMemcpyDeviceToHost, s));
  DLM_CUDA(ctx, cudaStreamSynchronize(s));
  if (mm->scorer) DLM_TRY(dlm_scorer_save(ctx, mm->scorer, h + L.scorer));
  if (mm->deep) DLM_TRY(dlm_deepnet_save(ctx, mm->deep, h + L.scorer));
  memcpy(h, &H, sizeof(H));
  return DLM_OK;
}

extern "C" dlm_status dlm_memetic_load(dlm_ctx* ctx, dlm_memetic* mm, const void* host) {
  if (!ctx || !mm || !host) return fail(ctx, DLM_EINVAL, "memetic_load: null argument");
  const CkptLayout L = ckpt_layout(mm);
  const uint8_t* h = (const uint8_t*)host;
  CkptHeader H;
  memcpy(&H, h, sizeof(H));
  if (memcmp(H.magic, kMagic, 8) != 0) return fail(ctx, DLM_EINVAL, "memetic_load: not a memetic checkpoint");
  if (H.n != mm->n || H.k != mm->prm.k || H.p != mm->prm.p || H.K != mm->prm.K ||
      H.use_scorer != mm->prm.use_scorer || H.total != (int64_t)L.total ||
      H.scorer_bytes != (mm->scorer ? dlm_scorer_state_bytes(mm->scorer)
                                    : (mm->deep ? dlm_deepnet_state_bytes(mm->deep) : 0)))
    return fail(ctx, DLM_EINVAL, "memetic_load: checkpoint of another configuration");
  if (H.fingerprint != mm->fingerprint)
    return fail(ctx, DLM_EINVAL, "memetic_load: checkpoint of another graph or parameter set (seed, budget, tenure, "
                                 "training)");
  const size_t p = (size_t)mm->prm.p, n = (size_t)mm->n;
  cudaStream_t s = ctx->stream;
  DLM_CUDA(ctx, cudaMemcpyAsync(mm->P, h + L.P, p * n * 2, cudaMemcpyHostToDevice, s));
  DLM_CUDA(ctx, cudaMemcpyAsync(mm->fP, h + L.fP, p * 8, cudaMemcpyHostToDevice, s));
  DLM_CUDA(ctx, cudaMemcpyAsync(mm->DP, h + L.DP, p * p * 2, cudaMemcpyHostToDevice, s));
  DLM_CUDA(ctx, cudaMemcpyAsync(mm->SO, h + L.SO, p * n * 2, cudaMemcpyHostToDevice, s));
  DLM_CUDA(ctx, cudaMemcpyAsync(mm->best_f, h + L.best_f, 8, cudaMemcpyHostToDevice, s));
  DLM_CUDA(ctx, cudaMemcpyAsync(mm->best_col, h + L.best_col, n * 2, cudaMemcpyHostToDevice, s));
  DLM_CUDA(ctx, cudaStreamSynchronize(s));
  if (mm->scorer) DLM_TRY(dlm_scorer_load(ctx, mm->scorer, h + L.scorer));
  if (mm->deep) DLM_TRY(dlm_deepnet_load(ctx, mm->deep, h + L.scorer));
  mm->gen = H.gen;
  return DLM_OK;
}

// ---- COL: k-COL with decreasing k ----------------------------------------------------------------
extern "C" dlm_status dlm_col_descend(dlm_ctx* ctx, const dlm_graph* g, const dlm_memetic_params* prm, int32_t max_gens,
                                      int32_t* k_best, int16_t* best_col, int32_t* gens_per_k) {
  if (!ctx || !g || !prm || !k_best || !best_col) return fail(ctx, DLM_EINVAL, "col_descend: null argument");
  if (max_gens < 1) return fail(ctx, DLM_EINVAL, "col_descend: max_gens must be positive");
  *k_best = -1;
  for (int k = prm->k; k >= 2; --k) {
    dlm_memetic_params q = *prm;
    q.k = k;
    dlm_memetic* mm = nullptr;
    DLM_TRY(dlm_memetic_create(ctx, g, &q, &mm));
    bool solved = false;
    int gens = 0;
    dlm_status st = DLM_OK;
    for (; gens < max_gens && st == DLM_OK && !solved; ++gens) {
      int64_t best = 0;
      st = dlm_memetic_step(ctx, mm, &best);
      solved = st == DLM_OK && best == 0;
    }
    if (gens_per_k) gens_per_k[k] = gens;
    if (st == DLM_OK && solved) {
      st = cuda_check(ctx, cudaMemcpyAsync(best_col, mm->best_col, (size_t)g->n * 2, cudaMemcpyDeviceToDevice, ctx->stream),
                      "copy");
      if (st == DLM_OK) st = dlm_sync(ctx);
    }
    dlm_memetic_destroy(mm);
    if (st != DLM_OK) return st;
    if (!solved) break;
    *k_best = k;
  }
  return DLM_OK;
}

extern "C" dlm_status dlm_memetic_found_ms(dlm_ctx* ctx, dlm_memetic* mm, double* ms) {
  if (!ctx || !mm || !ms) return fail(ctx, DLM_EINVAL, "memetic_found_ms: null argument");
  if (mm->gen == 0) return fail(ctx, DLM_EINVAL, "memetic_found_ms: no generation has run");
  DLM_CUDA(ctx, cudaEventSynchronize(mm->ev_found));
  float e = 0.f;
  DLM_CUDA(ctx, cudaEventElapsedTime(&e, mm->ev_gen, mm->ev_found));
  *ms = (double)e;
  return DLM_OK;
}

extern "C" dlm_status dlm_memetic_profile(dlm_ctx* ctx, dlm_memetic* mm, int32_t enable, double* stage_ms) {
  if (!ctx || !mm) return fail(ctx, DLM_EINVAL, "memetic_profile: null argument");
  if (stage_ms) {
    for (int i = 0; i < 7; ++i) stage_ms[i] = mm->prof_gens ? mm->stage_ms[i] / (double)mm->prof_gens : 0.0;
    stage_ms[7] = (double)mm->prof_gens;
    for (int i = 7; i < 10; ++i) stage_ms[i + 1] = mm->prof_gens ? mm->stage_ms[i] / (double)mm->prof_gens : 0.0;
  }
  for (auto& x : mm->stage_ms) x = 0.0;
  mm->prof_gens = 0;
  if (enable && !mm->pev[0]) {
    for (auto& e : mm->pev) DLM_CUDA(ctx, cudaEventCreate(&e));
    for (auto& e : mm->tev) DLM_CUDA(ctx, cudaEventCreate(&e));
  }
  mm->prof = enable != 0;
  return DLM_OK;
}
