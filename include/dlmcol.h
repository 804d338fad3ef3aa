/*
 * libdlmcol -- C-ABI of the GB300 (sm_103a) implementation of the hot path of DLMCOL, the deep
 * learning guided memetic framework for graph colouring (Goudet, Grelier, Hao, arXiv 2109.05948).
 *
 * Conventions (all entry points):
 *  - Colours are 0-based: the paper's colours 1..k are 0..k-1 here.
 *  - Every pointer argument is owned by the caller. Pointers documented "device" must be device
 *    memory of the context's GPU; "host" pointers are ordinary host memory. The library allocates
 *    only inside the objects it creates (dlm_ctx, dlm_graph, dlm_scorer, dlm_memetic), which own
 *    their memory until destroyed.
 *  - Work is asynchronous on the context's CUDA stream. Argument validation happens synchronously
 *    and returns DLM_EINVAL / DLM_EUNSUPPORTED before anything is launched. Errors detected by a
 *    kernel (e.g. a tabu tenure outside the representable range) are recorded in the context and
 *    returned by the next dlm_sync().
 *  - Calls are thread-compatible: use one context per host thread.
 *  - Randomness: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed; counter words
 *    (a, b, c, tag) with tags INIT=1, TABU=2, GPX=3, SELECT=4, NNINIT=7, BATCH=8, WINIT=9. Each
 *    entry point states the counter it uses, so results are reproducible bit for bit.
 */
#ifndef DLMCOL_H
#define DLMCOL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dlm_status;
#define DLM_OK 0
#define DLM_EINVAL (-1)        /* bad argument (null pointer, size out of range, ...) */
#define DLM_ENOMEM (-2)        /* device allocation inside a library object failed */
#define DLM_ECUDA (-3)         /* a CUDA runtime call failed; dlm_last_error has the text */
#define DLM_ETIMEOUT (-4)      /* a bounded device-side wait gave up */
#define DLM_ECANCELLED (-5)    /* cancelled through the context's cancel flag */
#define DLM_EUNSUPPORTED (-6)  /* valid input this build does not handle (sizes, ranges) */

typedef struct dlm_ctx dlm_ctx;
typedef struct dlm_graph dlm_graph;
typedef struct dlm_scorer dlm_scorer;
typedef struct dlm_memetic dlm_memetic;

/* ---------------------------------------------------------------------------------------------
 * Context. `stream` is a cudaStream_t (NULL = the legacy default stream) on `device`.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_create(dlm_ctx** out, int32_t device, void* stream);
void dlm_destroy(dlm_ctx* ctx);
dlm_status dlm_set_stream(dlm_ctx* ctx, void* stream);
/* Cancellation (no counterpart in the paper): flag is a device-readable int32 (device or managed
 * memory, or pinned host memory, which is polled through its device mapping) or NULL to disable;
 * pageable host memory returns DLM_EINVAL. The TabuCol kernels launched
 * afterwards through ctx (batch, uneven batch, plans created afterwards) read it every 1024
 * iterations of each individual; once it is nonzero each search stops after the current
 * iteration's selection, writes its best colouring and conflicts so far, and dlm_sync returns
 * DLM_ECANCELLED. The caller owns the flag and keeps it valid while such launches run. */
dlm_status dlm_set_cancel_flag(dlm_ctx* ctx, const int32_t* flag);
/* Text of the last error on this context (valid until the next call on it). */
const char* dlm_last_error(const dlm_ctx* ctx);
/* Waits for the context's stream and returns (then clears) the device-side status. */
dlm_status dlm_sync(dlm_ctx* ctx);

/* ---------------------------------------------------------------------------------------------
 * Graph (paper: G = (V, E), section "Introduction"; the graph is held in global memory and shared
 * by all searches, section "Parallel iterated feasible and infeasible Tabu Search").
 * edges: device, [m][2] int32 vertex pairs (u != v, each undirected edge once, 0 <= u,v < n).
 * weights: device [n] int32 vertex weights (> 0) for the WVCP, or NULL.
 * The library builds CSR neighbour lists (ascending) and bit-packed adjacency rows on the GPU.
 * Limits: 2 <= n <= 2048. Duplicated edges are merged.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_graph_create(dlm_ctx* ctx, int32_t n, int64_t m, const int32_t* edges, const int32_t* weights,
                            dlm_graph** out);
void dlm_graph_destroy(dlm_graph* g);
int32_t dlm_graph_n(const dlm_graph* g);
int64_t dlm_graph_m(const dlm_graph* g); /* number of distinct edges after the build (valid after dlm_sync) */
/* Copies the CSR (off: device [n+1], idx: device [2m] int32) and bit rows (device [n][ceil(n/32)]). */
dlm_status dlm_graph_export(dlm_ctx* ctx, const dlm_graph* g, int32_t* off, int32_t* idx, uint32_t* bits);

/* ---------------------------------------------------------------------------------------------
 * Random initialisation for k-COL (section "Adaptations of the algorithm for the vertex coloring
 * problem": each vertex receives a uniform random colour). col: device [pop][n] int16 output;
 * col[i][v] = high word of r0 * k, r = Philox(a = v, b = 0, c = ind_base + i, tag = INIT).
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_init_colors(dlm_ctx* ctx, int32_t n, int32_t k, int32_t pop, uint64_t seed, uint32_t ind_base,
                           int16_t* col);

/* Conflict table gamma[v][c] = #neighbours of v coloured c and the k-COL objective f (Eq. f):
 * the number of edges whose end points share a colour. col: device [pop][n]; gamma: device
 * [pop][n][k] int32 or NULL; f: device [pop] int64. */
dlm_status dlm_gamma(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, const int16_t* col,
                     int32_t* gamma, int64_t* f);

/* ---------------------------------------------------------------------------------------------
 * Tabu tenure rule. k-COL (Table params-COL, alpha = 0.6): after moving v away from colour c the
 * pair (v, c) is tabu for tt = U{0..L_max} + floor(alpha_num * f / alpha_den) iterations, f the
 * conflicts after the move. WVCP (section "Parallel iterated feasible and infeasible Tabu Search",
 * alpha = 0.2): the vertex is frozen for tt = U{0..L_max} + floor(alpha_num * n / alpha_den).
 * U{0..L_max} = high word of r1 * (L_max + 1) of the iteration's Philox block.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  int32_t L_max;     /* paper: 9 */
  int32_t alpha_num; /* 6 (k-COL) or 2 (WVCP) */
  int32_t alpha_den; /* 10 */
} dlm_tenure;

/* TabuCol for k-COL on a population (paper: TabuCOL of Hertz & de Werra in the implementation of
 * Galinier & Hao, run on every individual in parallel; section "Adaptations ... vertex coloring",
 * Table params-COL). Iteration `it` of individual i draws r = Philox(a = it, b = generation,
 * c = ind_base + i, tag = TABU). Among the moves (v, c) of conflicting vertices v to colours
 * c != col(v), with delta = gamma[v][c] - gamma[v][col(v)], a move is admissible when (v, c) is not
 * tabu or f + delta < best f so far (aspiration); the search takes the j-th admissible move of
 * minimum delta in (v ascending, c ascending) order, j = high word of r0 * (number of such moves),
 * and makes no move when none is admissible. It stops early when f reaches 0.
 *   col     device [pop][n] int16: in the start colourings (values in 0..k-1), out the best
 *           colouring each search visited.
 *   best_f  device [pop] int64 out: conflicts of that colouring.
 *   moves   device [pop] int64 out (or NULL): iterations that made a move.
 *   iters   iteration budget per individual (paper: 128 |V|).
 * State: each individual's conflict table gamma (2 n k bytes, the tabu flag of every (v, c) in its
 * top bit), row summaries and a ring of tabu entries live in shared memory, several individuals
 * per CTA sharing the graph's bit rows; tabu entries whose tenure does not fit the ring go to a
 * per-individual list in the context's workspace. When one individual's gamma does not fit in
 * shared memory (n k above about 110 000), the search runs one individual per CTA with a separate
 * expiry table, its last rows in a per-CTA slab of global memory (L2 resident).
 * Limits: k <= 128 (DLM_EUNSUPPORTED above); iters + L_max + alpha_num |E| / alpha_den below 2^32
 * (DLM_EUNSUPPORTED); on the one-individual-per-CTA path, tenures above 32766 iterations stop the
 * search with DLM_EUNSUPPORTED at dlm_sync. */
dlm_status dlm_tabucol_batch(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                             int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                             uint32_t generation, uint32_t ind_base);

/* As dlm_tabucol_batch, with warps_per_individual forced (1, 2, 4, 8, 16 or 32; 0 = autotuned or
 * the library's default; a 32-warp CTA holds all of an SM's registers, so one runs per SM), an
 * optional per-iteration trace -- device [pop][iters][4] int32 of (v, c, delta, #tied moves),
 * (-1, -1, 0, 0) for an iteration without a move, entries after an early stop untouched -- and an
 * optional work count -- device [pop][3] int64: the number of conflicting rows evaluated, the sum
 * of the degrees of the moved vertices and the number of rows whose summary was recomputed (the
 * algorithmic work of the selection, of the update and of the re-summaries). */
dlm_status dlm_tabucol_batch_ex(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                                uint32_t generation, uint32_t ind_base, int32_t warps_per_individual,
                                int32_t* trace, int64_t* work);

/* Launch options of dlm_tabucol_batch_opts (all zero = the library's choice). */
typedef struct {
  int32_t warps_per_individual; /* 1, 2, 4, 8, 16 or 32; 0 = autotuned or default */
  int32_t ring;                 /* tabu ring entries per individual: a power of two in 64..8192, or 0 =
                                   the largest that fits beside the most individuals per CTA; entries
                                   with longer tenures go to the global list (tests use small rings) */
  int32_t legacy;               /* 1 = one individual per CTA with an expiry table (the spill path) */
  int32_t entry_bits;           /* conflict-table entries of the grouped kernel: 16, 8 (a 7-bit count
                                   and the tabu flag, valid while every colour class holds at most
                                   126 vertices; an individual whose search would exceed that is
                                   searched again with 16-bit entries, with the same result), or 0 =
                                   8 when it fits more individuals on an SM */
} dlm_tabu_opts;

/* dlm_tabucol_batch_ex with launch options (opts may be NULL); same results for every option. */
dlm_status dlm_tabucol_batch_opts(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                  int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                                  uint32_t generation, uint32_t ind_base, const dlm_tabu_opts* opts,
                                  int32_t* trace, int64_t* work);

/* Uneven batch: several graphs, each with its own k, population and budget, in one persistent
 * launch (individuals ordered by decreasing work and handed to resident blocks from a device
 * queue). Arrays of length n_graphs are host arrays; col[g], best_f[g], moves[g] are device
 * pointers as in dlm_tabucol_batch (moves[g] may be NULL). Individual j of graph g uses the
 * Philox stream c = ind_base + (sum of pop[0..g-1]) + j. */
dlm_status dlm_tabucol_multi(dlm_ctx* ctx, int32_t n_graphs, const dlm_graph* const* graphs, const int32_t* k,
                             const int32_t* pop, int16_t* const* col, int64_t* const* best_f,
                             int64_t* const* moves, const int64_t* iters, dlm_tenure tenure, uint64_t seed,
                             uint32_t generation, uint32_t ind_base);

/* dlm_tabucol_multi without any device allocation. The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory -- code on a latency-critical path where
 * cudaMalloc's implicit device synchronisation is unacceptable, or a process whose device memory
 * is owned by another allocator (a framework's caching allocator, a fixed memory budget), where a
 * raw cudaMalloc may fail or fragment the pool. The job list and the work queue of the persistent
 * kernel live in a file-scope device array of the library (1 MiB plus 256 bytes, held on every GPU
 * that loads the library until the process exits) instead of the context's workspace.
 * Arguments and results are those of dlm_tabucol_multi. Limit: at most 16384 individuals in total
 * per call (DLM_EUNSUPPORTED above, nothing launched). The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. All calls share the one array, which keeps the last call's contents:
 * the queue counter is cleared by every call, and calls that overlap on the GPU (other streams or
 * other contexts on the same device) race on it -- serialise them. */
dlm_status dlm_tabucol_multi_noalloc(dlm_ctx* ctx, int32_t n_graphs, const dlm_graph* const* graphs, const int32_t* k,
                                     const int32_t* pop, int16_t* const* col, int64_t* const* best_f,
                                     int64_t* const* moves, const int64_t* iters, dlm_tenure tenure, uint64_t seed,
                                     uint32_t generation, uint32_t ind_base);

/* The uneven batch of dlm_tabucol_multi as a reusable plan: the job list (individuals by decreasing
 * work), the work queue and the slab of spilled rows are built once in plan-owned device memory,
 * and the launch (queue reset + persistent kernel) is captured into a CUDA graph; each
 * dlm_tabucol_multi_plan_launch replays it on the context's stream with the arguments given at
 * creation (the colourings are searched in place: col holds the best colourings afterwards).
 * The warps per individual come from the autotuner's cache (dlm_tabucol_autotune) when present. */
typedef struct dlm_multi_plan dlm_multi_plan;
dlm_status dlm_tabucol_multi_plan_create(dlm_ctx* ctx, int32_t n_graphs, const dlm_graph* const* graphs,
                                         const int32_t* k, const int32_t* pop, int16_t* const* col,
                                         int64_t* const* best_f, int64_t* const* moves, const int64_t* iters,
                                         dlm_tenure tenure, uint64_t seed, uint32_t generation, uint32_t ind_base,
                                         dlm_multi_plan** out);
dlm_status dlm_tabucol_multi_plan_launch(dlm_ctx* ctx, dlm_multi_plan* plan);
void dlm_tabucol_multi_plan_destroy(dlm_multi_plan* plan);

/* Autotuner for the tabu kernel: times warps_per_individual in {1, 2, 4, 8, 16} on a short run of
 * the given problem and caches the fastest for (n, k) in the context; returns it in *best. */
dlm_status dlm_tabucol_autotune(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int64_t iters,
                                int32_t* best);

/* ---------------------------------------------------------------------------------------------
 * GPX crossover (Galinier & Hao 1999; section "Parent matching and selection of crossovers").
 * For child t with parents A = parents[pairs[t][0]], B = parents[pairs[t][1]]: for l = 0..k-1 the
 * child gives label l to the largest class (smallest colour on ties) not yet inherited of A (l even)
 * or B (l odd); those vertices leave both parents. Vertices left over get the label high word of
 * r0 * k, r = Philox(a = v, b = generation, c = child_id[t], tag = GPX).
 *   parents  device [pop][n] int16;  pairs device [m][2] int32;  child_id device [m] uint32 or
 *   NULL (child_id = t);  children device [m][n] int16 out.  Limits: k <= 255, n <= 2048.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_gpx_batch(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* parents, int32_t pop,
                         const int32_t* pairs, const uint32_t* child_id, int32_t m, int16_t* children,
                         uint64_t seed, uint32_t generation);

/* ---------------------------------------------------------------------------------------------
 * Approximate set-theoretic partition distance (section "Distance computation"): with
 * M[c][c'] = |A_c intersect B_c'|, D = n - min(sum_c max_c' M, sum_c' max_c M), a symmetric lower
 * bound of the exact (Hungarian) distance, exact when the best-match map is injective.
 *   X device [a][n], Y device [b][n] int16 colourings; D device out, D[i * ldD + j] = D(X_i, Y_j).
 *   upper != 0 with X == Y computes only j > i (and writes those entries). Limits: k <= 255.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_distance_batch(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* X, int32_t a, const int16_t* Y,
                              int32_t b, int16_t* D, int64_t ldD, int32_t upper);
/* As dlm_distance_batch with the kernel chosen by the caller (same results; the paper has no
 * counterpart: measurement and testing support). method 1: one warp per pair counts M in a k x k
 * table and scans it for the row and column maxima, O(n + k^2) per pair; method 2: the CTA
 * counts one pair at a time and takes the maxima with atomic maxima while counting, O(n) per
 * pair; method 3: every M as a block of one-hot matrix products on the tcgen05 tensor cores
 * (bf16 0/1 operands, exact FP32 counts), row maxima from X . Y^T and column maxima from
 * Y . X^T, 2 (a + b) kp n_64 + 8 a b B of context workspace (kp = 64 for k <= 64, 128 for
 * k <= 128; n_64 = n rounded up to 64; k > 128: DLM_EUNSUPPORTED), O(n kp^2) per pair; method
 * 0: the library's
 * choice (method 2 from k = 72 on). */
dlm_status dlm_distance_batch_ex(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* X, int32_t a,
                                 const int16_t* Y, int32_t b, int16_t* D, int64_t ldD, int32_t upper,
                                 int32_t method);
/* Exact partition distance (section "Distance computation"): D = n - the largest total overlap
 * sum_c M[c][pi(c)] over one-to-one matchings pi of the classes, i.e. the fewest vertices to
 * recolour to turn one partition into the other up to colour names. One warp per pair: counting
 * for M, then the Hungarian algorithm (shortest augmenting paths with integer potentials),
 * O(n + k^3) per pair. Arguments as for dlm_distance_batch; k <= 128 (DLM_EUNSUPPORTED). The
 * approximate D of dlm_distance_batch is a lower bound of this value and equal to it when the
 * best-match map is one-to-one. */
dlm_status dlm_distance_exact_batch(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* X, int32_t a,
                                    const int16_t* Y, int32_t b, int16_t* D, int64_t ldD, int32_t upper);

/* Distance-and-quality pool update (section "Population update"): the 2p candidates (index < p:
 * the population, >= p: the improved individuals) are visited by increasing fit, ties by lower
 * index; a candidate is kept when its distance to every candidate kept so far is > n / 10; if
 * fewer than p are kept the best remaining ones (same order) fill the population.
 *   fit device [2p] int64 in 0..2^43 - 1 (else DLM_EINVAL at dlm_sync);
 *   D   device [2p][2p] int16, 4-byte aligned (DLM_EINVAL otherwise), row x read in full;
 *   sel device [p] int32 out (in keep order).
 * The visit runs in blocks of 1024 candidates: every SM scans the block's rows of D against the
 * members kept in earlier blocks, then one warp settles the block in order; the result is that of
 * the one-at-a-time visit. Scratch (about 9 m + 130 KB bytes, m = 2p) comes from the context's
 * workspace. Limits: p <= 8192 (the sort runs in one CTA's shared memory; DLM_EUNSUPPORTED). */
dlm_status dlm_pool_update(dlm_ctx* ctx, int32_t p, int32_t n, const int64_t* fit, const int16_t* D, int32_t* sel);

/* Parent matching (section "Parent matching ..."): the K nearest j != i of every i by D (device
 * [p][p] int16), nearest first, ties by lower index. nbr device [p][K] int32 out. K <= 64. */
dlm_status dlm_knn(dlm_ctx* ctx, int32_t p, const int16_t* D, int32_t K, int32_t* nbr);

/* ---------------------------------------------------------------------------------------------
 * Offspring scorer f_theta (section "Deep neural network training"): a colour-permutation
 * invariant deep-set network. Layer 0 sums the 64-d embedding rows E[v] over each colour class
 * (plus bias, LeakyReLU 0.2); three layers H' = LeakyReLU_0.2(beta + H Lambda + rho(H) Gamma) of
 * width 256, rho the mean over the k classes; output = mean over classes of the linear head.
 * Matrix products run on the tcgen05 tensor cores in BF16 with FP32 accumulation; parameters
 * are kept in FP32. Flat parameter order: E[n][64], b0[64], for l = 1..3 (din = 64, 256, 256):
 * Lambda_l[din][256], Gamma_l[din][256], beta_l[256]; then w_head[256], b_head[1].
 * Each candidate occupies 64 ceil(k / 64) class rows of the tensor-core tiles (rows at and above
 * k are empty and masked out of rho and of the head mean). Limits: k <= 256, n <= 2048.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_scorer_create(dlm_ctx* ctx, int32_t n, int32_t k, uint64_t seed, dlm_scorer** out);
void dlm_scorer_destroy(dlm_scorer* s);
int64_t dlm_scorer_nparams(const dlm_scorer* s);
/* params: device [nparams] float32 (copy out / copy in; set also resets the Adam state). */
dlm_status dlm_scorer_get_params(dlm_ctx* ctx, dlm_scorer* s, float* params);
dlm_status dlm_scorer_set_params(dlm_ctx* ctx, dlm_scorer* s, const float* params);
/* Scores c colourings: col device [c][n] int16, out device [c] float32. By default the
 * activations between layers are kept as bf16 hi + lo pairs (about 16 mantissa bits, three MMA
 * passes per layer product), which holds every score's colour-dependent part (score minus the
 * head bias) within 1e-2 of FP64. */
dlm_status dlm_score_offspring(dlm_ctx* ctx, dlm_scorer* s, const int16_t* col, int32_t c, float* out);
/* split = 1 (default): scoring activations as bf16 hi + lo; split = 0: bf16 activations alone
 * (two MMA passes, half the activation traffic; the colour-dependent part of a score then carries
 * about 3e-2 relative error). The paper has no counterpart: a precision/speed choice of this
 * implementation. Waits for the context's stream and frees the scoring buffers. */
dlm_status dlm_scorer_set_scoring_precision(dlm_ctx* ctx, dlm_scorer* s, int32_t split);
/* Mean squared error of B samples (col device [B][n], y device [B]) and its gradient
 * (grad device [nparams] float32, out device [B] float32 predictions, loss device [1]). */
dlm_status dlm_scorer_loss_grad(dlm_ctx* ctx, dlm_scorer* s, const int16_t* col, const float* y, int32_t B,
                                float* grad, float* out, float* loss);
/* Online training: N epochs of Adam (lr, betas 0.9/0.999, eps 1e-8) over p samples (cols device
 * [p][n], targets fvals device [p] int64 standardised by their mean and std) in batches of b;
 * epoch e visits the samples sorted by the keys Philox(a = i, b = e, c = generation,
 * tag = BATCH).r0 (ties by i). */
dlm_status dlm_scorer_train(dlm_ctx* ctx, dlm_scorer* s, const int16_t* cols, const int64_t* fvals, int32_t p,
                            int32_t epochs, int32_t b, float lr, uint64_t seed, uint32_t generation);
/* Scorer state to or from caller-owned host memory of dlm_scorer_state_bytes bytes: parameters,
 * Adam first and second moments (nparams float32 each) and the Adam step counter (int64). Both
 * wait for the copies; load also refreshes the bf16 weight copies the forward pass reads. */
int64_t dlm_scorer_state_bytes(const dlm_scorer* s);
dlm_status dlm_scorer_save(dlm_ctx* ctx, dlm_scorer* s, void* host);
dlm_status dlm_scorer_load(dlm_ctx* ctx, dlm_scorer* s, const void* host);

/* ---------------------------------------------------------------------------------------------
 * Paper-size offspring scorer (section "Deep neural network training" with its invariant batch
 * normalisation; section "Implementation and parameter setting": hidden widths 10|V|, 5|V|,
 * 2|V| x 5, |V|, |V|//2 for k-COL, 5|V|, 2|V|, |V|, |V|//2 for the WVCP), any depth and widths.
 * Layer 0 sums the rows E[v] over each class (+ beta_0); layer l >= 1 computes
 * Z = H Lambda_l + rho(H) Gamma_l + beta_l on the tcgen05 tensor cores; every layer normalises
 * each feature over the batch and the k classes (training: batch mean and biased variance,
 * running estimates updated with momentum 0.1, the variance unbiased; evaluation: the running
 * estimates), y = x^ gamma + mu, then LeakyReLU_0.2; the output is the mean over the classes of
 * a linear head. eps = 1e-5.
 * Flat parameter order (float32): E[n][h0], b0[h0], g0[h0], mu0[h0]; for l = 1 .. nh-1:
 * Lambda_l[h_l-1][h_l], Gamma_l[h_l-1][h_l], beta_l[h_l], g_l[h_l], mu_l[h_l]; then w_head[h_nh-1],
 * b_head[1]. Statistics (float32): per layer, running mean[h_l] then running variance[h_l].
 * Initial parameters: weights and biases uniform in +-1/sqrt(fan_in) from Philox(a = index,
 * b = 1, c = 0, tag = NNINIT), gamma = 1, mu = 0; running mean 0, variance 1.
 * GEMM operands are bf16 hi + lo pairs by default (dlm_deepnet_set_precision: split = 0 for
 * bf16 alone). Limits: n <= 2048, k <= 256, 1..16 hidden layers of 1..16384 features; a
 * training batch (or a training-mode forward) holds at most 8192 candidates. Buffers grow with
 * the largest batch (evaluation: chunks of about 4 GB of activations).
 * ------------------------------------------------------------------------------------------- */
typedef struct dlm_deepnet dlm_deepnet;
/* widths: host [nh] int32, the hidden widths h_0 .. h_nh-1. Waits for its initialisation. */
dlm_status dlm_deepnet_create(dlm_ctx* ctx, int32_t n, int32_t k, int32_t nh, const int32_t* widths, uint64_t seed,
                              dlm_deepnet** out);
void dlm_deepnet_destroy(dlm_deepnet* net);
int64_t dlm_deepnet_nparams(const dlm_deepnet* net);
int64_t dlm_deepnet_nstats(const dlm_deepnet* net);
/* which = 0: parameters (set also resets the Adam state), 1: running statistics; device float32. */
dlm_status dlm_deepnet_get(dlm_ctx* ctx, dlm_deepnet* net, int32_t which, float* dst);
dlm_status dlm_deepnet_set(dlm_ctx* ctx, dlm_deepnet* net, int32_t which, const float* src);
dlm_status dlm_deepnet_set_precision(dlm_ctx* ctx, dlm_deepnet* net, int32_t split);
/* Scores of c colourings (col device [c][n] int16, colours 0..k-1; out device [c] float32).
 * train = 0: evaluation (running statistics); train = 1: one training-mode batch (its own
 * statistics, running estimates updated), c <= 8192. */
dlm_status dlm_deepnet_forward(dlm_ctx* ctx, dlm_deepnet* net, const int16_t* col, int32_t c, int32_t train,
                               float* out);
/* Training-mode forward (running estimates updated) and backward of B samples: mean squared
 * error against y (device [B] float32), its gradient (grad device [nparams] or NULL), the
 * predictions (out device [B] or NULL) and the loss (loss device [1] or NULL). */
dlm_status dlm_deepnet_loss_grad(dlm_ctx* ctx, dlm_deepnet* net, const int16_t* col, const float* y, int32_t B,
                                 float* grad, float* out, float* loss);
/* One Adam step (lr, betas 0.9 / 0.999, eps 1e-8) with a given gradient (device [nparams]). */
dlm_status dlm_deepnet_adam_step(dlm_ctx* ctx, dlm_deepnet* net, const float* grad, float lr);
/* Online training as dlm_scorer_train: targets fvals (device [p] int64) standardised by their
 * mean and population standard deviation, N epochs of Adam over batches of b in the epoch order
 * (samples sorted by Philox(a = i, b = epoch, c = generation, tag = BATCH).r0, ties by i). */
dlm_status dlm_deepnet_train(dlm_ctx* ctx, dlm_deepnet* net, const int16_t* cols, const int64_t* fvals, int32_t p,
                             int32_t epochs, int32_t b, float lr, uint64_t seed, uint32_t generation);
/* State to or from caller-owned host memory of dlm_deepnet_state_bytes bytes: parameters, Adam
 * moments, running statistics (float32 each) and the Adam step counter (int64); both wait. */
int64_t dlm_deepnet_state_bytes(const dlm_deepnet* net);
dlm_status dlm_deepnet_save(dlm_ctx* ctx, dlm_deepnet* net, void* host);
dlm_status dlm_deepnet_load(dlm_ctx* ctx, dlm_deepnet* net, const void* host);

/* ---------------------------------------------------------------------------------------------
 * Memetic loop (Algorithm 1). dlm_memetic_step runs one generation: the local search of every
 * offspring (TabuCol for k-COL, the iterated tabu search for the WVCP), best-so-far update,
 * scorer training (use_scorer), distances between P and P' and within P', pool update, K nearest
 * neighbours, and offspring: with use_scorer the best-scored of the K GPX
 * children of i (parent 2 = its j-th neighbour, child id i*K + j); without, one GPX child with a
 * neighbour drawn uniformly (Philox(a = i, b = generation, c = 0, tag = SELECT)), the ablation of
 * section "Benefits of the neural network based crossover selection".
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  int32_t k, p, K;
  int64_t iters;          /* tabu iterations per generation (paper: 128 |V|) */
  dlm_tenure tenure;      /* paper: {9, 6, 10} */
  int32_t use_scorer;     /* 1 = learned selection with the 64-d + 3 x 256 scorer (dlm_scorer_*),
                             2 = learned selection with the paper-size network with invariant
                             batch normalisation (dlm_deepnet_*; hidden widths 10|V|, 5|V|, 2|V| x 5,
                             |V|, |V|//2 for k-COL, 5|V|, 2|V|, |V|, |V|//2 for the WVCP),
                             0 = random GPX */
  int32_t epochs, batch;  /* paper: 5, 100 (k-COL), 20, 100 (WVCP) */
  float lr;               /* paper: 1e-3 */
  uint64_t seed;
  int32_t problem;        /* 0 = k-COL; 1 = WVCP (the graph needs vertex weights): the initial
                             population from the randomised greedy initialisation (individual i
                             from stream i; it must open at most k colours, k <= 255), fitness =
                             the WVCP score f, the local search = the iterated feasible and
                             infeasible tabu search of dlm_wvcp_iterated (max_ls searches of iters
                             iterations, fscale 256, phi0 = round(256 k max w / (2 |V|)),
                             phi_last = 256 * 2 max w); an offspring none of whose searches ended
                             legal gets the fitness sum(w) + 1 */
  int32_t max_ls;         /* WVCP: searches per generation (paper: 10); ignored for k-COL */
} dlm_memetic_params;

dlm_status dlm_memetic_create(dlm_ctx* ctx, const dlm_graph* g, const dlm_memetic_params* prm, dlm_memetic** out);
void dlm_memetic_destroy(dlm_memetic* mm);
/* One generation; *best_f_host (host, may be NULL) receives f(S*) after it (this waits). */
dlm_status dlm_memetic_step(dlm_ctx* ctx, dlm_memetic* mm, int64_t* best_f_host);
/* Copies a state array to device memory dst: 0 = P [p][n] int16, 1 = f(P) [p] int64,
 * 2 = D(P,P) [p][p] int16, 3 = offspring S^O [p][n] int16, 4 = best colouring [n] int16,
 * 5 = f(S'_i) of the last generation [p] int64, 6 = chosen candidate j [p] int32,
 * 7 = candidate scores of the last generation [p][K] float32 (use_scorer only),
 * 8 = scorer parameters [nparams] float32 (of the paper-size network with use_scorer = 2),
 * 9 = its running statistics [nstats] float32 (use_scorer = 2 only). */
dlm_status dlm_memetic_get(dlm_ctx* ctx, dlm_memetic* mm, int32_t which, void* dst);

/* Diagnostics of the last generation (section "Analysis of the contributions of deep learning":
 * predicted against actual fitness, and the population's spread), host out[8]: the generation
 * index; the Pearson correlation between the scorer's prediction for each offspring searched in
 * that generation (chosen by the previous generation's learned selection) and its post-tabu
 * conflicts f(S'_i); the mean of |prediction * sd + mean - f(S'_i)| / max(f(S'_i), 1), the
 * prediction mapped back through the standardisation of the targets it was trained on; the mean
 * and the minimum of f(S'_i); the mean, minimum and maximum distance between distinct members of
 * the new population. The two prediction entries are NaN without the scorer and in generation 0.
 * Waits for the context's stream. */
dlm_status dlm_memetic_stats(dlm_ctx* ctx, dlm_memetic* mm, double* out);
/* Overwrites the population state (which = 0..3 as above) from device memory src. */
dlm_status dlm_memetic_set(dlm_ctx* ctx, dlm_memetic* mm, int32_t which, const void* src);

/* Measurement utility (no counterpart in the paper): while enabled, dlm_memetic_step records CUDA
 * events at its stage boundaries (and waits for its last one). dlm_memetic_profile returns in
 * stage_ms (host [11] double, or NULL) the mean ms per generation since the previous call of:
 * 0 tabu search, 1 best so far, 2 distances, 3 pool update and gathers, 4 matching, 5 offspring
 * (GPX, and scoring and selection with the scorer), 6 scorer training (on its side stream,
 * overlapping 2-4), 7 the number of generations averaged, and with the scorer the parts of
 * stage 5: 8 GPX of the K candidates, 9 the wait for the training, 10 scoring and selection;
 * then clears them and sets the recording state to enable. */
dlm_status dlm_memetic_profile(dlm_ctx* ctx, dlm_memetic* mm, int32_t enable, double* stage_ms);
/* Measurement utility: host *ms = device time from the start of the last dlm_memetic_step to the
 * end of its best-so-far update (Algorithm 1 records S* right after the local search), i.e. how
 * far into that generation its best colouring was known; the rest of the generation (training,
 * distances, pool update, offspring) prepares the next one. Waits for that point of the stream;
 * DLM_EINVAL before the first generation. */
dlm_status dlm_memetic_found_ms(dlm_ctx* ctx, dlm_memetic* mm, double* ms);

/* The vertex colouring problem (section "Adaptations of the algorithm for the vertex coloring
 * problem"): k-COL with decreasing k. Starting at k = prm->k, a memetic search (fresh random
 * population, parameters prm with that k) runs up to max_gens generations; when it reaches a
 * legal k-colouring, its colouring goes to best_col (device [n] int16) and k is decreased by one;
 * the first k without a legal colouring within max_gens generations ends the descent. k_best
 * (host) receives the last k with a legal colouring (-1: none); gens_per_k (host [prm->k + 1],
 * or NULL) the generations run at each k. Waits for every generation. */
dlm_status dlm_col_descend(dlm_ctx* ctx, const dlm_graph* g, const dlm_memetic_params* prm, int32_t max_gens,
                           int32_t* k_best, int16_t* best_col, int32_t* gens_per_k);

/* Checkpoint and resume (the paper runs last up to 138 h and describes no checkpoint; this is
 * the state Algorithm 1 carries from one generation to the next). dlm_memetic_state_bytes gives
 * the size of the blob; dlm_memetic_save writes it to caller-owned host memory (a 64-byte header
 * with the configuration, the generation counter and a 64-bit FNV-1a fingerprint of the graph's
 * bit rows and of every parameter (k, p, K, iters, tenure, use_scorer, epochs, batch, lr, seed,
 * problem; for the WVCP also the vertex weights and max_ls), then
 * P, f(P), D(P,P), the offspring S^O, f(S*) and S*, and, with the scorer, its parameters, Adam
 * moments and step counter) and waits; dlm_memetic_load restores it into an object created on the
 * same graph with the same parameters (DLM_EINVAL otherwise) and waits. Every random draw is keyed
 * by (seed, individual, generation, iteration), so a resumed run continues bit-identically to an
 * uninterrupted one. The diagnostics of dlm_memetic_stats restart after a load. */
int64_t dlm_memetic_state_bytes(const dlm_memetic* mm);
dlm_status dlm_memetic_save(dlm_ctx* ctx, dlm_memetic* mm, void* host);
dlm_status dlm_memetic_load(dlm_ctx* ctx, dlm_memetic* mm, const void* host);

/* ---------------------------------------------------------------------------------------------
 * Weighted vertex colouring (WVCP; Eq. score_WVCP: f(S) = sum over classes of the largest vertex
 * weight in the class). The graph must carry vertex weights (1..255).
 *
 * dlm_wvcp_greedy: randomised greedy initialisation (section "Initialization with a greedy random
 * algorithm"). Vertices are visited by decreasing weight, then decreasing degree, then increasing
 * index; vertex number pos of that order takes the colour at index high word of r0 * m among the
 * m already-opened colours (ascending) that none of its coloured neighbours uses, with
 * r = Philox(a = pos, b = 0, c = ind_base + i, tag = WINIT), or opens a new colour when m = 0.
 *   col   device [pop][n] int16 out;  used  device [pop] int32 out (colours opened) or NULL.
 * More than 255 colours raises DLM_EUNSUPPORTED at dlm_sync. This call waits for its kernel.
 *
 * dlm_wvcp_tabu_batch: feasible and infeasible tabu search with a fixed penalty phi (section
 * "Parallel iterated feasible and infeasible Tabu Search", Eq. AFISA_score; Algorithm 2 with its
 * last-run setting phi = 2 max w). It minimises g = f + phi * c, c the conflicting edges, over all
 * one-moves (v, c') of all vertices. A vertex that moves is frozen for
 * tt = U{0..L_max} + floor(alpha_num * n / alpha_den) iterations (Table params-WVCP: alpha = 0.2);
 * a move of a frozen vertex is admissible only when g + delta < best g of the run. Iteration it
 * draws r = Philox(a = it, b = generation, c = ind_base + i, tag = TABU); ties: the j-th admissible
 * minimum in (v, c') order, j = high word of r0 * (number of ties); U{0..L_max} from r1.
 *   col      device [pop][n] int16: in start colourings (0..k-1), out the best-g colouring visited
 *   best_g   device [pop] int64 out;  best_fc  device [pop][2] int64 out (f, c of it) or NULL
 *   moves    device [pop] int64 out or NULL;  iters  iterations per individual (paper: 10 |V|)
 * Limits: k <= 255; max w + phi * (max degree + 1) < 2^30; tenure < 2^14. */
dlm_status dlm_wvcp_greedy(dlm_ctx* ctx, const dlm_graph* g, int32_t pop, uint64_t seed, uint32_t ind_base,
                           int16_t* col, int32_t* used);
dlm_status dlm_wvcp_tabu_batch(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                               int64_t* best_g, int64_t* best_fc, int64_t* moves, int64_t iters, dlm_tenure tenure,
                               int64_t phi, uint64_t seed, uint32_t generation, uint32_t ind_base);
/* As dlm_wvcp_tabu_batch with a per-iteration trace: device [pop][iters][4] int32 of
 * (v, c', delta, #ties), (-1, -1, 0, 0) for an iteration without a move, or NULL; and the entry
 * size of the per-individual conflict table: 0 automatic (as dlm_wvcp_entry_bits reports), 8 or
 * 16. With 8-bit entries the whole table stays in shared memory; an individual whose start
 * colouring has a class of more than 255 vertices, or whose search would grow one past 255, is
 * searched again from its start colouring with 16-bit entries (same draws, same result). 16 puts
 * the colours that do not fit shared memory in an L2-resident slab per CTA. 8 returns
 * DLM_EUNSUPPORTED when the u8 table does not fit. The result never depends on the entry size. */
dlm_status dlm_wvcp_tabu_batch_ex(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                  int64_t* best_g, int64_t* best_fc, int64_t* moves, int64_t iters,
                                  dlm_tenure tenure, int64_t phi, uint64_t seed, uint32_t generation,
                                  uint32_t ind_base, int32_t* trace, int32_t entry_bits);
/* The entry size (8 or 16; 0 when the state does not fit at all) the weighted tabu search takes
 * on graph g with k colours: 8 when only 8-bit entries keep the whole conflict table in shared
 * memory, else 16.   bits  host int32 out. */
dlm_status dlm_wvcp_entry_bits(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t* bits);

/* Parallel iterated feasible and infeasible tabu search (Algorithm 2): max_ls (paper: 10, at most
 * 16) successive searches of iters iterations (paper: 10 |V|) per individual, each from the
 * previous one's best colouring (by g), on g = fscale f + phi c, phi held in fixed point with
 * resolution 1 / fscale (a reading: the paper's phi is real). phi starts at phi0 (paper:
 * k max w / (2 |V|), times fscale); after search t, while t + 1 < max_ls - 1, it is halved (floor,
 * at least 1) when that search's best colouring is legal and doubled otherwise; the last search
 * uses phi_last (paper: 2 max w, times fscale). Search t draws Philox blocks of generation
 * generation * 16 + t. col (device [pop][n] int16, in: start, out: the last search's best);
 * best_col (device [pop][n] int16 out): the legal colouring with the smallest f over the
 * searches, or the last search's best when none was legal; best_f (device [pop] int64 out): its
 * f, or -1. Move keys are 32-bit: fscale max w + phi (max degree + 1) must stay below 2^30 for
 * the largest phi of the schedule (DLM_EUNSUPPORTED otherwise). Allocates and frees a pop * 32
 * byte scratch and waits for the searches. */
dlm_status dlm_wvcp_iterated(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                             int16_t* best_col, int64_t* best_f, int64_t iters, int32_t max_ls, dlm_tenure tenure,
                             int32_t fscale, int64_t phi0, int64_t phi_last, uint64_t seed, uint32_t generation,
                             uint32_t ind_base);

/* ---------------------------------------------------------------------------------------------
 * Building block of the scorer, exported for testing: C = A . B^T on the tcgen05 tensor cores.
 * A: device [M][K] bf16 row-major, B: device [N][K] bf16 row-major, C: device [M][N] float32.
 * K must be a multiple of 64 and N a multiple of 64; FP32 accumulation.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_gemm_bf16(dlm_ctx* ctx, const void* A, const void* B, float* C, int32_t M, int32_t N, int32_t K);

/* ---------------------------------------------------------------------------------------------
 * Measurement utility (no counterpart in the paper): streams conflict-free 16-byte shared-memory
 * loads on every SM and returns the achieved bandwidth in GB/s (host double). It is the
 * denominator of the tabu kernel's roofline, whose state is held in shared memory.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_probe_smem_bandwidth(dlm_ctx* ctx, double* gbps);

/* L2 read bandwidth of this GPU in GB/s (the paper has no counterpart: measurement support): every
 * SM streams 16-byte loads that bypass L1 over a 32 MB buffer held in L2, 16 passes after a warm-up
 * pass; uses the context's workspace and synchronises its stream. */
dlm_status dlm_probe_l2_bandwidth(dlm_ctx* ctx, double* gbps);

/* How dlm_tabucol_batch would run a problem (the paper has no counterpart: measurement support).
 * info (host, 8 int32): [0] 1 = several individuals per CTA (tabu flags inside gamma), 2 = the
 * same with 8-bit conflict-table entries, 0 = one individual per CTA; [1] warps per individual; [2] individuals per CTA; [3] tabu ring entries;
 * [4] vertices per thread; [5] 1 = the graph's bit rows in shared memory; [6] CTAs launched;
 * [7] individual slots (CTAs x individuals per CTA). warps = 0: the library's choice. */
dlm_status dlm_tabucol_launch_info(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int32_t warps,
                                   int32_t* info);

/* ---------------------------------------------------------------------------------------------
 * Measurement utility (no counterpart in the paper): while enabled (enable != 0), every launch of
 * the tensor-core GEMM kernel made through ctx (scorer forward, scorer backward, dlm_gemm_bf16)
 * is bracketed by two CUDA events recorded on the context's stream. dlm_gemm_profile_read waits
 * for the stream, returns in host memory the summed launch time (ms), the executed tensor-core
 * FLOPs (2 M N K per MMA pass: 1 pass, 2 with one split operand, 3 with both) and the number of
 * launches recorded, then clears the record. Recording adds two event records per launch.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_gemm_profile(dlm_ctx* ctx, int32_t enable);
dlm_status dlm_gemm_profile_read(dlm_ctx* ctx, double* ms, double* flops, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* DLMCOL_H */
