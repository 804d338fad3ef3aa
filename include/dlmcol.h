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
 * Limits: k <= 128 (DLM_EUNSUPPORTED above); the per-individual state must fit the GPU's shared
 * memory: 4 * n * k bytes plus small arrays, about 227 KB (n = 1000 with k <= 52, n = 500 with
 * k <= 108). Tenures above 32766 iterations stop the search with DLM_EUNSUPPORTED at dlm_sync. */
dlm_status dlm_tabucol_batch(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                             int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                             uint32_t generation, uint32_t ind_base);

/* As dlm_tabucol_batch, with warps_per_individual forced (1, 2, 4 or 8; 0 = autotuned), an
 * optional per-iteration trace -- device [pop][iters][4] int32 of (v, c, delta, #tied moves),
 * (-1, -1, 0, 0) for an iteration without a move, entries after an early stop untouched -- and an
 * optional work count -- device [pop][2] int64: the number of conflicting rows scanned and the sum
 * of the degrees of the moved vertices (the algorithmic work of the scan and of the update). */
dlm_status dlm_tabucol_batch_ex(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                                uint32_t generation, uint32_t ind_base, int32_t warps_per_individual,
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

/* Autotuner for the tabu kernel: times warps_per_individual in {1, 2, 4, 8} on a short run of
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
 *   NULL (child_id = t);  children device [m][n] int16 out.  Limits: k <= 128, n <= 2048.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_gpx_batch(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* parents, int32_t pop,
                         const int32_t* pairs, const uint32_t* child_id, int32_t m, int16_t* children,
                         uint64_t seed, uint32_t generation);

/* ---------------------------------------------------------------------------------------------
 * Approximate set-theoretic partition distance (section "Distance computation"): with
 * M[c][c'] = |A_c intersect B_c'|, D = n - min(sum_c max_c' M, sum_c' max_c M), a symmetric lower
 * bound of the exact (Hungarian) distance, exact when the best-match map is injective.
 *   X device [a][n], Y device [b][n] int16 colourings; D device out, D[i * ldD + j] = D(X_i, Y_j).
 *   upper != 0 with X == Y computes only j > i (and writes those entries). Limits: k <= 128.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_distance_batch(dlm_ctx* ctx, int32_t n, int32_t k, const int16_t* X, int32_t a, const int16_t* Y,
                              int32_t b, int16_t* D, int64_t ldD, int32_t upper);

/* Distance-and-quality pool update (section "Population update"): the 2p candidates (index < p:
 * the population, >= p: the improved individuals) are visited by increasing fit, ties by lower
 * index; a candidate is kept when its distance to every candidate kept so far is > n / 10; if
 * fewer than p are kept the best remaining ones (same order) fill the population.
 *   fit device [2p] int64;  D device [2p][2p] int16;  sel device [p] int32 out (in keep order). */
dlm_status dlm_pool_update(dlm_ctx* ctx, int32_t p, int32_t n, const int64_t* fit, const int16_t* D, int32_t* sel);

/* Parent matching (section "Parent matching ..."): the K nearest j != i of every i by D (device
 * [p][p] int16), nearest first, ties by lower index. nbr device [p][K] int32 out. K <= 64. */
dlm_status dlm_knn(dlm_ctx* ctx, int32_t p, const int16_t* D, int32_t K, int32_t* nbr);

/* ---------------------------------------------------------------------------------------------
 * Measurement utility (no counterpart in the paper): streams conflict-free 16-byte shared-memory
 * loads on every SM and returns the achieved bandwidth in GB/s (host double). It is the
 * denominator of the tabu kernel's roofline, whose state is held in shared memory.
 * ------------------------------------------------------------------------------------------- */
dlm_status dlm_probe_smem_bandwidth(dlm_ctx* ctx, double* gbps);

#ifdef __cplusplus
}
#endif

#endif /* DLMCOL_H */
