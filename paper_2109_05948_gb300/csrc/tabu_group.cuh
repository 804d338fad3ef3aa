// TabuCol with several individuals per CTA (tabu_group.cu): launch arguments, shared-memory plan.
#pragma once

#include "common.cuh"

namespace dlm {

// gamma row stride in u16 entries: ks / 2 odd, so that rows of different vertices start in
// different shared-memory banks
__host__ __device__ inline int group_row_stride(int k) {
  int kw = (k + 1) / 2;
  if ((kw & 1) == 0) kw += 1;
  return 2 * kw;
}

// gamma row stride in u8 entries: ks / 4 odd (the same bank rule for byte entries)
__host__ __device__ inline int group_row_stride8(int k) {
  int kw = (k + 3) / 4;
  if ((kw & 1) == 0) kw += 1;
  return 4 * kw;
}

// byte offsets of one individual's arrays within its group's shared memory
struct GroupLayout {
  size_t gam, csz, col, best, ring, due, red, sc, total;
};

struct GroupArgs {
  int32_t n, k, ks, words, pop, W, G, R, per;
  const uint32_t* bits;  // device [n][words] adjacency bit rows
  int16_t* col;          // [pop][n] in: start colourings, out: best colourings
  int64_t* best_f;       // [pop]
  int64_t* moves;        // [pop] or null
  int32_t* trace;        // [pop][iters][4] or null
  int64_t* work;         // [pop][3] or null
  int64_t iters;
  uint32_t ind_base;
  uint32_t L1;           // L_max + 1
  int32_t an, ad;        // alpha = an / ad
  uint64_t ad_recip;     // ceil(2^64 / ad) for ad >= 2
  uint64_t seed;
  uint32_t gen;
  int32_t* status;
  const int32_t* cancel;
  uint2* far;            // per slot far_cap entries, or null
  int32_t far_cap;
  size_t group_bytes, bits_bytes;
  int32_t* redo;         // [pop] individuals a u8 launch gave up
  int32_t redo_mode;     // 0: none; 1 (u8 launch): flag the individuals given up; 2: only those
};

// W warps per individual, G individuals per CTA, ring of R tabu entries, per vertices a thread,
// the graph's bit rows in shared memory (bsm) or read from global memory
struct GroupPlan {
  int W, G, R, per;
  bool bsm;
  int eb;                // bits of a gamma entry: 16, or 8 (counts up to 126, u16 fallback)
  size_t group_bytes, bits_bytes, smem;
};

// Shared-memory plan for n vertices, k colours, W warps per individual within `optin` bytes
// (ring_force > 0 forces the ring size); false when one individual's state does not fit.
bool group_plan(int n, int k, int words, int W, size_t optin, int pop, int num_sms, int ring_force, int eb,
                GroupPlan* out);
// resident CTAs of the plan's kernel on one SM
int group_ctas_per_sm(const GroupPlan& plan);

// CTAs the grouped launch of `pop` individuals uses (resident CTAs at most; each loops over its
// individuals)
int group_grid(dlm_ctx* ctx, const GroupPlan& plan, int pop);

dlm_status tabucol_group_launch(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int16_t* col,
                                int64_t* best_f, int64_t* moves, int64_t iters, dlm_tenure tenure, uint64_t seed,
                                uint32_t generation, uint32_t ind_base, const GroupPlan& plan, int32_t* trace,
                                int64_t* work, void* far_mem = nullptr, int32_t** redo_out = nullptr);
// (redo_out: with u8 entries and no u16 plan of the grouped kernel, only the u8 pass runs and
// *redo_out receives the device flags [pop] of the individuals it gave up, for the caller to
// search with the one-individual-per-CTA kernel)
// bytes of far-list memory a launch needs (0 when every tenure fits the ring); far_mem of
// tabucol_group_launch: that much device memory, or null to take it from the context's workspace
int64_t group_far_cap(const dlm_graph* g, int32_t k, int64_t iters, dlm_tenure tenure, const GroupPlan& plan);
size_t group_far_bytes(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, int64_t iters, dlm_tenure tenure,
                       const GroupPlan& plan);

}  // namespace dlm
