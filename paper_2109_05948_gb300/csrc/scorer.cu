// Offspring scorer f_theta (section "Deep neural network training"): colour-permutation
// invariant deep-set network, trained online with Adam, scoring the K GPX candidates of every
// individual (Eq. select_cross).
//
// Network (the sizes of the benchmarked workload): layer 0 sums the 64-d embedding rows E[v]
// over each colour class (V_i Lambda_0; the rho(S) Gamma_0 term is the same for every partition
// and is part of beta_0), LeakyReLU_0.2; layers 1..3: H' = LeakyReLU_0.2(beta + H Lambda +
// rho(H) Gamma) with width 256 and rho the mean over the k classes; output = mean over classes of
// the linear head. In a training batch each candidate occupies R = 64 ceil(k / 64) rows (rows
// k..R-1 are zero); a scoring chunk keeps k rows per candidate.
//
// Where the work runs:
//   tcgen05 BF16 GEMMs (FP32 accumulate in TMEM): H Lambda for layers 1..3 (fused epilogue:
//     + per-candidate (rho Gamma + beta), LeakyReLU, row mask, bf16 store, head dot product),
//     the backward dH = dZ Lambda^T (fused: + per-candidate term, LeakyReLU derivative, row mask),
//     the weight gradients dLambda = H^T dZ (split-K) and, for scoring chunks, the per-candidate
//     rho(H) Gamma terms (both operands split). Lambda enters as two bf16 matrices (hi + lo):
//     two MMAs per K step keep the weights at ~16 mantissa bits, since rounding the weights to
//     bf16 shifts every row of a layer the same way and dominates the error.
//   CUDA cores (FP32): the class pooling of layer 0 (a gather, not a contraction), per-candidate
//     means and column sums, the rho(H) Gamma terms of small and training batches (fused into
//     the pooling and the class-mean kernels), the embedding gradient (scatter by colour), Adam
//     (which also writes the bf16 operand copies). A training step is one CUDA graph: 16 launches
//     on the chain forward -> dZ_3 -> ... -> dZ_0 -> Adam, and side branches for the layers'
//     weight gradients, the head gradient and loss, the embedding bias and Adam's bias
//     corrections.
// All reductions run in a fixed order: results are deterministic run to run.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tcgemm.cuh"

using bf16 = __nv_bfloat16;

namespace dlm {
constexpr int kD0 = 64, kD = 256, kNL = 3, kRMax = 256;  // rows per candidate: 64 ceil(k / 64) <= 256
}

struct dlm_scorer {
  int n = 0, k = 0;
  int R = 64;  // rows per candidate in the training layer matrices: k rounded up to a multiple of 64
  int Rs = 64;  // rows per candidate when scoring: k (no padding rows; rows are independent in every
                // layer GEMM, so the scores are the same)
  int64_t np = 0;
  int64_t t = 0;  // Adam step counter
  size_t oE = 0, ob0 = 0, olam[4] = {}, ogam[4] = {}, ob[4] = {}, owh = 0, obh = 0;
  float *theta = nullptr, *am = nullptr, *av = nullptr, *grad = nullptr;
  bf16* E16 = nullptr;
  bf16 *LamT[4] = {}, *Lam[4] = {}, *LamTlo[4] = {}, *Lamlo[4] = {};
  bf16 *GamT[4] = {}, *GamTlo[4] = {};  // Gamma^T [kD][din], bf16 hi and lo
  // forward work buffers for up to `cap` candidates
  int cap = 0;
  bf16* H[4] = {};
  bf16* Hlo[4] = {};  // lo parts of the scoring activations (split_act)
  int split_act = 1;  // scoring activations as bf16 hi + lo (three MMA passes) or bf16 alone
  bf16* Mb[4] = {};
  bf16* Mblo[4] = {};
  float* Mf[4] = {};
  float* G[4] = {};
  float* rowdot = nullptr;
  // backward buffers for up to `capb` candidates
  int capb = 0;
  bf16* Hb[4] = {};
  bf16* Hblo[4] = {};  // lo parts of the training activations (hi + lo carries ~16 mantissa bits)
  bf16* HT[4] = {};
  bf16* HTlo[4] = {};
  bf16* Mbb[4] = {};
  bf16* Mbblo[4] = {};
  float* Mfb[4] = {};
  float* Gbf[4] = {};
  bf16* dZ[4] = {};
  bf16* dZT[4] = {};
  float* S[4] = {};
  float* Gb = nullptr;
  float* part[4] = {};  // split-K partial sums of dLambda_l, one buffer per layer
  // the weight gradients of layer l (dLambda_l GEMM, its split-K sum, dGamma_l, dbeta_l) run on a
  // side branch forked after the layer's transposes and joined before the Adam step, off the
  // chain dZ_l -> dZ_{l-1} of the backward pass
  // branch streams: [1..3] one per layer (the branches of a step overlap), [0] the head's gradient
  // and the loss, then the embedding bias gradient
  cudaStream_t side[4] = {};
  // fork / join events: [1..3] the layers' weight gradients, [4] the head's gradient and the loss,
  // [5] the embedding bias gradient
  cudaEvent_t ev_fork[6] = {}, ev_join[6] = {};
  float* sqerr = nullptr;  // squared error of each candidate of a training batch
  // Adam's bias corrections of the coming step, formed on the side branch ([0] 1 - 0.9^t,
  // [1] sqrt(1 - 0.999^t))
  float* d_bc = nullptr;
  cudaEvent_t ev_bc_fork = nullptr, ev_bc_join = nullptr;
  float* rowdotb = nullptr;
  float* outb = nullptr;
  float* dout = nullptr;
  float* lossd = nullptr;
  // training
  float* y = nullptr;         // standardised targets
  int32_t* perm = nullptr;
  int capp = 0;
  // training step replayed from a CUDA graph: the batch offset within the epoch's permutation and
  // the Adam step counter live on the device ([0] offset, [1] t)
  int32_t* d_step = nullptr;
  cudaStream_t cap_stream = nullptr;
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    int B = 0, b = 0;
    float lr = 0.f;
    const int16_t* cols = nullptr;
  } sg[2];
  int sg_next = 0;
  bool stepped = false;  // one eager step has run (first-use attributes are set outside capture)
};

namespace dlm {

static int din_of(int l) { return l == 1 ? kD0 : kD; }

// ------------------------------------------------------------------------------------------------
// parameter conversion: fp32 master -> bf16 operands in GEMM layouts
// ------------------------------------------------------------------------------------------------
struct ConvArgs {
  const float* theta;
  int n;
  size_t oE, olam[4], ogam[4];
  bf16* E16;
  bf16 *LamT[4], *Lam[4], *LamTlo[4], *Lamlo[4];
  bf16 *GamT[4], *GamTlo[4];
};

__global__ void k_convert(ConvArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nE = (int64_t)a.n * kD0;
  if (t < nE) { a.E16[t] = __float2bfloat16_rn(a.theta[a.oE + t]); return; }
  int64_t r = t - nE;
  for (int l = 1; l <= kNL; ++l) {
    const int din = l == 1 ? kD0 : kD;
    const int64_t sz = (int64_t)din * kD;
    if (r < sz) {
      const int f = (int)(r / kD), o = (int)(r % kD);
      const float lam = a.theta[a.olam[l] + r];
      const bf16 hi = __float2bfloat16_rn(lam);
      const bf16 lo = __float2bfloat16_rn(lam - __bfloat162float(hi));
      a.Lam[l][r] = hi;
      a.Lamlo[l][r] = lo;
      a.LamT[l][(size_t)o * din + f] = hi;
      a.LamTlo[l][(size_t)o * din + f] = lo;
      return;
    }
    r -= sz;
    if (r < sz) {
      const int f = (int)(r / kD), o = (int)(r % kD);
      const float gam = a.theta[a.ogam[l] + r];
      const bf16 hi = __float2bfloat16_rn(gam);
      a.GamT[l][(size_t)o * din + f] = hi;
      a.GamTlo[l][(size_t)o * din + f] = __float2bfloat16_rn(gam - __bfloat162float(hi));
      return;
    }
    r -= sz;
  }
}

// G[o] = beta[o] + sum_f m[f] Gamma[f][o] for the 256 threads o of a block (m in shared memory,
// f ascending; thirty-two Gamma loads in flight; din a multiple of 32)
__device__ __forceinline__ float gterm_col(const float* m, int din, const float* gam, const float* beta, int o) {
  float acc = 0.f;
  for (int f = 0; f < din; f += 32) {
    float g[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) g[u] = gam[(size_t)(f + u) * kD + o];
#pragma unroll
    for (int u = 0; u < 32; ++u) acc += m[f + u] * g[u];
  }
  return acc + beta[o];
}

// ------------------------------------------------------------------------------------------------
// layer 0: class pooling. One CTA of kPoolWarps warps per candidate (grid-stride): a stable
// counting sort puts the vertices of each class in ascending order, then warp w sums the FP32
// embedding rows of classes w, w + kPoolWarps, ... with lane = feature pair (fixed summation order;
// E is read through L1/L2).
// A training batch reads its candidates through the epoch permutation (candidate b = sample
// perm[step[0] + b]) and, with G1 set, ends with layer 1's per-candidate term
// G1 = beta_1 + mean_c(H0) Gamma_1.
// ------------------------------------------------------------------------------------------------
constexpr int kPoolWarps = 8;
__global__ void __launch_bounds__(32 * kPoolWarps) k_pool(int n, int k, int R, const int16_t* cols, int c, const int32_t* perm,
                                              const int32_t* step, const float* E, const float* b0, bf16* H0,
                                              bf16* H0lo, float* Mf0, bf16* Mb0, bf16* Mb0lo, const float* gam1,
                                              const float* beta1, float* G1, int32_t* status) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint8_t* col = sm;                                        // [n]
  uint16_t* mem = (uint16_t*)(sm + ((n + 15) & ~15));       // [n]
  int* cnt = (int*)(mem + ((n + 7) & ~7));                  // [256]
  int* off = cnt + kRMax;                                   // [257]
  int* cur = off + kRMax + 1;                               // [256]
  float* part = (float*)(cur + kRMax);                      // [kPoolWarps][64]
  float* mvec = part + kPoolWarps * 64;                     // [64]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int cand = blockIdx.x; cand < c; cand += gridDim.x) {
    const int srow = perm ? perm[step[0] + cand] : cand;
    const int16_t* cc = cols + (size_t)srow * n;
    if (tid < kRMax) cnt[tid] = 0;  // every class counter
    __syncthreads();
    for (int v = tid; v < n; v += 32 * kPoolWarps) {
      int q = cc[v];
      if (q < 0 || q >= k) { raise_status(status, DLM_EINVAL); q = 0; }
      col[v] = (uint8_t)q;
      atomicAdd(cnt + q, 1);
    }
    __syncthreads();
    if (warp == 0) {
      // exclusive prefix of the class sizes: lane l holds classes 8 l .. 8 l + 7
      int x[8], loc = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) { x[u] = cnt[8 * lane + u]; loc += x[u]; }
      int incl = loc;
      for (int d = 1; d < 32; d <<= 1) {
        const int a = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += a;
      }
      int o = incl - loc;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        off[8 * lane + u] = o;
        cur[8 * lane + u] = o;
        o += x[u];
      }
      if (lane == 31) off[kRMax] = incl;
      // stable scatter: chunks of 32 vertices in order, rank among equal colours by lane order
      for (int v0 = 0; v0 < n; v0 += 32) {
        const int v = v0 + lane;
        const int q = v < n ? col[v] : kRMax + lane;
        const unsigned same = __match_any_sync(0xFFFFFFFFu, q);
        const int rank = __popc(same & ((1u << lane) - 1u));
        int base = 0;
        if (v < n) base = cur[q];
        __syncwarp();
        if (v < n) {
          mem[base + rank] = (uint16_t)v;
          if (rank == __popc(same) - 1) cur[q] = base + rank + 1;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    float2 msum = make_float2(0.f, 0.f);
    const float2 bb = make_float2(b0[2 * lane], b0[2 * lane + 1]);
    for (int q = warp; q < R; q += kPoolWarps) {
      float2 acc = make_float2(0.f, 0.f);
      if (q < k) {
        // members in ascending order; sixteen (then eight) embedding rows are loaded before they are added (the
        // rows come from L2, so the loads of a class overlap), the sum keeps the member order
        int j = off[q];
        const int je = off[q + 1];
        for (; j + 16 <= je; j += 16) {
          float2 ef[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) ef[u] = *reinterpret_cast<const float2*>(E + (size_t)mem[j + u] * kD0 + 2 * lane);
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            acc.x += ef[u].x;
            acc.y += ef[u].y;
          }
        }
        for (; j + 8 <= je; j += 8) {
          float2 ef[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) ef[u] = *reinterpret_cast<const float2*>(E + (size_t)mem[j + u] * kD0 + 2 * lane);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            acc.x += ef[u].x;
            acc.y += ef[u].y;
          }
        }
        for (; j < je; ++j) {
          const float2 ef = *reinterpret_cast<const float2*>(E + (size_t)mem[j] * kD0 + 2 * lane);
          acc.x += ef.x;
          acc.y += ef.y;
        }
        float zx = acc.x + bb.x, zy = acc.y + bb.y;
        acc.x = zx > 0.f ? zx : 0.2f * zx;
        acc.y = zy > 0.f ? zy : 0.2f * zy;
        msum.x += acc.x;
        msum.y += acc.y;
      }
      const __nv_bfloat162 hi = __floats2bfloat162_rn(acc.x, acc.y);
      *reinterpret_cast<__nv_bfloat162*>(H0 + ((size_t)cand * R + q) * kD0 + 2 * lane) = hi;
      if (H0lo) {
        const float2 hf = __bfloat1622float2(hi);
        *reinterpret_cast<__nv_bfloat162*>(H0lo + ((size_t)cand * R + q) * kD0 + 2 * lane) =
            __floats2bfloat162_rn(acc.x - hf.x, acc.y - hf.y);
      }
    }
    part[warp * 64 + 2 * lane] = msum.x;
    part[warp * 64 + 2 * lane + 1] = msum.y;
    __syncthreads();
    if (tid < 64) {
      float s = 0.f;
      for (int w = 0; w < kPoolWarps; ++w) s += part[w * 64 + tid];
      s /= (float)k;
      Mf0[(size_t)cand * kD0 + tid] = s;
      mvec[tid] = s;
      const bf16 hi = __float2bfloat16_rn(s);
      Mb0[(size_t)cand * kD0 + tid] = hi;
      Mb0lo[(size_t)cand * kD0 + tid] = __float2bfloat16_rn(s - __bfloat162float(hi));
    }
    __syncthreads();
    if (G1 && tid < kD) G1[(size_t)cand * kD + tid] = gterm_col(mvec, kD0, gam1, beta1, tid);
  }
}

// per-candidate term G[cand][o] = beta[o] + sum_f M[cand][f] Gamma[f][o] in FP32 on CUDA cores,
// for small batches (a training step's 100 candidates), where a tensor-core GEMM of one tile is
// latency bound; a block of 256 threads (thread = o) handles one candidate.
__global__ void __launch_bounds__(256) k_gterm(int c, int din, const float* M, const float* theta, size_t ogam,
                                               size_t ob, float* G) {
  __shared__ float ms[256];
  const int cand = blockIdx.x, o = threadIdx.x;
  if (o < din) ms[o] = M[(size_t)cand * din + o];
  __syncthreads();
  G[(size_t)cand * kD + o] = gterm_col(ms, din, theta + ogam, theta + ob, o);
}

// per-candidate mean (or sum) over the k valid rows of a bf16 [c*R][w] matrix, column col of
// candidate cand; returns the value written to outf
__device__ __forceinline__ float segment_col(const bf16* X, const bf16* Xlo, int w, int k, int R, float scale,
                                             float* outf, bf16* outb, bf16* outblo, int cand, int col) {
  const bf16* x = X + (size_t)cand * R * w + col;
  const bf16* xl = Xlo ? Xlo + (size_t)cand * R * w + col : nullptr;
  float s = 0.f;
  int r = 0;
  for (; r + 16 <= k; r += 16) {  // sixteen rows loaded before they are added, sum in row order
    float t[16];
#pragma unroll
    for (int u = 0; u < 16; ++u)
      t[u] = __bfloat162float(x[(size_t)(r + u) * w]) + (xl ? __bfloat162float(xl[(size_t)(r + u) * w]) : 0.f);
#pragma unroll
    for (int u = 0; u < 16; ++u) s += t[u];
  }
  for (; r < k; ++r) s += __bfloat162float(x[(size_t)r * w]) + (xl ? __bfloat162float(xl[(size_t)r * w]) : 0.f);
  s *= scale;
  outf[(size_t)cand * w + col] = s;
  if (outb) {
    const bf16 hi = __float2bfloat16_rn(s);
    outb[(size_t)cand * w + col] = hi;
    outblo[(size_t)cand * w + col] = __float2bfloat16_rn(s - __bfloat162float(hi));
  }
  return s;
}

// block = w threads, one candidate per block
__global__ void k_segment_reduce(const bf16* X, const bf16* Xlo, int w, int k, int R, float scale, float* outf,
                                 bf16* outb, bf16* outblo) {
  segment_col(X, Xlo, w, k, R, scale, outf, outb, outblo, blockIdx.x, threadIdx.x);
}

// a training batch between layers l and l + 1: the class mean of H_l (written as segment_col
// writes it), then the next layer's per-candidate term G = beta + mean Gamma. One candidate per
// block of kMgGroups x kD threads: group g sums its contiguous share of the k rows (in row order)
// and then its share of the rows f of Gamma; the groups' parts are added in group order. Two
// groups (512 threads): in a memetic generation the training runs beside the distance kernel, whose
// CTAs leave about 768 threads of an SM free, so a 1024-thread block would wait for one to finish.
constexpr int kMgGroups = 2;
__global__ void __launch_bounds__(kMgGroups * kD) k_mean_gterm(const bf16* X, const bf16* Xlo, int k, int R,
                                                               float* outf, bf16* outb, bf16* outblo, const float* gam,
                                                               const float* beta, float* G) {
  __shared__ float ms[kD];
  __shared__ float part[kMgGroups][kD];
  const int cand = blockIdx.x, o = threadIdx.x % kD, grp = threadIdx.x / kD;
  {  // class mean: rows [r0, r1) of this group, eight loads in flight
    const int share = (k + kMgGroups - 1) / kMgGroups;
    const int r0 = min(k, grp * share), r1 = min(k, r0 + share);
    const bf16* x = X + (size_t)cand * R * kD + o;
    const bf16* xl = Xlo ? Xlo + (size_t)cand * R * kD + o : nullptr;
    float sum = 0.f;
    int r = r0;
    for (; r + 8 <= r1; r += 8) {
      float t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        t[u] = __bfloat162float(x[(size_t)(r + u) * kD]) + (xl ? __bfloat162float(xl[(size_t)(r + u) * kD]) : 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) sum += t[u];
    }
    for (; r < r1; ++r) sum += __bfloat162float(x[(size_t)r * kD]) + (xl ? __bfloat162float(xl[(size_t)r * kD]) : 0.f);
    part[grp][o] = sum;
  }
  __syncthreads();
  if (grp == 0) {
    float m = part[0][o];
#pragma unroll
    for (int g = 1; g < kMgGroups; ++g) m += part[g][o];
    m *= 1.f / (float)k;
    ms[o] = m;
    outf[(size_t)cand * kD + o] = m;
    const bf16 hi = __float2bfloat16_rn(m);
    outb[(size_t)cand * kD + o] = hi;
    outblo[(size_t)cand * kD + o] = __float2bfloat16_rn(m - __bfloat162float(hi));
  }
  __syncthreads();
  {  // this group's rows f of Gamma, thirty-two loads in flight
    constexpr int FQ = kD / kMgGroups;
    float acc = 0.f;
    for (int f = grp * FQ; f < (grp + 1) * FQ; f += 32) {
      float g[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) g[u] = gam[(size_t)(f + u) * kD + o];
#pragma unroll
      for (int u = 0; u < 32; ++u) acc += ms[f + u] * g[u];
    }
    part[grp][o] = acc;
  }
  __syncthreads();
  if (grp == 0) {
    float acc = part[0][o];
#pragma unroll
    for (int g = 1; g < kMgGroups; ++g) acc += part[g][o];
    G[(size_t)cand * kD + o] = acc + beta[o];
  }
}

// output = head bias + mean over the k class rows of the head dot, whose row values come in
// `parts` column slices of M = c * R rows each (summed in slice order). One warp per candidate:
// lane l sums rows l, l + 32, ... in order, then a fixed butterfly over the lanes.
constexpr int kHeadOutWarps = 8;
__global__ void __launch_bounds__(32 * kHeadOutWarps) k_head_out(int c, int k, int R, const float* rowdot, int parts,
                                                                 const float* theta, size_t obh, float* out) {
  const int cand = blockIdx.x * kHeadOutWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (cand >= c) return;
  const size_t M = (size_t)c * R;
  float s = 0.f;
  for (int r = lane; r < k; r += 32) {
    float t = rowdot[(size_t)cand * R + r];
    for (int q = 1; q < parts; ++q) t += rowdot[q * M + (size_t)cand * R + r];
    s += t;
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
  if (lane == 0) out[cand] = theta[obh] + s / (float)k;
}

// 32x32 tile (bx, by) of the transpose of a bf16 [rows][cols] matrix into [cols][rows]; 256
// threads as 32 x 8
__device__ __forceinline__ void transpose_tile(const bf16* X, int rows, int cols, bf16* Y, int bx, int by,
                                               bf16 (&tile)[32][33]) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8) {
    const int r = by + i, c = bx + tx;
    if (r < rows && c < cols) tile[i][tx] = X[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int c = bx + i, r = by + tx;
    if (r < rows && c < cols) Y[(size_t)c * rows + r] = tile[tx][i];
  }
}

// backward layer l, before its weight-gradient GEMM (256 threads a block):
//   blocks [0, B)            column sums S = sum over the k valid rows of dZ_l, per candidate
//   next ceil(rows/32) * 8   tiles of dZ_l^T
//   next 2 ceil(rows/32) (din/32)  tiles of H_{l-1}^T and of its lo part
__global__ void __launch_bounds__(256) k_bwd_prep(int B, int k, int R, int rows, int din, const bf16* dZ, float* S,
                                                  bf16* dZT, const bf16* H, const bf16* Hlo, bf16* HT, bf16* HTlo) {
  __shared__ bf16 tile[32][33];
  int t = blockIdx.x;
  if (t < B) {  // (B = 0: the transposes alone)
    segment_col(dZ, nullptr, kD, k, R, 1.f, S, nullptr, nullptr, t, threadIdx.x);
    return;
  }
  t -= B;
  const int ty = (rows + 31) / 32;
  const int tz = ty * (kD / 32);
  if (t < tz) {
    transpose_tile(dZ, rows, kD, dZT, (t % (kD / 32)) * 32, (t / (kD / 32)) * 32, tile);
    return;
  }
  t -= tz;
  const int xh = din / 32, th = ty * xh;
  const bf16* src = t < th ? H : Hlo;
  bf16* dst = t < th ? HT : HTlo;
  if (t >= th) t -= th;
  transpose_tile(src, rows, din, dst, (t % xh) * 32, (t / xh) * 32, tile);
}

// ------------------------------------------------------------------------------------------------
// GEMM epilogues
// ------------------------------------------------------------------------------------------------
struct EpiPlain {  // out[row][col] = alpha * acc + bias[col]
  __device__ void tile(int, int) {}
  float* out;
  int ld, M;
  float alpha;
  const float* bias;
  __device__ void operator()(int row, int col0, const float (&v)[16]) const {
    if (row >= M) return;
    float* o = out + (size_t)row * ld + col0;
#pragma unroll
    for (int i = 0; i < 16; ++i) o[i] = alpha * v[i] + (bias ? bias[col0 + i] : 0.f);
  }
  __device__ void finish(int) const {}
};

struct EpiBias {  // G[row][col] = acc + beta[col] (the per-candidate Gamma term of a layer)
  __device__ void tile(int, int) {}
  float* G;
  int M;
  const float* beta;
  __device__ void operator()(int row, int col0, const float (&v)[16]) const {
    if (row >= M) return;
    float* o = G + (size_t)row * kD + col0;
#pragma unroll
    for (int i = 0; i < 16; i += 4)
      *reinterpret_cast<float4*>(o + i) =
          make_float4(v[i] + beta[col0 + i], v[i + 1] + beta[col0 + i + 1], v[i + 2] + beta[col0 + i + 2],
                      v[i + 3] + beta[col0 + i + 3]);
  }
  __device__ void finish(int) const {}
};

struct EpiPartial {  // split-K slice z: part[z][row][col] = acc
  float* part;
  int ld, M;
  size_t zstride;
  int z = 0;
  __device__ void tile(int zz, int) { z = zz; }
  __device__ void operator()(int row, int col0, const float (&v)[16]) const {
    if (row >= M) return;
    float* o = part + (size_t)z * zstride + (size_t)row * ld + col0;
#pragma unroll
    for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4*>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  }
  __device__ void finish(int) const {}
};

struct EpiLayer {  // H[row][col] = mask(LeakyReLU(acc + G[cand][col])); optional head dot
  bf16* H;    // may be null (scoring the last layer)
  bf16* Hlo;  // lo part (training) or null
  int M, kv, R;
  const float* G;
  const float* wh;
  float* rowdot;  // [256 / pbn][M]: the head dot of each row over the pbn columns one epilogue warp drains
  float dot;
  int pbn;        // half the GEMM's N tile width
  int part;
  // G[cand][gnext - 1 ..] for the next call, loaded during this one (gnext = 0: nothing loaded)
  float4 gq[4];
  int gnext;
  __device__ void tile(int, int n0) { part = n0 / pbn; }
  __device__ void operator()(int row, int col0, const float (&v)[16]) {
    if (row >= M) return;
    const int cand = row / R;
    const bool valid = row - cand * R < kv;
    const float4* gsrc = reinterpret_cast<const float4*>(G + (size_t)cand * kD);
    float4 gc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) gc[i] = gnext == col0 + 1 ? gq[i] : gsrc[col0 / 4 + i];
    gnext = 0;
    if (col0 + 16 < kD) {  // the next 16 columns of this row's G (the call after this one)
#pragma unroll
      for (int i = 0; i < 4; ++i) gq[i] = gsrc[(col0 + 16) / 4 + i];
      gnext = col0 + 17;
    }
    const float* g = reinterpret_cast<const float*>(gc);
    float h[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float z = v[i] + g[i];
      h[i] = valid ? (z > 0.f ? z : 0.2f * z) : 0.f;
    }
    if (wh) {
#pragma unroll
      for (int i = 0; i < 16; ++i) dot += h[i] * wh[col0 + i];
    }
    if (H) {
      uint4 pk[2];
      uint32_t* p = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(h[2 * i], h[2 * i + 1]);
        p[i] = *reinterpret_cast<const uint32_t*>(&b2);
      }
      uint4* dst = reinterpret_cast<uint4*>(H + (size_t)row * kD + col0);
      dst[0] = pk[0];
      dst[1] = pk[1];
      if (Hlo) {
        const bf16* hb = reinterpret_cast<const bf16*>(pk);
        uint4 lk[2];
        uint32_t* q = reinterpret_cast<uint32_t*>(lk);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const __nv_bfloat162 b2 =
              __floats2bfloat162_rn(h[2 * i] - __bfloat162float(hb[2 * i]), h[2 * i + 1] - __bfloat162float(hb[2 * i + 1]));
          q[i] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        uint4* dl = reinterpret_cast<uint4*>(Hlo + (size_t)row * kD + col0);
        dl[0] = lk[0];
        dl[1] = lk[1];
      }
    }
  }
  __device__ void finish(int row) const {
    if (rowdot && row < M) rowdot[(size_t)part * M + row] = dot;
  }
};

struct EpiBwd {  // dZprev[row][col] = mask((acc + Gb[cand][col]) * LeakyReLU'(Hprev[row][col]))
  __device__ void tile(int, int) {}
  bf16* dZ;
  int ld, M, kv, R;
  const float* Gb;
  const bf16* Hp;
  __device__ void operator()(int row, int col0, const float (&v)[16]) const {
    if (row >= M) return;
    const int cand = row / R;
    const bool valid = row - cand * R < kv;
    const float* g = Gb + (size_t)cand * ld + col0;
    const uint4* hsrc = reinterpret_cast<const uint4*>(Hp + (size_t)row * ld + col0);
    uint4 hv[2] = {hsrc[0], hsrc[1]};
    const bf16* hb = reinterpret_cast<const bf16*>(hv);
    uint4 pk[2];
    uint32_t* p = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float d0 = v[2 * i] + g[2 * i], d1 = v[2 * i + 1] + g[2 * i + 1];
      d0 *= __bfloat162float(hb[2 * i]) > 0.f ? 1.f : 0.2f;
      d1 *= __bfloat162float(hb[2 * i + 1]) > 0.f ? 1.f : 0.2f;
      if (!valid) { d0 = 0.f; d1 = 0.f; }
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(d0, d1);
      p[i] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    uint4* dst = reinterpret_cast<uint4*>(dZ + (size_t)row * ld + col0);
    dst[0] = pk[0];
    dst[1] = pk[1];
  }
  __device__ void finish(int) const {}
};

// ------------------------------------------------------------------------------------------------
// backward helpers (batch of B candidates)
// ------------------------------------------------------------------------------------------------
// end of a training batch's forward pass, one candidate per block of kD threads: the class mean of
// H3 (Mf3 and its bf16 hi / lo, as segment_col writes them), the output out = head bias + mean over
// the k class rows of the head dot (warp 0, in the order of k_head_out), the loss gradient
// dout = 2 (out - y) / B and the squared error; with perm, candidate i is sample perm[step[0] + i]
// (target y of that sample)
__global__ void __launch_bounds__(kD) k_head_fwd(int B, int k, int R, const bf16* H3, const bf16* H3lo, float* Mf3,
                                                 bf16* Mb3, bf16* Mb3lo, const float* rowdot, int parts,
                                                 const float* theta, size_t obh, const float* y, const int32_t* perm,
                                                 const int32_t* step, float* out, float* dout, float* sqerr) {
  const int cand = blockIdx.x, o = threadIdx.x;
  segment_col(H3, H3lo, kD, k, R, 1.f / k, Mf3, Mb3, Mb3lo, cand, o);
  if (o < 32) {
    const size_t M = (size_t)B * R;
    float sum = 0.f;
    for (int r = o; r < k; r += 32) {
      float t = rowdot[(size_t)cand * R + r];
      for (int q = 1; q < parts; ++q) t += rowdot[q * M + (size_t)cand * R + r];
      sum += t;
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, d);
    if (o == 0) {
      const float ov = theta[obh] + sum / (float)k;
      out[cand] = ov;
      const float e = ov - y[perm ? perm[step[0] + cand] : cand];
      dout[cand] = 2.f * e / (float)B;
      sqerr[cand] = e * e;
    }
  }
}

// dZ3 = (dout/k * wh) * LeakyReLU'(H3) on valid rows; block = one candidate row chunk
__device__ __forceinline__ void head_back_row(int k, int R, const float* dout, const float* theta, size_t owh,
                                              const bf16* H3, bf16* dZ3, int row, int o) {
  const int cand = row / R;
  const bool valid = row - cand * R < k;
  float d = 0.f;
  if (valid) {
    d = dout[cand] / (float)k * theta[owh + o];
    d *= __bfloat162float(H3[(size_t)row * kD + o]) > 0.f ? 1.f : 0.2f;
  }
  dZ3[(size_t)row * kD + o] = __float2bfloat16_rn(d);
}

// grad of the head: wh[o] = sum_cand dout * mean(H3)[cand][o]; bh = sum dout
__device__ __forceinline__ void head_grad_col(int B, const float* dout, const float* Mf3, float* grad, size_t owh,
                                              size_t obh, int o) {
  float s = 0.f;
  int c = 0;
  for (; c + 8 <= B; c += 8) {
    float m[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] = Mf3[(size_t)(c + u) * kD + o];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += dout[c + u] * m[u];
  }
  for (; c < B; ++c) s += dout[c] * Mf3[(size_t)c * kD + o];
  grad[owh + o] = s;
  if (o == 0) {
    float b = 0.f;
    for (int c = 0; c < B; ++c) b += dout[c];
    grad[obh] = b;
  }
}

// dZ3 = (dout/k * wh) * LeakyReLU'(H3) on valid rows (thread = column, kHeadRows rows a block)
constexpr int kHeadRows = 8;
__global__ void __launch_bounds__(kD) k_head_bwd(int k, int R, int rows, const float* dout, const float* theta,
                                                 size_t owh, const bf16* H3, bf16* dZ3) {
  const int rb = (int)blockIdx.x * kHeadRows;
#pragma unroll
  for (int i = 0; i < kHeadRows; ++i)
    if (rb + i < rows) head_back_row(k, R, dout, theta, owh, H3, dZ3, rb + i, threadIdx.x);
}

// the head's gradient (wh[o] = sum_cand dout * mean(H3)[cand][o], bh = sum dout) and the batch's
// MSE loss; one block of kD threads, on a side branch
__global__ void __launch_bounds__(kD) k_head_grad(int B, const float* dout, const float* Mf3, float* grad, size_t owh,
                                                  size_t obh, const float* sqerr, float* loss) {
  head_grad_col(B, dout, Mf3, grad, owh, obh, threadIdx.x);
  if (threadIdx.x >= 32 && threadIdx.x < 64) {  // warp 1: lane-strided sums, then a fixed butterfly
    const int lane = threadIdx.x - 32;
    float t = 0.f;
    for (int i = lane; i < B; i += 32) t += sqerr[i];
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, d);
    if (lane == 0) *loss = t / (float)B;
  }
}

// dGamma[f][o] = sum_cand Mprev[cand][f] * S[cand][o]; dbeta[o] = sum_cand S[cand][o]
__device__ __forceinline__ void dgamma_col(int B, int din, const float* Mprev, const float* S, float* grad,
                                           size_t ogam, size_t ob, int f, int o) {
  float s = 0.f;
  int c = 0;
  for (; c + 8 <= B; c += 8) {  // eight candidates' loads in flight, sum in candidate order
    float a[8], b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      a[u] = Mprev[(size_t)(c + u) * din + f];
      b[u] = S[(size_t)(c + u) * kD + o];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u] * b[u];
  }
  for (; c < B; ++c) s += Mprev[(size_t)c * din + f] * S[(size_t)c * kD + o];
  grad[ogam + (size_t)f * kD + o] = s;
  if (f == 0) {
    float b = 0.f;
    for (int c = 0; c < B; ++c) b += S[(size_t)c * kD + o];
    grad[ob + o] = b;
  }
}

// backward layer l, after its weight-gradient GEMM (256 threads a block):
//   blocks [0, cnt / 256)   dLambda = sum of the split-K slices (fixed slice order)
//   next din blocks         dGamma row f and (f = 0) dbeta
__global__ void __launch_bounds__(kD) k_bwd_grads(int B, int din, int64_t cnt, int splits, const float* part,
                                                  float* dlam, const float* Mprev, const float* S, float* grad,
                                                  size_t ogam, size_t ob) {
  const int64_t nr = (cnt + 255) / 256;
  const int64_t t = blockIdx.x;
  if (t < nr) {
    const int64_t i = t * 256 + threadIdx.x;
    if (i >= cnt) return;
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * cnt + i];
    dlam[i] = s;
    return;
  }
  dgamma_col(B, din, Mprev, S, grad, ogam, ob, (int)(t - nr), threadIdx.x);
}

// backward layer l on the chain dZ_l -> dZ_{l-1}, one candidate per block of kMgGroups x kD
// threads: the column sums S of its k valid rows of dZ_l (group g sums its contiguous share of the
// rows in order, the groups' parts are added in group order; written out for dGamma_l and
// dbeta_l), then the per-candidate term Gb[cand][f] = (1/k) sum_o S[o] Gamma[f][o] of dH_{l-1}:
// warp w takes rows f = w, w + 32, ..., its lanes read a Gamma row contiguously and reduce by a
// fixed butterfly
__global__ void __launch_bounds__(kMgGroups * kD) k_bwd_sums_gb(int din, int k, int R, const bf16* dZ, float* S,
                                                                const float* theta, size_t ogam, float* Gb) {
  __shared__ float ss[kD];
  __shared__ float part[kMgGroups][kD];
  const int cand = blockIdx.x, o = threadIdx.x % kD, grp = threadIdx.x / kD;
  {
    const int share = (k + kMgGroups - 1) / kMgGroups;
    const int r0 = min(k, grp * share), r1 = min(k, r0 + share);
    const bf16* x = dZ + (size_t)cand * R * kD + o;
    float sum = 0.f;
    int r = r0;
    for (; r + 8 <= r1; r += 8) {
      float t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = __bfloat162float(x[(size_t)(r + u) * kD]);
#pragma unroll
      for (int u = 0; u < 8; ++u) sum += t[u];
    }
    for (; r < r1; ++r) sum += __bfloat162float(x[(size_t)r * kD]);
    part[grp][o] = sum;
  }
  __syncthreads();
  if (grp == 0) {
    float m = part[0][o];
#pragma unroll
    for (int g = 1; g < kMgGroups; ++g) m += part[g][o];
    ss[o] = m;
    S[(size_t)cand * kD + o] = m;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kMgGroups * kD / 32;  // warps of the block
  const float* gam = theta + ogam;
  for (int f0 = warp; f0 < din; f0 += 4 * NW) {  // four rows in flight
    float gv[4][kD / 32];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int i = 0; i < kD / 32; ++i)
        gv[q][i] = f0 + q * NW < din ? gam[(size_t)(f0 + q * NW) * kD + lane + 32 * i] : 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float acc = 0.f;
#pragma unroll
      for (int i = 0; i < kD / 32; ++i) acc += ss[lane + 32 * i] * gv[q][i];
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, d);
      if (lane == 0 && f0 + q * NW < din) Gb[(size_t)cand * din + f0 + q * NW] = acc / (float)k;
    }
  }
}

// embedding gradient: dE[v][f] = sum_cand dZ0[cand*R + col_cand[v]][f]; db0[f] = sum_cand S0[cand][f]
// (with perm, candidate c of the batch is sample perm[step[0] + c] of cols). Block v - vbase (256
// threads = kDembGroups groups of kD0 features): group g sums the candidates of its contiguous
// share in order, eight loads in flight, then the groups' sums are added in group order.
constexpr int kDembGroups = 256 / kD0;
__global__ void __launch_bounds__(256) k_demb(int n, int B, int R, const int16_t* cols, const int32_t* perm,
                                              const int32_t* step, const bf16* dZ0, const float* S0, float* grad,
                                              size_t oE, size_t ob0, int vbase) {
  __shared__ float ps[kDembGroups][kD0];
  const int v = vbase + (int)blockIdx.x, f = threadIdx.x % kD0, grp = threadIdx.x / kD0;
  const int share = (B + kDembGroups - 1) / kDembGroups;
  const int c0 = min(B, grp * share), c1 = min(B, c0 + share);
  auto row = [&](int c) -> size_t { return (size_t)(perm ? perm[step[0] + c] : c) * n; };
  float s = 0.f;
  if (v < n) {
    int c = c0;
    for (; c + 8 <= c1; c += 8) {  // eight candidates' colour and gradient loads in flight
      int q[8];
      float z[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) q[u] = cols[row(c + u) + v];
#pragma unroll
      for (int u = 0; u < 8; ++u) z[u] = __bfloat162float(dZ0[((size_t)(c + u) * R + q[u]) * kD0 + f]);
#pragma unroll
      for (int u = 0; u < 8; ++u) s += z[u];
    }
    for (; c < c1; ++c) {
      const int q = cols[row(c) + v];
      s += __bfloat162float(dZ0[((size_t)c * R + q) * kD0 + f]);
    }
  } else {
    for (int c = c0; c < c1; ++c) s += S0[(size_t)c * kD0 + f];
  }
  ps[grp][f] = s;
  __syncthreads();
  if (grp == 0) {
    float t = ps[0][f];
#pragma unroll
    for (int g = 1; g < kDembGroups; ++g) t += ps[g][f];
    grad[(v < n ? oE + (size_t)v * kD0 : ob0) + f] = t;
  }
}

// Adam's bias corrections of step t + 1 (t = step[1]) in double, by one thread: 1 - 0.9^(t+1) and
// sqrt(1 - 0.999^(t+1)), rounded to float
__global__ void k_adam_bias(const int32_t* step, float* bc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double t = (double)(step[1] + 1);
    bc[0] = (float)(1.0 - pow(0.9, t));
    bc[1] = (float)sqrt(1.0 - pow(0.999, t));
  }
}

// Adam step t + 1 (t = step[1]) of every parameter with the bias corrections bc of k_adam_bias,
// then the parameter's bf16 operand copies (those k_convert writes); thread 0 then advances the
// batch offset step[0] by b and Adam's counter step[1] (nothing of this step reads them any more).
__global__ void __launch_bounds__(256) k_adam_convert(int64_t np, float* th, float* m, float* v, const float* g,
                                                      float lr, const float* bc, ConvArgs a, int32_t* step, int b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && step) {  // the step's end: the next batch starts b samples later, Adam's counter advances
    step[0] += b;
    step[1] += 1;
  }
  if (i >= np) return;
  const float bc1 = bc[0], sbc2 = bc[1];  // the same two words for every thread (L1 broadcast)
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float denom = sqrtf(vi) / sbc2 + 1e-8f;
  const float tn = th[i] - (lr / bc1) * mi / denom;
  th[i] = tn;
  const int64_t nE = (int64_t)a.n * kD0;
  if (i >= (int64_t)a.oE && i < (int64_t)a.oE + nE) {
    a.E16[i - a.oE] = __float2bfloat16_rn(tn);
    return;
  }
  for (int l = 1; l <= kNL; ++l) {
    const int din = l == 1 ? kD0 : kD;
    const int64_t sz = (int64_t)din * kD;
    int64_t r = i - (int64_t)a.olam[l];
    if (r >= 0 && r < sz) {
      const int f = (int)(r / kD), o = (int)(r % kD);
      const bf16 hi = __float2bfloat16_rn(tn);
      const bf16 lo = __float2bfloat16_rn(tn - __bfloat162float(hi));
      a.Lam[l][r] = hi;
      a.Lamlo[l][r] = lo;
      a.LamT[l][(size_t)o * din + f] = hi;
      a.LamTlo[l][(size_t)o * din + f] = lo;
      return;
    }
    r = i - (int64_t)a.ogam[l];
    if (r >= 0 && r < sz) {
      const int f = (int)(r / kD), o = (int)(r % kD);
      const bf16 hi = __float2bfloat16_rn(tn);
      a.GamT[l][(size_t)o * din + f] = hi;
      a.GamTlo[l][(size_t)o * din + f] = __float2bfloat16_rn(tn - __bfloat162float(hi));
      return;
    }
  }
}


__global__ void k_init_params(int64_t np, uint64_t seed, float* th, const float* bound_of, const int64_t* seg_end, int nseg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  int s = 0;
  while (s < nseg - 1 && i >= seg_end[s]) ++s;
  const U4 r = rng(seed, (uint32_t)i, 0u, 0u, kTagNnInit);
  const float u = (float)(r.x >> 8) * (1.0f / 16777216.0f);
  th[i] = (2.f * u - 1.f) * bound_of[s];
}

// ---- training data: standardised targets, epoch permutation, batch gather ----------------------
__global__ void k_standardise(int p, const int64_t* f, float* y) {
  __shared__ double s1[256], s2[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) a += (double)f[i];
  s1[threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += s1[i];
    s1[0] = t / p;
  }
  __syncthreads();
  const double mean = s1[0];
  double b = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) b += ((double)f[i] - mean) * ((double)f[i] - mean);
  s2[threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += s2[i];
    double sd = sqrt(t / p);
    if (!(sd > 1e-12)) sd = 1.0;
    s2[0] = sd;
  }
  __syncthreads();
  const double sd = s2[0];
  for (int i = threadIdx.x; i < p; i += blockDim.x) y[i] = (float)(((double)f[i] - mean) / sd);
}

// one CTA: sort of the 64-bit keys (Philox(i, epoch, gen, BATCH).r0 << 32 | i); p <= 8192
__global__ void k_epoch_perm(int p, uint64_t seed, uint32_t epoch, uint32_t gen, int32_t* perm) {
  extern __shared__ __align__(16) uint64_t keys[];
  int mp = 1;
  while (mp < p) mp <<= 1;
  for (int i = threadIdx.x; i < mp; i += blockDim.x) {
    if (i < p) {
      const U4 r = rng(seed, (uint32_t)i, epoch, gen, kTagBatch);
      keys[i] = ((uint64_t)r.x << 32) | (uint32_t)i;
    } else {
      keys[i] = ~0ull;
    }
  }
  __syncthreads();
  for (int size = 2; size <= mp; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = threadIdx.x; q < mp; q += blockDim.x) {
        const int r = q ^ stride;
        if (r > q) {
          const bool up = (q & size) == 0;
          const uint64_t x = keys[q], y = keys[r];
          if ((x > y) == up) { keys[q] = y; keys[r] = x; }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < p; i += blockDim.x) perm[i] = (int32_t)(keys[i] & 0xFFFFFFFFu);
}


// ------------------------------------------------------------------------------------------------
// host plumbing
// ------------------------------------------------------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                              const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
  }
  return fn;
}

namespace tc {
dlm_status make_map_bf16(dlm_ctx* ctx, CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                         uint32_t box_rows) {
  EncodeFn fn = encode_fn();
  if (!fn) return fail(ctx, DLM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  if (((uintptr_t)base & 15) || (ld * 2) % 16) return fail(ctx, DLM_EINVAL, "tensor map: misaligned operand");
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, DLM_ECUDA, "cuTensorMapEncodeTiled failed");
  return DLM_OK;
}
}  // namespace tc

// C[M][N] = (A + A2)[M][K] . (B + B2)[N][K]^T through the tcgen05 kernel, A2 / B2 the lo parts
// of split operands (or null); kc = 64-wide K chunks per CTA (split-K along grid z)
// ST = 0: two pipeline stages (split operands) or four; ST > 0: that many (one keeps the shared
// memory of a 128 x 64 tile at about 50 KB)
// training batches of at least this many class rows (100 samples at k > 64) run their GEMMs as
// 128 x 256 tiles with two pipeline stages, as the scoring pass does
constexpr int kWideRows = 12288;
// below that, the training GEMMs run as 128 x 128 tiles with one pipeline stage: one tile per CTA
// for a batch of 100 samples at k <= 64 (100 CTAs), where 128 x 64 tiles give some CTAs two tiles
// in sequence; about 66 KB of shared memory each, so that the CTAs also find room beside the
// distance kernel that runs at the same time in a memetic generation
constexpr int kTrainBN = 128;

template <int BN, int ST = 0, class Epi>
static dlm_status gemm(dlm_ctx* ctx, const bf16* A, const bf16* A2, int M, int K, int lda, const bf16* B, const bf16* B2,
                       int N, int ldb, int kc, Epi epi) {
  constexpr int S2 = ST ? ST : 2, S4 = ST ? ST : 4;
  if (M <= 0) return DLM_OK;
  if (K % tc::BK || N % BN) return fail(ctx, DLM_EINVAL, "gemm: K must be a multiple of 64 and N of the tile");
  CUtensorMap ma, ma2, mb, mb2;
  DLM_TRY(tc::make_map_bf16(ctx, &ma, A, (uint64_t)M, (uint64_t)K, (uint64_t)lda, tc::BM));
  DLM_TRY(tc::make_map_bf16(ctx, &mb, B, (uint64_t)N, (uint64_t)K, (uint64_t)ldb, BN));
  if (A2) DLM_TRY(tc::make_map_bf16(ctx, &ma2, A2, (uint64_t)M, (uint64_t)K, (uint64_t)lda, tc::BM));
  else ma2 = ma;
  if (B2) DLM_TRY(tc::make_map_bf16(ctx, &mb2, B2, (uint64_t)N, (uint64_t)K, (uint64_t)ldb, BN));
  else mb2 = mb;
  const int nchunks = K / tc::BK;
  if (kc <= 0) kc = nchunks;
  tc::GemmShape sh{M, N, K, kc};
  // persistent: one CTA per SM (TMEM holds two BN-column accumulators), looping over the tiles
  const int tiles = ((M + tc::BM - 1) / tc::BM) * (N / BN) * ((nchunks + kc - 1) / kc);
  dim3 grid(std::min(tiles, ctx->num_sms));
  auto launch = [&](auto kfn, size_t smem, PerDeviceOnce& attr) -> dlm_status {
    if (attr.need(ctx->device)) {
      DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr.mark(ctx->device);
    }
    dlm_ctx::GemmRec rec{nullptr, nullptr, 0.0};
    if (ctx->gemm_prof && cudaEventCreate(&rec.a) == cudaSuccess && cudaEventCreate(&rec.b) == cudaSuccess) {
      // executed tensor-core work: one pass of 2 M N K per MMA (hi.hi, plus hi.lo / lo.hi for split operands)
      rec.flops = 2.0 * M * N * K * (1 + (A2 ? 1 : 0) + (B2 ? 1 : 0));
      cudaEventRecord(rec.a, ctx->stream);
    }
    kfn<<<grid, tc::kThreads, smem, ctx->stream>>>(ma, ma2, mb, mb2, sh, epi, ctx->d_status);
    if (rec.b) {
      cudaEventRecord(rec.b, ctx->stream);
      ctx->gemm_recs.push_back(rec);
    }
    return launch_check(ctx, "gemm_kernel");
  };
  if (A2 && B2) {
    static PerDeviceOnce attr;
    return launch(tc::gemm_kernel<BN, S2, 2, 2, Epi>, tc::gemm_smem_bytes<BN, S2, 2, 2>(), attr);
  }
  if (A2) {
    static PerDeviceOnce attr;
    return launch(tc::gemm_kernel<BN, S2, 2, 1, Epi>, tc::gemm_smem_bytes<BN, S2, 2, 1>(), attr);
  }
  if (B2) {
    static PerDeviceOnce attr;
    return launch(tc::gemm_kernel<BN, S2, 1, 2, Epi>, tc::gemm_smem_bytes<BN, S2, 1, 2>(), attr);
  }
  static PerDeviceOnce attr;
  return launch(tc::gemm_kernel<BN, S4, 1, 1, Epi>, tc::gemm_smem_bytes<BN, S4, 1, 1>(), attr);
}

template <typename T>
static dlm_status dalloc(dlm_ctx* ctx, T** p, size_t count) {
  if (cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DLM_ENOMEM, "scorer: device allocation failed");
  }
  return DLM_OK;
}

static ConvArgs conv_args(const dlm_scorer* s, int64_t* tot_out) {
  ConvArgs a;
  a.theta = s->theta;
  a.n = s->n;
  a.oE = s->oE;
  a.E16 = s->E16;
  int64_t tot = (int64_t)s->n * kD0;
  for (int l = 1; l <= kNL; ++l) {
    a.olam[l] = s->olam[l];
    a.ogam[l] = s->ogam[l];
    a.LamT[l] = s->LamT[l];
    a.Lam[l] = s->Lam[l];
    a.LamTlo[l] = s->LamTlo[l];
    a.Lamlo[l] = s->Lamlo[l];
    a.GamT[l] = s->GamT[l];
    a.GamTlo[l] = s->GamTlo[l];
    tot += 2 * (int64_t)din_of(l) * kD;
  }
  if (tot_out) *tot_out = tot;
  return a;
}

static dlm_status convert_params(dlm_ctx* ctx, dlm_scorer* s) {
  int64_t tot = 0;
  const ConvArgs a = conv_args(s, &tot);
  k_convert<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(a);
  return launch_check(ctx, "k_convert");
}

static size_t pool_smem(int n) {
  return ((n + 15) & ~15) + ((n + 7) & ~7) * 2 + (3 * kRMax + 1) * 4 + (kPoolWarps + 1) * 64 * 4 + 64;
}

// forward over c candidates with the given buffers; train = a training batch: keep every
// activation (and H3), candidate b being sample perm[step[0] + b] of cols when perm is given
static dlm_status forward(dlm_ctx* ctx, dlm_scorer* s, const int16_t* cols, int c, int R, float* out, bf16** H,
                          bf16** Hlo, bf16** Mb, bf16** Mblo, float** Mf, float** G, float* rowdot, bool train,
                          const int32_t* perm = nullptr, const int32_t* step = nullptr) {
  const int rows = c * R;
  const size_t psm = pool_smem(s->n);  // < 10 KB for n <= 2048
  const int pgrid = std::min(c, ctx->num_sms * 4);
  // per-candidate term rho(H_{l-1}) Gamma_l + beta_l: on the tensor cores for a scoring chunk,
  // both operands split into bf16 hi + lo (three MMA passes, about 16 mantissa bits each); in
  // FP32 on CUDA cores for a small batch, for a training batch fused into the kernel that forms
  // the class means (k_pool for layer 1, k_mean_gterm for layers 2 and 3)
  k_pool<<<pgrid, 32 * kPoolWarps, psm, ctx->stream>>>(s->n, s->k, R, cols, c, perm, step, s->theta + s->oE, s->theta + s->ob0, H[0],
                                           Hlo ? Hlo[0] : nullptr, Mf[0], Mb[0], Mblo[0],
                                           s->theta + s->ogam[1], s->theta + s->ob[1], train ? G[1] : nullptr,
                                           ctx->d_status);
  DLM_TRY(launch_check(ctx, "k_pool"));
  for (int l = 1; l <= kNL; ++l) {
    const int din = din_of(l);
    if (!train) {
      if (c >= 1024) {
        DLM_TRY(gemm<256>(ctx, Mb[l - 1], Mblo[l - 1], c, din, din, s->GamT[l], s->GamTlo[l], kD, din, 0,
                          EpiBias{G[l], c, s->theta + s->ob[l]}));
      } else {
        k_gterm<<<c, 256, 0, ctx->stream>>>(c, din, Mf[l - 1], s->theta, s->ogam[l], s->ob[l], G[l]);
        DLM_TRY(launch_check(ctx, "k_gterm"));
      }
    }
    const bool last = l == kNL;
    // a training batch of a few thousand rows runs its layer GEMMs as 128 x kTrainBN tiles with
    // one pipeline stage (twice the CTAs of a 128 x 256 tile, and a third of its shared memory);
    // from kWideRows rows on (k > 64) 128 x 256 tiles fill the SMs
    const bool narrow = train && rows < kWideRows;
    EpiLayer e{(last && !train) ? nullptr : H[l], Hlo ? Hlo[l] : nullptr, rows, s->k, R, G[l],
               last ? s->theta + s->owh : nullptr, last ? rowdot : nullptr, 0.f, narrow ? kTrainBN / 2 : 128, 0};
    if (narrow)
      DLM_TRY((gemm<kTrainBN, 1>(ctx, H[l - 1], Hlo ? Hlo[l - 1] : nullptr, rows, din, din, s->LamT[l], s->LamTlo[l], kD, din,
                          0, e)));
    else
      DLM_TRY(gemm<256>(ctx, H[l - 1], Hlo ? Hlo[l - 1] : nullptr, rows, din, din, s->LamT[l], s->LamTlo[l], kD, din, 0,
                        e));
    if (train && !last) {
      k_mean_gterm<<<c, kMgGroups * kD, 0, ctx->stream>>>(H[l], Hlo ? Hlo[l] : nullptr, s->k, R, Mf[l], Mb[l], Mblo[l],
                                              s->theta + s->ogam[l + 1], s->theta + s->ob[l + 1], G[l + 1]);
      DLM_TRY(launch_check(ctx, "k_mean_gterm"));
    } else if (!last) {
      k_segment_reduce<<<c, kD, 0, ctx->stream>>>(H[l], Hlo ? Hlo[l] : nullptr, kD, s->k, R, 1.f / s->k, Mf[l], Mb[l],
                                                  Mblo[l]);
      DLM_TRY(launch_check(ctx, "k_segment_reduce"));
    }
  }
  if (train) return DLM_OK;  // the training batch's class means of H3 and output: k_head_fwd
  k_head_out<<<(c + kHeadOutWarps - 1) / kHeadOutWarps, 32 * kHeadOutWarps, 0, ctx->stream>>>(c, s->k, R, rowdot,
                                                                                             kD / 128, s->theta, s->obh,
                                                                                             out);
  return launch_check(ctx, "k_head_out");
}

// forward + backward of one batch; gradient into s->grad (overwritten), predictions into outb.
// With perm, candidate b of the batch is sample perm[step[0] + b] of cols (target y of that
// sample); otherwise cols and y hold the batch itself.
static dlm_status loss_grad(dlm_ctx* ctx, dlm_scorer* s, const int16_t* cols, const float* y, int B,
                            const int32_t* perm = nullptr, const int32_t* step = nullptr) {
  DLM_TRY(forward(ctx, s, cols, B, s->R, s->outb, s->Hb, s->Hblo, s->Mbb, s->Mbblo, s->Mfb, s->Gbf, s->rowdotb, true, perm,
                  step));
  const int rows = B * s->R;
  const int parts = rows < kWideRows ? kD / (kTrainBN / 2) : kD / 128;  // head-dot slices of the layer-3 GEMM
  k_head_fwd<<<(unsigned)B, kD, 0, ctx->stream>>>(B, s->k, s->R, s->Hb[kNL], s->Hblo[kNL], s->Mfb[kNL], s->Mbb[kNL],
                                                  s->Mbblo[kNL], s->rowdotb, parts, s->theta, s->obh, y, perm, step,
                                                  s->outb, s->dout, s->sqerr);
  DLM_TRY(launch_check(ctx, "k_head_fwd"));
  cudaStream_t main_stream = ctx->stream;
  // side branch: the head's gradient and the loss
  DLM_CUDA(ctx, cudaEventRecord(s->ev_fork[4], main_stream));
  DLM_CUDA(ctx, cudaStreamWaitEvent(s->side[0], s->ev_fork[4], 0));
  k_head_grad<<<1, kD, 0, s->side[0]>>>(B, s->dout, s->Mfb[kNL], s->grad, s->owh, s->obh, s->sqerr, s->lossd);
  DLM_TRY(launch_check(ctx, "k_head_grad"));
  DLM_CUDA(ctx, cudaEventRecord(s->ev_join[4], s->side[0]));
  k_head_bwd<<<(unsigned)((rows + kHeadRows - 1) / kHeadRows), kD, 0, ctx->stream>>>(s->k, s->R, rows, s->dout, s->theta,
                                                                                     s->owh, s->Hb[kNL], s->dZ[kNL]);
  DLM_TRY(launch_check(ctx, "k_head_bwd"));
  for (int l = kNL; l >= 1; --l) {
    const int din = din_of(l);
    // main chain: the column sums S_l of dZ_l per candidate (valid rows are the only nonzero ones)
    // and the per-candidate term Gb of dH_{l-1} (from S_l and Gamma_l), in one launch
    k_bwd_sums_gb<<<(unsigned)B, kMgGroups * kD, 0, ctx->stream>>>(din, s->k, s->R, s->dZ[l], s->S[l], s->theta, s->ogam[l], s->Gb);
    DLM_TRY(launch_check(ctx, "k_bwd_sums_gb"));
    // side branch: the transposes of dZ_l and H_{l-1} (hi and lo), dLambda_l = H_{l-1}^T dZ_l
    // (split-K over rows, fixed-order reduction; the tile width does not change any sum), then the
    // split sums into dLambda_l, dGamma_l and dbeta_l. It reads dZ_l, S_l and this step's
    // activations, and writes only layer l's gradient blocks, transposes and partial sums.
    const int ty = (rows + 31) / 32;
    const int nchunks = rows / tc::BK, kc = 4, splits = (nchunks + kc - 1) / kc;
    const int64_t cnt = (int64_t)din * kD;
    DLM_CUDA(ctx, cudaEventRecord(s->ev_fork[l], main_stream));
    DLM_CUDA(ctx, cudaStreamWaitEvent(s->side[l], s->ev_fork[l], 0));
    ctx->stream = s->side[l];
    {
      k_bwd_prep<<<ty * (kD / 32) + 2 * ty * (din / 32), 256, 0, ctx->stream>>>(
          0, s->k, s->R, rows, din, s->dZ[l], nullptr, s->dZT[l], s->Hb[l - 1], s->Hblo[l - 1], s->HT[l - 1],
          s->HTlo[l - 1]);
      dlm_status st = launch_check(ctx, "k_bwd_prep");
      const EpiPartial ep{s->part[l], kD, din, (size_t)din * kD};
      if (st == DLM_OK)
        st = rows < kWideRows ? gemm<kTrainBN, 1>(ctx, s->HT[l - 1], s->HTlo[l - 1], din, rows, rows, s->dZT[l], nullptr, kD,
                                            rows, kc, ep)
                              : gemm<256>(ctx, s->HT[l - 1], s->HTlo[l - 1], din, rows, rows, s->dZT[l], nullptr, kD,
                                          rows, kc, ep);
      if (st == DLM_OK) {
        k_bwd_grads<<<(unsigned)((cnt + 255) / 256 + din), kD, 0, ctx->stream>>>(
            B, din, cnt, splits, s->part[l], s->grad + s->olam[l], s->Mfb[l - 1], s->S[l], s->grad, s->ogam[l],
            s->ob[l]);
        st = launch_check(ctx, "k_bwd_grads");
      }
      if (st == DLM_OK) st = cuda_check(ctx, cudaEventRecord(s->ev_join[l], s->side[l]), "event");
      ctx->stream = main_stream;
      DLM_TRY(st);
    }
    // dZ_{l-1} = (dZ_l Lambda_l^T + Gb) * LeakyReLU'(H_{l-1})
    EpiBwd e{s->dZ[l - 1], din, rows, s->k, s->R, s->Gb, s->Hb[l - 1]};
    if (rows < kWideRows && din % kTrainBN == 0)
      DLM_TRY((gemm<kTrainBN, 1>(ctx, s->dZ[l], nullptr, rows, kD, kD, s->Lam[l], s->Lamlo[l], din, kD, 0, e)));
    else if (rows < kWideRows || din % 256)
      DLM_TRY((gemm<64, 1>(ctx, s->dZ[l], nullptr, rows, kD, kD, s->Lam[l], s->Lamlo[l], din, kD, 0, e)));
    else
      DLM_TRY((gemm<256>(ctx, s->dZ[l], nullptr, rows, kD, kD, s->Lam[l], s->Lamlo[l], din, kD, 0, e)));
  }
  // side branch: the embedding bias gradient db0 = sum over candidates of the column sums of dZ0
  DLM_CUDA(ctx, cudaEventRecord(s->ev_fork[5], main_stream));
  DLM_CUDA(ctx, cudaStreamWaitEvent(s->side[0], s->ev_fork[5], 0));
  k_segment_reduce<<<B, kD0, 0, s->side[0]>>>(s->dZ[0], nullptr, kD0, s->k, s->R, 1.f, s->S[0], nullptr, nullptr);
  k_demb<<<1, 256, 0, s->side[0]>>>(s->n, B, s->R, cols, perm, step, s->dZ[0], s->S[0], s->grad, s->oE, s->ob0, s->n);
  DLM_TRY(launch_check(ctx, "k_demb"));
  DLM_CUDA(ctx, cudaEventRecord(s->ev_join[5], s->side[0]));
  // the embedding gradient dE on the main chain
  k_demb<<<(unsigned)s->n, 256, 0, ctx->stream>>>(s->n, B, s->R, cols, perm, step, s->dZ[0], s->S[0], s->grad, s->oE,
                                                  s->ob0, 0);
  DLM_TRY(launch_check(ctx, "k_demb"));
  for (int l = 1; l < 6; ++l) DLM_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, s->ev_join[l], 0));
  return DLM_OK;
}

static dlm_status ensure_train_buffers(dlm_ctx* ctx, dlm_scorer* s, int B) {
  if (B <= s->capb) return DLM_OK;
  if (B > 256) return fail(ctx, DLM_EUNSUPPORTED, "scorer: training batches are limited to 256 samples");
  const int cb = 256, rows = cb * s->R, cpad = cb;
  for (int l = 0; l <= kNL; ++l) {
    const int w = l == 0 ? kD0 : kD;
    DLM_TRY(dalloc(ctx, &s->Hb[l], (size_t)rows * w));
    DLM_TRY(dalloc(ctx, &s->Hblo[l], (size_t)rows * w));
    DLM_TRY(dalloc(ctx, &s->HT[l], (size_t)rows * w));
    DLM_TRY(dalloc(ctx, &s->HTlo[l], (size_t)rows * w));
    DLM_TRY(dalloc(ctx, &s->Mbb[l], (size_t)cpad * w));
    DLM_TRY(dalloc(ctx, &s->Mbblo[l], (size_t)cpad * w));
    DLM_TRY(dalloc(ctx, &s->Mfb[l], (size_t)cb * w));
    DLM_TRY(dalloc(ctx, &s->Gbf[l], (size_t)cb * kD));
    DLM_TRY(dalloc(ctx, &s->dZ[l], (size_t)rows * w));
    DLM_TRY(dalloc(ctx, &s->dZT[l], (size_t)rows * w));
    DLM_TRY(dalloc(ctx, &s->S[l], (size_t)cb * w));
  }
  DLM_TRY(dalloc(ctx, &s->Gb, (size_t)cb * kD));
  for (int l = 1; l <= kNL; ++l) DLM_TRY(dalloc(ctx, &s->part[l], (size_t)(rows / tc::BK / 4 + 1) * kD * kD));
  if (!s->side[0]) {
    for (int l = 0; l <= kNL; ++l)
      if (cudaStreamCreateWithFlags(&s->side[l], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, DLM_ECUDA, "scorer: side stream");
      }
    for (int l = 0; l < 6; ++l)
      if (cudaEventCreateWithFlags(&s->ev_fork[l], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&s->ev_join[l], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, DLM_ECUDA, "scorer: events");
      }
    if (cudaEventCreateWithFlags(&s->ev_bc_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_bc_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, DLM_ECUDA, "scorer: events");
    }
    DLM_TRY(dalloc(ctx, &s->d_bc, 2));
  }
  DLM_TRY(dalloc(ctx, &s->sqerr, (size_t)cb));
  DLM_TRY(dalloc(ctx, &s->rowdotb, (size_t)rows * (kD / 32)));
  DLM_TRY(dalloc(ctx, &s->outb, (size_t)cb));
  DLM_TRY(dalloc(ctx, &s->dout, (size_t)cb));
  DLM_TRY(dalloc(ctx, &s->lossd, 1));
  s->capb = cb;
  return DLM_OK;
}

static dlm_status ensure_fwd_buffers(dlm_ctx* ctx, dlm_scorer* s) {
  if (s->cap) return DLM_OK;
  const int cap = 8192 * 64 / s->Rs, rows = cap * s->Rs;  // about the same bytes for every k
  for (int l = 0; l <= kNL; ++l) {
    const int w = l == 0 ? kD0 : kD;
    if (l < kNL) DLM_TRY(dalloc(ctx, &s->H[l], (size_t)rows * w));
    if (l < kNL && s->split_act) DLM_TRY(dalloc(ctx, &s->Hlo[l], (size_t)rows * w));
    DLM_TRY(dalloc(ctx, &s->Mb[l], (size_t)cap * w));
    DLM_TRY(dalloc(ctx, &s->Mblo[l], (size_t)cap * w));
    DLM_TRY(dalloc(ctx, &s->Mf[l], (size_t)cap * w));
    DLM_TRY(dalloc(ctx, &s->G[l], (size_t)cap * kD));
  }
  DLM_TRY(dalloc(ctx, &s->rowdot, (size_t)rows * (kD / 128)));
  s->cap = cap;
  return DLM_OK;
}

// one Adam step of batch size B (batch offset and step counter on the device): the batch is read
// through the epoch permutation, the Adam update writes the bf16 operand copies too
static dlm_status train_step(dlm_ctx* ctx, dlm_scorer* s, const int16_t* cols, int B, int b, float lr) {
  // the bias corrections (a short double-precision chain) on the side branch, off the critical path
  DLM_CUDA(ctx, cudaEventRecord(s->ev_bc_fork, ctx->stream));
  DLM_CUDA(ctx, cudaStreamWaitEvent(s->side[0], s->ev_bc_fork, 0));
  k_adam_bias<<<1, 32, 0, s->side[0]>>>(s->d_step, s->d_bc);
  DLM_TRY(launch_check(ctx, "k_adam_bias"));
  DLM_CUDA(ctx, cudaEventRecord(s->ev_bc_join, s->side[0]));
  DLM_TRY(loss_grad(ctx, s, cols, s->y, B, s->perm, s->d_step));
  DLM_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, s->ev_bc_join, 0));
  k_adam_convert<<<(unsigned)((s->np + 255) / 256), 256, 0, ctx->stream>>>(s->np, s->theta, s->am, s->av, s->grad, lr,
                                                                          s->d_bc, conv_args(s, nullptr), s->d_step, b);
  return launch_check(ctx, "k_adam_convert");
}

// the training step of batch size B as an instantiated CUDA graph (captured on a private stream,
// replayed on the context's stream); cached for the last two (B, b, lr, cols) keys
static dlm_status step_graph(dlm_ctx* ctx, dlm_scorer* s, const int16_t* cols, int B, int b, float lr,
                             cudaGraphExec_t* exec) {
  for (auto& g : s->sg)
    if (g.exec && g.B == B && g.b == b && g.lr == lr && g.cols == cols) { *exec = g.exec; return DLM_OK; }
  if (!s->cap_stream) DLM_CUDA(ctx, cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = ctx->stream;
  const bool prof = ctx->gemm_prof;
  ctx->gemm_prof = false;  // no event records inside the graph
  ctx->stream = s->cap_stream;
  cudaGraph_t graph = nullptr;
  dlm_status st = cuda_check(ctx, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal), "capture");
  if (st == DLM_OK) {
    st = train_step(ctx, s, cols, B, b, lr);
    const cudaError_t e = cudaStreamEndCapture(s->cap_stream, &graph);
    if (st == DLM_OK) st = cuda_check(ctx, e, "end capture");
  }
  ctx->stream = user;
  ctx->gemm_prof = prof;
  cudaGraphExec_t ge = nullptr;
  if (st == DLM_OK) st = cuda_check(ctx, cudaGraphInstantiate(&ge, graph, 0), "graph instantiate");
  if (graph) cudaGraphDestroy(graph);
  if (st != DLM_OK) return st;
  auto& slot = s->sg[s->sg_next];
  s->sg_next ^= 1;
  if (slot.exec) cudaGraphExecDestroy(slot.exec);
  slot.exec = ge;
  slot.B = B;
  slot.b = b;
  slot.lr = lr;
  slot.cols = cols;
  *exec = ge;
  return DLM_OK;
}

}  // namespace dlm

using namespace dlm;

extern "C" void dlm_scorer_destroy(dlm_scorer* s) {
  if (!s) return;
  for (auto& g : s->sg)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  for (int l = 0; l < 4; ++l) cudaFree(s->part[l]);
  for (int l = 0; l < 6; ++l) {
    if (s->ev_fork[l]) cudaEventDestroy(s->ev_fork[l]);
    if (s->ev_join[l]) cudaEventDestroy(s->ev_join[l]);
  }
  cudaFree(s->sqerr);
  for (auto st : s->side)
    if (st) cudaStreamDestroy(st);
  if (s->ev_bc_fork) cudaEventDestroy(s->ev_bc_fork);
  if (s->ev_bc_join) cudaEventDestroy(s->ev_bc_join);
  cudaFree(s->d_bc);
  cudaFree(s->d_step);
  cudaFree(s->theta); cudaFree(s->am); cudaFree(s->av); cudaFree(s->grad); cudaFree(s->E16);
  for (int l = 0; l <= kNL; ++l) {
    cudaFree(s->LamT[l]); cudaFree(s->Lam[l]); cudaFree(s->LamTlo[l]); cudaFree(s->Lamlo[l]);
    cudaFree(s->GamT[l]); cudaFree(s->GamTlo[l]); cudaFree(s->Mblo[l]); cudaFree(s->Mbblo[l]);
    cudaFree(s->H[l]); cudaFree(s->Hlo[l]); cudaFree(s->Mb[l]); cudaFree(s->Mf[l]); cudaFree(s->G[l]);
    cudaFree(s->Hb[l]); cudaFree(s->Hblo[l]); cudaFree(s->HT[l]); cudaFree(s->HTlo[l]); cudaFree(s->Mbb[l]); cudaFree(s->Mfb[l]); cudaFree(s->Gbf[l]);
    cudaFree(s->dZ[l]); cudaFree(s->dZT[l]); cudaFree(s->S[l]);
  }
  cudaFree(s->rowdot); cudaFree(s->Gb); cudaFree(s->rowdotb); cudaFree(s->outb); cudaFree(s->dout);
  cudaFree(s->lossd); cudaFree(s->y); cudaFree(s->perm);
  delete s;
}

extern "C" dlm_status dlm_scorer_create(dlm_ctx* ctx, int32_t n, int32_t k, uint64_t seed, dlm_scorer** out) {
  if (!ctx || !out) return fail(ctx, DLM_EINVAL, "scorer_create: null argument");
  *out = nullptr;
  if (n < 1 || n > 2048 || k < 1) return fail(ctx, DLM_EINVAL, "scorer_create: bad sizes");
  if (k > kRMax) return fail(ctx, DLM_EUNSUPPORTED, "scorer_create: k must be <= 256");
  dlm_scorer* s = new dlm_scorer();
  s->n = n;
  s->k = k;
  s->R = 64 * ((k + 63) / 64);
  s->Rs = k;
  size_t o = 0;
  s->oE = o; o += (size_t)n * kD0;
  s->ob0 = o; o += kD0;
  for (int l = 1; l <= kNL; ++l) {
    s->olam[l] = o; o += (size_t)din_of(l) * kD;
    s->ogam[l] = o; o += (size_t)din_of(l) * kD;
    s->ob[l] = o; o += kD;
  }
  s->owh = o; o += kD;
  s->obh = o; o += 1;
  s->np = (int64_t)o;
  dlm_status st = DLM_OK;
  auto A = [&](auto** p, size_t cnt) { if (st == DLM_OK) st = dalloc(ctx, p, cnt); };
  A(&s->theta, o); A(&s->am, o); A(&s->av, o); A(&s->grad, o); A(&s->E16, (size_t)n * kD0);
  for (int l = 1; l <= kNL; ++l) {
    A(&s->LamT[l], (size_t)din_of(l) * kD); A(&s->Lam[l], (size_t)din_of(l) * kD);
    A(&s->LamTlo[l], (size_t)din_of(l) * kD); A(&s->Lamlo[l], (size_t)din_of(l) * kD);
    A(&s->GamT[l], (size_t)din_of(l) * kD); A(&s->GamTlo[l], (size_t)din_of(l) * kD);
  }
  if (st != DLM_OK) { dlm_scorer_destroy(s); return st; }
  // uniform +-1/sqrt(fan_in) per parameter block (fan_in of E and b0: n)
  std::vector<float> bound;
  std::vector<int64_t> seg_end;
  auto seg = [&](size_t end, int fan) { seg_end.push_back((int64_t)end); bound.push_back(1.f / std::sqrt((float)fan)); };
  seg(s->ob0, n);
  seg(s->ob0 + kD0, n);
  for (int l = 1; l <= kNL; ++l) {
    seg(s->ogam[l], din_of(l));
    seg(s->ob[l], din_of(l));
    seg(s->ob[l] + kD, din_of(l));
  }
  seg(s->obh, kD);
  seg(o, kD);
  float* dbound = nullptr;
  int64_t* dseg = nullptr;
  void* ws = nullptr;
  st = ctx_workspace(ctx, bound.size() * 4 + 64 + seg_end.size() * 8, &ws);
  if (st == DLM_OK) {
    dbound = (float*)ws;
    dseg = (int64_t*)((uint8_t*)ws + ((bound.size() * 4 + 63) & ~(size_t)63));
    cudaMemcpyAsync(dbound, bound.data(), bound.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dseg, seg_end.data(), seg_end.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
    k_init_params<<<(unsigned)((o + 255) / 256), 256, 0, ctx->stream>>>((int64_t)o, seed, s->theta, dbound, dseg,
                                                                          (int)seg_end.size());
    st = launch_check(ctx, "k_init_params");
  }
  if (st == DLM_OK) st = cuda_check(ctx, cudaMemsetAsync(s->am, 0, o * 4, ctx->stream), "memset");
  if (st == DLM_OK) st = cuda_check(ctx, cudaMemsetAsync(s->av, 0, o * 4, ctx->stream), "memset");
  if (st == DLM_OK) st = convert_params(ctx, s);
  if (st == DLM_OK) st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sync");
  if (st != DLM_OK) { dlm_scorer_destroy(s); return st; }
  *out = s;
  return DLM_OK;
}

extern "C" int64_t dlm_scorer_nparams(const dlm_scorer* s) { return s ? s->np : 0; }

extern "C" dlm_status dlm_scorer_get_params(dlm_ctx* ctx, dlm_scorer* s, float* params) {
  if (!ctx || !s || !params) return fail(ctx, DLM_EINVAL, "scorer_get_params: null argument");
  DLM_CUDA(ctx, cudaMemcpyAsync(params, s->theta, (size_t)s->np * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  return DLM_OK;
}

extern "C" dlm_status dlm_scorer_set_params(dlm_ctx* ctx, dlm_scorer* s, const float* params) {
  if (!ctx || !s || !params) return fail(ctx, DLM_EINVAL, "scorer_set_params: null argument");
  DLM_CUDA(ctx, cudaMemcpyAsync(s->theta, params, (size_t)s->np * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  DLM_CUDA(ctx, cudaMemsetAsync(s->am, 0, (size_t)s->np * 4, ctx->stream));
  DLM_CUDA(ctx, cudaMemsetAsync(s->av, 0, (size_t)s->np * 4, ctx->stream));
  s->t = 0;
  return convert_params(ctx, s);
}

extern "C" dlm_status dlm_score_offspring(dlm_ctx* ctx, dlm_scorer* s, const int16_t* col, int32_t c, float* out) {
  if (!ctx || !s) return fail(ctx, DLM_EINVAL, "score_offspring: null argument");
  if (c < 0) return fail(ctx, DLM_EINVAL, "score_offspring: negative count");
  if (c == 0) return DLM_OK;
  if (!col || !out) return fail(ctx, DLM_EINVAL, "score_offspring: null pointer");
  DLM_TRY(ensure_fwd_buffers(ctx, s));
  for (int c0 = 0; c0 < c; c0 += s->cap) {
    const int cc = std::min(s->cap, c - c0);
    DLM_TRY(forward(ctx, s, col + (size_t)c0 * s->n, cc, s->Rs, out + c0, s->H, s->split_act ? s->Hlo : nullptr, s->Mb,
                    s->Mblo, s->Mf, s->G, s->rowdot, false));
  }
  return DLM_OK;
}

extern "C" dlm_status dlm_scorer_set_scoring_precision(dlm_ctx* ctx, dlm_scorer* s, int32_t split) {
  if (!ctx || !s || (split != 0 && split != 1)) return fail(ctx, DLM_EINVAL, "scorer_set_scoring_precision: bad argument");
  if (split == s->split_act) return DLM_OK;
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the buffers may be in use by queued work
  for (int l = 0; l <= kNL; ++l) {
    cudaFree(s->H[l]); cudaFree(s->Hlo[l]); cudaFree(s->Mb[l]); cudaFree(s->Mblo[l]); cudaFree(s->Mf[l]);
    cudaFree(s->G[l]);
    s->H[l] = s->Hlo[l] = s->Mb[l] = s->Mblo[l] = nullptr;
    s->Mf[l] = s->G[l] = nullptr;
  }
  cudaFree(s->rowdot);
  s->rowdot = nullptr;
  s->cap = 0;  // reallocated by the next scoring call
  s->split_act = split;
  return DLM_OK;
}

extern "C" dlm_status dlm_scorer_loss_grad(dlm_ctx* ctx, dlm_scorer* s, const int16_t* col, const float* y, int32_t B,
                                           float* grad, float* out, float* loss) {
  if (!ctx || !s || !col || !y) return fail(ctx, DLM_EINVAL, "scorer_loss_grad: null argument");
  if (B < 1) return fail(ctx, DLM_EINVAL, "scorer_loss_grad: empty batch");
  DLM_TRY(ensure_train_buffers(ctx, s, B));
  DLM_TRY(loss_grad(ctx, s, col, y, B));
  if (grad) DLM_CUDA(ctx, cudaMemcpyAsync(grad, s->grad, (size_t)s->np * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (out) DLM_CUDA(ctx, cudaMemcpyAsync(out, s->outb, (size_t)B * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (loss) DLM_CUDA(ctx, cudaMemcpyAsync(loss, s->lossd, 4, cudaMemcpyDeviceToDevice, ctx->stream));
  return DLM_OK;
}

extern "C" dlm_status dlm_scorer_train(dlm_ctx* ctx, dlm_scorer* s, const int16_t* cols, const int64_t* fvals, int32_t p,
                                       int32_t epochs, int32_t b, float lr, uint64_t seed, uint32_t generation) {
  if (!ctx || !s || !cols || !fvals) return fail(ctx, DLM_EINVAL, "scorer_train: null argument");
  if (p < 1 || p > 8192 || epochs < 0 || b < 1) return fail(ctx, DLM_EINVAL, "scorer_train: bad sizes (p <= 8192)");
  const int bb = std::min(b, p);
  DLM_TRY(ensure_train_buffers(ctx, s, bb));
  if (p > s->capp) {
    cudaFree(s->y);
    cudaFree(s->perm);
    s->y = nullptr;
    s->perm = nullptr;
    DLM_TRY(dalloc(ctx, &s->y, 8192));
    DLM_TRY(dalloc(ctx, &s->perm, 8192));
    s->capp = 8192;
  }
  k_standardise<<<1, 256, 0, ctx->stream>>>(p, fvals, s->y);
  DLM_TRY(launch_check(ctx, "k_standardise"));
  int mp = 1;
  while (mp < p) mp <<= 1;
  static PerDeviceOnce attr;
  if (attr.need(ctx->device)) {
    DLM_CUDA(ctx, cudaFuncSetAttribute(k_epoch_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8));
    attr.mark(ctx->device);
  }
  if (!s->d_step) {
    DLM_TRY(dalloc(ctx, &s->d_step, 2));
  }
  // the device counters start from the host mirror of Adam's step counter; the call waits for its
  // stream here (init lives on the host stack). In a memetic generation that wait ends with the
  // local search, so the training steps are submitted before the distance kernels: a learned
  // generation measured about 8 ms shorter than with the counters set by a kernel and no wait.
  int32_t init[2] = {0, (int32_t)s->t};
  DLM_CUDA(ctx, cudaMemcpyAsync(s->d_step, init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int ep = 0; ep < epochs; ++ep) {
    k_epoch_perm<<<1, 1024, (size_t)mp * 8, ctx->stream>>>(p, seed, (uint32_t)ep, generation, s->perm);
    DLM_TRY(launch_check(ctx, "k_epoch_perm"));
    DLM_CUDA(ctx, cudaMemsetAsync(s->d_step, 0, sizeof(int32_t), ctx->stream));  // batch offset 0
    for (int s0 = 0; s0 < p; s0 += b) {
      const int B = std::min(b, p - s0);
      if (!s->stepped) {  // the first step ever runs eagerly (it sets the kernels' attributes)
        DLM_TRY(train_step(ctx, s, cols, B, b, lr));
        s->stepped = true;
      } else {
        cudaGraphExec_t ge = nullptr;
        DLM_TRY(step_graph(ctx, s, cols, B, b, lr, &ge));
        DLM_CUDA(ctx, cudaGraphLaunch(ge, ctx->stream));
      }
      s->t += 1;
    }
  }
  return DLM_OK;
}

extern "C" dlm_status dlm_gemm_bf16(dlm_ctx* ctx, const void* A, const void* B, float* C, int32_t M, int32_t N, int32_t K) {
  if (!ctx || !A || !B || !C) return fail(ctx, DLM_EINVAL, "gemm_bf16: null argument");
  if (M < 1 || N < 64 || K < 64 || K % 64 || N % 64) return fail(ctx, DLM_EINVAL, "gemm_bf16: need K, N multiples of 64");
  if (N % 256 == 0)
    return gemm<256>(ctx, (const bf16*)A, nullptr, M, K, K, (const bf16*)B, nullptr, N, K, 0, EpiPlain{C, N, M, 1.f, nullptr});
  return gemm<64>(ctx, (const bf16*)A, nullptr, M, K, K, (const bf16*)B, nullptr, N, K, 0, EpiPlain{C, N, M, 1.f, nullptr});
}

extern "C" dlm_status dlm_gemm_profile(dlm_ctx* ctx, int32_t enable) {
  if (!ctx) return DLM_EINVAL;
  ctx->gemm_prof = enable != 0;
  return DLM_OK;
}

extern "C" dlm_status dlm_gemm_profile_read(dlm_ctx* ctx, double* ms, double* flops, int64_t* launches) {
  if (!ctx || !ms || !flops || !launches) return fail(ctx, DLM_EINVAL, "gemm_profile_read: null argument");
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double t = 0.0, f = 0.0;
  for (auto& r : ctx->gemm_recs) {
    float e = 0.f;
    if (cudaEventElapsedTime(&e, r.a, r.b) == cudaSuccess) t += e;
    f += r.flops;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  *ms = t;
  *flops = f;
  *launches = (int64_t)ctx->gemm_recs.size();
  ctx->gemm_recs.clear();
  return DLM_OK;
}

extern "C" int64_t dlm_scorer_state_bytes(const dlm_scorer* s) { return s ? 3 * s->np * 4 + 8 : 0; }

// theta, Adam m, Adam v (np float32 each) and the Adam step counter, to or from host memory
extern "C" dlm_status dlm_scorer_save(dlm_ctx* ctx, dlm_scorer* s, void* host) {
  if (!ctx || !s || !host) return fail(ctx, DLM_EINVAL, "scorer_save: null argument");
  uint8_t* h = (uint8_t*)host;
  const size_t b = (size_t)s->np * 4;
  DLM_CUDA(ctx, cudaMemcpyAsync(h, s->theta, b, cudaMemcpyDeviceToHost, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(h + b, s->am, b, cudaMemcpyDeviceToHost, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(h + 2 * b, s->av, b, cudaMemcpyDeviceToHost, ctx->stream));
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  memcpy(h + 3 * b, &s->t, 8);
  return DLM_OK;
}

extern "C" dlm_status dlm_scorer_load(dlm_ctx* ctx, dlm_scorer* s, const void* host) {
  if (!ctx || !s || !host) return fail(ctx, DLM_EINVAL, "scorer_load: null argument");
  const uint8_t* h = (const uint8_t*)host;
  const size_t b = (size_t)s->np * 4;
  int64_t t = 0;
  memcpy(&t, h + 3 * b, 8);
  if (t < 0) return fail(ctx, DLM_EINVAL, "scorer_load: negative Adam step counter");
  DLM_CUDA(ctx, cudaMemcpyAsync(s->theta, h, b, cudaMemcpyHostToDevice, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(s->am, h + b, b, cudaMemcpyHostToDevice, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(s->av, h + 2 * b, b, cudaMemcpyHostToDevice, ctx->stream));
  s->t = t;
  DLM_TRY(convert_params(ctx, s));
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return DLM_OK;
}
