// The paper-size colour-permutation invariant network with invariant batch normalisation
// (section "Deep neural network training": the layer equation, the colour average rho, the
// invariant batch normalisation, LeakyReLU_0.2, the mean over the k classes; section
// "Implementation and parameter setting": 9 hidden layers of 10|V| ... |V|//2 for k-COL, 4 of
// 5|V| ... |V|//2 for the WVCP), any depth and widths.
//
// Rows are (candidate, class) pairs, R = c k. Layer 0 sums the rows E[v] of each class (the
// classes' vertex lists come from a stable counting sort per candidate); layer l >= 1 is
// Z = H Lambda_l + rho(H) Gamma_l + beta_l with both products on the tcgen05 tensor cores; every
// layer then normalises each feature over the R rows (training: batch statistics, running
// estimates updated with momentum 0.1; evaluation: the running estimates), applies gamma, mu and
// LeakyReLU_0.2. The linear head is averaged over the classes. Operands enter the GEMMs as bf16
// hi + lo pairs by default (three MMA passes, about 16 mantissa bits) or as bf16 alone; feature
// statistics are accumulated in FP64, everything else in FP32. Widths are padded to multiples
// of 64 with zero columns.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tcgemm_launch.cuh"

using bf16 = __nv_bfloat16;

namespace dlm {
namespace dn {

constexpr float kEps = 1e-5f;
constexpr double kMomentum = 0.1;
constexpr float kSlope = 0.2f;
constexpr int kMaxLayers = 16;
constexpr int kMaxWidth = 16384;

__host__ __device__ inline int pad64(int x) { return 64 * ((x + 63) / 64); }

__device__ __forceinline__ void split_bf16(float x, bf16& hi, bf16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// stable counting sort of every candidate's vertices by colour: idx[cand][.] lists the vertices
// of class 0, then class 1, ..., each in increasing order; off[cand][c] is where class c starts
__global__ void k_sort(int c, int n, int k, const int16_t* cols, int32_t* idx, int32_t* off, int32_t* status) {
  __shared__ int cnt[4][257];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cand = blockIdx.x * 4 + w;
  if (cand >= c) return;
  int* ct = cnt[w];
  for (int q = lane; q <= k; q += 32) ct[q] = 0;
  __syncwarp();
  const int16_t* s = cols + (size_t)cand * n;
  for (int v = lane; v < n; v += 32) {
    int col = s[v];
    if (col < 0 || col >= k) { raise_status(status, DLM_EINVAL); col = 0; }
    atomicAdd(ct + col, 1);
  }
  __syncwarp();
  if (lane == 0) {
    int run = 0;
    for (int q = 0; q < k; ++q) {
      const int x = ct[q];
      ct[q] = run;
      off[(size_t)cand * (k + 1) + q] = run;
      run += x;
    }
    off[(size_t)cand * (k + 1) + k] = run;
  }
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
  for (int base = 0; base < n; base += 32) {
    const int v = base + lane;
    const bool act = v < n;
    const unsigned am = __ballot_sync(0xFFFFFFFFu, act);
    int col = act ? (int)s[v] : -1;
    col = (col < 0 || col >= k) ? 0 : col;
    if (act) {
      const unsigned grp = __match_any_sync(am, col);
      const int rank = __popc(grp & lt);
      idx[(size_t)cand * n + ct[col] + rank] = v;
      __syncwarp(am);
      if (rank == 0) ct[col] += __popc(grp);
    }
    __syncwarp();
  }
}

// Z0[row][j] = beta0[j] + sum of E[v][j] over the row's class (j < h0; 0 in the padding)
__global__ void k_embed(int R, int n, int k, int h0, int hp0, const float* E, const float* b0, const int32_t* idx,
                        const int32_t* off, float* Z) {
  const int row = blockIdx.x;
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= hp0) return;
  float s = 0.f;
  if (j < h0) {
    const int cand = row / k, cl = row - cand * k;
    const int32_t* o = off + (size_t)cand * (k + 1);
    const int32_t* ix = idx + (size_t)cand * n;
    s = b0[j];
    for (int t = o[cl]; t < o[cl + 1]; ++t) s += E[(size_t)ix[t] * h0 + j];
  }
  Z[(size_t)row * hp0 + j] = s;
}

struct EpiStore {  // out[row][col] = acc for row < M, col < Nv (ld elements a row)
  float* out;
  int ld, M, Nv;
  __device__ void tile(int, int) {}
  __device__ void operator()(int row, int col0, const float (&v)[16]) const {
    if (row >= M) return;
    float* o = out + (size_t)row * ld;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (col0 + i < Nv) o[col0 + i] = v[i];
  }
  __device__ void finish(int) const {}
};

// Z[row][j] += G[cand][j] + beta[j] (j < h); padding columns to 0
__global__ void k_add_term(int R, int k, int h, int hp, float* Z, const float* G, const float* beta) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)R * hp) return;
  const int row = (int)(t / hp), j = (int)(t % hp);
  Z[t] = j < h ? Z[t] + G[(size_t)(row / k) * hp + j] + beta[j] : 0.f;
}

// per-feature column sums over R rows in FP64: sum[j] = sum_rows f(X[row][j]) for j < h, where
// f is x (mode 0), (x - mean[j])^2 (mode 1)
__global__ void k_colsum(int R, int h, int hp, const float* X, const double* mean, int mode, double* out) {
  __shared__ double red[32][33];
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  const int ry = threadIdx.x >> 5;  // 32 row groups
  double s = 0.0;
  if (j < h) {
    const double m = mode ? mean[j] : 0.0;
    for (int row = ry; row < R; row += 32) {
      const double x = X[(size_t)row * hp + j];
      s += mode ? (x - m) * (x - m) : x;
    }
  }
  red[ry][threadIdx.x & 31] = s;
  __syncthreads();
  if (ry == 0) {
    double t = 0.0;
    for (int q = 0; q < 32; ++q) t += red[q][threadIdx.x & 31];
    if (j < h) out[j] = t;
  }
}

// statistics -> (mean, 1 / sqrt(var + eps)) as FP32; training: from the batch mean and the
// centred sum of squares (biased variance), updating the running estimates when asked;
// evaluation: from the running estimates
__global__ void k_bn_finish(int h, int R, int train, int update, const double* dmean, const double* sq, float* rmean,
                            float* rvar, float* mean, float* inv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= h) return;
  if (train) {
    const double m = dmean[j], var = sq[j] / R;
    mean[j] = (float)m;
    inv[j] = (float)(1.0 / sqrt(var + (double)kEps));
    if (update) {
      rmean[j] = (float)((1.0 - kMomentum) * rmean[j] + kMomentum * m);
      rvar[j] = (float)((1.0 - kMomentum) * rvar[j] + kMomentum * var * ((double)R / (double)(R > 1 ? R - 1 : 1)));
    }
  } else {
    mean[j] = rmean[j];
    inv[j] = (float)(1.0 / sqrt((double)rvar[j] + (double)kEps));
  }
}

__global__ void k_div(int h, double d, const double* x, double* y) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < h) y[j] = x[j] / d;
}

// x^ = (Z - mean) inv, y = x^ gamma + mu, H = LeakyReLU_0.2(y): FP32 H, bf16 hi / lo copies
__global__ void k_bn_act(int R, int h, int hp, const float* Z, const float* mean, const float* inv, const float* g,
                         const float* mu, float* XH, float* HF, bf16* H16, bf16* H16lo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)R * hp) return;
  const int j = (int)(t % hp);
  float hv = 0.f, xh = 0.f;
  if (j < h) {
    xh = (Z[t] - mean[j]) * inv[j];
    const float y = xh * g[j] + mu[j];
    hv = y > 0.f ? y : kSlope * y;
  }
  if (XH) XH[t] = xh;
  HF[t] = hv;
  bf16 hi, lo;
  split_bf16(hv, hi, lo);
  H16[t] = hi;
  if (H16lo) H16lo[t] = lo;
}

// rho[cand][j] = mean over the candidate's k rows of H (bf16 hi / lo), rows cand >= c zero up to cp
__global__ void k_rowmean(int c, int cp, int k, int hp, const float* HF, bf16* rho, bf16* rholo, float* rhof) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)cp * hp) return;
  const int cand = (int)(t / hp), j = (int)(t % hp);
  float s = 0.f;
  if (cand < c) {
    for (int i = 0; i < k; ++i) s += HF[((size_t)cand * k + i) * hp + j];
    s /= (float)k;
  }
  bf16 hi, lo;
  split_bf16(s, hi, lo);
  rho[t] = hi;
  if (rholo) rholo[t] = lo;
  if (rhof) rhof[t] = s;
}

// out[cand] = (1 / k) sum_i H[cand, i] . wh + bh
__global__ void k_head(int k, int h, int hp, const float* HF, const float* wh, const float* bh, float* out) {
  __shared__ double red[32];
  const int cand = blockIdx.x;
  double s = 0.0;
  for (int q = threadIdx.x; q < k * h; q += blockDim.x) {
    const int i = q / h, j = q - i * h;
    s += (double)HF[((size_t)cand * k + i) * hp + j] * (double)wh[j];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[cand] = (float)(t / k + bh[0]);
  }
}

// loss, dout = 2 (out - y) / B, d bh (one block)
__global__ void k_loss(int B, const float* out, const float* y, float* dout, float* loss, float* gbh) {
  __shared__ double r1[32], r2[32];
  double s = 0.0, d = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double e = (double)out[b] - (double)y[b];
    s += e * e;
    d += 2.0 * e / B;
    dout[b] = (float)(2.0 * e / B);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    d += __shfl_xor_sync(0xFFFFFFFFu, d, o);
  }
  if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = s; r2[threadIdx.x >> 5] = d; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += r1[w]; c += r2[w]; }
    if (loss) loss[0] = (float)(a / B);
    gbh[0] = (float)c;
  }
}

// d wh[j] = sum_b dout_b (1/k) sum_i H[b,i,j]; dH[row][j] = dout_b wh[j] / k
__global__ void k_head_bwd(int B, int k, int h, int hp, const float* HF, const float* dout, const float* wh, float* gwh,
                           float* dH) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < h) {
    const int j = (int)t;
    double s = 0.0;
    for (int b = 0; b < B; ++b) {
      double m = 0.0;
      for (int i = 0; i < k; ++i) m += HF[((size_t)b * k + i) * hp + j];
      s += (double)dout[b] * m / k;
    }
    gwh[j] = (float)s;
  }
  if (t < (int64_t)B * k * hp) {
    const int row = (int)(t / hp), j = (int)(t % hp);
    dH[t] = j < h ? dout[row / k] * wh[j] / (float)k : 0.f;
  }
}

// column sums of dy = dH LeakyReLU'(y) and of dy x^ (FP64), y = x^ gamma + mu
__global__ void k_bn_bwd_sums(int R, int h, int hp, const float* dH, const float* XH, const float* g, const float* mu,
                              double* sdy, double* sdyx) {
  __shared__ double r1[32][33], r2[32][33];
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  const int ry = threadIdx.x >> 5;
  double a = 0.0, b = 0.0;
  if (j < h) {
    for (int row = ry; row < R; row += 32) {
      const size_t t = (size_t)row * hp + j;
      const float xh = XH[t], y = xh * g[j] + mu[j];
      const double dy = (double)dH[t] * (y > 0.f ? 1.0 : (double)kSlope);
      a += dy;
      b += dy * xh;
    }
  }
  r1[ry][threadIdx.x & 31] = a;
  r2[ry][threadIdx.x & 31] = b;
  __syncthreads();
  if (ry == 0) {
    double s1 = 0.0, s2 = 0.0;
    for (int q = 0; q < 32; ++q) { s1 += r1[q][threadIdx.x & 31]; s2 += r2[q][threadIdx.x & 31]; }
    if (j < h) { sdy[j] = s1; sdyx[j] = s2; }
  }
}

// dZ = inv gamma (dy - sum dy / R - x^ sum(dy x^) / R) in place of dH; bf16 hi / lo copies;
// d gamma = sum dy x^, d mu = sum dy
__global__ void k_bn_bwd(int R, int h, int hp, float* dH, const float* XH, const float* g, const float* mu,
                         const float* inv, const double* sdy, const double* sdyx, bf16* d16, bf16* d16lo, float* gg,
                         float* gmu) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < h) {
    gg[t] = (float)sdyx[t];
    gmu[t] = (float)sdy[t];
  }
  if (t >= (int64_t)R * hp) return;
  const int j = (int)(t % hp);
  float dz = 0.f;
  if (j < h) {
    const float xh = XH[t], y = xh * g[j] + mu[j];
    const float dy = dH[t] * (y > 0.f ? 1.f : kSlope);
    dz = inv[j] * g[j] * (dy - (float)(sdy[j] / R) - xh * (float)(sdyx[j] / R));
  }
  dH[t] = dz;
  if (d16) {
    bf16 hi, lo;
    split_bf16(dz, hi, lo);
    d16[t] = hi;
    if (d16lo) d16lo[t] = lo;
  }
}

// dst[col][r] = src[r][col] (r < rows), 0 for rows <= r < ldT; bf16
__global__ void k_transpose(int rows, int cols, int ldT, const bf16* src, int lds, bf16* dst) {
  __shared__ bf16 tile[32][34];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int q = ty; q < 32; q += 8) {
    const int r = r0 + q, c = c0 + tx;
    tile[q][tx] = (r < rows && c < cols) ? src[(size_t)r * lds + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    const int c = c0 + q, r = r0 + tx;
    if (c < cols && r < ldT) dst[(size_t)c * ldT + r] = tile[tx][q];
  }
}

// drho[cand][j] = sum_i dZ[cand, i][j] (bf16 hi / lo) for cand < c, zero up to cp
__global__ void k_candsum(int c, int cp, int k, int hp, const float* dZ, bf16* d16, bf16* d16lo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)cp * hp) return;
  const int cand = (int)(t / hp), j = (int)(t % hp);
  float s = 0.f;
  if (cand < c)
    for (int i = 0; i < k; ++i) s += dZ[((size_t)cand * k + i) * hp + j];
  bf16 hi, lo;
  split_bf16(s, hi, lo);
  d16[t] = hi;
  if (d16lo) d16lo[t] = lo;
}

// dH[row][j] += T[cand][j] / k (the colour-average term of the input gradient)
__global__ void k_add_rho_grad(int R, int k, int hp, float* dH, const float* T) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)R * hp) return;
  const int row = (int)(t / hp), j = (int)(t % hp);
  dH[t] += T[(size_t)(row / k) * hp + j] / (float)k;
}

// d beta[j] = sum over rows of dZ[row][j] (FP64 accumulation)
__global__ void k_colsum_f(int R, int h, int hp, const float* X, float* out) {
  __shared__ double red[32][33];
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  const int ry = threadIdx.x >> 5;
  double s = 0.0;
  if (j < h)
    for (int row = ry; row < R; row += 32) s += X[(size_t)row * hp + j];
  red[ry][threadIdx.x & 31] = s;
  __syncthreads();
  if (ry == 0) {
    double t = 0.0;
    for (int q = 0; q < 32; ++q) t += red[q][threadIdx.x & 31];
    if (j < h) out[j] = (float)t;
  }
}

// dE[v][j] = sum over the batch of dZ0[(b, colour of v in b)][j]
__global__ void k_demb(int B, int n, int k, int h0, int hp0, const int16_t* cols, const float* dZ, float* gE) {
  const int v = blockIdx.x;
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= h0) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) {
    int c = cols[(size_t)b * n + v];
    c = (c < 0 || c >= k) ? 0 : c;
    s += dZ[((size_t)b * k + c) * hp0 + j];
  }
  gE[(size_t)v * h0 + j] = s;
}

// Adam (betas 0.9 / 0.999, eps 1e-8), bias corrections bc1 = 1 - 0.9^t, sbc2 = sqrt(1 - 0.999^t)
__global__ void k_adam(int64_t P, float* th, float* m, float* v, const float* g, float lr_bc1, float sbc2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr_bc1 * mi / (sqrtf(vi) / sbc2 + 1e-8f);
}

// bf16 hi / lo operand copies of a [din][dout] weight: T[o][i] (transposed, [doutp][dinp]) and
// N[i][o] ([dinp][doutp]), zero padding
__global__ void k_convert(int din, int dout, int dinp, int doutp, const float* W, bf16* T, bf16* Tlo, bf16* N,
                          bf16* Nlo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)dinp * doutp) return;
  const int i = (int)(t / doutp), o = (int)(t % doutp);
  const float w = (i < din && o < dout) ? W[(size_t)i * dout + o] : 0.f;
  bf16 hi, lo;
  split_bf16(w, hi, lo);
  N[(size_t)i * doutp + o] = hi;
  Nlo[(size_t)i * doutp + o] = lo;
  T[(size_t)o * dinp + i] = hi;
  Tlo[(size_t)o * dinp + i] = lo;
}

__global__ void k_fill_uniform(int64_t off, int64_t cnt, float bound, uint64_t seed, float* th) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  const U4 r = rng(seed, (uint32_t)(off + i), 1u, 0u, kTagNnInit);
  const float u = (float)(r.x >> 8) * (1.0f / 16777216.0f);
  th[off + i] = (2.0f * u - 1.0f) * bound;
}

__global__ void k_fill_const(int64_t off, int64_t cnt, float val, float* th) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) th[off + i] = val;
}

__global__ void k_standardise(int p, const int64_t* f, float* y) {
  __shared__ double s[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) a += (double)f[i];
  s[threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += s[i];
    s[0] = t / p;
  }
  __syncthreads();
  const double mean = s[0];
  __syncthreads();
  double b = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) b += ((double)f[i] - mean) * ((double)f[i] - mean);
  s[threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += s[i];
    const double sd = sqrt(t / p);
    s[0] = sd > 0.0 ? sd : 1.0;
  }
  __syncthreads();
  const double sd = s[0];
  for (int i = threadIdx.x; i < p; i += blockDim.x) y[i] = (float)(((double)f[i] - mean) / sd);
}

// the epoch order: samples sorted by Philox(a = i, b = epoch, c = generation, tag = BATCH).r0, ties by i
__global__ void k_perm(int p, uint64_t seed, uint32_t epoch, uint32_t gen, int32_t* perm) {
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

// batch gather: bc[t] = cols[perm[s0 + t]], by[t] = y[perm[s0 + t]]
__global__ void k_gather(int B, int n, int s0, const int32_t* perm, const int16_t* cols, const float* y, int16_t* bc,
                         float* by) {
  const int t = blockIdx.x;
  const int src = perm[s0 + t];
  for (int v = threadIdx.x; v < n; v += blockDim.x) bc[(size_t)t * n + v] = cols[(size_t)src * n + v];
  if (threadIdx.x == 0) by[t] = y[src];
}

template <typename T>
dlm_status dalloc(dlm_ctx* ctx, T** p, size_t count) {
  if (cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DLM_ENOMEM, "deepnet: device allocation failed");
  }
  return DLM_OK;
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace dn
}  // namespace dlm

using namespace dlm;
using namespace dlm::dn;

struct dlm_deepnet {
  int n = 0, k = 0, nh = 0;
  std::vector<int> h, hp;
  int64_t np = 0, nst = 0;
  std::vector<int64_t> og, omu, ob, olam, ogam, ost;  // per layer (olam / ogam for l >= 1); ost: stats
  int64_t oE = 0, owh = 0, obh = 0;
  float *theta = nullptr, *am = nullptr, *av = nullptr, *grad = nullptr, *stats = nullptr;
  int64_t t = 0;
  bool split = true;
  // bf16 operands of layer l >= 1 (hi, lo): Lambda^T, Lambda, Gamma^T, Gamma
  std::vector<bf16*> LT, LTl, LN, LNl, GT, GTl, GN, GNl;
  // activations for cap_c candidates (cap_c k rows): per layer Z, x^, H (FP32), H bf16 hi / lo,
  // rho bf16 hi / lo
  int cap_c = 0;
  std::vector<float*> Z, XH, HF;
  std::vector<bf16*> H16, H16l, rho16, rho16l;
  float *G = nullptr, *T = nullptr, *dA = nullptr, *dB = nullptr;
  bf16 *d16 = nullptr, *d16l = nullptr, *tA = nullptr, *tAl = nullptr, *tB = nullptr, *tBl = nullptr;
  bf16 *c16 = nullptr, *c16l = nullptr;
  std::vector<float*> MU, IV;  // per layer: the mean and 1 / sqrt(var + eps) the normalisation used
  float *mean = nullptr, *inv = nullptr, *outb = nullptr, *dout = nullptr, *lossd = nullptr, *y = nullptr, *by = nullptr;
  double *s1 = nullptr, *s2 = nullptr, *s3 = nullptr;
  int32_t *idx = nullptr, *off = nullptr, *perm = nullptr;
  int16_t* bcols = nullptr;
};

namespace {

dlm_status convert_weights(dlm_ctx* ctx, dlm_deepnet* s) {
  for (int l = 1; l < s->nh; ++l) {
    const int din = s->h[l - 1], dout = s->h[l], dinp = s->hp[l - 1], doutp = s->hp[l];
    const int64_t tot = (int64_t)dinp * doutp;
    k_convert<<<blocks_for(tot), 256, 0, ctx->stream>>>(din, dout, dinp, doutp, s->theta + s->olam[l], s->LT[l], s->LTl[l],
                                                      s->LN[l], s->LNl[l]);
    DLM_TRY(launch_check(ctx, "k_convert"));
    k_convert<<<blocks_for(tot), 256, 0, ctx->stream>>>(din, dout, dinp, doutp, s->theta + s->ogam[l], s->GT[l], s->GTl[l],
                                                      s->GN[l], s->GNl[l]);
    DLM_TRY(launch_check(ctx, "k_convert"));
  }
  return DLM_OK;
}

void free_cap(dlm_deepnet* s) {
  auto F = [](auto*& p) { cudaFree(p); p = nullptr; };
  for (int l = 0; l < s->nh; ++l) {
    F(s->Z[l]); F(s->XH[l]); F(s->HF[l]); F(s->H16[l]); F(s->H16l[l]); F(s->rho16[l]); F(s->rho16l[l]);
  }
  F(s->G); F(s->T); F(s->dA); F(s->dB); F(s->d16); F(s->d16l); F(s->tA); F(s->tAl); F(s->tB); F(s->tBl);
  F(s->c16); F(s->c16l); F(s->outb); F(s->dout); F(s->by); F(s->idx); F(s->off); F(s->bcols);
  s->cap_c = 0;
}

dlm_status ensure_cap(dlm_ctx* ctx, dlm_deepnet* s, int c) {
  if (c <= s->cap_c) return DLM_OK;
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  free_cap(s);
  const int k = s->k, n = s->n;
  const size_t R = (size_t)c * k, Rp = (size_t)pad64((int)R), cp = (size_t)pad64(c);
  size_t hmax = 0;
  for (int x : s->hp) hmax = std::max(hmax, (size_t)x);
  for (int l = 0; l < s->nh; ++l) {
    const size_t w = (size_t)s->hp[l];
    DLM_TRY(dalloc(ctx, &s->Z[l], R * w));
    DLM_TRY(dalloc(ctx, &s->XH[l], R * w));
    DLM_TRY(dalloc(ctx, &s->HF[l], R * w));
    DLM_TRY(dalloc(ctx, &s->H16[l], R * w));
    DLM_TRY(dalloc(ctx, &s->H16l[l], R * w));
    DLM_TRY(dalloc(ctx, &s->rho16[l], cp * w));
    DLM_TRY(dalloc(ctx, &s->rho16l[l], cp * w));
  }
  DLM_TRY(dalloc(ctx, &s->G, cp * hmax));
  DLM_TRY(dalloc(ctx, &s->T, cp * hmax));
  DLM_TRY(dalloc(ctx, &s->dA, R * hmax));
  DLM_TRY(dalloc(ctx, &s->dB, R * hmax));
  DLM_TRY(dalloc(ctx, &s->d16, R * hmax));
  DLM_TRY(dalloc(ctx, &s->d16l, R * hmax));
  DLM_TRY(dalloc(ctx, &s->tA, Rp * hmax));
  DLM_TRY(dalloc(ctx, &s->tAl, Rp * hmax));
  DLM_TRY(dalloc(ctx, &s->tB, Rp * hmax));
  DLM_TRY(dalloc(ctx, &s->tBl, Rp * hmax));
  DLM_TRY(dalloc(ctx, &s->c16, cp * hmax));
  DLM_TRY(dalloc(ctx, &s->c16l, cp * hmax));
  DLM_TRY(dalloc(ctx, &s->outb, (size_t)c));
  DLM_TRY(dalloc(ctx, &s->dout, (size_t)c));
  DLM_TRY(dalloc(ctx, &s->by, (size_t)c));
  DLM_TRY(dalloc(ctx, &s->idx, (size_t)c * n));
  DLM_TRY(dalloc(ctx, &s->off, (size_t)c * (k + 1)));
  DLM_TRY(dalloc(ctx, &s->bcols, (size_t)c * n));
  s->cap_c = c;
  return DLM_OK;
}

// column reductions: one CTA of 32 columns x 32 row groups per 32 features, a fixed order
dim3 colgrid(int h, int) { return dim3((unsigned)((h + 31) / 32)); }

// the feature statistics of layer l over the R rows in Z[l] -> MU[l], IV[l]
dlm_status bn_stats(dlm_ctx* ctx, dlm_deepnet* s, int l, int R, bool train, bool update) {
  const int h = s->h[l], hp = s->hp[l];
  float* rmean = s->stats + s->ost[l];
  float* rvar = rmean + h;
  cudaStream_t st = ctx->stream;
  if (train) {
    k_colsum<<<colgrid(h, R), 1024, 0, st>>>(R, h, hp, s->Z[l], nullptr, 0, s->s1);
    DLM_TRY(launch_check(ctx, "k_colsum"));
    k_div<<<blocks_for(h), 256, 0, st>>>(h, (double)R, s->s1, s->s3);
    DLM_TRY(launch_check(ctx, "k_div"));
    k_colsum<<<colgrid(h, R), 1024, 0, st>>>(R, h, hp, s->Z[l], s->s3, 1, s->s2);
    DLM_TRY(launch_check(ctx, "k_colsum"));
  }
  k_bn_finish<<<blocks_for(h), 256, 0, st>>>(h, R, train ? 1 : 0, update ? 1 : 0, s->s3, s->s2, rmean, rvar, s->MU[l],
                                           s->IV[l]);
  return launch_check(ctx, "k_bn_finish");
}

// forward pass of c <= cap_c candidates: activations of every layer kept, scores in s->outb
dlm_status forward_rows(dlm_ctx* ctx, dlm_deepnet* s, const int16_t* cols, int c, bool train, bool update) {
  cudaStream_t st = ctx->stream;
  const int k = s->k, n = s->n, R = c * k, cp = pad64(c);
  const bool sp = s->split;
  k_sort<<<(c + 3) / 4, 128, 0, st>>>(c, n, k, cols, s->idx, s->off, ctx->d_status);
  DLM_TRY(launch_check(ctx, "k_sort"));
  for (int l = 0; l < s->nh; ++l) {
    const int h = s->h[l], hp = s->hp[l];
    if (l == 0) {
      k_embed<<<dim3((unsigned)R, (unsigned)((hp + 127) / 128)), 128, 0, st>>>(R, n, k, h, hp, s->theta + s->oE,
                                                                            s->theta + s->ob[0], s->idx, s->off, s->Z[0]);
      DLM_TRY(launch_check(ctx, "k_embed"));
    } else {
      const int hin = s->hp[l - 1];
      // Z = H Lambda (rows), G = rho(H) Gamma (candidates)
      DLM_TRY(tc::gemm_run(ctx, s->H16[l - 1], sp ? s->H16l[l - 1] : nullptr, R, hin, hin, s->LT[l],
                           sp ? s->LTl[l] : nullptr, hp, hin, EpiStore{s->Z[l], hp, R, hp}));
      k_rowmean<<<blocks_for((int64_t)cp * hin), 256, 0, st>>>(c, cp, k, hin, s->HF[l - 1], s->rho16[l - 1],
                                                             s->rho16l[l - 1], nullptr);
      DLM_TRY(launch_check(ctx, "k_rowmean"));
      DLM_TRY(tc::gemm_run(ctx, s->rho16[l - 1], sp ? s->rho16l[l - 1] : nullptr, c, hin, hin, s->GT[l],
                           sp ? s->GTl[l] : nullptr, hp, hin, EpiStore{s->G, hp, c, hp}));
      k_add_term<<<blocks_for((int64_t)R * hp), 256, 0, st>>>(R, k, h, hp, s->Z[l], s->G, s->theta + s->ob[l]);
      DLM_TRY(launch_check(ctx, "k_add_term"));
    }
    DLM_TRY(bn_stats(ctx, s, l, R, train, update));
    k_bn_act<<<blocks_for((int64_t)R * hp), 256, 0, st>>>(R, h, hp, s->Z[l], s->MU[l], s->IV[l], s->theta + s->og[l],
                                                        s->theta + s->omu[l], train ? s->XH[l] : nullptr, s->HF[l],
                                                        s->H16[l], sp ? s->H16l[l] : nullptr);
    DLM_TRY(launch_check(ctx, "k_bn_act"));
  }
  const int L = s->nh - 1;
  k_head<<<c, 256, 0, st>>>(k, s->h[L], s->hp[L], s->HF[L], s->theta + s->owh, s->theta + s->obh, s->outb);
  return launch_check(ctx, "k_head");
}

// backward pass of a training-mode forward over B candidates (cols, the same batch), given the
// targets y; the gradient (parameter order) in s->grad, the loss in s->lossd
dlm_status backward_rows(dlm_ctx* ctx, dlm_deepnet* s, const int16_t* cols, int B, const float* y) {
  cudaStream_t st = ctx->stream;
  const int k = s->k, n = s->n, R = B * k, Rp = pad64(R), cp = pad64(B);
  const bool sp = s->split;
  const int L = s->nh - 1;
  DLM_CUDA(ctx, cudaMemsetAsync(s->grad, 0, (size_t)s->np * 4, st));
  k_loss<<<1, 256, 0, st>>>(B, s->outb, y, s->dout, s->lossd, s->grad + s->obh);
  DLM_TRY(launch_check(ctx, "k_loss"));
  {
    const int64_t tot = std::max<int64_t>((int64_t)R * s->hp[L], s->h[L]);
    k_head_bwd<<<blocks_for(tot), 256, 0, st>>>(B, k, s->h[L], s->hp[L], s->HF[L], s->dout, s->theta + s->owh,
                                              s->grad + s->owh, s->dA);
    DLM_TRY(launch_check(ctx, "k_head_bwd"));
  }
  float* dH = s->dA;  // gradient w.r.t. H of the current layer
  float* dN = s->dB;  // gradient w.r.t. H of the layer below
  for (int l = L; l >= 0; --l) {
    const int h = s->h[l], hp = s->hp[l];
    k_bn_bwd_sums<<<colgrid(h, R), 1024, 0, st>>>(R, h, hp, dH, s->XH[l], s->theta + s->og[l], s->theta + s->omu[l],
                                                 s->s1, s->s2);
    DLM_TRY(launch_check(ctx, "k_bn_bwd_sums"));
    k_bn_bwd<<<blocks_for(std::max<int64_t>((int64_t)R * hp, h)), 256, 0, st>>>(
        R, h, hp, dH, s->XH[l], s->theta + s->og[l], s->theta + s->omu[l], s->IV[l], s->s1, s->s2, s->d16,
        sp ? s->d16l : nullptr, s->grad + s->og[l], s->grad + s->omu[l]);
    DLM_TRY(launch_check(ctx, "k_bn_bwd"));
    k_colsum_f<<<(h + 31) / 32, 1024, 0, st>>>(R, h, hp, dH, s->grad + s->ob[l]);
    DLM_TRY(launch_check(ctx, "k_colsum_f"));
    if (l == 0) {
      k_demb<<<dim3((unsigned)n, (unsigned)((h + 127) / 128)), 128, 0, st>>>(B, n, k, h, hp, cols, dH, s->grad + s->oE);
      DLM_TRY(launch_check(ctx, "k_demb"));
      break;
    }
    const int hin = s->hp[l - 1], hi_real = s->h[l - 1];
    // d Lambda = H^T dZ over the R rows (both transposed so that the rows are the contraction)
    {
      dim3 gA((unsigned)((hin + 31) / 32), (unsigned)((Rp + 31) / 32));
      k_transpose<<<gA, 256, 0, st>>>(R, hin, Rp, s->H16[l - 1], hin, s->tA);
      if (sp) k_transpose<<<gA, 256, 0, st>>>(R, hin, Rp, s->H16l[l - 1], hin, s->tAl);
      dim3 gB((unsigned)((hp + 31) / 32), (unsigned)((Rp + 31) / 32));
      k_transpose<<<gB, 256, 0, st>>>(R, hp, Rp, s->d16, hp, s->tB);
      if (sp) k_transpose<<<gB, 256, 0, st>>>(R, hp, Rp, s->d16l, hp, s->tBl);
      DLM_TRY(launch_check(ctx, "k_transpose"));
      DLM_TRY(tc::gemm_run(ctx, s->tA, sp ? s->tAl : nullptr, hi_real, Rp, Rp, s->tB, sp ? s->tBl : nullptr, hp, Rp,
                           EpiStore{s->grad + s->olam[l], h, hi_real, h}));
    }
    // d Gamma = rho^T drho over the candidates; drho = per-candidate sums of dZ
    {
      k_candsum<<<blocks_for((int64_t)cp * hp), 256, 0, st>>>(B, cp, k, hp, dH, s->c16, sp ? s->c16l : nullptr);
      DLM_TRY(launch_check(ctx, "k_candsum"));
      dim3 gA((unsigned)((hin + 31) / 32), (unsigned)((cp + 31) / 32));
      k_transpose<<<gA, 256, 0, st>>>(cp, hin, cp, s->rho16[l - 1], hin, s->tA);
      if (sp) k_transpose<<<gA, 256, 0, st>>>(cp, hin, cp, s->rho16l[l - 1], hin, s->tAl);
      dim3 gB((unsigned)((hp + 31) / 32), (unsigned)((cp + 31) / 32));
      k_transpose<<<gB, 256, 0, st>>>(cp, hp, cp, s->c16, hp, s->tB);
      if (sp) k_transpose<<<gB, 256, 0, st>>>(cp, hp, cp, s->c16l, hp, s->tBl);
      DLM_TRY(launch_check(ctx, "k_transpose"));
      DLM_TRY(tc::gemm_run(ctx, s->tA, sp ? s->tAl : nullptr, hi_real, cp, cp, s->tB, sp ? s->tBl : nullptr, hp, cp,
                           EpiStore{s->grad + s->ogam[l], h, hi_real, h}));
    }
    // dH below = dZ Lambda^T + (1 / k) drho Gamma^T (broadcast over the candidate's rows)
    DLM_TRY(tc::gemm_run(ctx, s->d16, sp ? s->d16l : nullptr, R, hp, hp, s->LN[l], sp ? s->LNl[l] : nullptr, hin, hp,
                         EpiStore{dN, hin, R, hin}));
    DLM_TRY(tc::gemm_run(ctx, s->c16, sp ? s->c16l : nullptr, B, hp, hp, s->GN[l], sp ? s->GNl[l] : nullptr, hin, hp,
                         EpiStore{s->T, hin, B, hin}));
    k_add_rho_grad<<<blocks_for((int64_t)R * hin), 256, 0, st>>>(R, k, hin, dN, s->T);
    DLM_TRY(launch_check(ctx, "k_add_rho_grad"));
    std::swap(dH, dN);
  }
  return DLM_OK;
}

dlm_status adam_step(dlm_ctx* ctx, dlm_deepnet* s, float lr) {
  s->t += 1;
  const double bc1 = 1.0 - std::pow(0.9, (double)s->t), bc2 = 1.0 - std::pow(0.999, (double)s->t);
  k_adam<<<blocks_for(s->np), 256, 0, ctx->stream>>>(s->np, s->theta, s->am, s->av, s->grad, (float)(lr / bc1),
                                                   (float)std::sqrt(bc2));
  DLM_TRY(launch_check(ctx, "k_adam"));
  return convert_weights(ctx, s);
}

}  // namespace

extern "C" void dlm_deepnet_destroy(dlm_deepnet* s) {
  if (!s) return;
  free_cap(s);
  cudaFree(s->theta); cudaFree(s->am); cudaFree(s->av); cudaFree(s->grad); cudaFree(s->stats);
  for (auto* v : {&s->LT, &s->LTl, &s->LN, &s->LNl, &s->GT, &s->GTl, &s->GN, &s->GNl})
    for (auto p : *v) cudaFree(p);
  for (auto p : s->MU) cudaFree(p);
  for (auto p : s->IV) cudaFree(p);
  cudaFree(s->mean); cudaFree(s->inv); cudaFree(s->lossd); cudaFree(s->y); cudaFree(s->s1); cudaFree(s->s2);
  cudaFree(s->s3); cudaFree(s->perm);
  delete s;
}

extern "C" dlm_status dlm_deepnet_create(dlm_ctx* ctx, int32_t n, int32_t k, int32_t nh, const int32_t* widths,
                                         uint64_t seed, dlm_deepnet** out) {
  if (!ctx || !out || !widths) return fail(ctx, DLM_EINVAL, "deepnet_create: null argument");
  *out = nullptr;
  if (n < 1 || n > 2048 || k < 1 || k > 256) return fail(ctx, DLM_EINVAL, "deepnet_create: need 1 <= n <= 2048, 1 <= k <= 256");
  if (nh < 1 || nh > kMaxLayers) return fail(ctx, DLM_EINVAL, "deepnet_create: 1 to 16 hidden layers");
  for (int l = 0; l < nh; ++l)
    if (widths[l] < 1 || widths[l] > kMaxWidth) return fail(ctx, DLM_EINVAL, "deepnet_create: widths in 1..16384");
  dlm_deepnet* s = new dlm_deepnet();
  s->n = n; s->k = k; s->nh = nh;
  s->h.assign(widths, widths + nh);
  for (int x : s->h) s->hp.push_back(pad64(x));
  s->og.resize(nh); s->omu.resize(nh); s->ob.resize(nh); s->olam.assign(nh, 0); s->ogam.assign(nh, 0); s->ost.resize(nh);
  int64_t o = 0;
  s->oE = o; o += (int64_t)n * s->h[0];
  s->ob[0] = o; o += s->h[0];
  s->og[0] = o; o += s->h[0];
  s->omu[0] = o; o += s->h[0];
  for (int l = 1; l < nh; ++l) {
    s->olam[l] = o; o += (int64_t)s->h[l - 1] * s->h[l];
    s->ogam[l] = o; o += (int64_t)s->h[l - 1] * s->h[l];
    s->ob[l] = o; o += s->h[l];
    s->og[l] = o; o += s->h[l];
    s->omu[l] = o; o += s->h[l];
  }
  s->owh = o; o += s->h[nh - 1];
  s->obh = o; o += 1;
  s->np = o;
  int64_t so = 0;
  for (int l = 0; l < nh; ++l) { s->ost[l] = so; so += 2 * (int64_t)s->h[l]; }
  s->nst = so;
  s->Z.assign(nh, nullptr); s->XH.assign(nh, nullptr); s->HF.assign(nh, nullptr); s->H16.assign(nh, nullptr);
  s->H16l.assign(nh, nullptr); s->rho16.assign(nh, nullptr); s->rho16l.assign(nh, nullptr);
  for (auto* v : {&s->LT, &s->LTl, &s->LN, &s->LNl, &s->GT, &s->GTl, &s->GN, &s->GNl}) v->assign(nh, nullptr);
  s->MU.assign(nh, nullptr);
  s->IV.assign(nh, nullptr);
  dlm_status st = DLM_OK;
  auto A = [&](auto** p, size_t cnt) { if (st == DLM_OK) st = dalloc(ctx, p, cnt); };
  A(&s->theta, (size_t)o); A(&s->am, (size_t)o); A(&s->av, (size_t)o); A(&s->grad, (size_t)o); A(&s->stats, (size_t)so);
  int hmax = 0;
  for (int x : s->hp) hmax = std::max(hmax, x);
  A(&s->mean, (size_t)hmax); A(&s->inv, (size_t)hmax); A(&s->lossd, 1); A(&s->y, 8192); A(&s->perm, 8192);
  A(&s->s1, (size_t)hmax); A(&s->s2, (size_t)hmax); A(&s->s3, (size_t)hmax);
  for (int l = 0; l < nh; ++l) { A(&s->MU[l], (size_t)s->hp[l]); A(&s->IV[l], (size_t)s->hp[l]); }
  for (int l = 1; l < nh && st == DLM_OK; ++l) {
    const size_t w = (size_t)s->hp[l - 1] * s->hp[l];
    A(&s->LT[l], w); A(&s->LTl[l], w); A(&s->LN[l], w); A(&s->LNl[l], w);
    A(&s->GT[l], w); A(&s->GTl[l], w); A(&s->GN[l], w); A(&s->GNl[l], w);
  }
  if (st != DLM_OK) { dlm_deepnet_destroy(s); return st; }
  // initial parameters: weights and biases uniform in +-1/sqrt(fan_in) from the NNINIT stream
  // (word b = 1), gamma = 1, mu = 0; running estimates mean 0, variance 1
  cudaStream_t cs = ctx->stream;
  auto U = [&](int64_t off, int64_t cnt, int fan) {
    if (st != DLM_OK || cnt == 0) return;
    k_fill_uniform<<<blocks_for(cnt), 256, 0, cs>>>(off, cnt, (float)(1.0 / std::sqrt((double)fan)), seed, s->theta);
    st = launch_check(ctx, "k_fill_uniform");
  };
  auto C = [&](float* base, int64_t off, int64_t cnt, float val) {
    if (st != DLM_OK || cnt == 0) return;
    k_fill_const<<<blocks_for(cnt), 256, 0, cs>>>(off, cnt, val, base);
    st = launch_check(ctx, "k_fill_const");
  };
  U(s->oE, (int64_t)n * s->h[0], n);
  U(s->ob[0], s->h[0], n);
  for (int l = 0; l < nh; ++l) { C(s->theta, s->og[l], s->h[l], 1.f); C(s->theta, s->omu[l], s->h[l], 0.f); }
  for (int l = 1; l < nh; ++l) {
    U(s->olam[l], (int64_t)s->h[l - 1] * s->h[l], s->h[l - 1]);
    U(s->ogam[l], (int64_t)s->h[l - 1] * s->h[l], s->h[l - 1]);
    U(s->ob[l], s->h[l], s->h[l - 1]);
  }
  U(s->owh, s->h[nh - 1], s->h[nh - 1]);
  U(s->obh, 1, s->h[nh - 1]);
  for (int l = 0; l < nh; ++l) { C(s->stats, s->ost[l], s->h[l], 0.f); C(s->stats, s->ost[l] + s->h[l], s->h[l], 1.f); }
  if (st == DLM_OK) st = cuda_check(ctx, cudaMemsetAsync(s->am, 0, (size_t)o * 4, cs), "memset");
  if (st == DLM_OK) st = cuda_check(ctx, cudaMemsetAsync(s->av, 0, (size_t)o * 4, cs), "memset");
  if (st == DLM_OK) st = convert_weights(ctx, s);
  if (st == DLM_OK) st = dlm_sync(ctx);
  if (st != DLM_OK) { dlm_deepnet_destroy(s); return st; }
  *out = s;
  return DLM_OK;
}

extern "C" int64_t dlm_deepnet_nparams(const dlm_deepnet* s) { return s ? s->np : 0; }
extern "C" int64_t dlm_deepnet_nstats(const dlm_deepnet* s) { return s ? s->nst : 0; }

extern "C" dlm_status dlm_deepnet_get(dlm_ctx* ctx, dlm_deepnet* s, int32_t which, float* dst) {
  if (!ctx || !s || !dst) return fail(ctx, DLM_EINVAL, "deepnet_get: null argument");
  if (which != 0 && which != 1) return fail(ctx, DLM_EINVAL, "deepnet_get: which is 0 (parameters) or 1 (statistics)");
  DLM_CUDA(ctx, cudaMemcpyAsync(dst, which ? s->stats : s->theta, (size_t)(which ? s->nst : s->np) * 4,
                                cudaMemcpyDeviceToDevice, ctx->stream));
  return DLM_OK;
}

extern "C" dlm_status dlm_deepnet_set(dlm_ctx* ctx, dlm_deepnet* s, int32_t which, const float* src) {
  if (!ctx || !s || !src) return fail(ctx, DLM_EINVAL, "deepnet_set: null argument");
  if (which != 0 && which != 1) return fail(ctx, DLM_EINVAL, "deepnet_set: which is 0 (parameters) or 1 (statistics)");
  DLM_CUDA(ctx, cudaMemcpyAsync(which ? s->stats : s->theta, src, (size_t)(which ? s->nst : s->np) * 4,
                                cudaMemcpyDeviceToDevice, ctx->stream));
  if (which == 0) {
    DLM_CUDA(ctx, cudaMemsetAsync(s->am, 0, (size_t)s->np * 4, ctx->stream));
    DLM_CUDA(ctx, cudaMemsetAsync(s->av, 0, (size_t)s->np * 4, ctx->stream));
    s->t = 0;
    DLM_TRY(convert_weights(ctx, s));
  }
  return DLM_OK;
}

extern "C" dlm_status dlm_deepnet_set_precision(dlm_ctx* ctx, dlm_deepnet* s, int32_t split) {
  if (!ctx || !s) return fail(ctx, DLM_EINVAL, "deepnet_set_precision: null argument");
  s->split = split != 0;
  return DLM_OK;
}

extern "C" dlm_status dlm_deepnet_forward(dlm_ctx* ctx, dlm_deepnet* s, const int16_t* col, int32_t c, int32_t train,
                                          float* out) {
  if (!ctx || !s || !col || !out) return fail(ctx, DLM_EINVAL, "deepnet_forward: null argument");
  if (c < 1) return c == 0 ? DLM_OK : fail(ctx, DLM_EINVAL, "deepnet_forward: c < 0");
  if (train) {  // one batch: the statistics couple its candidates
    if (c > 8192) return fail(ctx, DLM_EUNSUPPORTED, "deepnet_forward: a training batch holds at most 8192 candidates");
    DLM_TRY(ensure_cap(ctx, s, c));
    DLM_TRY(forward_rows(ctx, s, col, c, true, true));
    DLM_CUDA(ctx, cudaMemcpyAsync(out, s->outb, (size_t)c * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    return DLM_OK;
  }
  // evaluation: independent candidates, in chunks whose activations take about 4 GB (16 B per
  // feature of every layer and row), at most 4096 candidates; the buffers of a larger training
  // batch are reused
  int64_t feat = 0;
  for (int x : s->hp) feat += x;
  const int64_t per_cand = 16 * (int64_t)s->k * feat;
  const int budget = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (int64_t)4e9 / std::max<int64_t>(1, per_cand)));
  const int chunk = std::max(s->cap_c, std::min(c, budget));
  DLM_TRY(ensure_cap(ctx, s, std::min(c, chunk)));
  for (int c0 = 0; c0 < c; c0 += s->cap_c) {
    const int cc = std::min(s->cap_c, c - c0);
    DLM_TRY(forward_rows(ctx, s, col + (size_t)c0 * s->n, cc, false, false));
    DLM_CUDA(ctx, cudaMemcpyAsync(out + c0, s->outb, (size_t)cc * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return DLM_OK;
}

extern "C" dlm_status dlm_deepnet_loss_grad(dlm_ctx* ctx, dlm_deepnet* s, const int16_t* col, const float* y, int32_t B,
                                            float* grad, float* out, float* loss) {
  if (!ctx || !s || !col || !y) return fail(ctx, DLM_EINVAL, "deepnet_loss_grad: null argument");
  if (B < 1 || B > 8192) return fail(ctx, DLM_EINVAL, "deepnet_loss_grad: 1 <= B <= 8192");
  DLM_TRY(ensure_cap(ctx, s, B));
  DLM_TRY(forward_rows(ctx, s, col, B, true, true));
  DLM_TRY(backward_rows(ctx, s, col, B, y));
  if (grad) DLM_CUDA(ctx, cudaMemcpyAsync(grad, s->grad, (size_t)s->np * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (out) DLM_CUDA(ctx, cudaMemcpyAsync(out, s->outb, (size_t)B * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (loss) DLM_CUDA(ctx, cudaMemcpyAsync(loss, s->lossd, 4, cudaMemcpyDeviceToDevice, ctx->stream));
  return DLM_OK;
}

extern "C" dlm_status dlm_deepnet_train(dlm_ctx* ctx, dlm_deepnet* s, const int16_t* cols, const int64_t* fvals,
                                        int32_t p, int32_t epochs, int32_t b, float lr, uint64_t seed,
                                        uint32_t generation) {
  if (!ctx || !s || !cols || !fvals) return fail(ctx, DLM_EINVAL, "deepnet_train: null argument");
  if (p < 1 || p > 8192 || epochs < 0 || b < 1) return fail(ctx, DLM_EINVAL, "deepnet_train: bad sizes (p <= 8192)");
  const int bb = std::min(b, p);
  DLM_TRY(ensure_cap(ctx, s, bb));
  cudaStream_t st = ctx->stream;
  k_standardise<<<1, 256, 0, st>>>(p, fvals, s->y);
  DLM_TRY(launch_check(ctx, "k_standardise"));
  int mp = 1;
  while (mp < p) mp <<= 1;
  static PerDeviceOnce attr;
  if (attr.need(ctx->device)) {
    DLM_CUDA(ctx, cudaFuncSetAttribute(k_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8));
    attr.mark(ctx->device);
  }
  for (int e = 0; e < epochs; ++e) {
    k_perm<<<1, 1024, (size_t)mp * 8, st>>>(p, seed, (uint32_t)e, generation, s->perm);
    DLM_TRY(launch_check(ctx, "k_perm"));
    for (int s0 = 0; s0 < p; s0 += b) {
      const int B = std::min(b, p - s0);
      k_gather<<<B, 128, 0, st>>>(B, s->n, s0, s->perm, cols, s->y, s->bcols, s->by);
      DLM_TRY(launch_check(ctx, "k_gather"));
      DLM_TRY(forward_rows(ctx, s, s->bcols, B, true, true));
      DLM_TRY(backward_rows(ctx, s, s->bcols, B, s->by));
      DLM_TRY(adam_step(ctx, s, lr));
    }
  }
  return DLM_OK;
}

extern "C" dlm_status dlm_deepnet_adam_step(dlm_ctx* ctx, dlm_deepnet* s, const float* grad, float lr) {
  if (!ctx || !s || !grad) return fail(ctx, DLM_EINVAL, "deepnet_adam_step: null argument");
  DLM_CUDA(ctx, cudaMemcpyAsync(s->grad, grad, (size_t)s->np * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  return adam_step(ctx, s, lr);
}

// state for checkpoints: parameters, Adam moments, running statistics (float32) and the Adam
// step counter (int64)
extern "C" int64_t dlm_deepnet_state_bytes(const dlm_deepnet* s) {
  return s ? (int64_t)((3 * s->np + s->nst) * 4 + 8) : 0;
}

extern "C" dlm_status dlm_deepnet_save(dlm_ctx* ctx, dlm_deepnet* s, void* host) {
  if (!ctx || !s || !host) return fail(ctx, DLM_EINVAL, "deepnet_save: null argument");
  uint8_t* h = (uint8_t*)host;
  const size_t P = (size_t)s->np * 4;
  DLM_CUDA(ctx, cudaMemcpyAsync(h, s->theta, P, cudaMemcpyDeviceToHost, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(h + P, s->am, P, cudaMemcpyDeviceToHost, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(h + 2 * P, s->av, P, cudaMemcpyDeviceToHost, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(h + 3 * P, s->stats, (size_t)s->nst * 4, cudaMemcpyDeviceToHost, ctx->stream));
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  memcpy(h + 3 * P + (size_t)s->nst * 4, &s->t, 8);
  return DLM_OK;
}

extern "C" dlm_status dlm_deepnet_load(dlm_ctx* ctx, dlm_deepnet* s, const void* host) {
  if (!ctx || !s || !host) return fail(ctx, DLM_EINVAL, "deepnet_load: null argument");
  const uint8_t* h = (const uint8_t*)host;
  const size_t P = (size_t)s->np * 4;
  DLM_CUDA(ctx, cudaMemcpyAsync(s->theta, h, P, cudaMemcpyHostToDevice, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(s->am, h + P, P, cudaMemcpyHostToDevice, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(s->av, h + 2 * P, P, cudaMemcpyHostToDevice, ctx->stream));
  DLM_CUDA(ctx, cudaMemcpyAsync(s->stats, h + 3 * P, (size_t)s->nst * 4, cudaMemcpyHostToDevice, ctx->stream));
  memcpy(&s->t, h + 3 * P + (size_t)s->nst * 4, 8);
  DLM_TRY(convert_weights(ctx, s));
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return DLM_OK;
}
