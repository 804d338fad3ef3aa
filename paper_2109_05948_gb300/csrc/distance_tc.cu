// Partition distances on the tensor cores (section "Distance computation"; the overlap-matrix
// approximation of the distance): the class-overlap matrices M(X_i, Y_j)[a][b] = |A_a ∩ B_b| of
// all pairs as one-hot matrix products. With O_X[(i, a)][v] = [X_i(v) = a] (bf16, exact),
// O_X . O_Y^T holds every M(X_i, Y_j) as a kp x kp block (kp = k rounded up to 64 or 128), and
// the counts (at most 2048) are exact in the FP32 accumulators. One product gives the row maxima:
// the epilogue takes, per accumulator row (class a of X_i) and partner block, the largest count,
// sums it over the warp's 32 rows and adds the sum into rs[i][j]; the transposed product
// O_Y . O_X^T gives the column maxima into cs[j][i] the same way; D = n - min(rs, cs).
// A product forms all kp^2 overlaps of a pair from n kp one-hot products, where counting touches n
// counters, so this path is a measured comparison point for the counting kernels, not the
// library's choice.
#include <algorithm>

#include "common.cuh"
#include "tcgemm.cuh"

namespace dlm {
namespace {

using bf16 = __nv_bfloat16;

// O[(i kp + a)][v] = [X_i(v) = a] for v < n, 0 for n <= v < np; rows of padding individuals
// (i >= rows) are zero. One thread writes 8 consecutive columns (16 bytes).
__global__ void k_onehot(int n, int k, int kp, int np, const int16_t* X, int rows, int rows_pad, bf16* O,
                         int32_t* status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int chunks = np / 8;
  const int64_t total = (int64_t)rows_pad * kp * chunks;
  if (t >= total) return;
  const int ch = (int)(t % chunks);
  const int64_t r = t / chunks;
  const int a = (int)(r % kp), i = (int)(r / kp);
  const uint16_t one = 0x3F80u;  // bf16 1.0
  uint16_t out[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int v = ch * 8 + q;
    uint16_t x = 0;
    if (i < rows && v < n) {
      const int c = X[(size_t)i * n + v];
      if (a == 0 && (c < 0 || c >= k)) raise_status(status, DLM_EINVAL);
      x = c == a ? one : (uint16_t)0;
    }
    out[q] = x;
  }
  uint4 w;
  w.x = out[0] | ((uint32_t)out[1] << 16);
  w.y = out[2] | ((uint32_t)out[3] << 16);
  w.z = out[4] | ((uint32_t)out[5] << 16);
  w.w = out[6] | ((uint32_t)out[7] << 16);
  *reinterpret_cast<uint4*>(O + (size_t)r * np + (size_t)ch * 8) = w;
}

// Epilogue: per accumulator row, the largest count in each partner block of the half tile
// (128 columns: two blocks of 64 or one of 128), summed over the warp's rows into acc[i][j].
// Every row of a warp belongs to the same individual i (kp is a multiple of 32).
struct EpiRowMax {
  int* acc;
  int ld, rows_valid, cols_valid, kp;
  int n0c;
  float rm0, rm1;
  __device__ void tile(int, int c) {
    n0c = c;
    rm0 = 0.f;
    rm1 = 0.f;
  }
  __device__ void operator()(int, int col0, const float (&v)[16]) {
    float m = v[0];
#pragma unroll
    for (int i = 1; i < 16; ++i) m = fmaxf(m, v[i]);
    if (col0 - n0c < kp) rm0 = fmaxf(rm0, m);
    else rm1 = fmaxf(rm1, m);
  }
  __device__ void finish(int row) {
    const int lane = threadIdx.x & 31;
    const int i = row / kp;
    const int nb = 128 / kp;
    for (int jb = 0; jb < nb; ++jb) {
      const int s = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)(int)(jb ? rm1 : rm0));
      const int j = n0c / kp + jb;
      if (lane == 0 && i < rows_valid && j < cols_valid && s != 0) atomicAdd(acc + (size_t)i * ld + j, s);
    }
  }
};

__global__ void k_dist_tc_final(int n, int a, int b, const int* rs, const int* cs, int16_t* D, int64_t ldD,
                                int upper) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)a * b) return;
  const int i = (int)(t / b), j = (int)(t % b);
  if (upper && j <= i) return;
  const int r = rs[(size_t)i * b + j], c = cs[(size_t)j * a + i];
  D[(size_t)i * ldD + j] = (int16_t)(n - (r < c ? r : c));
}

dlm_status rowmax_gemm(dlm_ctx* ctx, const bf16* A, int Mrows, const bf16* B, int Nrows, int K, EpiRowMax epi) {
  using namespace tc;
  CUtensorMap ma, mb;
  DLM_TRY(make_map_bf16(ctx, &ma, A, (uint64_t)Mrows, (uint64_t)K, (uint64_t)K, BM));
  DLM_TRY(make_map_bf16(ctx, &mb, B, (uint64_t)Nrows, (uint64_t)K, (uint64_t)K, 256));
  GemmShape sh{Mrows, Nrows, K, K / BK};
  const int tiles = ((Mrows + BM - 1) / BM) * (Nrows / 256);
  auto kfn = gemm_kernel<256, 4, 1, 1, EpiRowMax>;
  const size_t smem = gemm_smem_bytes<256, 4, 1, 1>();
  static PerDeviceOnce attr;
  if (attr.need(ctx->device)) {
    DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr.mark(ctx->device);
  }
  kfn<<<std::min(tiles, ctx->num_sms), kThreads, smem, ctx->stream>>>(ma, ma, mb, mb, sh, epi, ctx->d_status);
  return launch_check(ctx, "gemm_kernel<EpiRowMax>");
}

}  // namespace

// the tensor-core path of dlm_distance_batch_ex (method 3); sizes already validated
dlm_status distance_tc(dlm_ctx* ctx, int n, int k, const int16_t* X, int a, const int16_t* Y, int b, int16_t* D,
                       int64_t ldD, int upper) {
  if (k > 128) return fail(ctx, DLM_EUNSUPPORTED, "distance (tensor cores): k must be <= 128");
  const int kp = k <= 64 ? 64 : 128;
  const int np = 64 * ((n + 63) / 64);
  const int per = 256 / kp;  // individuals per 256-column tile: pad both sides to a multiple
  const int ap = per * ((a + per - 1) / per), bp = per * ((b + per - 1) / per);
  const size_t ox = (size_t)ap * kp * np * 2, oy = (size_t)bp * kp * np * 2;
  const size_t rsb = (size_t)a * b * 4;
  uint8_t* ws = nullptr;
  DLM_TRY(ctx_workspace(ctx, ox + oy + 2 * rsb + 64, (void**)&ws));
  bf16* OX = (bf16*)ws;
  bf16* OY = (bf16*)(ws + ox);
  int* rs = (int*)(ws + ox + oy);
  int* cs = (int*)(ws + ox + oy + rsb);
  DLM_CUDA(ctx, cudaMemsetAsync(rs, 0, 2 * rsb, ctx->stream));
  const int chunks = np / 8;
  {
    const int64_t tx = (int64_t)ap * kp * chunks, ty = (int64_t)bp * kp * chunks;
    k_onehot<<<(unsigned)((tx + 255) / 256), 256, 0, ctx->stream>>>(n, k, kp, np, X, a, ap, OX, ctx->d_status);
    DLM_TRY(launch_check(ctx, "k_onehot"));
    k_onehot<<<(unsigned)((ty + 255) / 256), 256, 0, ctx->stream>>>(n, k, kp, np, Y, b, bp, OY, ctx->d_status);
    DLM_TRY(launch_check(ctx, "k_onehot"));
  }
  EpiRowMax e1{rs, b, a, b, kp, 0, 0.f, 0.f};
  DLM_TRY(rowmax_gemm(ctx, OX, ap * kp, OY, bp * kp, np, e1));
  EpiRowMax e2{cs, a, b, a, kp, 0, 0.f, 0.f};
  DLM_TRY(rowmax_gemm(ctx, OY, bp * kp, OX, ap * kp, np, e2));
  const int64_t tot = (int64_t)a * b;
  k_dist_tc_final<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(n, a, b, rs, cs, D, ldD, upper);
  return launch_check(ctx, "k_dist_tc_final");
}

}  // namespace dlm
