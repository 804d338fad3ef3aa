// Host launcher of the tcgen05 GEMM kernel (tcgemm.cuh) for callers outside the scorer:
// C = (A + A2)[M][K] . (B + B2)[N][K]^T, A2 / B2 the bf16 lo parts of split operands (or null),
// every row K-major with leading dimensions lda / ldb (elements, multiples of 8), K a multiple of
// 64, N a multiple of 64 (256-column tiles when N is a multiple of 256). The epilogue functor
// receives the FP32 accumulators (see gemm_kernel).
#pragma once

#include <algorithm>

#include "tcgemm.cuh"

namespace dlm {
namespace tc {

template <int BN, int S, int NA, int NB, class Epi>
inline dlm_status gemm_launch_one(dlm_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& ma2, const CUtensorMap& mb,
                                  const CUtensorMap& mb2, GemmShape sh, Epi epi) {
  auto kfn = gemm_kernel<BN, S, NA, NB, Epi>;
  constexpr size_t smem = gemm_smem_bytes<BN, S, NA, NB>();
  static PerDeviceOnce attr;
  if (attr.need(ctx->device)) {
    DLM_CUDA(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr.mark(ctx->device);
  }
  const int tiles = ((sh.M + BM - 1) / BM) * (sh.N / BN);
  kfn<<<std::min(tiles, ctx->num_sms), kThreads, smem, ctx->stream>>>(ma, ma2, mb, mb2, sh, epi, ctx->d_status);
  return launch_check(ctx, "gemm_kernel");
}

template <int BN, class Epi>
inline dlm_status gemm_launch_bn(dlm_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& ma2, const CUtensorMap& mb,
                                 const CUtensorMap& mb2, bool a2, bool b2, GemmShape sh, Epi epi) {
  constexpr int S2 = BN == 256 ? 2 : 4;
  if (a2 && b2) return gemm_launch_one<BN, S2, 2, 2>(ctx, ma, ma2, mb, mb2, sh, epi);
  if (a2) return gemm_launch_one<BN, S2, 2, 1>(ctx, ma, ma2, mb, mb2, sh, epi);
  if (b2) return gemm_launch_one<BN, S2, 1, 2>(ctx, ma, ma2, mb, mb2, sh, epi);
  return gemm_launch_one<BN, 4, 1, 1>(ctx, ma, ma2, mb, mb2, sh, epi);
}

template <class Epi>
inline dlm_status gemm_run(dlm_ctx* ctx, const __nv_bfloat16* A, const __nv_bfloat16* A2, int M, int K, int lda,
                           const __nv_bfloat16* B, const __nv_bfloat16* B2, int N, int ldb, Epi epi) {
  if (M <= 0) return DLM_OK;
  if (K % BK || N % 64) return fail(ctx, DLM_EINVAL, "gemm: K and N must be multiples of 64");
  const bool wide = N % 256 == 0;
  CUtensorMap ma, ma2, mb, mb2;
  DLM_TRY(make_map_bf16(ctx, &ma, A, (uint64_t)M, (uint64_t)K, (uint64_t)lda, BM));
  DLM_TRY(make_map_bf16(ctx, &mb, B, (uint64_t)N, (uint64_t)K, (uint64_t)ldb, wide ? 256 : 64));
  if (A2) DLM_TRY(make_map_bf16(ctx, &ma2, A2, (uint64_t)M, (uint64_t)K, (uint64_t)lda, BM));
  else ma2 = ma;
  if (B2) DLM_TRY(make_map_bf16(ctx, &mb2, B2, (uint64_t)N, (uint64_t)K, (uint64_t)ldb, wide ? 256 : 64));
  else mb2 = mb;
  GemmShape sh{M, N, K, K / BK};
  if (wide) return gemm_launch_bn<256>(ctx, ma, ma2, mb, mb2, A2 != nullptr, B2 != nullptr, sh, epi);
  return gemm_launch_bn<64>(ctx, ma, ma2, mb, mb2, A2 != nullptr, B2 != nullptr, sh, epi);
}

}  // namespace tc
}  // namespace dlm
