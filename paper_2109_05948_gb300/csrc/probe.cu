// Shared-memory bandwidth probe: the denominator of the tabu kernel's roofline (its state lives
// in shared memory, so neither the HBM copy nor the GEMM peak bounds it).
#include "common.cuh"

namespace dlm {

// Every thread streams 16-byte loads over a 32 KB shared buffer (conflict-free: a quarter warp
// reads 128 contiguous bytes), folding the data into a register so nothing is optimised away.
__global__ void __launch_bounds__(1024) k_smem_probe(int reps, uint4* sink) {
  __shared__ uint4 buf[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x)
    buf[i] = make_uint4(i, i * 3u, i * 5u, i * 7u);
  __syncthreads();
  uint4 acc = make_uint4(0, 0, 0, 0);
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
  uint32_t idx = threadIdx.x;
#pragma unroll 4
  for (int r = 0; r < reps; ++r) {
    uint4 v;
    // volatile: every iteration really reads shared memory
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(base + 16u * idx));
    acc.x ^= v.x; acc.y += v.y; acc.z ^= v.z; acc.w += v.w;
    idx = (idx + 1024u + (uint32_t)(r & 1)) & 2047u;
  }
  if (acc.x == 0x12345678u && acc.y == 0x9abcdef0u) sink[blockIdx.x] = acc;
}

}  // namespace dlm

using namespace dlm;

extern "C" dlm_status dlm_probe_smem_bandwidth(dlm_ctx* ctx, double* gbps) {
  if (!ctx || !gbps) return fail(ctx, DLM_EINVAL, "probe: null argument");
  uint4* sink = nullptr;
  DLM_TRY(ctx_workspace(ctx, 16 * 4096, (void**)&sink));
  const int blocks = ctx->num_sms * 2, threads = 1024, reps = 1 << 14;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_smem_probe<<<blocks, threads, 0, ctx->stream>>>(reps, sink);  // warm-up
  cudaEventRecord(e0, ctx->stream);
  k_smem_probe<<<blocks, threads, 0, ctx->stream>>>(reps, sink);
  cudaEventRecord(e1, ctx->stream);
  dlm_status st = launch_check(ctx, "k_smem_probe");
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DLM_OK) return st;
  *gbps = (double)blocks * threads * reps * 16.0 / (ms * 1e-3) / 1e9;
  return DLM_OK;
}
