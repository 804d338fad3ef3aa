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

// L2 bandwidth probe: 16-byte loads that bypass L1 (ld.global.cg) streaming over a buffer that
// fits in L2, every warp reading consecutive 512-byte lines, so each pass after the first is
// served by L2. The tabu kernel's L2 traffic (adjacency bit rows when they are not held in shared
// memory, long-tenure entries) is reported against it.
__global__ void __launch_bounds__(512) k_l2_probe(const uint4* __restrict__ buf, size_t n16, int passes,
                                                  uint4* sink) {
  uint4 acc = make_uint4(0, 0, 0, 0);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
      uint4 v;
      asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                   : "l"(buf + i));
      acc.x ^= v.x; acc.y += v.y; acc.z ^= v.z; acc.w += v.w;
    }
  }
  if (acc.x == 0x12345678u && acc.y == 0x9abcdef0u) sink[blockIdx.x] = acc;
}

}  // namespace dlm

using namespace dlm;

extern "C" dlm_status dlm_probe_l2_bandwidth(dlm_ctx* ctx, double* gbps) {
  if (!ctx || !gbps) return fail(ctx, DLM_EINVAL, "probe: null argument");
  const size_t bytes = (size_t)32 << 20;  // well inside the 129 MB L2
  uint8_t* ws = nullptr;
  DLM_TRY(ctx_workspace(ctx, bytes + 16 * 8192, (void**)&ws));
  const uint4* buf = (const uint4*)ws;
  uint4* sink = (uint4*)(ws + bytes);
  DLM_CUDA(ctx, cudaMemsetAsync(ws, 1, bytes, ctx->stream));
  const int blocks = ctx->num_sms * 4, threads = 512, passes = 16;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_l2_probe<<<blocks, threads, 0, ctx->stream>>>(buf, bytes / 16, 1, sink);  // brings the buffer into L2
  cudaEventRecord(e0, ctx->stream);
  k_l2_probe<<<blocks, threads, 0, ctx->stream>>>(buf, bytes / 16, passes, sink);
  cudaEventRecord(e1, ctx->stream);
  dlm_status st = launch_check(ctx, "k_l2_probe");
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DLM_OK) return st;
  *gbps = (double)bytes * passes / (ms * 1e-3) / 1e9;
  return DLM_OK;
}

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
