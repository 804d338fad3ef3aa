// Shared device/host helpers of the DLMCOL CUDA library (sm_103a only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/dlmcol.h"

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ < 1000)
#error "libdlmcol is written for sm_103a (GB300) only"
#endif

namespace dlm {

// ------------------------------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11). Key = the 64-bit
// seed split into two words; counter = (a, b, c, tag), the tag naming the use of the draw.
// ------------------------------------------------------------------------------------------------
enum : uint32_t { kTagInit = 1, kTagTabu = 2, kTagGpx = 3, kTagSelect = 4, kTagNnInit = 7,
                  kTagBatch = 8, kTagWInit = 9 };

struct U4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
  for (int r = 0; r < 10; ++r) {
#if defined(__CUDA_ARCH__)
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
#else
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

__host__ __device__ __forceinline__ U4 rng(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t tag) {
  return philox10(a, b, c, tag, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// uniform integer in [0, m): high word of r * m
__host__ __device__ __forceinline__ uint32_t below(uint32_t r, uint32_t m) {
  return (uint32_t)(((uint64_t)r * (uint64_t)m) >> 32);
}

// ------------------------------------------------------------------------------------------------
// Device-side error reporting: the first nonzero code wins; read back by dlm_sync.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void raise_status(int32_t* status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
}

}  // namespace dlm

// ------------------------------------------------------------------------------------------------
// Host-side objects behind the opaque C handles.
// ------------------------------------------------------------------------------------------------
struct dlm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int32_t* d_status = nullptr;  // device status word (DLM_OK or an error code)
  int num_sms = 0;
  size_t smem_optin = 0;
  std::string last_error;
  // autotune cache for the tabu kernel: warps per individual keyed by (n, k)
  struct TuneEntry { int n, k, warps; };
  TuneEntry tune[64];
  int n_tune = 0;
  // grow-only device workspace for calls that need scratch (job lists, queues, tuning buffers)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // optional CUDA-event timing of every tensor-core GEMM launch (dlm_gemm_profile)
  struct GemmRec { cudaEvent_t a, b; double flops; };
  bool gemm_prof = false;
  std::vector<GemmRec> gemm_recs;
  // cancellation flag polled by the long-running search kernels (dlm_set_cancel_flag)
  const int32_t* cancel = nullptr;
  // streams and events for launches that run side by side (the uneven batch: one launch per
  // graph), created on first use
  static constexpr int kPool = 16;
  cudaStream_t pool[kPool] = {};
  cudaEvent_t pool_ev[kPool + 1] = {};
};

struct dlm_graph {
  int32_t n = 0;
  int64_t m = 0;
  int32_t max_degree = 0;
  int32_t words = 0;           // ceil(n / 32)
  int32_t* d_off = nullptr;    // [n + 1]
  uint16_t* d_idx = nullptr;   // [2m], ascending per vertex
  uint32_t* d_bits = nullptr;  // [n][words]
  int32_t* d_weight = nullptr; // [n] or null
  int32_t max_weight = 0;
};

namespace dlm {

inline dlm_status fail(dlm_ctx* ctx, dlm_status code, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return code;
}

inline dlm_status cuda_check(dlm_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DLM_OK;
  return fail(ctx, DLM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define DLM_TRY(expr)                    \
  do {                                   \
    dlm_status _s = (expr);              \
    if (_s != DLM_OK) return _s;         \
  } while (0)

#define DLM_CUDA(ctx, expr) DLM_TRY(::dlm::cuda_check((ctx), (expr), #expr))

// Returns a device workspace of at least `bytes`, owned by the context. Growing it waits for the
// context's stream (work queued earlier may still use the old buffer).
inline dlm_status ctx_workspace(dlm_ctx* ctx, size_t bytes, void** out) {
  if (bytes > ctx->ws_bytes) {
    if (ctx->ws) {
      DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      cudaFree(ctx->ws);
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
    }
    const size_t want = bytes < (1u << 20) ? (1u << 20) : bytes;
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, DLM_ENOMEM, "workspace allocation failed");
    }
    ctx->ws_bytes = want;
  }
  *out = ctx->ws;
  return DLM_OK;
}

inline dlm_status launch_check(dlm_ctx* ctx, const char* what) {
  return cuda_check(ctx, cudaGetLastError(), what);
}

// A kernel attribute (such as its dynamic shared-memory limit) belongs to one device: the devices
// (0..63) on which a call site has set it; devices beyond 63 set it on every call.
struct PerDeviceOnce {
  std::atomic<uint64_t> done{0};
  bool need(int device) const { return device < 0 || device >= 64 || !((done.load() >> device) & 1u); }
  void mark(int device) {
    if (device >= 0 && device < 64) done.fetch_or(1ull << device);
  }
};

}  // namespace dlm
