// Context, graph build (CSR + bit rows on the GPU), random initialisation and conflict table.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace dlm {

// ---- graph build -------------------------------------------------------------------------------
__global__ void k_edges_to_bits(int32_t n, int64_t m, const int32_t* edges, uint32_t* bits, int32_t words,
                                int32_t* status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const int u = edges[2 * e], v = edges[2 * e + 1];
  if (u < 0 || v < 0 || u >= n || v >= n || u == v) {
    raise_status(status, DLM_EINVAL);
    return;
  }
  atomicOr(bits + (size_t)u * words + (v >> 5), 1u << (v & 31));
  atomicOr(bits + (size_t)v * words + (u >> 5), 1u << (u & 31));
}

// one block: degrees (popcounts of the bit rows) and their exclusive scan into off[0..n]
__global__ void k_degree_scan(int32_t n, const uint32_t* bits, int32_t words, int32_t* off) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  int local[4] = {0, 0, 0, 0};  // n <= 2048 and blockDim = 1024 -> per <= 2
  int sum = 0;
  for (int q = 0; q < per; ++q) {
    const int v = t * per + q;
    int d = 0;
    if (v < n)
      for (int w = 0; w < words; ++w) d += __popc(bits[(size_t)v * words + w]);
    local[q] = d;
    sum += d;
  }
  part[t] = sum;
  __syncthreads();
  for (int s = 1; s < (int)blockDim.x; s <<= 1) {
    const int x = t >= s ? part[t - s] : 0;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  int run = part[t] - sum;
  for (int q = 0; q < per; ++q) {
    const int v = t * per + q;
    if (v < n) off[v] = run;
    run += local[q];
  }
  if (t == blockDim.x - 1) off[n] = part[t];
}

// one warp per vertex: expand the bit row into ascending neighbour ids
__global__ void k_fill_csr(int32_t n, const uint32_t* bits, int32_t words, const int32_t* off, uint16_t* idx) {
  const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= n) return;
  int base = off[v];
  for (int w0 = 0; w0 < words; w0 += 32) {
    const int w = w0 + lane;
    const uint32_t x = w < words ? bits[(size_t)v * words + w] : 0u;
    const int c = __popc(x);
    int incl = c;
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= d) incl += y;
    }
    uint32_t m = x;
    int pos = base + incl - c;
    while (m) {
      idx[pos++] = (uint16_t)(32 * w + __ffs(m) - 1);
      m &= m - 1;
    }
    base += __shfl_sync(0xFFFFFFFFu, incl, 31);
  }
}

// ---- initialisation and conflict table ---------------------------------------------------------
__global__ void k_init_colors(int32_t n, int32_t k, int32_t pop, uint64_t seed, uint32_t ind_base, int16_t* col) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * pop) return;
  const int i = (int)(t / n), v = (int)(t % n);
  const U4 r = rng(seed, (uint32_t)v, 0u, ind_base + (uint32_t)i, kTagInit);
  col[t] = (int16_t)below(r.x, (uint32_t)k);
}

// one block per individual, one thread per row
__global__ void k_gamma(int32_t n, int32_t k, const uint32_t* bits, int32_t words, const int16_t* col,
                        int32_t* gamma, int64_t* f, int32_t* status) {
  const int i = blockIdx.x;
  const int16_t* c = col + (size_t)i * n;
  __shared__ long long part[32];
  long long loc = 0;
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    int32_t* grow = gamma ? gamma + ((size_t)i * n + v) * k : nullptr;
    if (grow)
      for (int q = 0; q < k; ++q) grow[q] = 0;
    const int cv = c[v];
    if (cv < 0 || cv >= k) { raise_status(status, DLM_EINVAL); continue; }
    int same = 0;
    for (int w = 0; w < words; ++w) {
      uint32_t m = bits[(size_t)v * words + w];
      while (m) {
        const int u = 32 * w + __ffs(m) - 1;
        m &= m - 1;
        const int cu = c[u];
        if (cu == cv) ++same;
        if (grow && cu >= 0 && cu < k) grow[cu]++;
      }
    }
    loc += same;
  }
  for (int d = 16; d >= 1; d >>= 1) loc += __shfl_down_sync(0xFFFFFFFFu, loc, d);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = loc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    f[i] = s / 2;
  }
}

}  // namespace dlm

using namespace dlm;

extern "C" {

dlm_status dlm_create(dlm_ctx** out, int32_t device, void* stream) {
  if (!out) return DLM_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return DLM_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return DLM_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return DLM_ECUDA;
  if (prop.major < 10) return DLM_EUNSUPPORTED;
  dlm_ctx* ctx = new dlm_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  ctx->num_sms = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  if (cudaMalloc(&ctx->d_status, sizeof(int32_t)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(int32_t)) != cudaSuccess) {
    delete ctx;
    return DLM_ENOMEM;
  }
  *out = ctx;
  return DLM_OK;
}

void dlm_destroy(dlm_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& r : ctx->gemm_recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  cudaFree(ctx->d_status);
  if (ctx->ws) cudaFree(ctx->ws);
  for (auto s : ctx->pool) if (s) cudaStreamDestroy(s);
  for (auto e : ctx->pool_ev) if (e) cudaEventDestroy(e);
  delete ctx;
}

dlm_status dlm_set_stream(dlm_ctx* ctx, void* stream) {
  if (!ctx) return DLM_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return DLM_OK;
}

dlm_status dlm_set_cancel_flag(dlm_ctx* ctx, const int32_t* flag) {
  if (!ctx) return DLM_EINVAL;
  if (!flag) {
    ctx->cancel = nullptr;
    return DLM_OK;
  }
  // only memory the device can address: device or managed memory as is, pinned host memory
  // through its device alias; pageable host memory is refused
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, flag) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DLM_EINVAL, "set_cancel_flag: pointer unknown to CUDA");
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    ctx->cancel = flag;
    return DLM_OK;
  }
  if (at.type == cudaMemoryTypeHost) {
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, (void*)flag, 0) != cudaSuccess || !d) {
      cudaGetLastError();
      return fail(ctx, DLM_EINVAL, "set_cancel_flag: pinned host memory without a device mapping");
    }
    ctx->cancel = (const int32_t*)d;
    return DLM_OK;
  }
  return fail(ctx, DLM_EINVAL, "set_cancel_flag: pageable host memory cannot be polled by the device");
}

const char* dlm_last_error(const dlm_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

dlm_status dlm_sync(dlm_ctx* ctx) {
  if (!ctx) return DLM_EINVAL;
  DLM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int32_t st = 0;
  DLM_CUDA(ctx, cudaMemcpy(&st, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (st != 0) {
    DLM_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int32_t)));
    return fail(ctx, st, "device-side status " + std::to_string(st));
  }
  return DLM_OK;
}

dlm_status dlm_graph_create(dlm_ctx* ctx, int32_t n, int64_t m, const int32_t* edges, const int32_t* weights,
                            dlm_graph** out) {
  if (!ctx || !out) return fail(ctx, DLM_EINVAL, "graph_create: null argument");
  *out = nullptr;
  if (n < 2 || n > 2048) return fail(ctx, DLM_EUNSUPPORTED, "graph_create: n must be in 2..2048");
  if (m < 0 || (m > 0 && !edges)) return fail(ctx, DLM_EINVAL, "graph_create: bad edge list");
  dlm_graph* g = new dlm_graph();
  g->n = n;
  g->words = (n + 31) / 32;
  auto cleanup = [&](dlm_status s, const char* msg) {
    cudaFree(g->d_off); cudaFree(g->d_idx); cudaFree(g->d_bits); cudaFree(g->d_weight);
    delete g;
    return fail(ctx, s, msg);
  };
  if (cudaMalloc(&g->d_bits, (size_t)n * g->words * 4) != cudaSuccess ||
      cudaMalloc(&g->d_off, (size_t)(n + 1) * 4) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(DLM_ENOMEM, "graph_create: allocation failed");
  }
  cudaMemsetAsync(g->d_bits, 0, (size_t)n * g->words * 4, ctx->stream);
  if (m > 0)
    k_edges_to_bits<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(n, m, edges, g->d_bits, g->words, ctx->d_status);
  k_degree_scan<<<1, 1024, 0, ctx->stream>>>(n, g->d_bits, g->words, g->d_off);
  std::vector<int32_t> off(n + 1);
  if (cudaMemcpyAsync(off.data(), g->d_off, (size_t)(n + 1) * 4, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return cleanup(DLM_ECUDA, "graph_create: build failed");
  int32_t st = 0;
  cudaMemcpy(&st, ctx->d_status, 4, cudaMemcpyDeviceToHost);
  if (st != 0) {
    cudaMemset(ctx->d_status, 0, 4);
    return cleanup(DLM_EINVAL, "graph_create: edge with an end point outside 0..n-1 or a self loop");
  }
  g->m = off[n] / 2;
  for (int v = 0; v < n; ++v) g->max_degree = std::max(g->max_degree, off[v + 1] - off[v]);
  if (cudaMalloc(&g->d_idx, std::max<size_t>(1, (size_t)off[n]) * 2) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(DLM_ENOMEM, "graph_create: allocation failed");
  }
  k_fill_csr<<<(n + 7) / 8, 256, 0, ctx->stream>>>(n, g->d_bits, g->words, g->d_off, g->d_idx);
  if (weights) {
    std::vector<int32_t> w(n);
    if (cudaMalloc(&g->d_weight, (size_t)n * 4) != cudaSuccess)
      return cleanup(DLM_ENOMEM, "graph_create: allocation failed");
    cudaMemcpyAsync(g->d_weight, weights, (size_t)n * 4, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(w.data(), weights, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    for (int v = 0; v < n; ++v) {
      if (w[v] <= 0) return cleanup(DLM_EINVAL, "graph_create: weights must be positive");
      g->max_weight = std::max(g->max_weight, w[v]);
    }
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return cleanup(DLM_ECUDA, "graph_create: build failed");
  *out = g;
  return DLM_OK;
}

void dlm_graph_destroy(dlm_graph* g) {
  if (!g) return;
  cudaFree(g->d_off);
  cudaFree(g->d_idx);
  cudaFree(g->d_bits);
  cudaFree(g->d_weight);
  delete g;
}

int32_t dlm_graph_n(const dlm_graph* g) { return g ? g->n : 0; }
int64_t dlm_graph_m(const dlm_graph* g) { return g ? g->m : 0; }

__global__ void k_widen_idx(int64_t cnt, const uint16_t* src, int32_t* dst) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < cnt) dst[t] = src[t];
}

dlm_status dlm_graph_export(dlm_ctx* ctx, const dlm_graph* g, int32_t* off, int32_t* idx, uint32_t* bits) {
  if (!ctx || !g) return fail(ctx, DLM_EINVAL, "graph_export: null argument");
  if (off) DLM_CUDA(ctx, cudaMemcpyAsync(off, g->d_off, (size_t)(g->n + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (idx && g->m > 0) {
    k_widen_idx<<<(unsigned)((2 * g->m + 255) / 256), 256, 0, ctx->stream>>>(2 * g->m, g->d_idx, idx);
    DLM_TRY(launch_check(ctx, "k_widen_idx"));
  }
  if (bits)
    DLM_CUDA(ctx, cudaMemcpyAsync(bits, g->d_bits, (size_t)g->n * g->words * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  return DLM_OK;
}

dlm_status dlm_init_colors(dlm_ctx* ctx, int32_t n, int32_t k, int32_t pop, uint64_t seed, uint32_t ind_base,
                           int16_t* col) {
  if (!ctx) return DLM_EINVAL;
  if (n <= 0 || k <= 0 || k > 32767 || pop < 0 || (pop > 0 && !col)) return fail(ctx, DLM_EINVAL, "init_colors: bad arguments");
  const int64_t total = (int64_t)n * pop;
  if (total == 0) return DLM_OK;
  k_init_colors<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(n, k, pop, seed, ind_base, col);
  return launch_check(ctx, "k_init_colors");
}

dlm_status dlm_gamma(dlm_ctx* ctx, const dlm_graph* g, int32_t k, int32_t pop, const int16_t* col, int32_t* gamma,
                     int64_t* f) {
  if (!ctx || !g) return fail(ctx, DLM_EINVAL, "gamma: null argument");
  if (k <= 0 || pop < 0 || (pop > 0 && (!col || !f))) return fail(ctx, DLM_EINVAL, "gamma: bad arguments");
  if (pop == 0) return DLM_OK;
  k_gamma<<<pop, 256, 0, ctx->stream>>>(g->n, k, g->d_bits, g->words, col, gamma, f, ctx->d_status);
  return launch_check(ctx, "k_gamma");
}

}  // extern "C"
