// tmbir_sfu_rate: the special-function throughput of the GPU the context runs on, measured
// rather than taken from a data sheet.  The prior stencil of the iteration (pass 3b) spends
// three special-function operations per neighbour pair (log2, exp2, reciprocal); this kernel
// runs independent chains of exactly those operations, enough of them per thread and enough
// threads per SM that the special-function unit, not latency, limits it.
#include "internal.h"

namespace tmbir {

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr int kRateChains = 8;

// per iteration and chain: a = log2 v in [0, 1], b = 2^a in [1, 2], c = 1 / b, v = c + 1 (three
// special-function operations and one add); the chains keep v in [1.5, 2]
__global__ void __launch_bounds__(256) k_sfu_rate(int iters, float* sink) {
  float v[kRateChains];
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) v[c] = 1.5f + 0.01f * (float)((threadIdx.x + c) & 31);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) v[c] = rcp_approx(ex2_approx(lg2_approx(v[c]))) + 1.0f;
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) s += v[c];
  if (s == 123.456f) sink[0] = s;  // keeps the chains live; never true for v in [1.5, 2]
}

}  // namespace tmbir

using namespace tmbir;

extern "C" int tmbir_sfu_rate(tmbir_ctx* ctx, int iters, double* h_ops_per_s) {
  TMBIR_TRACE("tmbir_sfu_rate");
  if (!ctx || !h_ops_per_s || iters < 1 || iters > (1 << 20))
    return set_error(TMBIR_ERR_ARG, "sfu_rate: need a context, an output and 1 <= iters <= 2^20");
  cudaStream_t s = ctx->c.stream;
  int dev = 0, sms = 0;
  TMBIR_CUDA(cudaGetDevice(&dev));
  TMBIR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;  // eight blocks of eight warps per SM: the most an SM holds
  cudaEvent_t e0, e1;
  TMBIR_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(TMBIR_ERR_CUDA, "sfu_rate: cudaEventCreate failed");
  }
  int rc = TMBIR_OK;
  float ms = 0.f;
  k_sfu_rate<<<blocks, 256, 0, s>>>(iters / 4 + 1, nullptr);  // warm-up
  if (cudaGetLastError() != cudaSuccess) rc = set_error(TMBIR_ERR_CUDA, "sfu_rate: launch failed");
  if (!rc) {
    __atomic_add_fetch(&g_launches, 1, __ATOMIC_RELAXED);
    cudaEventRecord(e0, s);
    k_sfu_rate<<<blocks, 256, 0, s>>>(iters, nullptr);
    if (cudaGetLastError() != cudaSuccess) rc = set_error(TMBIR_ERR_CUDA, "sfu_rate: launch failed");
    __atomic_add_fetch(&g_launches, 1, __ATOMIC_RELAXED);
    cudaEventRecord(e1, s);
    if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = set_error(TMBIR_ERR_CUDA, "sfu_rate: event timing failed");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  *h_ops_per_s = 3.0 * kRateChains * (double)iters * blocks * 256 / (ms * 1e-3);
  return TMBIR_OK;
}
