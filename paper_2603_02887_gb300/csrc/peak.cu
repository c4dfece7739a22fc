// Throughput microbenchmarks of the pipes the compositing kernels run on: the denominators of their
// roofline fractions. The compositing forward and replay are bound by FP32 issue (FMA and packed FMA) and
// by the MUFU ex2 of each alpha; nothing on the path is a dense contraction, so no tensor-core figure is
// involved. Each kernel runs eight independent dependency chains per thread on every SM at full
// occupancy, so that the pipe, not latency, limits it.
#include <algorithm>

#include "ngs_internal.cuh"

namespace ngs {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kThreads) peak_kernel(float* __restrict__ out, int iters, float seed) {
  const float b = 0.99993896484375f, c = 6.103515625e-05f;  // a <- a b + c converges to 1: no overflow
  float acc = 0.f;
  if constexpr (KIND == NGS_PEAK_FFMA) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = seed + 0.125f * (float)(j + threadIdx.x % 7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = __fmaf_rn(a[j], b, c);
    }
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += a[j];
  } else if constexpr (KIND == NGS_PEAK_FFMA2) {
    float2 a[kChains];
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = make_float2(seed + 0.125f * (float)j, seed - 0.0625f * (float)j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = __ffma2_rn(a[j], b2, c2);
    }
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += a[j].x + a[j].y;
  } else {
    // a <- 2^-a stays in [1/2, 1] for a in [0, 1]: the chains never leave the normal range
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 0.0625f * (float)(j + threadIdx.x % 5) * seed;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fast_exp2(-a[j]);
    }
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += a[j];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;  // keeps every chain live
}

// Operations one launch performs: FLOPs (an FMA counts 2, a packed FMA 4) or ex2 results.
double ops_per_launch(int kind, unsigned blocks, int iters) {
  const double per = kind == NGS_PEAK_FFMA ? 2.0 : kind == NGS_PEAK_FFMA2 ? 4.0 : 1.0;
  return per * kChains * (double)iters * (double)blocks * kThreads;
}

void launch_peak(int kind, float* out, unsigned blocks, int iters, cudaStream_t s) {
  if (kind == NGS_PEAK_FFMA) peak_kernel<NGS_PEAK_FFMA><<<blocks, kThreads, 0, s>>>(out, iters, 0.5f);
  else if (kind == NGS_PEAK_FFMA2) peak_kernel<NGS_PEAK_FFMA2><<<blocks, kThreads, 0, s>>>(out, iters, 0.5f);
  else peak_kernel<NGS_PEAK_EX2><<<blocks, kThreads, 0, s>>>(out, iters, 0.5f);
}

}  // namespace
}  // namespace ngs

using namespace ngs;

extern "C" NGS_API int ngs_measure_peak(ngs_ctx* ctx, int32_t kind, double seconds, double* rate, void* stream) {
  if (!ctx || !rate) return NGS_ERR_INVALID_ARG;
  if (kind != NGS_PEAK_FFMA && kind != NGS_PEAK_FFMA2 && kind != NGS_PEAK_EX2)
    return fail(ctx, NGS_ERR_INVALID_ARG, "unknown peak kind");
  if (!(seconds >= 0.01 && seconds <= 60.0)) return fail(ctx, NGS_ERR_INVALID_ARG, "seconds must be in [0.01, 60]");
  cudaStream_t s = (cudaStream_t)stream;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, kind == NGS_PEAK_FFMA ? peak_kernel<NGS_PEAK_FFMA>
                                     : kind == NGS_PEAK_FFMA2 ? peak_kernel<NGS_PEAK_FFMA2> : peak_kernel<NGS_PEAK_EX2>,
      kThreads, 0);
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  const unsigned blocks = (unsigned)(per_sm * ctx->num_sms);
  const int arc = ensure(ctx, ctx->flush, sizeof(float) * blocks * kThreads);
  if (arc != NGS_OK) return arc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(ctx, NGS_ERR_CUDA, "peak: cudaEventCreate failed");
  }
  // calibrate the iteration count on a short launch, then time launches of about `seconds` / 4 each
  int iters = 1024;
  float ms = 0.f;
  double best = 0.0;
  int rc = NGS_OK;
  for (int round = 0; round < 5 && rc == NGS_OK; ++round) {
    cudaEventRecord(e0, s);
    launch_peak(kind, ctx->flush.as<float>(), blocks, iters, s);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = fail(ctx, NGS_ERR_CUDA, std::string("peak: ") + cudaGetErrorString(e));
      break;
    }
    if (round > 0) best = std::max(best, ops_per_launch(kind, blocks, iters) / (ms * 1e-3));
    const double target_ms = 1e3 * seconds / 4.0;
    iters = (int)std::min(2.0e9, std::max(1024.0, iters * target_ms / std::max(ms, 1e-3f)));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != NGS_OK) return rc;
  ctx->launches += 5;
  *rate = best;
  return NGS_OK;
}
