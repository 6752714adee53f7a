// Measured FMA rates of the CUDA cores (FP64 DFMA, FP32 FFMA), used as the
// denominators of the roofline fractions of the FP64 path and of the
// CUDA-core share of the mixed path.  The paper has no counterpart: it
// reports GFLOP/s of its FP64 batched kernels (Sec. 8.1) without a peak.
//
// Every thread runs 8 independent FMA chains x = x * a + b (|a| < 1, so the
// values stay bounded and finite); the grid fills every SM with 8 CTAs of 256
// threads, enough warps and independent chains to keep the FMA pipes busy.
// Flops counted: 2 per FMA.
#include <cuda_runtime.h>

#include <algorithm>

#include "sbv_internal.cuh"

namespace sbv {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 16;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS)
fma_probe_kernel(T* out, int iters, T a, T b) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
      for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
static int run_probe(sbv_ctx* ctx, int iters, double* tflops) {
  int st = 0;
  const int grid = ctx->num_sms * 8;
  T* out = (T*)ws_get(ctx, WS_EXTRA, (size_t)grid * PROBE_THREADS * sizeof(T), &st);
  if (!out) return st;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SBV_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(s);
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cleanup();
    return fail(ctx, SBV_ECUDA, "cudaEventCreate");
  }
  const T a = (T)0.999999, b = (T)1e-6;
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {   // the first launch is a warm-up
    cudaEventRecord(e0, s);
    fma_probe_kernel<T><<<grid, PROBE_THREADS, 0, s>>>(out, iters, a, b);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      cleanup();
      return cuda_fail(ctx, e, "fma_probe_kernel");
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * (double)grid * PROBE_THREADS * PROBE_CHAINS * PROBE_UNROLL * iters;
    if (rep > 0 && ms > 0.0f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  cleanup();
  *tflops = best;
  return SBV_OK;
}

}  // namespace sbv

using namespace sbv;

extern "C" int sbv_peak_probe(sbv_ctx* ctx, int32_t kind, double* tflops) {
  if (!ctx || !tflops) return SBV_EINVAL;
  if (kind != 0 && kind != 1) return fail(ctx, SBV_EINVAL, "kind=%d: 0 (FP64) or 1 (FP32)", kind);
  SBV_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  // about 10-20 ms per launch on a GB300 at either precision
  return kind == 0 ? run_probe<double>(ctx, 256, tflops) : run_probe<float>(ctx, 8192, tflops);
}
