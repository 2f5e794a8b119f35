// sphdvr_measure_fp32_peak: FP32 FMA throughput of the device, measured.
//
// The render path is bound by FP32/ALU issue, not by HBM or tensor cores, so
// its roofline denominator is the FP32 FMA rate.  This kernel runs eight
// independent FMA chains per thread on every resident thread of the device
// and is timed with CUDA events: the same clocks, power and thermal state the
// render kernel sees.  It sets no clock and no other device setting.
#include <algorithm>

#include "sphdvr_internal.h"

namespace sphdvr {
namespace {

constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(256) k_ffma_loop(int iters, float b, float c, float* sink) {
  float a[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
#pragma unroll 1
  for (int i = 0; i < iters; i += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += a[k];
  if (s == 1234.5678f) sink[threadIdx.x] = s;  // keeps the chains alive; practically never taken
}

}  // namespace
}  // namespace sphdvr

using namespace sphdvr;

extern "C" sphdvr_status sphdvr_measure_fp32_peak(sphdvr_ctx* ctx, void* stream, double* tflops) {
  if (!ctx || !tflops) return SPHDVR_EINVAL;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0, per_sm = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma_loop, 256, 0)) != cudaSuccess)
    return cuda_err(ctx, e, "fp32 peak: occupancy");
  const int grid = std::max(1, sms * per_sm);
  const int iters = 1 << 18;
  sphdvr_status s = ensure(ctx, ctx->work, 4 * sizeof(unsigned) + 256 * sizeof(float));
  if (s != SPHDVR_OK) return s;
  float* sink = (float*)((unsigned*)ctx->work.p + 4);
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_err(ctx, e, "fp32 peak: event");
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_err(ctx, e, "fp32 peak: event");
  }
  double best_ms = 1e30;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, st);
    k_ffma_loop<<<grid, 256, 0, st>>>(iters, 0.99999f, 1e-5f, sink);
    ++ctx->launches;
    cudaEventRecord(e1, st);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
    if (rep > 0) best_ms = std::min(best_ms, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_err(ctx, e, "fp32 peak: kernel");
  const double flop = 2.0 * kPeakChains * (double)iters * 256.0 * grid;
  *tflops = flop / (best_ms * 1e-3) / 1e12;
  return SPHDVR_OK;
}
