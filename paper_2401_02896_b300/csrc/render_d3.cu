// Instantiations of the render kernel for polynomial degree D = 3.
#include "render.cuh"

namespace sphdvr {

template <typename S, int NW, bool DBG, bool RE, bool BT = false, bool QT = false>
static sphdvr_status launch(sphdvr_ctx* ctx, const RenderParams& p, int grid, size_t smem, cudaStream_t st) {
  auto kern = k_render<3, S, NW, DBG, RE, BT, QT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_err(ctx, e, "render smem attribute");
  if (!ctx->ev_ready) {
    if (cudaEventCreate(&ctx->ev_render0) != cudaSuccess || cudaEventCreate(&ctx->ev_render1) != cudaSuccess)
      return cuda_err(ctx, cudaGetLastError(), "render events");
    ctx->ev_ready = true;
  }
  cudaEventRecord(ctx->ev_render0, st);
  kern<<<grid, NW * 32, smem, st>>>(p);
  ++ctx->launches;
  cudaEventRecord(ctx->ev_render1, st);
  return cuda_err(ctx, cudaGetLastError(), "k_render");
}

template <typename S, int NW, bool DBG>
static int occupancy(size_t smem) {
  auto kern = k_render<3, S, NW, DBG, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NW * 32, smem) != cudaSuccess) return 0;
  return nb;
}

sphdvr_status launch_render_d3(sphdvr_ctx* ctx, bool f64, bool dbg, bool batch, bool qt, const RenderParams& p,
                                int grid, size_t smem, cudaStream_t st) {
  const bool re = p.reinit_dt > 0.f;  // FP32 only
  if (qt) {  // quantised path: integer knots and coefficients, FP32 compositing
    if (dbg) return launch<float, 1, true, false, false, true>(ctx, p, grid, smem, st);
    if (batch) return launch<float, kRenderWarps, false, false, true, true>(ctx, p, grid, smem, st);
    return launch<float, kRenderWarps, false, false, false, true>(ctx, p, grid, smem, st);
  }
  if (batch) {  // several frames, one work queue
    if (f64) return launch<double, kRenderWarps, false, false, true>(ctx, p, grid, smem, st);
    return re ? launch<float, kRenderWarps, false, true, true>(ctx, p, grid, smem, st)
              : launch<float, kRenderWarps, false, false, true>(ctx, p, grid, smem, st);
  }
  if (dbg) {
    if (f64) return launch<double, 1, true, false>(ctx, p, grid, smem, st);
    return re ? launch<float, 1, true, true>(ctx, p, grid, smem, st) : launch<float, 1, true, false>(ctx, p, grid, smem, st);
  }
  if (f64) return launch<double, kRenderWarps, false, false>(ctx, p, grid, smem, st);
  return re ? launch<float, kRenderWarps, false, true>(ctx, p, grid, smem, st)
            : launch<float, kRenderWarps, false, false>(ctx, p, grid, smem, st);
}

int render_occupancy_d3(bool f64, bool dbg, size_t smem) {
  if (dbg) return f64 ? occupancy<double, 1, true>(smem) : occupancy<float, 1, true>(smem);
  return f64 ? occupancy<double, kRenderWarps, false>(smem) : occupancy<float, kRenderWarps, false>(smem);
}

}  // namespace sphdvr
