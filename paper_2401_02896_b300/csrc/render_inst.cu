// Instantiations of the render kernels for one polynomial degree D.
//
// The build compiles this one file once per degree, with -DSPHDVR_D=1 ... 6,
// into separate objects (each holds the launchers launch_render_d<D> and
// render_occupancy_d<D>), so that the six degrees compile in parallel and
// share one source.
//
// Precision modes FP32_ANCHORED, FP32_NAIVE and FP32_KAHAN run the lean window
// kernel k_ray (ray.cuh); FP64_NAIVE, FP32_REINIT and INT64_QUANT run k_render
// (render.cuh), which carries their variants.
#include "ray.cuh"

#ifndef SPHDVR_D
#error "compile with -DSPHDVR_D=<degree>"
#endif

#define SPHDVR_CAT2(a, b) a##b
#define SPHDVR_CAT(a, b) SPHDVR_CAT2(a, b)

namespace sphdvr {
namespace {

constexpr int kD = SPHDVR_D;

sphdvr_status ensure_events(sphdvr_ctx* ctx) {
  if (!ctx->ev_ready) {
    if (cudaEventCreate(&ctx->ev_render0) != cudaSuccess || cudaEventCreate(&ctx->ev_render1) != cudaSuccess)
      return cuda_err(ctx, cudaGetLastError(), "render events");
    ctx->ev_ready = true;
  }
  return SPHDVR_OK;
}

// The render events bracket a frame's render kernels: a second pass (the
// fallback of k_ray) only moves the end event.
template <typename Kern>
sphdvr_status launch_kernel(sphdvr_ctx* ctx, Kern kern, int nw, const RenderParams& p, int grid, size_t smem,
                            cudaStream_t st, const char* name, bool second_pass = false) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_err(ctx, e, "render smem attribute");
  sphdvr_status s = ensure_events(ctx);
  if (s != SPHDVR_OK) return s;
  if (!second_pass) cudaEventRecord(ctx->ev_render0, st);
  kern<<<grid, nw * 32, smem, st>>>(p);
  ++ctx->launches;
  cudaEventRecord(ctx->ev_render1, st);
  return cuda_err(ctx, cudaGetLastError(), name);
}

template <typename S, int NW, bool DBG, bool RE, bool BT = false, bool QT = false>
sphdvr_status launch_old(sphdvr_ctx* ctx, const RenderParams& p, int grid, size_t smem, cudaStream_t st) {
  return launch_kernel(ctx, k_render<kD, S, NW, DBG, RE, BT, QT>, NW, p, grid, smem, st, "k_render");
}

template <int NW, bool DBG, bool BT, bool FB = false, bool GR = false, bool CP = false>
sphdvr_status launch_ray(sphdvr_ctx* ctx, const RenderParams& p, int grid, size_t smem, cudaStream_t st) {
  return launch_kernel(ctx, k_ray<kD, NW, DBG, BT, FB, GR, CP>, NW, p, grid, smem, st,
                       FB ? "k_ray fallback" : "k_ray", FB);
}

template <typename Kern>
int occupancy_of(Kern kern, int nw, size_t smem) {
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nw * 32, smem) != cudaSuccess) return 0;
  return nb;
}

}  // namespace

sphdvr_status SPHDVR_CAT(launch_render_d, SPHDVR_D)(sphdvr_ctx* ctx, int kind, bool dbg, bool batch,
                                                     const RenderParams& p, int grid, size_t smem, cudaStream_t st) {
  switch (kind) {
    case kKernRay:
      if (dbg) return launch_ray<1, true, false>(ctx, p, grid, smem, st);
      if (batch) return launch_ray<kRayWarps, false, true>(ctx, p, grid, smem, st);
      return launch_ray<kRayWarps, false, false>(ctx, p, grid, smem, st);
    case kKernRayFB:  // one warp per CTA, rays from the frame pass's list
      if (batch) return launch_ray<1, false, true, true>(ctx, p, grid, smem, st);
      return launch_ray<1, false, false, true>(ctx, p, grid, smem, st);
    case kKernRaySh:  // shaded: single frames and the parity hook
      if (batch) return set_err(ctx, SPHDVR_EINVAL, "render: shading is not available in batched launches");
      if (dbg) return launch_ray<1, true, false, false, true>(ctx, p, grid, smem, st);
      return launch_ray<kRayWarps, false, false, false, true>(ctx, p, grid, smem, st);
    case kKernRayShFB:
      if (batch) return set_err(ctx, SPHDVR_EINVAL, "render: shading is not available in batched launches");
      return launch_ray<1, false, false, true, true>(ctx, p, grid, smem, st);
    case kKernRayCp:  // compensated running sums
      if (dbg) return launch_ray<1, true, false, false, false, true>(ctx, p, grid, smem, st);
      if (batch) return launch_ray<kRayWarps, false, true, false, false, true>(ctx, p, grid, smem, st);
      return launch_ray<kRayWarps, false, false, false, false, true>(ctx, p, grid, smem, st);
    case kKernRayCpFB:
      if (batch) return launch_ray<1, false, true, true, false, true>(ctx, p, grid, smem, st);
      return launch_ray<1, false, false, true, false, true>(ctx, p, grid, smem, st);
    case kKernQuant:  // integer knots and coefficients, FP32 compositing
      if (dbg) return launch_old<float, 1, true, false, false, true>(ctx, p, grid, smem, st);
      if (batch) return launch_old<float, kRenderWarps, false, false, true, true>(ctx, p, grid, smem, st);
      return launch_old<float, kRenderWarps, false, false, false, true>(ctx, p, grid, smem, st);
    case kKernF64:  // FP64 running coefficients
      if (dbg) return launch_old<double, 1, true, false>(ctx, p, grid, smem, st);
      if (batch) return launch_old<double, kRenderWarps, false, false, true>(ctx, p, grid, smem, st);
      return launch_old<double, kRenderWarps, false, false>(ctx, p, grid, smem, st);
    case kKernReinit:  // FP32 with reinitialisation knots
      if (dbg) return launch_old<float, 1, true, true>(ctx, p, grid, smem, st);
      if (batch) return launch_old<float, kRenderWarps, false, true, true>(ctx, p, grid, smem, st);
      return launch_old<float, kRenderWarps, false, true>(ctx, p, grid, smem, st);
  }
  return set_err(ctx, SPHDVR_EINVAL, "render: unknown kernel kind");
}

int SPHDVR_CAT(render_occupancy_d, SPHDVR_D)(int kind, bool dbg, size_t smem) {
  switch (kind) {
    case kKernRay:
      return dbg ? occupancy_of(k_ray<kD, 1, true, false>, 1, smem)
                 : occupancy_of(k_ray<kD, kRayWarps, false, false>, kRayWarps, smem);
    case kKernRaySh:
      return dbg ? occupancy_of(k_ray<kD, 1, true, false, false, true>, 1, smem)
                 : occupancy_of(k_ray<kD, kRayWarps, false, false, false, true>, kRayWarps, smem);
    case kKernRayCp:
      return dbg ? occupancy_of(k_ray<kD, 1, true, false, false, false, true>, 1, smem)
                 : occupancy_of(k_ray<kD, kRayWarps, false, false, false, false, true>, kRayWarps, smem);
    case kKernQuant:
      return dbg ? occupancy_of(k_render<kD, float, 1, true, false, false, true>, 1, smem)
                 : occupancy_of(k_render<kD, float, kRenderWarps, false, false, false, true>, kRenderWarps, smem);
    case kKernF64:
      return dbg ? occupancy_of(k_render<kD, double, 1, true, false>, 1, smem)
                 : occupancy_of(k_render<kD, double, kRenderWarps, false, false>, kRenderWarps, smem);
    default:
      return dbg ? occupancy_of(k_render<kD, float, 1, true, true>, 1, smem)
                 : occupancy_of(k_render<kD, float, kRenderWarps, false, true>, kRenderWarps, smem);
  }
}

}  // namespace sphdvr
