// Frame plans: every buffer of a frame allocated up front and the transfer
// function uploaded once, so that rendering a frame neither allocates,
// synchronises with the host nor copies from the host -- the frame can be
// captured into a CUDA graph and replayed.  The binning is capacity-bound:
// the chunk-tile pairs go into buffers of a fixed number of entries (the pair
// count is never read back), the unused entries are padded with the largest
// key and sorted along, and pairs beyond the capacity are dropped with a
// device flag set (sphdvr_frame_plan_overflowed).
#include <algorithm>
#include <new>

#include "sphdvr_internal.h"

struct sphdvr_frame_plan {
  sphdvr_ctx* ctx = nullptr;
  const sphdvr_dataset* ds = nullptr;
  const sphdvr_lut* lut = nullptr;
  sphdvr_render_opts opts{};
  bool has_opts = false;
  int tf_n = 0;
  float tf_lo = 0.f, tf_hi = 1.f;
  int max_w = 0, max_h = 0, grid = 0;
  size_t pair_cap = 0;
  sphdvr::DevBuf chunk_rect, chunk_front, chunk_ntile, chunk_off, pair_key, pair_val, pair_key2, pair_val2,
      tile_range, tmp, stats, tf, table, work, ovf, fb_table, fb_list;
  int fb_warps = 0;
};

namespace sphdvr {
namespace {

void plan_free(sphdvr_frame_plan* P) {
  DevBuf* bufs[] = {&P->chunk_rect, &P->chunk_front, &P->chunk_ntile, &P->chunk_off, &P->pair_key,
                    &P->pair_val,   &P->pair_key2,   &P->pair_val2,   &P->tile_range, &P->tmp,
                    &P->stats,      &P->tf,          &P->table,       &P->work,       &P->ovf,
                    &P->fb_table,   &P->fb_list};
  for (DevBuf* b : bufs)
    if (b->p) {
      cudaFree(b->p);
      b->p = nullptr;
      b->bytes = 0;
    }
}

RenderArgs plan_args(const sphdvr_frame_plan* P, const DevCamera& cam, float* out) {
  RenderArgs a{};
  a.ds = P->ds;
  a.lut = &P->lut->d;
  a.cam = cam;
  a.tf_n = P->tf_n;
  a.tf_lo = P->tf_lo;
  a.tf_hi = P->tf_hi;
  a.tf_host = nullptr;
  a.opts = P->has_opts ? &P->opts : nullptr;
  a.out = out;
  return a;
}

}  // namespace
}  // namespace sphdvr

using namespace sphdvr;

extern "C" {

sphdvr_status sphdvr_frame_plan_create(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                       const sphdvr_tf* tf, const sphdvr_render_opts* opts, int max_width,
                                       int max_height, int64_t pair_cap, sphdvr_frame_plan** out) {
  if (!ctx) return SPHDVR_EINVAL;
  if (!out) return set_err(ctx, SPHDVR_EINVAL, "frame_plan_create: out is NULL");
  *out = nullptr;
  sphdvr_status s = check_common(ctx, ds, lut);
  if (s != SPHDVR_OK) return s;
  if ((s = check_opts(ctx, opts)) != SPHDVR_OK || (s = reject_shading(ctx, opts, "frame_plan")) != SPHDVR_OK) return s;
  if (max_width < 1 || max_height < 1 || max_width > 32768 || max_height > 32768)
    return set_err(ctx, SPHDVR_EINVAL, "frame_plan_create: max size out of [1, 32768]");
  if (pair_cap < 2 || pair_cap > 0x7fffffffLL)
    return set_err(ctx, SPHDVR_EINVAL, "frame_plan_create: pair_cap out of [2, 2^31 - 1]");
  std::vector<float4> tfh;
  if ((s = pack_tf(ctx, tf, tfh)) != SPHDVR_OK) return s;
  sphdvr_frame_plan* P = new (std::nothrow) sphdvr_frame_plan();
  if (!P) return set_err(ctx, SPHDVR_ENOMEM, "frame_plan_create: out of host memory");
  P->ctx = ctx;
  P->ds = ds;
  P->lut = lut;
  if (opts) {
    P->opts = *opts;
    P->has_opts = true;
  }
  P->tf_n = tf->n;
  P->tf_lo = (float)tf->lo;
  P->tf_hi = (float)tf->hi;
  P->max_w = max_width;
  P->max_h = max_height;
  P->pair_cap = (size_t)pair_cap;
  // the render grid of the largest frame (also sets the kernel's shared-memory attribute)
  DevCamera big{};
  big.width = max_width;
  big.height = max_height;
  RenderArgs a = plan_args(P, big, nullptr);
  P->grid = render_grid(ctx, a);
  {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    P->fb_warps = sms > 0 ? sms : 1;  // fallback pass: one warp per SM
  }
  const size_t nc = (size_t)ds->n_chunks;
  const size_t tiles = (size_t)((max_width + kTile - 1) / kTile) * ((max_height + kTile - 1) / kTile);
  const size_t tmp_words = std::max(scan_tmp_words((int64_t)nc), sort_tmp_words(pair_cap));
  if ((s = ensure(ctx, P->chunk_rect, nc * sizeof(float4))) != SPHDVR_OK ||
      (s = ensure(ctx, P->chunk_front, nc * sizeof(unsigned))) != SPHDVR_OK ||
      (s = ensure(ctx, P->chunk_ntile, nc * sizeof(uint32_t) + 16)) != SPHDVR_OK ||
      (s = ensure(ctx, P->chunk_off, nc * sizeof(uint32_t) + 16)) != SPHDVR_OK ||
      (s = ensure(ctx, P->pair_key, P->pair_cap * 8)) != SPHDVR_OK ||
      (s = ensure(ctx, P->pair_val, P->pair_cap * 4)) != SPHDVR_OK ||
      (s = ensure(ctx, P->pair_key2, P->pair_cap * 8)) != SPHDVR_OK ||
      (s = ensure(ctx, P->pair_val2, P->pair_cap * 4)) != SPHDVR_OK ||
      (s = ensure(ctx, P->tile_range, tiles * sizeof(int2))) != SPHDVR_OK ||
      (s = ensure(ctx, P->tmp, tmp_words * sizeof(uint32_t))) != SPHDVR_OK ||
      (s = ensure(ctx, P->stats, 32 * sizeof(unsigned long long))) != SPHDVR_OK ||
      (s = ensure(ctx, P->tf, (size_t)P->tf_n * sizeof(float4))) != SPHDVR_OK ||
      (s = ensure(ctx, P->table, render_table_floats(P->grid, false) * sizeof(float))) != SPHDVR_OK ||
      (s = ensure(ctx, P->work, 4 * sizeof(unsigned))) != SPHDVR_OK ||
      (s = ensure(ctx, P->ovf, sizeof(unsigned))) != SPHDVR_OK ||
      (s = ensure(ctx, P->fb_table, fallback_floats(P->fb_warps) * sizeof(float))) != SPHDVR_OK ||
      (s = ensure(ctx, P->fb_list, (size_t)(kFallbackList + 1) * sizeof(unsigned))) != SPHDVR_OK) {
    plan_free(P);
    delete P;
    return s;
  }
  cudaError_t e = cudaMemcpy(P->tf.p, tfh.data(), (size_t)P->tf_n * sizeof(float4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(P->ovf.p, 0, sizeof(unsigned));
  if (e == cudaSuccess && !ctx->ev_ready) {
    // the render launch records these events; create them now rather than inside a capture
    e = cudaEventCreate(&ctx->ev_render0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev_render1);
    if (e == cudaSuccess) ctx->ev_ready = true;
  }
  if (e != cudaSuccess) {
    plan_free(P);
    delete P;
    return cuda_err(ctx, e, "frame_plan_create");
  }
  *out = P;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_frame_plan_render(sphdvr_frame_plan* P, const sphdvr_camera* cam, float* rgba_out,
                                       void* stream) {
  if (!P) return SPHDVR_EINVAL;
  sphdvr_ctx* ctx = P->ctx;
  if (!rgba_out) return set_err(ctx, SPHDVR_EINVAL, "frame_plan_render: rgba_out is NULL");
  DevCamera c;
  sphdvr_status s = check_camera(ctx, cam, &c);
  if (s != SPHDVR_OK) return s;
  if (c.width > P->max_w || c.height > P->max_h)
    return set_err(ctx, SPHDVR_EINVAL, "frame_plan_render: camera larger than the plan's maximum size");
  FrameWork w;
  w.chunk_rect = (float4*)P->chunk_rect.p;
  w.chunk_front = (unsigned*)P->chunk_front.p;
  w.chunk_ntile = (uint32_t*)P->chunk_ntile.p;
  w.chunk_off = (uint32_t*)P->chunk_off.p;
  w.pair_key = (uint64_t*)P->pair_key.p;
  w.pair_val = (uint32_t*)P->pair_val.p;
  w.pair_key2 = (uint64_t*)P->pair_key2.p;
  w.pair_val2 = (uint32_t*)P->pair_val2.p;
  w.pair_cap = P->pair_cap;
  w.tile_range = (int2*)P->tile_range.p;
  w.tmp = (uint32_t*)P->tmp.p;
  w.tmp_words = P->tmp.bytes / sizeof(uint32_t);
  w.stats = (unsigned long long*)P->stats.p;
  w.tf = (float4*)P->tf.p;
  w.table = (float*)P->table.p;
  w.table_ctas = P->grid;
  w.work = (unsigned*)P->work.p;
  w.fb_table = (float*)P->fb_table.p;
  w.fb_warps = P->fb_warps;
  w.fb_list = (unsigned*)P->fb_list.p;
  w.fb_cap = kFallbackList;
  const RenderArgs a = plan_args(P, c, rgba_out);
  return render_frame_planned(ctx, a, w, P->grid, (unsigned*)P->ovf.p, (cudaStream_t)stream);
}

sphdvr_status sphdvr_frame_plan_overflowed(sphdvr_frame_plan* P, int* overflowed) {
  if (!P || !overflowed) return SPHDVR_EINVAL;
  unsigned v = 0;
  cudaError_t e = cudaMemcpy(&v, P->ovf.p, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(P->ovf.p, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_err(P->ctx, e, "frame_plan_overflowed");
  *overflowed = v ? 1 : 0;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_frame_plan_destroy(sphdvr_frame_plan* P) {
  if (!P) return SPHDVR_EINVAL;
  cudaSetDevice(P->ctx->device);
  plan_free(P);
  delete P;
  return SPHDVR_OK;
}

}  // extern "C"
