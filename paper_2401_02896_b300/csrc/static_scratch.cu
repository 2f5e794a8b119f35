// sphdvr_render_static_scratch: a render entry point that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they render: a
// serving loop whose memory is all handed to its own pool, a process that
// has reached its memory limit, or a latency-bound caller that cannot take the
// device-wide synchronisation a cudaMalloc or cudaFree may bring.  This entry
// point renders the same frame as sphdvr_render, through the same binning and
// render kernels, with every scratch buffer carved from one file-scope device
// array of fixed size instead of the context's grow-only buffers.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "sphdvr_internal.h"

namespace sphdvr {
namespace {

// Limits of the static scratch.
constexpr int64_t kStMaxChunks = int64_t(1) << 20;  // dataset chunks (<= 32 particles each)
constexpr int kStMaxTiles = 1 << 16;                // 16x16-pixel tiles (4096 x 4096 pixels)
constexpr size_t kStMaxPairs = size_t(1) << 21;     // chunk-tile pairs of one frame
constexpr int kStTableCtas = 64;                    // render CTAs whose per-ray scratch fits
constexpr int kStFbWarps = 16;                      // warps of the fallback pass
constexpr size_t kStBytes = size_t(192) << 20;      // 192 MiB
constexpr int kStMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStBytes];

std::mutex g_mu;
unsigned char* g_base[kStMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
sphdvr_status scratch_base(sphdvr_ctx* ctx, unsigned char** out) {
  if (ctx->device < 0 || ctx->device >= kStMaxDevices)
    return set_err(ctx, SPHDVR_EINVAL, "static scratch: device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_base[ctx->device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_err(ctx, e, "static scratch: cudaGetSymbolAddress");
    g_base[ctx->device] = (unsigned char*)p;
  }
  *out = g_base[ctx->device];
  return SPHDVR_OK;
}

struct Carver {
  unsigned char* base;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = (T*)(base + used);
    used += (count * sizeof(T) + 255) & ~size_t(255);
    return p;
  }
};

// Fixed layout of the array (independent of the frame).
sphdvr_status carve(sphdvr_ctx* ctx, unsigned char* base, FrameWork& w) {
  Carver c{base};
  w.chunk_rect = c.take<float4>(kStMaxChunks);
  w.chunk_front = c.take<unsigned>(kStMaxChunks);
  w.chunk_ntile = c.take<uint32_t>(kStMaxChunks + 4);
  w.chunk_off = c.take<uint32_t>(kStMaxChunks + 4);
  w.tile_range = c.take<int2>(kStMaxTiles);
  w.stats = c.take<unsigned long long>(32);
  w.tf = c.take<float4>(kMaxTf);
  w.work = c.take<unsigned>(4);
  w.pair_key = c.take<uint64_t>(kStMaxPairs);
  w.pair_key2 = c.take<uint64_t>(kStMaxPairs);
  w.pair_val = c.take<uint32_t>(kStMaxPairs);
  w.pair_val2 = c.take<uint32_t>(kStMaxPairs);
  w.pair_cap = kStMaxPairs;
  w.tmp_words = std::max(scan_tmp_words(kStMaxChunks), sort_tmp_words((int64_t)kStMaxPairs));
  w.tmp = c.take<uint32_t>(w.tmp_words);
  w.table_ctas = kStTableCtas;
  w.table = c.take<float>(render_table_floats(kStTableCtas, false));
  w.fb_warps = kStFbWarps;
  w.fb_table = c.take<float>(fallback_floats(kStFbWarps));
  w.fb_cap = kFallbackList;
  w.fb_list = c.take<unsigned>(kFallbackList + 1);
  if (c.used > kStBytes) return set_err(ctx, SPHDVR_EINVAL, "static scratch: layout exceeds the array");
  return SPHDVR_OK;
}

// Transfer-function validation and packing into a caller-provided array.
sphdvr_status pack_tf_fixed(sphdvr_ctx* ctx, const sphdvr_tf* tf, float4* out) {
  if (!tf || !tf->rgba) return set_err(ctx, SPHDVR_EINVAL, "transfer function is NULL");
  if (tf->n < 2 || tf->n > kMaxTf) return set_err(ctx, SPHDVR_EINVAL, "transfer function: n out of [2, 4096]");
  if (!(tf->lo < tf->hi) || !std::isfinite(tf->lo) || !std::isfinite(tf->hi))
    return set_err(ctx, SPHDVR_EINVAL, "transfer function: need finite lo < hi");
  if (!(tf->sigma_scale >= 0) || !std::isfinite(tf->sigma_scale))
    return set_err(ctx, SPHDVR_EINVAL, "transfer function: sigma_scale must be finite and >= 0");
  for (int i = 0; i < tf->n; ++i) {
    const float* v = tf->rgba + 4 * i;
    for (int k = 0; k < 4; ++k)
      if (!std::isfinite(v[k]) || v[k] < 0)
        return set_err(ctx, SPHDVR_EINVAL, "transfer function: entries must be finite and >= 0");
    out[i] = make_float4(v[0], v[1], v[2], (float)(v[3] * tf->sigma_scale));
  }
  return SPHDVR_OK;
}

}  // namespace
}  // namespace sphdvr

using namespace sphdvr;

extern "C" sphdvr_status sphdvr_render_static_scratch(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                                      const sphdvr_camera* cam, const sphdvr_tf* tf,
                                                      const sphdvr_render_opts* opts, float* rgba_out, void* stream) {
  if (!ctx) return SPHDVR_EINVAL;
  if (!rgba_out) return set_err(ctx, SPHDVR_EINVAL, "render_static_scratch: rgba_out is NULL");
  sphdvr_status s = check_common(ctx, ds, lut);
  if (s != SPHDVR_OK) return s;
  if ((s = check_opts(ctx, opts)) != SPHDVR_OK || (s = reject_shading(ctx, opts, "render_static_scratch")) != SPHDVR_OK) return s;
  RenderArgs a;
  a.ds = ds;
  a.lut = &lut->d;
  if ((s = check_camera(ctx, cam, &a.cam)) != SPHDVR_OK) return s;
  const int64_t tiles = (int64_t)((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
  if (tiles > kStMaxTiles)
    return set_err(ctx, SPHDVR_EINVAL, "render_static_scratch: " + std::to_string(tiles) +
                                           " tiles of 16x16 pixels; the static scratch holds at most 65536");
  if (ds->n_chunks > kStMaxChunks)
    return set_err(ctx, SPHDVR_EINVAL, "render_static_scratch: dataset has " + std::to_string(ds->n_chunks) +
                                           " chunks; the static scratch holds at most 1048576");
  float4 tfh[kMaxTf];
  if ((s = pack_tf_fixed(ctx, tf, tfh)) != SPHDVR_OK) return s;
  a.tf_n = tf->n;
  a.tf_lo = (float)tf->lo;
  a.tf_hi = (float)tf->hi;
  a.tf_host = tfh;
  a.opts = opts;
  a.out = rgba_out;
  unsigned char* base = nullptr;
  if ((s = scratch_base(ctx, &base)) != SPHDVR_OK) return s;
  FrameWork w;
  if ((s = carve(ctx, base, w)) != SPHDVR_OK) return s;
  ctx->frame_launch0 = ctx->launches;
  ctx->stats_pending = false;
  for (auto& v : ctx->last_stats) v = 0;
  s = render_frame_ws(ctx, a, w, nullptr, nullptr, (cudaStream_t)stream);
  if (s == SPHDVR_EOVERFLOW && ctx->last_pairs > (int64_t)kStMaxPairs)
    return set_err(ctx, SPHDVR_EOVERFLOW, "render_static_scratch: frame has " + std::to_string(ctx->last_pairs) +
                                              " chunk-tile pairs; the static scratch holds at most 2097152");
  if (s != SPHDVR_OK) return s;
  // the frame's counters and flags live in the static array until the next
  // call on it: sphdvr_frame_stats reads them from there
  ctx->last_stream = (cudaStream_t)stream;
  ctx->stats_src = w.stats;
  ctx->stats_pending = true;
  return SPHDVR_OK;
}
