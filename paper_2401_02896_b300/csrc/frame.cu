// Per-frame work: bin chunks into 16x16-pixel tiles, order each tile's chunks
// by a lower bound on every knot position their particles can produce on any
// ray through the tile, and launch the render kernel.
//
// Lower bound.  Let R be the table's largest outer knot theta_m (optimal outer
// knots may sit slightly beyond the support).  Perspective: a candidate at
// r = |chi - eye| > q h from the eye and d < q h from the ray has its first
// knot at t_chi - theta_m h with t_chi = sqrt(r^2 - d^2) >= r - d^2 / r >
// r - q^2 h^2 / r (and >= r - q h for any r), so every knot is above
// r - R h - min(q h, q^2 h^2 / r), which grows with r.  Orthographic: t_chi =
// (chi - eye).f on every ray.  Hence, with the chunk's tight box and h_max,
// front = dist(eye, box) - R h_max - min(q h_max, q^2 h_max^2 / dist), resp.
// min over the box of (x - eye).f - R h_max, bounds every knot of the chunk's
// particles from below; once a tile's chunks are consumed in order of front,
// every knot below the next chunk's front is final.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "ray.cuh"

namespace sphdvr {
namespace {

__device__ __forceinline__ unsigned f2ord(float x) {
  unsigned b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void k_chunk_project(int n_chunks, const float4* clo, const float4* chi, DevCamera cam, float q,
                                float reach, int tiles_x, int tiles_y, float4* rect, unsigned* front_ord,
                                uint32_t* ntile) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  float4 lo = clo[c], hi = chi[c];
  float rho = q * lo.w;          // a candidate's centre lies within rho of the ray
  float rfront = reach * lo.w;   // its knots lie within rfront of its t_chi
  float bl[3] = {lo.x - rho, lo.y - rho, lo.z - rho}, bh[3] = {hi.x + rho, hi.y + rho, hi.z + rho};
  float ex[3] = {(float)cam.eye[0], (float)cam.eye[1], (float)cam.eye[2]};
  float fr[3] = {(float)cam.f[0], (float)cam.f[1], (float)cam.f[2]};
  float rr[3] = {(float)cam.r[0], (float)cam.r[1], (float)cam.r[2]};
  float uu[3] = {(float)cam.u[0], (float)cam.u[1], (float)cam.u[2]};
  const float W = (float)cam.width, H = (float)cam.height;
  float x0 = 1e30f, x1 = -1e30f, y0 = 1e30f, y1 = -1e30f, front;
  bool full = false, behind = true;
  if (cam.proj == 0) {
    // distance from the eye to the tight box, minus the dilation
    float dd = 0.f;
    float lb[3] = {lo.x, lo.y, lo.z}, hb[3] = {hi.x, hi.y, hi.z};
    for (int k = 0; k < 3; ++k) {
      float d = fmaxf(fmaxf(lb[k] - ex[k], ex[k] - hb[k]), 0.f);
      dd += d * d;
    }
    float dist = sqrtf(dd);
    front = dist - rfront - (dist > rho ? rho * rho / dist : rho);
    front = front - 1e-5f * fabsf(front) - 1e-6f;
    const float sxk = 1.f / (float)(cam.tan_half * cam.aspect), syk = 1.f / (float)cam.tan_half;
    for (int i = 0; i < 8; ++i) {
      float p[3] = {(i & 1) ? bh[0] : bl[0], (i & 2) ? bh[1] : bl[1], (i & 4) ? bh[2] : bl[2]};
      float d0 = p[0] - ex[0], d1 = p[1] - ex[1], d2 = p[2] - ex[2];
      float z = d0 * fr[0] + d1 * fr[1] + d2 * fr[2];
      float x = d0 * rr[0] + d1 * rr[1] + d2 * rr[2];
      float y = d0 * uu[0] + d1 * uu[1] + d2 * uu[2];
      if (z > 0.f) behind = false;
      if (z <= 1e-6f * (fabsf(x) + fabsf(y) + 1e-3f)) { full = true; continue; }
      float px = (x / z * sxk + 1.f) * 0.5f * W - 0.5f;
      float py = (1.f - y / z * syk) * 0.5f * H - 0.5f;
      x0 = fminf(x0, px); x1 = fmaxf(x1, px); y0 = fminf(y0, py); y1 = fmaxf(y1, py);
    }
  } else {
    float zmin = 0.f;
    float lb[3] = {lo.x, lo.y, lo.z}, hb[3] = {hi.x, hi.y, hi.z};
    for (int k = 0; k < 3; ++k) zmin += fminf((lb[k] - ex[k]) * fr[k], (hb[k] - ex[k]) * fr[k]);
    front = zmin - rfront;
    front = front - 1e-5f * fabsf(front) - 1e-6f;
    behind = false;
    const float sxk = 1.f / (float)cam.half_w, syk = 1.f / (float)cam.half_h;
    for (int i = 0; i < 8; ++i) {
      float p[3] = {(i & 1) ? bh[0] : bl[0], (i & 2) ? bh[1] : bl[1], (i & 4) ? bh[2] : bl[2]};
      float d0 = p[0] - ex[0], d1 = p[1] - ex[1], d2 = p[2] - ex[2];
      float x = d0 * rr[0] + d1 * rr[1] + d2 * rr[2];
      float y = d0 * uu[0] + d1 * uu[1] + d2 * uu[2];
      float px = (x * sxk + 1.f) * 0.5f * W - 0.5f;
      float py = (1.f - y * syk) * 0.5f * H - 0.5f;
      x0 = fminf(x0, px); x1 = fmaxf(x1, px); y0 = fminf(y0, py); y1 = fmaxf(y1, py);
    }
  }
  uint32_t cnt = 0;
  if (behind) {
    x0 = 1.f; x1 = -1.f; y0 = 1.f; y1 = -1.f;
  } else {
    if (full) { x0 = -1.f; y0 = -1.f; x1 = W; y1 = H; }
    // conservative margin for FP32 rounding of the projection
    float mx = 1.f + 1e-4f * (fabsf(x0) + fabsf(x1)), my = 1.f + 1e-4f * (fabsf(y0) + fabsf(y1));
    x0 -= mx; x1 += mx; y0 -= my; y1 += my;
    if (x1 >= 0.f && y1 >= 0.f && x0 <= W - 1.f && y0 <= H - 1.f) {
      int tx0 = max(0, (int)floorf(x0 / kTile)), tx1 = min(tiles_x - 1, (int)floorf(x1 / kTile));
      int ty0 = max(0, (int)floorf(y0 / kTile)), ty1 = min(tiles_y - 1, (int)floorf(y1 / kTile));
      if (tx1 >= tx0 && ty1 >= ty0) cnt = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
    }
  }
  rect[c] = make_float4(x0, y0, x1, y1);
  front_ord[c] = f2ord(front);
  ntile[c] = cnt;
}

// cap: pairs beyond it are dropped (capacity-bound binning sets *ovf instead)
__global__ void k_emit_pairs(int n_chunks, const float4* rect, const unsigned* front_ord, const uint32_t* ntile,
                             const uint32_t* off, int tiles_x, int tiles_y, uint64_t* keys, uint32_t* vals,
                             uint32_t cap, unsigned* ovf) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  uint32_t n = ntile[c];
  if (!n) return;
  if ((uint64_t)off[c] + n > cap) {
    if (ovf) atomicOr(ovf, 1u);
    n = off[c] < cap ? cap - off[c] : 0;
  }
  float4 r = rect[c];
  int tx0 = max(0, (int)floorf(r.x / kTile)), tx1 = min(tiles_x - 1, (int)floorf(r.z / kTile));
  int ty0 = max(0, (int)floorf(r.y / kTile));
  int w = tx1 - tx0 + 1;
  uint32_t o = off[c];
  uint64_t fo = front_ord[c];
  for (uint32_t i = 0; i < n; ++i) {
    int tx = tx0 + (int)(i % w), ty = ty0 + (int)(i / w);
    keys[o + i] = ((uint64_t)(ty * tiles_x + tx) << 32) | fo;
    vals[o + i] = (uint32_t)c;
  }
}

// [first, end) of each tile's pairs, as indices into the pair arrays that
// start `base` entries before `keys`
// Capacity-bound binning: the entries [min(*total, cap), cap) get the largest
// key, so that a sort of all cap entries leaves the frame's pairs in front.
__global__ void k_pad_pairs(const uint32_t* total, uint32_t cap, uint64_t* keys, uint32_t* vals) {
  const uint32_t n = min(*total, cap);
  for (uint32_t i = n + blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
    keys[i] = ~0ull;
    vals[i] = 0;
  }
}

// k_tile_ranges for the first min(*total, cap) of cap sorted entries
__global__ void k_tile_ranges_dev(const uint32_t* total, uint32_t cap, const uint64_t* keys, int2* range) {
  const int64_t n = min(*total, cap);
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int t = (int)(keys[i] >> 32);
  if (i == 0 || (int)(keys[i - 1] >> 32) != t) range[t].x = (int)i;
  if (i == n - 1 || (int)(keys[i + 1] >> 32) != t) range[t].y = (int)(i + 1);
}

__global__ void k_tile_ranges(int64_t n, const uint64_t* keys, int2* range, int base) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int t = (int)(keys[i] >> 32);
  if (i == 0 || (int)(keys[i - 1] >> 32) != t) range[t].x = base + (int)i;
  if (i == n - 1 || (int)(keys[i + 1] >> 32) != t) range[t].y = base + (int)(i + 1);
}

}  // namespace

// per-degree launchers (render_inst.cu, compiled once per degree)
#define SPHDVR_DECL(D)                                                                                         \
  sphdvr_status launch_render_d##D(sphdvr_ctx* ctx, int kind, bool dbg, bool batch, const RenderParams& p,   \
                                   int grid, size_t smem, cudaStream_t st);                                  \
  int render_occupancy_d##D(int kind, bool dbg, size_t smem);
SPHDVR_DECL(1)
SPHDVR_DECL(2)
SPHDVR_DECL(3)
SPHDVR_DECL(4)
SPHDVR_DECL(5)
SPHDVR_DECL(6)
#undef SPHDVR_DECL

// The render kernel of a precision mode (and of shaded rendering).
static int kernel_kind(const sphdvr_render_opts* o) {
  if (o && o->shading) return kKernRaySh;
  switch (o ? o->precision : SPHDVR_PREC_FP32_ANCHORED) {
    case SPHDVR_PREC_FP64_NAIVE: return kKernF64;
    case SPHDVR_PREC_FP32_REINIT: return kKernReinit;
    case SPHDVR_PREC_INT64_QUANT: return kKernQuant;
    case SPHDVR_PREC_FP32_KAHAN: return kKernRayCp;
    default: return kKernRay;
  }
}

// Dynamic shared memory of a render launch.
static size_t kernel_smem(int kind, int tf_n, bool dbg) {
  if (kind == kKernRayFB || kind == kKernRayShFB || kind == kKernRayCpFB)
    return ray_smem_bytes(tf_n, 1, true, kind == kKernRayShFB);
  const bool ray = kind == kKernRay || kind == kKernRaySh || kind == kKernRayCp;
  const int nw = dbg ? 1 : (ray ? kRayWarps : kRenderWarps);
  return ray ? ray_smem_bytes(tf_n, nw, dbg, kind == kKernRaySh) : render_smem_bytes(tf_n, nw);
}

static sphdvr_status dispatch_render(sphdvr_ctx* ctx, int D, int kind, bool dbg, bool batch, const RenderParams& p,
                                     int grid, size_t smem, cudaStream_t st) {
  switch (D) {
    case 1: return launch_render_d1(ctx, kind, dbg, batch, p, grid, smem, st);
    case 2: return launch_render_d2(ctx, kind, dbg, batch, p, grid, smem, st);
    case 3: return launch_render_d3(ctx, kind, dbg, batch, p, grid, smem, st);
    case 4: return launch_render_d4(ctx, kind, dbg, batch, p, grid, smem, st);
    case 5: return launch_render_d5(ctx, kind, dbg, batch, p, grid, smem, st);
    case 6: return launch_render_d6(ctx, kind, dbg, batch, p, grid, smem, st);
  }
  return set_err(ctx, SPHDVR_EINVAL, "D out of range");
}

static int render_occupancy(int D, int kind, bool dbg, size_t smem) {
  switch (D) {
    case 1: return render_occupancy_d1(kind, dbg, smem);
    case 2: return render_occupancy_d2(kind, dbg, smem);
    case 3: return render_occupancy_d3(kind, dbg, smem);
    case 4: return render_occupancy_d4(kind, dbg, smem);
    case 5: return render_occupancy_d5(kind, dbg, smem);
    case 6: return render_occupancy_d6(kind, dbg, smem);
  }
  return 0;
}

static int frame_tiles(const DevCamera& c) { return ((c.width + kTile - 1) / kTile) * ((c.height + kTile - 1) / kTile); }

// Persistent grid: resident CTAs on every SM, no more CTAs than work items.
static int grid_for_items(sphdvr_ctx* ctx, const RenderArgs& a, int64_t items) {
  const bool dbg = a.n_dbg > 0;
  const int kind = kernel_kind(a.opts);
  const size_t smem = kernel_smem(kind, a.tf_n, dbg);
  int nb = render_occupancy(a.lut->D, kind, dbg, smem);
  if (!dbg && a.opts && a.opts->ctas_per_sm > 0) nb = std::min(nb, a.opts->ctas_per_sm);
  if (ctx->num_sms <= 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device);
    ctx->num_sms = n > 0 ? n : 1;
  }
  const int64_t grid = (int64_t)std::max(1, nb) * ctx->num_sms;
  return (int)std::max<int64_t>(1, std::min(grid, items));
}

int render_grid(sphdvr_ctx* ctx, const RenderArgs& a) {
  const int64_t items = a.n_dbg > 0 ? a.n_dbg
                                    : ((int64_t)frame_tiles(a.cam) * kTile * kTile + kRenderWarps - 1) / kRenderWarps;
  return grid_for_items(ctx, a, items);
}

int render_grid_batch(sphdvr_ctx* ctx, const RenderArgs* a, int n) {
  int64_t rays = 0;
  for (int f = 0; f < n; ++f) rays += (int64_t)frame_tiles(a[f].cam) * kTile * kTile;
  return grid_for_items(ctx, a[0], (rays + kRenderWarps - 1) / kRenderWarps);
}

size_t render_table_floats(int grid, bool dbg, bool shaded) {
  static_assert(kRayWarps == kRenderWarps, "both render kernels run the same warps per CTA");
  // the parity hook runs k_ray with the fallback's larger per-ray capacities
  const int ray = shaded ? (dbg ? kRayWordsBigGR : kRayWordsGR) : (dbg ? kRayWordsBig : kRayWords);
  return (size_t)grid * (dbg ? 1 : kRenderWarps) * (size_t)std::max(kTableWords, ray);
}

size_t fallback_floats(int warps, bool shaded) { return (size_t)warps * (shaded ? kRayWordsBigGR : kRayWordsBig); }

// warps of the fallback pass (one per SM)
static int fallback_warps(sphdvr_ctx* ctx) {
  if (ctx->num_sms <= 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device);
    ctx->num_sms = n > 0 ? n : 1;
  }
  return ctx->num_sms;
}

// grow the context's pair buffers once the pair count is known
sphdvr_status ctx_pair_sizer(sphdvr_ctx* ctx, FrameWork& w, size_t pairs, void*) {
  const size_t np = std::max<size_t>(pairs, 1);
  sphdvr_status s;
  if ((s = ensure(ctx, ctx->pair_key, np * 8)) != SPHDVR_OK || (s = ensure(ctx, ctx->pair_val, np * 4)) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->pair_key2, np * 8)) != SPHDVR_OK || (s = ensure(ctx, ctx->pair_val2, np * 4)) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->sort_tmp, sort_tmp_words((int64_t)np) * sizeof(uint32_t))) != SPHDVR_OK)
    return s;
  w.pair_key = (uint64_t*)ctx->pair_key.p;
  w.pair_val = (uint32_t*)ctx->pair_val.p;
  w.pair_key2 = (uint64_t*)ctx->pair_key2.p;
  w.pair_val2 = (uint32_t*)ctx->pair_val2.p;
  w.pair_cap = np;
  w.tmp = (uint32_t*)ctx->sort_tmp.p;
  w.tmp_words = ctx->sort_tmp.bytes / sizeof(uint32_t);
  return SPHDVR_OK;
}

// size of a grow-only buffer after ensure(b, bytes)
static size_t grown(const DevBuf& b, size_t bytes) {
  return (b.bytes >= bytes && b.p) ? b.bytes : bytes + bytes / 4 + 256;
}

size_t held_after_pair_sizer(const sphdvr_ctx* ctx, size_t pairs) {
  const size_t np = std::max<size_t>(pairs, 1);
  const DevBuf* b[] = {&ctx->pair_key, &ctx->pair_val, &ctx->pair_key2, &ctx->pair_val2, &ctx->sort_tmp};
  const size_t want[] = {np * 8, np * 4, np * 8, np * 4, sort_tmp_words((int64_t)np) * sizeof(uint32_t)};
  size_t t = ctx_held_bytes(ctx);
  for (int i = 0; i < 5; ++i) t = t - b[i]->bytes + grown(*b[i], want[i]);
  return t;
}

size_t pair_bytes(size_t pairs) {
  const size_t np = std::max<size_t>(pairs, 1);
  return np * 24 + sort_tmp_words((int64_t)np) * sizeof(uint32_t);
}

// Bytes shared by the frames of a batch (chunk scratch, statistics, table
// scratch of the grid, transfer function, work counter, frame records, the
// fallback pass's scratch and list).
static size_t shared_fixed_bytes(const RenderArgs& a, int grid, int n, int ctx_fallback_warps) {
  const size_t nc = a.ds->n_chunks;
  return nc * (sizeof(unsigned) + 2 * sizeof(uint32_t)) + 32 + 32 * sizeof(unsigned long long) +
         scan_tmp_words(nc) * sizeof(uint32_t) + (size_t)a.tf_n * sizeof(float4) +
         render_table_floats(grid, a.n_dbg > 0, a.opts && a.opts->shading) * sizeof(float) + 4 * sizeof(unsigned) +
         (n > 1 ? (size_t)n * sizeof(RenderFrame) : 0) + (size_t)(kFallbackList + 1) * sizeof(unsigned) +
         fallback_floats(ctx_fallback_warps, a.opts && a.opts->shading) * sizeof(float);
}

size_t frame_fixed_bytes(sphdvr_ctx* ctx, const RenderArgs& a) {
  return (size_t)a.ds->n_chunks * sizeof(float4) + (size_t)frame_tiles(a.cam) * sizeof(int2) +
         shared_fixed_bytes(a, render_grid(ctx, a), 1, fallback_warps(ctx));
}

size_t batch_fixed_bytes(sphdvr_ctx* ctx, const RenderArgs* a, int n) {
  size_t t = shared_fixed_bytes(a[0], render_grid_batch(ctx, a, n), n, fallback_warps(ctx)) +
             (size_t)n * a[0].ds->n_chunks * sizeof(float4);
  for (int f = 0; f < n; ++f) t += (size_t)frame_tiles(a[f].cam) * sizeof(int2);
  return t;
}

sphdvr_status render_frame(sphdvr_ctx* ctx, const RenderArgs& a, cudaStream_t st) {
  return render_frame_sized(ctx, a, st, ctx_pair_sizer, nullptr);
}

// Grow the buffers the frames of a batch share and point `w` at them.
static sphdvr_status shared_work(sphdvr_ctx* ctx, const RenderArgs& a, int grid, FrameWork& w) {
  const int nc = a.ds->n_chunks;
  sphdvr_status s;
  if ((s = ensure(ctx, ctx->chunk_front, (size_t)nc * sizeof(unsigned))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->chunk_ntile, (size_t)nc * sizeof(uint32_t) + 16)) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->chunk_off, (size_t)nc * sizeof(uint32_t) + 16)) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->stats, 32 * sizeof(unsigned long long))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->scan_tmp, scan_tmp_words(nc) * sizeof(uint32_t))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->tf, (size_t)a.tf_n * sizeof(float4))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->table, render_table_floats(grid, a.n_dbg > 0, a.opts && a.opts->shading) * sizeof(float))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->work, 4 * sizeof(unsigned))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->fb_table, fallback_floats(fallback_warps(ctx), a.opts && a.opts->shading) * sizeof(float))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->fb_list, (size_t)(kFallbackList + 1) * sizeof(unsigned))) != SPHDVR_OK)
    return s;
  w.fb_table = (float*)ctx->fb_table.p;
  w.fb_warps = fallback_warps(ctx);
  w.fb_list = (unsigned*)ctx->fb_list.p;
  w.fb_cap = kFallbackList;
  w.table = (float*)ctx->table.p;
  w.table_ctas = grid;
  w.work = (unsigned*)ctx->work.p;
  w.chunk_front = (unsigned*)ctx->chunk_front.p;
  w.chunk_ntile = (uint32_t*)ctx->chunk_ntile.p;
  w.chunk_off = (uint32_t*)ctx->chunk_off.p;
  w.stats = (unsigned long long*)ctx->stats.p;
  w.tf = (float4*)ctx->tf.p;
  w.tmp = (uint32_t*)ctx->scan_tmp.p;
  w.tmp_words = ctx->scan_tmp.bytes / sizeof(uint32_t);
  return SPHDVR_OK;
}

// Grow the chunk rectangles (n_rect frames) and tile ranges (tiles) and point `w` at them.
static sphdvr_status rect_range_work(sphdvr_ctx* ctx, const RenderArgs& a, int n_rect, int64_t tiles, FrameWork& w) {
  sphdvr_status s;
  if ((s = ensure(ctx, ctx->chunk_rect, (size_t)n_rect * a.ds->n_chunks * sizeof(float4))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->tile_range, (size_t)tiles * sizeof(int2))) != SPHDVR_OK)
    return s;
  w.chunk_rect = (float4*)ctx->chunk_rect.p;
  w.tile_range = (int2*)ctx->tile_range.p;
  return SPHDVR_OK;
}

sphdvr_status render_frame_sized(sphdvr_ctx* ctx, const RenderArgs& a, cudaStream_t st, PairSizer sizer, void* user) {
  FrameWork w;
  sphdvr_status s;
  if ((s = shared_work(ctx, a, render_grid(ctx, a), w)) != SPHDVR_OK ||
      (s = rect_range_work(ctx, a, 1, frame_tiles(a.cam), w)) != SPHDVR_OK)
    return s;
  return render_frame_ws(ctx, a, w, sizer, user, st);
}

// Binning, first half: project the chunks into the frame (rectangles into
// `rect`, fronts and tile counts into w's chunk scratch) and scan the counts
// into offsets; with `total` non-null, read the frame's pair count back.
static sphdvr_status project_frame(sphdvr_ctx* ctx, const RenderArgs& a, float4* rect, const FrameWork& w,
                                   cudaStream_t st, uint32_t* total) {
  const sphdvr_dataset* ds = a.ds;
  const int tiles_x = (a.cam.width + kTile - 1) / kTile, tiles_y = (a.cam.height + kTile - 1) / kTile;
  const int nc = ds->n_chunks;
  cudaError_t e;
  k_chunk_project<<<(nc + 255) / 256, 256, 0, st>>>(nc, ds->chunk_lo, ds->chunk_hi, a.cam, a.lut->q, a.lut->reach,
                                                    tiles_x, tiles_y, rect, w.chunk_front, w.chunk_ntile);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_chunk_project");
  uint32_t* d_total = w.chunk_off + nc;
  if (w.tmp_words < scan_tmp_words(nc)) return set_err(ctx, SPHDVR_EOVERFLOW, "frame scratch too small for the scan");
  sphdvr_status s = scan_exclusive_u32(ctx, w.chunk_ntile, w.chunk_off, nc, d_total, w.tmp, st);
  if (s != SPHDVR_OK || !total) return s;
  if ((e = cudaMemcpyAsync(total, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_err(ctx, e, "pair count");
  return SPHDVR_OK;
}

// Binning, second half: emit the frame's `total` chunk-tile pairs at entry
// `base` of w's pair arrays, sort them by (tile, front) and write each tile's
// range (indices into the pair arrays) to `trange`.
static sphdvr_status sort_frame(sphdvr_ctx* ctx, const RenderArgs& a, const float4* rect, const FrameWork& w,
                                uint32_t total, int64_t base, int2* trange, cudaStream_t st) {
  const int tiles_x = (a.cam.width + kTile - 1) / kTile, tiles_y = (a.cam.height + kTile - 1) / kTile;
  const int n_tiles = tiles_x * tiles_y;
  const int nc = a.ds->n_chunks;
  cudaError_t e;
  if ((int64_t)w.pair_cap < base + total || w.tmp_words < sort_tmp_words(total))
    return set_err(ctx, SPHDVR_EOVERFLOW, "frame scratch too small for " + std::to_string(total) + " chunk-tile pairs");
  uint64_t* keys = w.pair_key + base;
  uint32_t* vals = w.pair_val + base;
  k_emit_pairs<<<(nc + 255) / 256, 256, 0, st>>>(nc, rect, w.chunk_front, w.chunk_ntile, w.chunk_off, tiles_x,
                                                 tiles_y, keys, vals, 0xffffffffu, nullptr);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_emit_pairs");
  int tbits = 0;
  while ((1 << tbits) < n_tiles) ++tbits;
  sphdvr_status s = radix_sort_u64(ctx, keys, vals, w.pair_key2, w.pair_val2, total, 32 + tbits, w.tmp, st);
  if (s != SPHDVR_OK) return s;
  if ((e = cudaMemsetAsync(trange, 0, (size_t)n_tiles * sizeof(int2), st)) != cudaSuccess)
    return cuda_err(ctx, e, "tile range memset");
  if (total) {
    k_tile_ranges<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(total, keys, trange, (int)base);
    ++ctx->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_tile_ranges");
  }
  return SPHDVR_OK;
}

// Kernel parameters common to every frame of a launch (data, table, transfer
// function, options, scratch).
static void common_params(const RenderArgs& a, const FrameWork& w, RenderParams& p) {
  const sphdvr_dataset* ds = a.ds;
  const DevLut* L = a.lut;
  std::memset(&p, 0, sizeof(p));
  p.pos = ds->pos;
  p.amp = ds->amp;
  p.orig = ds->orig;
  p.chunk = ds->chunk;
  p.chunk_lo = ds->chunk_lo;
  p.chunk_hi = ds->chunk_hi;
  p.K = L->K;
  p.m = L->m;
  p.n_lambda = L->n_lambda;
  p.q = L->q;
  p.lam_scale = (float)((L->n_lambda - 1) / (double)L->q);
  p.theta = L->theta;
  p.jump = L->jump;
  p.piece = L->piece;
  p.gjump = L->gjump;
  p.gpiece = L->gpiece;
  p.shade_ka = (a.opts && a.opts->shading) ? a.opts->shade_ka : 1.f;
  p.shade_kd = (a.opts && a.opts->shading) ? a.opts->shade_kd : 0.f;
  p.shade_g2 = (a.opts && a.opts->shading) ? a.opts->shade_g0 * a.opts->shade_g0 : 0.f;
  p.tf_n = a.tf_n;
  p.tf_lo = a.tf_lo;
  p.tf_dv = (a.tf_hi - a.tf_lo) / (a.tf_n - 1);
  p.tf_inv_dv = (float)((a.tf_n - 1) / ((double)a.tf_hi - (double)a.tf_lo));
  p.tf = w.tf;
  const sphdvr_render_opts* o = a.opts;
  int prec = o ? o->precision : SPHDVR_PREC_FP32_ANCHORED;
  p.anchor_every = (prec == SPHDVR_PREC_FP32_ANCHORED) ? std::max(1, o ? o->anchor_every : 2) : 0;
  p.window_h = (o && o->window_h > 0.f) ? o->window_h : 1.0f;
  p.window_fill = (o && o->window_fill > 0.f) ? o->window_fill : 0.85f;
  p.reinit_dt = (prec == SPHDVR_PREC_FP32_REINIT) ? o->reinit_dt : 0.f;
  const bool qt = prec == SPHDVR_PREC_INT64_QUANT;
  p.q_tau = qt ? o->quant_tau : 1.0;
  p.q_inv_tau = 1.0 / p.q_tau;
  p.q_sigma = qt ? o->quant_sigma : 1.0;
  float eps = o ? o->ert_eps : 1e-5f;
  p.tau_ert = eps > 0.f ? -std::log(eps) : 0.f;
  p.stats = w.stats;
  p.scratch = w.table;
  p.work = w.work;
  p.dynamic = o ? (o->persistent ? 1 : 0) : 1;
}

static sphdvr_status upload_tf(sphdvr_ctx* ctx, const RenderArgs& a, const FrameWork& w, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(w.tf, a.tf_host, (size_t)a.tf_n * sizeof(float4), cudaMemcpyHostToDevice, st);
  return e == cudaSuccess ? SPHDVR_OK : cuda_err(ctx, e, "transfer function upload");
}

static sphdvr_status clear_counters(sphdvr_ctx* ctx, const FrameWork& w, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.stats, 0, 32 * sizeof(unsigned long long), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(w.work, 0, sizeof(unsigned), st)) != cudaSuccess ||
      (w.fb_list && (e = cudaMemsetAsync(w.fb_list, 0, sizeof(unsigned), st)) != cudaSuccess))
    return cuda_err(ctx, e, "stats memset");
  return SPHDVR_OK;
}

// The frame pass of k_ray and, after it, the fallback pass over the rays it
// abandoned (a launch that ends at once when there are none).
static sphdvr_status launch_frame(sphdvr_ctx* ctx, const RenderArgs& a, const FrameWork& w, RenderParams p,
                                  bool batch, int grid, cudaStream_t st) {
  const int kind = kernel_kind(a.opts);
  const bool fb = (kind == kKernRay || kind == kKernRaySh || kind == kKernRayCp) && w.fb_table && w.fb_list &&
                  w.fb_warps > 0;
  p.ray_cap = a.opts ? a.opts->ray_capacity : 0;
  p.ovf = fb ? w.fb_list : nullptr;
  p.ovf_cap = fb ? w.fb_cap : 0;
  sphdvr_status s =
      dispatch_render(ctx, a.lut->D, kind, false, batch, p, grid, kernel_smem(kind, a.tf_n, false), st);
  if (s != SPHDVR_OK || !fb) return s;
  p.scratch = w.fb_table;
  const int fk = kind == kKernRaySh ? kKernRayShFB : (kind == kKernRayCp ? kKernRayCpFB : kKernRayFB);
  return dispatch_render(ctx, a.lut->D, fk, false, batch, p, w.fb_warps, kernel_smem(fk, a.tf_n, false), st);
}

sphdvr_status render_frame_ws(sphdvr_ctx* ctx, const RenderArgs& a, FrameWork& w, PairSizer sizer, void* user,
                              cudaStream_t st) {
  sphdvr_status s;
  uint32_t pairs = 0;
  if ((s = upload_tf(ctx, a, w, st)) != SPHDVR_OK || (s = project_frame(ctx, a, w.chunk_rect, w, st, &pairs)) != SPHDVR_OK)
    return s;
  ctx->last_pairs = pairs;
  if (sizer && (s = sizer(ctx, w, pairs, user)) != SPHDVR_OK) return s;
  if ((s = sort_frame(ctx, a, w.chunk_rect, w, pairs, 0, w.tile_range, st)) != SPHDVR_OK ||
      (s = clear_counters(ctx, w, st)) != SPHDVR_OK)
    return s;
  RenderParams p;
  common_params(a, w, p);
  p.cam = a.cam;
  p.chunk_rect = w.chunk_rect;
  p.pair_key = w.pair_key;
  p.pair_val = w.pair_val;
  p.tile_range = w.tile_range;
  p.tiles_x = (a.cam.width + kTile - 1) / kTile;
  p.tiles_y = (a.cam.height + kTile - 1) / kTile;
  p.out = a.out;
  p.n_items = frame_tiles(a.cam) * kTile * kTile;
  p.n_dbg = a.n_dbg;
  p.dbg_pix = a.dbg_pix;
  p.dbg_rgba = a.dbg_rgba;
  p.dbg_counts = a.dbg_counts;
  p.dbg_cands = a.dbg_cands;
  p.cand_cap = a.cand_cap;
  p.dbg_field = a.dbg_field;
  p.field_cap = a.field_cap;
  p.dbg_grad = a.dbg_grad;
  const bool dbg = a.n_dbg > 0;
  const int kind = kernel_kind(a.opts);
  const int grid = std::min(render_grid(ctx, a), w.table_ctas);
  if (!dbg) return launch_frame(ctx, a, w, p, false, grid, st);
  return dispatch_render(ctx, a.lut->D, kind, true, false, p, grid, kernel_smem(kind, a.tf_n, true), st);
}

sphdvr_status project_chunk_rects(sphdvr_ctx* ctx, const RenderArgs& a, float4* rect, unsigned* front, uint32_t* ntile,
                                  cudaStream_t st) {
  const int tiles_x = (a.cam.width + kTile - 1) / kTile, tiles_y = (a.cam.height + kTile - 1) / kTile;
  const int nc = a.ds->n_chunks;
  k_chunk_project<<<(nc + 255) / 256, 256, 0, st>>>(nc, a.ds->chunk_lo, a.ds->chunk_hi, a.cam, a.lut->q, a.lut->reach,
                                                    tiles_x, tiles_y, rect, front, ntile);
  ++ctx->launches;
  return cuda_err(ctx, cudaGetLastError(), "k_chunk_project");
}

sphdvr_status render_frame_planned(sphdvr_ctx* ctx, const RenderArgs& a, const FrameWork& w, int grid, unsigned* ovf,
                                   cudaStream_t st) {
  const sphdvr_dataset* ds = a.ds;
  const int tiles_x = (a.cam.width + kTile - 1) / kTile, tiles_y = (a.cam.height + kTile - 1) / kTile;
  const int n_tiles = tiles_x * tiles_y;
  const int nc = ds->n_chunks;
  const uint32_t cap = (uint32_t)std::min<size_t>(w.pair_cap, 0xffffffffu);
  if (cap < 2 || w.tmp_words < sort_tmp_words(cap)) return set_err(ctx, SPHDVR_EINVAL, "plan: pair buffers too small");
  sphdvr_status s;
  cudaError_t e;
  if ((s = project_frame(ctx, a, w.chunk_rect, w, st, nullptr)) != SPHDVR_OK) return s;
  const uint32_t* d_total = w.chunk_off + nc;
  k_emit_pairs<<<(nc + 255) / 256, 256, 0, st>>>(nc, w.chunk_rect, w.chunk_front, w.chunk_ntile, w.chunk_off, tiles_x,
                                                 tiles_y, w.pair_key, w.pair_val, cap, ovf);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_emit_pairs");
  k_pad_pairs<<<std::max(1u, std::min(1024u, (cap + 255) / 256)), 256, 0, st>>>(d_total, cap, w.pair_key, w.pair_val);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_pad_pairs");
  int tbits = 0;
  while ((1 << tbits) < n_tiles) ++tbits;
  if ((s = radix_sort_u64(ctx, w.pair_key, w.pair_val, w.pair_key2, w.pair_val2, cap, 32 + tbits, w.tmp, st)) !=
      SPHDVR_OK)
    return s;
  if ((e = cudaMemsetAsync(w.tile_range, 0, (size_t)n_tiles * sizeof(int2), st)) != cudaSuccess)
    return cuda_err(ctx, e, "tile range memset");
  k_tile_ranges_dev<<<(cap + 255) / 256, 256, 0, st>>>(d_total, cap, w.pair_key, w.tile_range);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_tile_ranges_dev");
  if ((s = clear_counters(ctx, w, st)) != SPHDVR_OK) return s;
  RenderParams p;
  common_params(a, w, p);
  p.cam = a.cam;
  p.chunk_rect = w.chunk_rect;
  p.pair_key = w.pair_key;
  p.pair_val = w.pair_val;
  p.tile_range = w.tile_range;
  p.tiles_x = tiles_x;
  p.tiles_y = tiles_y;
  p.out = a.out;
  p.n_items = n_tiles * kTile * kTile;
  return launch_frame(ctx, a, w, p, false, std::min(grid, w.table_ctas), st);
}

sphdvr_status render_batch_sized(sphdvr_ctx* ctx, const RenderArgs* a, int n, cudaStream_t st, PairSizer sizer,
                                 void* user) {
  if (n < 1 || n > SPHDVR_MAX_BATCH) return set_err(ctx, SPHDVR_EINVAL, "batch: frame count out of range");
  if (n == 1) return render_frame_sized(ctx, a[0], st, sizer, user);
  const int grid = render_grid_batch(ctx, a, n);
  const int nc = a[0].ds->n_chunks;
  int64_t tiles = 0, rays = 0;
  for (int f = 0; f < n; ++f) {
    tiles += frame_tiles(a[f].cam);
    rays += (int64_t)frame_tiles(a[f].cam) * kTile * kTile;
  }
  if (rays > INT32_MAX) return set_err(ctx, SPHDVR_EINVAL, "batch: more than 2^31 rays");
  FrameWork w;
  sphdvr_status s;
  if ((s = shared_work(ctx, a[0], grid, w)) != SPHDVR_OK || (s = rect_range_work(ctx, a[0], n, tiles, w)) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->frames, (size_t)n * sizeof(RenderFrame))) != SPHDVR_OK ||
      (s = upload_tf(ctx, a[0], w, st)) != SPHDVR_OK)
    return s;
  // pass 1: each frame's pair count (the chunk scratch is reused frame after frame)
  uint32_t cnt[SPHDVR_MAX_BATCH];
  int64_t pairs = 0;
  for (int f = 0; f < n; ++f) {
    if ((s = project_frame(ctx, a[f], w.chunk_rect + (size_t)f * nc, w, st, &cnt[f])) != SPHDVR_OK) return s;
    pairs += cnt[f];
  }
  if (pairs > INT32_MAX) return set_err(ctx, SPHDVR_EOVERFLOW, "batch: more than 2^31 chunk-tile pairs");
  ctx->last_pairs = pairs;
  if (sizer && (s = sizer(ctx, w, (size_t)pairs, user)) != SPHDVR_OK) return s;
  // pass 2: project again and sort each frame's pairs into its part of the common arrays
  RenderFrame fr[SPHDVR_MAX_BATCH];
  int64_t base = 0, tile_base = 0, items = 0;
  for (int f = 0; f < n; ++f) {
    const float4* rect = w.chunk_rect + (size_t)f * nc;
    if ((s = project_frame(ctx, a[f], w.chunk_rect + (size_t)f * nc, w, st, nullptr)) != SPHDVR_OK ||
        (s = sort_frame(ctx, a[f], rect, w, cnt[f], base, w.tile_range + tile_base, st)) != SPHDVR_OK)
      return s;
    std::memset(&fr[f], 0, sizeof(RenderFrame));
    fr[f].cam = a[f].cam;
    fr[f].tiles_x = (a[f].cam.width + kTile - 1) / kTile;
    fr[f].tiles_y = (a[f].cam.height + kTile - 1) / kTile;
    fr[f].tile_base = (int)tile_base;
    items += (int64_t)frame_tiles(a[f].cam) * kTile * kTile;
    fr[f].item_end = (int)items;
    fr[f].out = a[f].out;
    base += cnt[f];
    tile_base += frame_tiles(a[f].cam);
  }
  cudaError_t e = cudaMemcpyAsync(ctx->frames.p, fr, (size_t)n * sizeof(RenderFrame), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "frame records upload");
  if ((s = clear_counters(ctx, w, st)) != SPHDVR_OK) return s;
  RenderParams p;
  common_params(a[0], w, p);
  p.chunk_rect = w.chunk_rect;
  p.pair_key = w.pair_key;
  p.pair_val = w.pair_val;
  p.tile_range = w.tile_range;
  p.frames = (const RenderFrame*)ctx->frames.p;
  p.n_frames = n;
  p.rect_stride = nc;
  p.n_items = (int)items;
  return launch_frame(ctx, a[0], w, p, true, std::min(grid, w.table_ctas), st);
}

}  // namespace sphdvr
