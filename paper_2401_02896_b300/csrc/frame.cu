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

#include "render.cuh"

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

__global__ void k_emit_pairs(int n_chunks, const float4* rect, const unsigned* front_ord, const uint32_t* ntile,
                             const uint32_t* off, int tiles_x, int tiles_y, uint64_t* keys, uint32_t* vals) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  uint32_t n = ntile[c];
  if (!n) return;
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

__global__ void k_tile_ranges(int64_t n, const uint64_t* keys, int2* range) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int t = (int)(keys[i] >> 32);
  if (i == 0 || (int)(keys[i - 1] >> 32) != t) range[t].x = (int)i;
  if (i == n - 1 || (int)(keys[i + 1] >> 32) != t) range[t].y = (int)(i + 1);
}

}  // namespace

// per-degree launchers (render_d<D>.cu)
#define SPHDVR_DECL(D)                                                                                         \
  sphdvr_status launch_render_d##D(sphdvr_ctx* ctx, bool f64, bool dbg, const RenderParams& p, int grid,    \
                                   size_t smem, cudaStream_t st);                                            \
  int render_occupancy_d##D(bool f64, bool dbg, size_t smem);
SPHDVR_DECL(1)
SPHDVR_DECL(2)
SPHDVR_DECL(3)
SPHDVR_DECL(4)
SPHDVR_DECL(5)
SPHDVR_DECL(6)
#undef SPHDVR_DECL

static sphdvr_status dispatch_render(sphdvr_ctx* ctx, int D, bool f64, bool dbg, const RenderParams& p, int grid,
                                     size_t smem, cudaStream_t st) {
  switch (D) {
    case 1: return launch_render_d1(ctx, f64, dbg, p, grid, smem, st);
    case 2: return launch_render_d2(ctx, f64, dbg, p, grid, smem, st);
    case 3: return launch_render_d3(ctx, f64, dbg, p, grid, smem, st);
    case 4: return launch_render_d4(ctx, f64, dbg, p, grid, smem, st);
    case 5: return launch_render_d5(ctx, f64, dbg, p, grid, smem, st);
    case 6: return launch_render_d6(ctx, f64, dbg, p, grid, smem, st);
  }
  return set_err(ctx, SPHDVR_EINVAL, "D out of range");
}

static int render_occupancy(int D, bool f64, bool dbg, size_t smem) {
  switch (D) {
    case 1: return render_occupancy_d1(f64, dbg, smem);
    case 2: return render_occupancy_d2(f64, dbg, smem);
    case 3: return render_occupancy_d3(f64, dbg, smem);
    case 4: return render_occupancy_d4(f64, dbg, smem);
    case 5: return render_occupancy_d5(f64, dbg, smem);
    case 6: return render_occupancy_d6(f64, dbg, smem);
  }
  return 0;
}

int render_grid(sphdvr_ctx* ctx, const RenderArgs& a) {
  const bool dbg = a.n_dbg > 0;
  const int prec = a.opts ? a.opts->precision : SPHDVR_PREC_FP32_ANCHORED;
  const bool f64 = prec == SPHDVR_PREC_FP64_NAIVE;
  const size_t smem = render_smem_bytes(a.tf_n, dbg ? 1 : kRenderWarps);
  int nb = render_occupancy(a.lut->D, f64, dbg, smem);
  if (ctx->num_sms <= 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device);
    ctx->num_sms = n > 0 ? n : 1;
  }
  int items;
  if (dbg) {
    items = a.n_dbg;
  } else {
    const int tiles = ((a.cam.width + kTile - 1) / kTile) * ((a.cam.height + kTile - 1) / kTile);
    items = (tiles * kTile * kTile + kRenderWarps - 1) / kRenderWarps;
  }
  int grid = std::max(1, nb) * ctx->num_sms;
  return std::max(1, std::min(grid, items));
}

size_t render_table_floats(int grid, bool dbg) { return (size_t)grid * (dbg ? 1 : kRenderWarps) * kTableWords; }



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

size_t pair_bytes(size_t pairs) {
  const size_t np = std::max<size_t>(pairs, 1);
  return np * 24 + sort_tmp_words((int64_t)np) * sizeof(uint32_t);
}

size_t frame_fixed_bytes(sphdvr_ctx* ctx, const RenderArgs& a) {
  const size_t tiles = (size_t)((a.cam.width + kTile - 1) / kTile) * ((a.cam.height + kTile - 1) / kTile);
  const size_t nc = a.ds->n_chunks;
  const int grid = render_grid(ctx, a);
  return nc * (sizeof(float4) + sizeof(unsigned) + 2 * sizeof(uint32_t)) + 32 + tiles * sizeof(int2) +
         32 * sizeof(unsigned long long) + scan_tmp_words(nc) * sizeof(uint32_t) + (size_t)a.tf_n * sizeof(float4) +
         render_table_floats(grid, a.n_dbg > 0) * sizeof(float) + 4 * sizeof(unsigned);
}

sphdvr_status render_frame(sphdvr_ctx* ctx, const RenderArgs& a, cudaStream_t st) {
  return render_frame_sized(ctx, a, st, ctx_pair_sizer, nullptr);
}

sphdvr_status render_frame_sized(sphdvr_ctx* ctx, const RenderArgs& a, cudaStream_t st, PairSizer sizer, void* user) {
  const int tiles = ((a.cam.width + kTile - 1) / kTile) * ((a.cam.height + kTile - 1) / kTile);
  const int nc = a.ds->n_chunks;
  sphdvr_status s;
  if ((s = ensure(ctx, ctx->chunk_rect, (size_t)nc * sizeof(float4))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->chunk_front, (size_t)nc * sizeof(unsigned))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->chunk_ntile, (size_t)nc * sizeof(uint32_t) + 16)) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->chunk_off, (size_t)nc * sizeof(uint32_t) + 16)) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->tile_range, (size_t)tiles * sizeof(int2))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->stats, 32 * sizeof(unsigned long long))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->scan_tmp, scan_tmp_words(nc) * sizeof(uint32_t))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->tf, (size_t)a.tf_n * sizeof(float4))) != SPHDVR_OK)
    return s;
  const int grid = render_grid(ctx, a);
  if ((s = ensure(ctx, ctx->table, render_table_floats(grid, a.n_dbg > 0) * sizeof(float))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->work, 4 * sizeof(unsigned))) != SPHDVR_OK)
    return s;
  FrameWork w;
  w.table = (float*)ctx->table.p;
  w.table_ctas = grid;
  w.work = (unsigned*)ctx->work.p;
  w.chunk_rect = (float4*)ctx->chunk_rect.p;
  w.chunk_front = (unsigned*)ctx->chunk_front.p;
  w.chunk_ntile = (uint32_t*)ctx->chunk_ntile.p;
  w.chunk_off = (uint32_t*)ctx->chunk_off.p;
  w.tile_range = (int2*)ctx->tile_range.p;
  w.stats = (unsigned long long*)ctx->stats.p;
  w.tf = (float4*)ctx->tf.p;
  w.tmp = (uint32_t*)ctx->scan_tmp.p;
  w.tmp_words = ctx->scan_tmp.bytes / sizeof(uint32_t);
  return render_frame_ws(ctx, a, w, sizer, user, st);
}

sphdvr_status render_frame_ws(sphdvr_ctx* ctx, const RenderArgs& a, FrameWork& w, PairSizer sizer, void* user,
                              cudaStream_t st) {
  const sphdvr_dataset* ds = a.ds;
  const DevLut* L = a.lut;
  const DevCamera& cam = a.cam;
  const int tiles_x = (cam.width + kTile - 1) / kTile, tiles_y = (cam.height + kTile - 1) / kTile;
  const int n_tiles = tiles_x * tiles_y;
  const int nc = ds->n_chunks;
  sphdvr_status s;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(w.tf, a.tf_host, (size_t)a.tf_n * sizeof(float4), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return cuda_err(ctx, e, "transfer function upload");
  float4* rect = w.chunk_rect;
  unsigned* front = w.chunk_front;
  uint32_t* ntile = w.chunk_ntile;
  uint32_t* off = w.chunk_off;
  int2* trange = w.tile_range;
  unsigned long long* stats = w.stats;
  k_chunk_project<<<(nc + 255) / 256, 256, 0, st>>>(nc, ds->chunk_lo, ds->chunk_hi, cam, L->q, L->reach, tiles_x,
                                                    tiles_y, rect, front, ntile);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_chunk_project");
  uint32_t* d_total = off + nc;
  if (w.tmp_words < scan_tmp_words(nc)) return set_err(ctx, SPHDVR_EOVERFLOW, "frame scratch too small for the scan");
  if ((s = scan_exclusive_u32(ctx, ntile, off, nc, d_total, w.tmp, st)) != SPHDVR_OK) return s;
  uint32_t total = 0;
  if ((e = cudaMemcpyAsync(&total, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_err(ctx, e, "pair count");
  ctx->last_pairs = total;
  if (sizer && (s = sizer(ctx, w, total, user)) != SPHDVR_OK) return s;
  if (w.pair_cap < total || w.tmp_words < sort_tmp_words(total))
    return set_err(ctx, SPHDVR_EOVERFLOW, "frame scratch too small for " + std::to_string(total) + " chunk-tile pairs");
  uint64_t* keys = w.pair_key;
  uint32_t* vals = w.pair_val;
  k_emit_pairs<<<(nc + 255) / 256, 256, 0, st>>>(nc, rect, front, ntile, off, tiles_x, tiles_y, keys, vals);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_emit_pairs");
  int tbits = 0;
  while ((1 << tbits) < n_tiles) ++tbits;
  if ((s = radix_sort_u64(ctx, keys, vals, w.pair_key2, w.pair_val2, total, 32 + tbits, w.tmp, st)) != SPHDVR_OK)
    return s;
  if ((e = cudaMemsetAsync(trange, 0, (size_t)n_tiles * sizeof(int2), st)) != cudaSuccess)
    return cuda_err(ctx, e, "tile range memset");
  if (total) {
    k_tile_ranges<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(total, keys, trange);
    ++ctx->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_tile_ranges");
  }
  if ((e = cudaMemsetAsync(stats, 0, 32 * sizeof(unsigned long long), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(w.work, 0, sizeof(unsigned), st)) != cudaSuccess)
    return cuda_err(ctx, e, "stats memset");

  RenderParams p;
  std::memset(&p, 0, sizeof(p));
  p.cam = cam;
  p.pos = ds->pos;
  p.amp = ds->amp;
  p.orig = ds->orig;
  p.chunk = ds->chunk;
  p.chunk_lo = ds->chunk_lo;
  p.chunk_hi = ds->chunk_hi;
  p.chunk_rect = rect;
  p.pair_key = keys;
  p.pair_val = vals;
  p.tile_range = trange;
  p.tiles_x = tiles_x;
  p.tiles_y = tiles_y;
  p.K = L->K;
  p.m = L->m;
  p.n_lambda = L->n_lambda;
  p.q = L->q;
  p.lam_scale = (float)((L->n_lambda - 1) / (double)L->q);
  p.theta = L->theta;
  p.jump = L->jump;
  p.piece = L->piece;
  p.tf_n = a.tf_n;
  p.tf_lo = a.tf_lo;
  p.tf_dv = (a.tf_hi - a.tf_lo) / (a.tf_n - 1);
  p.tf_inv_dv = (float)((a.tf_n - 1) / ((double)a.tf_hi - (double)a.tf_lo));
  p.tf = w.tf;
  const sphdvr_render_opts* o = a.opts;
  int prec = o ? o->precision : SPHDVR_PREC_FP32_ANCHORED;
  p.anchor_every = (prec == SPHDVR_PREC_FP32_ANCHORED) ? std::max(1, o ? o->anchor_every : 2) : 0;
  p.window_h = (o && o->window_h > 0.f) ? o->window_h : 1.0f;
  p.reinit_dt = (prec == SPHDVR_PREC_FP32_REINIT) ? o->reinit_dt : 0.f;
  float eps = o ? o->ert_eps : 1e-5f;
  p.tau_ert = eps > 0.f ? -std::log(eps) : 0.f;
  p.out = a.out;
  p.stats = stats;
  p.n_dbg = a.n_dbg;
  p.dbg_pix = a.dbg_pix;
  p.dbg_rgba = a.dbg_rgba;
  p.dbg_counts = a.dbg_counts;
  p.dbg_cands = a.dbg_cands;
  p.cand_cap = a.cand_cap;
  p.dbg_field = a.dbg_field;
  p.field_cap = a.field_cap;
  const bool f64 = prec == SPHDVR_PREC_FP64_NAIVE;
  const bool dbg = a.n_dbg > 0;
  const int grid = std::min(render_grid(ctx, a), w.table_ctas);
  p.scratch = w.table;
  p.work = w.work;
  p.n_items = n_tiles * kTile * kTile;
  p.dynamic = o ? (o->persistent ? 1 : 0) : 1;
  size_t smem = render_smem_bytes(a.tf_n, dbg ? 1 : kRenderWarps);
  return dispatch_render(ctx, L->D, f64, dbg, p, grid, smem, st);
}

}  // namespace sphdvr
