// The particle-centric pass order the paper states (Sec. 2, "Method
// Overview"): (1) every particle approximates its contribution to every ray
// it meets and scatters that ray's knots into a frame-wide knot list; (2) the
// list is sorted by (ray, position), which puts each ray's knots in order;
// (3) every ray runs the coefficient update over its sorted knots and
// classifies and composites the pieces.  The knots of a whole frame are held
// at once (12 bytes each, twice for the sort), so this order suits frames of
// modest knot counts; it is kept beside the ray-gathering kernel as the
// paper's own formulation and for comparison.
//
// Pass 1 runs one warp per chunk (a lane per particle) over the pixels of the
// chunk's screen rectangle: a conservative FP32 distance test skips clear
// misses, then the candidate test is the oracle's, in FP64 (distance from the
// ray below q h, far exit beyond t_near), and a hit emits
// the particle's K + 1 knots with the key (ray << 32 | ordered FP32 position).
// Pass 3 runs one warp per ray over its knots, 32 at a time: each lane
// rebuilds its knot's localized difference coefficients from the particle
// and the table (Sec. 2, 3.1), a warp scan of the Taylor-shift operator with
// the carry from the previous 32 gives every knot's coefficients (FP64
// running coefficients and FP64 differences of the table's pieces, the plain
// recurrence), and each lane composites its
// piece up to the next knot; the lanes' optical depths are combined in order.
#include <algorithm>
#include <cmath>
#include <string>

#include "render.cuh"

namespace sphdvr {
namespace {

__device__ __forceinline__ unsigned ord_key(float x) {
  unsigned b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ void pixel_ray(const DevCamera& c, int px, int py, double* o, double* v) {
  const double sx = 2.0 * (px + 0.5) / c.width - 1.0, sy = 1.0 - 2.0 * (py + 0.5) / c.height;
  if (c.proj == 0) {
    const double ax = sx * c.tan_half * c.aspect, ay = sy * c.tan_half;
    double n = 0;
    for (int i = 0; i < 3; ++i) {
      v[i] = c.f[i] + ax * c.r[i] + ay * c.u[i];
      n += v[i] * v[i];
    }
    n = sqrt(n);
    for (int i = 0; i < 3; ++i) {
      v[i] /= n;
      o[i] = c.eye[i];
    }
  } else {
    for (int i = 0; i < 3; ++i) {
      o[i] = c.eye[i] + sx * c.half_w * c.r[i] + sy * c.half_h * c.u[i];
      v[i] = c.f[i];
    }
  }
}

// FP32 ray of a pixel, for a conservative pre-test only
__device__ __forceinline__ void pixel_ray_f(const DevCamera& c, int px, int py, float* o, float* v) {
  const float sx = 2.f * (px + 0.5f) / c.width - 1.f, sy = 1.f - 2.f * (py + 0.5f) / c.height;
  if (c.proj == 0) {
    const float ax = sx * (float)(c.tan_half * c.aspect), ay = sy * (float)c.tan_half;
    float n = 0.f;
    for (int i = 0; i < 3; ++i) {
      v[i] = (float)c.f[i] + ax * (float)c.r[i] + ay * (float)c.u[i];
      n += v[i] * v[i];
    }
    n = rsqrtf(n);
    for (int i = 0; i < 3; ++i) {
      v[i] *= n;
      o[i] = (float)c.eye[i];
    }
  } else {
    for (int i = 0; i < 3; ++i) {
      o[i] = (float)(c.eye[i] + sx * c.half_w * c.r[i] + sy * c.half_h * c.u[i]);
      v[i] = (float)c.f[i];
    }
  }
}

struct Hit {
  double tc, d;
};

// the oracle's candidate test in FP64; t_chi and the ray-centre distance on a hit
__device__ __forceinline__ bool hit_test(const double* o, const double* v, float4 P, float q, double t_near, Hit& h) {
  const double p0 = (double)P.x - o[0], p1 = (double)P.y - o[1], p2 = (double)P.z - o[2];
  const double w0 = p1 * v[2] - p2 * v[1], w1 = p2 * v[0] - p0 * v[2], w2 = p0 * v[1] - p1 * v[0];
  const double d = sqrt(w0 * w0 + w1 * w1 + w2 * w2), R = (double)q * (double)P.w;
  if (!(d < R)) return false;
  const double tc = p0 * v[0] + p1 * v[1] + p2 * v[2];
  if (!(tc + sqrt(R * R - d * d) > t_near)) return false;
  h.tc = tc;
  h.d = d;
  return true;
}

// Localized coefficients, in ray units, of piece pc (0..K-1, between sorted
// knots pc and pc+1) of a particle with table entry j, smoothing length h and
// amplitude c, expanded at its sorted knot k -- in FP64 from the table's pieces.
template <int D>
__device__ void piece_at_knot(const RenderParams& p, int j, double h, double c, int pc, int k, double* A) {
  const int K = p.K, m = p.m;
  int kp;
  double sg;
  if (!(K & 1)) {
    if (pc < m) { kp = m - pc; sg = -1.0; } else { kp = pc - m + 1; sg = 1.0; }
  } else {
    if (pc < m - 1) { kp = m - pc; sg = -1.0; }
    else if (pc == m - 1) { kp = 1; sg = 1.0; }
    else { kp = pc - m + 2; sg = 1.0; }
  }
  const float2 th = __ldg(p.theta + j);
  const double th0 = kp == 1 ? 0.0 : (double)th.x;
  const double z = sg * (double)knot_sigma(K, m, th, k) - th0;
  const float* pr = p.piece + (size_t)j * 2 * (D + 1) + (kp - 1) * (D + 1);
  double q[D + 1];
  for (int d = 0; d <= D; ++d) q[d] = (double)__ldg(pr + d);
  taylor_shift<D, double>(q, z);
  double f = c;
  for (int d = 0; d <= D; ++d) {
    A[d] = q[d] * f;
    f *= sg / h;
  }
}

// Localized difference coefficients of sorted knot k (Sec. 2): the piece after
// the knot minus the piece before it, both expanded at the knot in FP64, so
// that a particle's differences sum to zero up to FP64 rounding (its pieces
// telescope) and the plain recurrence keeps no FP32 residue of it.
template <int D>
__device__ void knot_jump_fp64(const RenderParams& p, int j, double h, double c, int k, double* J) {
  double L[D + 1], R[D + 1];
  for (int d = 0; d <= D; ++d) L[d] = R[d] = 0.0;
  if (k >= 1) piece_at_knot<D>(p, j, h, c, k - 1, k, L);
  if (k <= p.K - 1) piece_at_knot<D>(p, j, h, c, k, k, R);
  for (int d = 0; d <= D; ++d) J[d] = R[d] - L[d];
}

struct ScatterParams {
  RenderParams rp;     // table, data set, transfer function, options
  const float4* rect;  // chunk pixel rectangles
  int n_chunks;
  const uint32_t* off;  // pass 1b: first knot slot of each particle
  uint32_t* cnt;        // pass 1a: knots of each particle
  uint64_t* keys;
  uint32_t* vals;  // particle << 3 | knot
  unsigned long long* total;  // pass 1a: all knots of the frame (64-bit, to detect a frame beyond 2^31)
  const int2* ray_range;
  int n_rays;
  float* out;
};

// pass 1: emit (emit = 1) or count (emit = 0) every particle's knots on every ray it meets
__global__ void k_scatter_knots(ScatterParams sp, int emit) {
  const RenderParams& p = sp.rp;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (c >= sp.n_chunks) return;
  const int2 ch = p.chunk[c];
  const bool mine = lane < ch.y;
  const int i = ch.x + lane;
  const float4 P = mine ? p.pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 r = sp.rect[c];
  const int x0 = max(0, (int)ceilf(r.x - 0.5f)), x1 = min(p.cam.width - 1, (int)floorf(r.z + 0.5f));
  const int y0 = max(0, (int)ceilf(r.y - 0.5f)), y1 = min(p.cam.height - 1, (int)floorf(r.w + 0.5f));
  const int K = p.K, nl = p.n_lambda;
  uint32_t n = 0, slot = (emit && mine) ? sp.off[i] : 0;
  if (mine && x0 <= x1 && y0 <= y1) {
    for (int py = y0; py <= y1; ++py)
      for (int px = x0; px <= x1; ++px) {
        {
          // FP32 pre-test: the squared ray-centre distance with a margin far above
          // its FP32 error (positions and distances of order 1 or below)
          float of[3], vf[3];
          pixel_ray_f(p.cam, px, py, of, vf);
          const float a0 = P.x - of[0], a1 = P.y - of[1], a2 = P.z - of[2];
          const float c0 = a1 * vf[2] - a2 * vf[1], c1 = a2 * vf[0] - a0 * vf[2], c2 = a0 * vf[1] - a1 * vf[0];
          const float R = p.q * P.w, mg = 1e-4f * (1.f + fabsf(a0) + fabsf(a1) + fabsf(a2));
          if (c0 * c0 + c1 * c1 + c2 * c2 > (R + mg) * (R + mg)) continue;
        }
        double o[3], v[3];
        pixel_ray(p.cam, px, py, o, v);
        Hit h;
        if (!hit_test(o, v, P, p.q, p.cam.t_near, h)) continue;
        n += K + 1;
        if (!emit) continue;
        const int j = min((int)floor(h.d / (double)P.w * (nl - 1) / (double)p.q + 0.5), nl - 1);
        const float2 th = __ldg(p.theta + j);
        const uint64_t ray = (uint64_t)py * p.cam.width + px;
        for (int k = 0; k <= K; ++k) {
          const double t = h.tc + (double)knot_sigma(K, p.m, th, k) * (double)P.w;
          sp.keys[slot] = (ray << 32) | ord_key((float)t);
          sp.vals[slot] = ((uint32_t)i << 3) | (uint32_t)k;
          ++slot;
        }
      }
  }
  if (!emit && mine) {
    sp.cnt[i] = n;
    if (n) atomicAdd(sp.total, (unsigned long long)n);
  }
}

// [first, end) of each ray's knots in the sorted list
__global__ void k_ray_ranges(int64_t n, const uint64_t* keys, int2* range) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t t = (uint32_t)(keys[i] >> 32);
  if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) range[t].x = (int)i;
  if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != t) range[t].y = (int)(i + 1);
}

// pass 3: the coefficient update and compositing per ray
template <int D>
__global__ void __launch_bounds__(128) k_scatter_composite(ScatterParams sp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const RenderParams& p = sp.rp;
  float4* s_tf = (float4*)smem;
  for (int t = threadIdx.x; t < p.tf_n; t += blockDim.x) s_tf[t] = p.tf[t];
  __syncthreads();
  const TfCtx tfc{s_tf, p.tf_n, p.tf_lo, p.tf_inv_dv, p.tf_dv};
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int nl = p.n_lambda, K = p.K;
  unsigned long long st_knots = 0, st_rays = 0, st_ert = 0;
  for (int ray = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ray < sp.n_rays; ray += warps) {
    const int px = ray % p.cam.width, py = ray / p.cam.width;
    const int2 rg = sp.ray_range[ray];
    float col[3] = {0.f, 0.f, 0.f}, tau_ray = 0.f;
    if (rg.y > rg.x) {
      double o[3], v[3];
      pixel_ray(p.cam, px, py, o, v);
      double carry[D + 1], tcar = 0.0, t_start = 0.0;
      for (int d = 0; d <= D; ++d) carry[d] = 0.0;
      bool first = true;
      for (int b = rg.x; b < rg.y; b += 32) {
        const int idx = b + lane;
        const bool valid = idx < rg.y;
        double A[D + 1], t = 0.0;
        for (int d = 0; d <= D; ++d) A[d] = 0.0;
        if (valid) {
          const uint32_t vv = sp.vals[idx];
          const int i = (int)(vv >> 3), k = (int)(vv & 7u);
          const float4 P = p.pos[i];
          Hit h{0.0, 0.0};
          hit_test(o, v, P, p.q, -INFINITY, h);  // passed in pass 1 with the same arithmetic
          const int j = min((int)floor(h.d / (double)P.w * (nl - 1) / (double)p.q + 0.5), nl - 1);
          const float2 th = __ldg(p.theta + j);
          t = h.tc + (double)knot_sigma(K, p.m, th, k) * (double)P.w;
          const double hw = (double)P.w;
          knot_jump_fp64<D>(p, j, hw, (double)p.amp[i] / (hw * hw * hw), k, A);
        }
        const int nv = min(32, rg.y - b);
        const double t0 = __shfl_sync(kFull, t, 0);
        if (first) {
          t_start = fmax(t0, p.cam.t_near);
          tcar = t0;
          first = false;
        }
        // lane 0 takes the carry: the polynomial after the previous knots, moved to its knot
        if (lane == 0) {
          double cs[D + 1];
          for (int d = 0; d <= D; ++d) cs[d] = carry[d];
          taylor_shift<D, double>(cs, t - tcar);
          for (int d = 0; d <= D; ++d) A[d] += cs[d];
        }
        // inclusive scan of (A, t): (X, tx) (+) (Y, ty) = (Shift(X, ty - tx) + Y, ty)
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
          double oa[D + 1];
          for (int d = 0; d <= D; ++d) oa[d] = __shfl_up_sync(kFull, A[d], o2);
          const double ot = __shfl_up_sync(kFull, t, o2);
          if (lane >= o2 && valid) {
            taylor_shift<D, double>(oa, t - ot);
            for (int d = 0; d <= D; ++d) A[d] += oa[d];
          }
        }
        // the piece from this knot to the next (the last one's end is the next 32's first knot)
        const double tn = __shfl_down_sync(kFull, t, 1);
        Acc acc{0.f, 0.f, 0.f, 0.f};
        // lane 0 also composites the piece before its knot: carry from tcar (previous 32's last knot)
        if (lane == 0 && b > rg.x) {
          const double a0 = fmax(tcar, t_start), L = t - a0;
          if (L > 0) {
            double cs[D + 1];
            for (int d = 0; d <= D; ++d) cs[d] = carry[d];
            taylor_shift<D, double>(cs, a0 - tcar);
            Poly<D> Pf;
            for (int d = 0; d <= D; ++d) Pf.c[d] = (float)cs[d];
            acc = composite_piece_v<D>(Pf, (float)L, tfc, acc);
          }
        }
        if (valid && lane < nv - 1) {
          const double a0 = fmax(t, t_start), L = tn - a0;
          if (L > 0) {
            double cs[D + 1];
            for (int d = 0; d <= D; ++d) cs[d] = A[d];
            taylor_shift<D, double>(cs, a0 - t);
            Poly<D> Pf;
            for (int d = 0; d <= D; ++d) Pf.c[d] = (float)cs[d];
            acc = composite_piece_v<D>(Pf, (float)L, tfc, acc);
          }
        }
        // combine the lanes in order: transmittance from the accumulated optical depth
        float tx = acc.tau;
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
          const float y = __shfl_up_sync(kFull, tx, o2);
          if (lane >= o2) tx += y;
        }
        const float w = __expf(-(tau_ray + tx - acc.tau));
        col[0] += warp_sum(w * acc.r);
        col[1] += warp_sum(w * acc.g);
        col[2] += warp_sum(w * acc.b);
        tau_ray += __shfl_sync(kFull, tx, 31);
        // carry: the last valid knot's coefficients
        for (int d = 0; d <= D; ++d) carry[d] = __shfl_sync(kFull, A[d], nv - 1);
        tcar = __shfl_sync(kFull, t, nv - 1);
        st_knots += nv;
        if (p.tau_ert > 0.f && tau_ray > p.tau_ert) {
          ++st_ert;
          break;
        }
      }
    }
    ++st_rays;
    if (lane == 0) {
      const float alpha = 1.f - __expf(-tau_ray);
      ((float4*)sp.out)[ray] = make_float4(col[0], col[1], col[2], alpha);
    }
  }
  if (lane == 0) {
    atomicAdd(p.stats + 0, st_rays);
    atomicAdd(p.stats + 1, st_knots / (K + 1));
    atomicAdd(p.stats + 2, st_knots);
    atomicAdd(p.stats + 8, st_ert);
  }
}

template <int D>
sphdvr_status launch_composite(sphdvr_ctx* ctx, const ScatterParams& sp, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_scatter_composite<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_err(ctx, e, "scatter smem attribute");
  k_scatter_composite<D><<<grid, 128, smem, st>>>(sp);
  ++ctx->launches;
  return cuda_err(ctx, cudaGetLastError(), "k_scatter_composite");
}

}  // namespace

sphdvr_status render_scatter(sphdvr_ctx* ctx, const RenderArgs& a, cudaStream_t st) {
  const sphdvr_dataset* ds = a.ds;
  const DevLut* L = a.lut;
  const int nc = ds->n_chunks;
  const int64_t n = ds->n;
  const int64_t rays = (int64_t)a.cam.width * a.cam.height;
  if (n >= (int64_t)1 << 29) return set_err(ctx, SPHDVR_EINVAL, "scatter: at most 2^29 particles");
  sphdvr_status s;
  if ((s = ensure(ctx, ctx->chunk_rect, (size_t)nc * sizeof(float4))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->chunk_front, (size_t)nc * sizeof(unsigned))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->chunk_ntile, (size_t)nc * sizeof(uint32_t) + 16)) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->chunk_off, (size_t)(n + 4) * sizeof(uint32_t))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->dbg_counts, (size_t)(n + 4) * sizeof(uint32_t))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->scan_tmp, scan_tmp_words(n) * sizeof(uint32_t))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->tile_range, (size_t)rays * sizeof(int2))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->stats, 32 * sizeof(unsigned long long))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->tf, (size_t)a.tf_n * sizeof(float4))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->work, 4 * sizeof(unsigned long long))) != SPHDVR_OK)
    return s;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(ctx->tf.p, a.tf_host, (size_t)a.tf_n * sizeof(float4), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return cuda_err(ctx, e, "transfer function upload");
  float4* rect = (float4*)ctx->chunk_rect.p;
  if ((s = project_chunk_rects(ctx, a, rect, (unsigned*)ctx->chunk_front.p, (uint32_t*)ctx->chunk_ntile.p, st)) !=
      SPHDVR_OK)
    return s;
  ScatterParams sp{};
  RenderParams& p = sp.rp;
  p.cam = a.cam;
  p.pos = ds->pos;
  p.amp = ds->amp;
  p.chunk = ds->chunk;
  p.K = L->K;
  p.m = L->m;
  p.n_lambda = L->n_lambda;
  p.q = L->q;
  p.theta = L->theta;
  p.jump = L->jump;
  p.piece = L->piece;
  p.tf_n = a.tf_n;
  p.tf_lo = a.tf_lo;
  p.tf_dv = (a.tf_hi - a.tf_lo) / (a.tf_n - 1);
  p.tf_inv_dv = (float)((a.tf_n - 1) / ((double)a.tf_hi - (double)a.tf_lo));
  p.tf = (const float4*)ctx->tf.p;
  const float eps = a.opts ? a.opts->ert_eps : 1e-5f;
  p.tau_ert = eps > 0.f ? -std::log(eps) : 0.f;
  p.stats = (unsigned long long*)ctx->stats.p;
  sp.rect = rect;
  sp.n_chunks = nc;
  sp.cnt = (uint32_t*)ctx->dbg_counts.p;  // (the parity hook's buffer, free outside its calls)
  sp.off = (uint32_t*)ctx->chunk_off.p;
  sp.total = (unsigned long long*)ctx->work.p;
  // pass 1a: knots per particle, then their offsets and the frame's total
  const int cgrid = (nc + 3) / 4;
  if ((e = cudaMemsetAsync(sp.cnt, 0, (size_t)n * sizeof(uint32_t), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(sp.total, 0, sizeof(unsigned long long), st)) != cudaSuccess)
    return cuda_err(ctx, e, "scatter count memset");
  k_scatter_knots<<<cgrid, 128, 0, st>>>(sp, 0);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_scatter_knots (count)");
  uint32_t* d_total = (uint32_t*)ctx->chunk_off.p + n;
  if ((s = scan_exclusive_u32(ctx, sp.cnt, (uint32_t*)ctx->chunk_off.p, n, d_total, (uint32_t*)ctx->scan_tmp.p, st)) !=
      SPHDVR_OK)
    return s;
  unsigned long long total64 = 0;
  if ((e = cudaMemcpyAsync(&total64, sp.total, sizeof(total64), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_err(ctx, e, "knot count");
  if (total64 > 0x7fffffffull)
    return set_err(ctx, SPHDVR_EOVERFLOW,
                   "scatter: " + std::to_string(total64) + " knots in the frame, more than 2^31 - 1");
  const uint32_t total = (uint32_t)total64;
  (void)d_total;
  ctx->last_pairs = total;
  // pass 1b: emit; pass 2: sort by (ray, position)
  const size_t nk = std::max<size_t>(total, 1);
  if ((s = ensure(ctx, ctx->pair_key, nk * 8)) != SPHDVR_OK || (s = ensure(ctx, ctx->pair_val, nk * 4)) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->pair_key2, nk * 8)) != SPHDVR_OK || (s = ensure(ctx, ctx->pair_val2, nk * 4)) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->sort_tmp, sort_tmp_words((int64_t)nk) * sizeof(uint32_t))) != SPHDVR_OK)
    return s;
  sp.keys = (uint64_t*)ctx->pair_key.p;
  sp.vals = (uint32_t*)ctx->pair_val.p;
  k_scatter_knots<<<cgrid, 128, 0, st>>>(sp, 1);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_scatter_knots (emit)");
  int rbits = 0;
  while (((int64_t)1 << rbits) < rays) ++rbits;
  if ((s = radix_sort_u64(ctx, sp.keys, sp.vals, (uint64_t*)ctx->pair_key2.p, (uint32_t*)ctx->pair_val2.p, total,
                          32 + rbits, (uint32_t*)ctx->sort_tmp.p, st)) != SPHDVR_OK)
    return s;
  int2* range = (int2*)ctx->tile_range.p;
  if ((e = cudaMemsetAsync(range, 0, (size_t)rays * sizeof(int2), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(p.stats, 0, 32 * sizeof(unsigned long long), st)) != cudaSuccess)
    return cuda_err(ctx, e, "scatter memset");
  if (total) {
    k_ray_ranges<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(total, sp.keys, range);
    ++ctx->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ctx, e, "k_ray_ranges");
  }
  // pass 3
  sp.ray_range = range;
  sp.n_rays = (int)rays;
  sp.out = a.out;
  if (ctx->num_sms <= 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device);
    ctx->num_sms = v > 0 ? v : 1;
  }
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->num_sms * 8, (rays + 3) / 4));
  const size_t smem = (size_t)a.tf_n * sizeof(float4);
  switch (L->D) {
    case 1: return launch_composite<1>(ctx, sp, grid, smem, st);
    case 2: return launch_composite<2>(ctx, sp, grid, smem, st);
    case 3: return launch_composite<3>(ctx, sp, grid, smem, st);
    case 4: return launch_composite<4>(ctx, sp, grid, smem, st);
    case 5: return launch_composite<5>(ctx, sp, grid, smem, st);
    case 6: return launch_composite<6>(ctx, sp, grid, smem, st);
  }
  return set_err(ctx, SPHDVR_EINVAL, "D out of range");
}

}  // namespace sphdvr
