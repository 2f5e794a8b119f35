// Per-ray field reconstruction and compositing kernel.
//
// One warp owns one viewing ray; a CTA of NW warps owns an NW-ray sub-tile of a
// 16x16 binning tile and streams that tile's chunk list (sorted by a lower
// bound F of every knot position a chunk's particles can produce) through
// shared memory.  Per ray:
//   1. candidate gathering: every staged particle is tested against the ray in
//      FP32, and in double-float (hi+lo FP32 pairs) near the decision; a
//      candidate has d < q h and its support ends after t_near (Sec. 3.1);
//   2. per-particle approximation: L = d/h picks the nearest table entry; the
//      particle's knots are t_chi + h * (+-theta_k, 0) with localized
//      difference coefficients a h^-3 * s_kd / h^d (Sec. 2, Sec. 3.1);
//      candidates are kept in a per-warp table in shared memory;
//   3. windows: all knots below the current bound F are final; up to W of them
//      (the window) are emitted from the table, bucket-sorted by position and
//      insertion-sorted within buckets;
//   4. segmented prefix sum: the coefficient-update recurrence of Sec. 2
//      (eq. Piecewise-Coefficients-Update) as an associative scan over the warp
//      -- (A, e_A) (+) (B, e_B) = (Shift(A, e_B - e_A) + B, e_B) -- seeded with
//      the field's exact coefficients at the window start, summed over the
//      active particles' own pieces (re-anchoring bounds the FP32 drift that
//      Sec. 4.1 describes);
//   5. classification + compositing per piece: pieces are split where the
//      field crosses transfer-function nodes, optical depth is integrated in
//      closed form, emission by 2-point Gauss-Legendre; transmittance is kept
//      as accumulated optical depth; early ray termination.
#pragma once

#include "device_common.cuh"
#include "sphdvr_internal.h"

#ifdef SPHDVR_PHASE_TIMING
#define PT_DECL long long pt_acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}; long long pt_t0 = 0;
#define PT_BEGIN pt_t0 = clock64();
#define PT_END(ph) pt_acc[ph] += clock64() - pt_t0;
#else
#define PT_DECL
#define PT_BEGIN
#define PT_END(ph)
#endif

namespace sphdvr {

constexpr int kCap = 4096;        // candidate table entries per ray (global scratch, L1-cached)
constexpr int kKpl = 8;           // knots per lane in a window
constexpr int kW = 32 * kKpl;     // window capacity (knots)
constexpr int kNb = 64;           // buckets of the window sort
constexpr int kStageChunks = 16;  // chunks staged per batch
constexpr int kStage = kStageChunks * kChunk;
constexpr int kDefer = 48;        // new candidates that trigger window processing
constexpr int kRenderWarps = 4;   // rays (warps) per CTA in normal rendering
constexpr int kTableWords = 7 * kCap;  // per-ray table: 7 arrays of kCap words

struct RenderParams {
  DevCamera cam;
  // data set
  const float4* pos;
  const float* amp;
  const int* orig;
  const int2* chunk;
  const float4* chunk_lo;  // tight box min, w = h_max
  const float4* chunk_hi;  // tight box max
  // binning
  const float4* chunk_rect;
  const uint64_t* pair_key;
  const uint32_t* pair_val;
  const int2* tile_range;
  int tiles_x, tiles_y;
  // table
  int K, m, n_lambda;
  float q, lam_scale;  // lam_scale = (n_lambda - 1) / q
  const float2* theta;
  const float* jump;
  const float* piece;
  // transfer function
  int tf_n;
  float tf_lo, tf_inv_dv, tf_dv;
  const float4* tf;
  // options
  int anchor_every;  // 0: never (naive recurrence)
  float window_h;    // window length limit in units of the smallest pending h
  float tau_ert;     // stop when accumulated optical depth exceeds this
  float* out;
  unsigned long long* stats;
  float* scratch;       // per-ray tables: (grid * NW) * kTableWords words
  unsigned* work;       // work-queue counter (dynamic scheduling), zeroed per frame
  int n_items;          // sub-tiles
  int dynamic;          // 1: atomic work queue, 0: static stride
  // debug
  int n_dbg;
  const int* dbg_pix;
  float* dbg_rgba;
  long long* dbg_counts;
  long long* dbg_cands;
  int cand_cap;
  double* dbg_field;
  int field_cap;
};

// ---------------------------------------------------------------------------
// small polynomial helpers
// ---------------------------------------------------------------------------

// In place: coefficients of p(y + s) from those of p(y) (Sec. 2 localized
// coefficients; this is the sum over j of binom(j,d) a_j s^(j-d)).
template <int D, typename T>
__device__ __forceinline__ void taylor_shift(T* c, T s) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = D - 1; j >= i; --j) c[j] = c[j] + s * c[j + 1];
}

template <int D>
__device__ __forceinline__ float horner(const float* c, float y) {
  float r = c[D];
#pragma unroll
  for (int d = D - 1; d >= 0; --d) r = fmaf(r, y, c[d]);
  return r;
}

// antiderivative from 0: sum_d c_d y^(d+1)/(d+1)
template <int D>
__device__ __forceinline__ float horner_int(const float* c, float y) {
  float r = c[D] * (1.f / (D + 1));
#pragma unroll
  for (int d = D - 1; d >= 0; --d) r = fmaf(r, y, c[d] * (1.f / (d + 1)));
  return r * y;
}

// ---------------------------------------------------------------------------
// transfer function / compositing
// ---------------------------------------------------------------------------

struct TfCtx {
  const float4* tf;
  int n;
  float lo, inv_dv, dv;
};

// cell -1: below lo; cell n-1: above hi; else [v_c, v_{c+1}]
__device__ __forceinline__ int tf_cell(const TfCtx& t, float f) {
  float x = (f - t.lo) * t.inv_dv;
  if (!(x >= 0.f)) return -1;
  if (x >= (float)(t.n - 1)) return t.n - 1;
  return (int)x;
}

// Composite y in [0, L] of a polynomial g (coefficients at the sub-piece start)
// lying within TF cell c.  tau_l: accumulated optical depth before the
// sub-piece (local to the lane); C: emitted colour (un-attenuated by the
// lane's incoming transmittance).
template <int D>
__device__ __forceinline__ void composite_cell(const float* Q, float L, int c, const TfCtx& t, float& tau_l,
                                               float* C) {
  if (!(L > 0.f)) return;
  if (c < 0 || c >= t.n - 1) {
    float4 k = t.tf[c < 0 ? 0 : t.n - 1];
    float tau = k.w * L;
    float w = __expf(-tau_l) * (-expm1f(-tau));
    C[0] += k.x * w;
    C[1] += k.y * w;
    C[2] += k.z * w;
    tau_l += tau;
    return;
  }
  float4 a = t.tf[c], b = t.tf[c + 1];
  float vc = t.lo + c * t.dv;
  float g[D + 1];
#pragma unroll
  for (int d = 0; d <= D; ++d) g[d] = Q[d];
  g[0] -= vc;
  float s1 = (b.w - a.w) * t.inv_dv;
  float cr = (b.x - a.x) * t.inv_dv, cg = (b.y - a.y) * t.inv_dv, cb = (b.z - a.z) * t.inv_dv;
  // sub-divide when the sub-piece is optically thick, so that 2-point
  // Gauss-Legendre stays accurate
  float tauL = a.w * L + s1 * horner_int<D>(g, L);
  int ns = 1;
  if (tauL > 0.25f) ns = min(32, (int)ceilf(tauL * 4.f));
  float h = L / ns;
  const float x0 = 0.21132486540518713f, x1 = 0.78867513459481287f;
  float Gprev = 0.f;
  for (int s = 0; s < ns; ++s) {
    float ya = s * h;
    float y0 = ya + x0 * h, y1 = ya + x1 * h;
    float G0 = horner_int<D>(g, y0), G1 = horner_int<D>(g, y1);
    float g0 = horner<D>(g, y0), g1 = horner<D>(g, y1);
    float e0 = __expf(-(tau_l + a.w * y0 + s1 * G0));
    float e1 = __expf(-(tau_l + a.w * y1 + s1 * G1));
    float sg0 = fmaxf(a.w + s1 * g0, 0.f) * e0, sg1 = fmaxf(a.w + s1 * g1, 0.f) * e1;
    float hw = 0.5f * h;
    C[0] += hw * ((a.x + cr * g0) * sg0 + (a.x + cr * g1) * sg1);
    C[1] += hw * ((a.y + cg * g0) * sg0 + (a.y + cg * g1) * sg1);
    C[2] += hw * ((a.z + cb * g0) * sg0 + (a.z + cb * g1) * sg1);
    (void)Gprev;
  }
  tau_l += tauL;
}

template <int D>
__device__ __noinline__ void composite_piece_slow(const float* P, float L, float f0, const TfCtx& t, float& tau_l,
                                                   float* C);

// Composite [0, L] of piece polynomial P (coefficients at the piece start).
template <int D>
__device__ __forceinline__ void composite_piece(const float* P, float L, const TfCtx& t, float& tau_l, float* C) {
  if (!(L > 0.f)) return;
  float f0 = P[0], f1 = horner<D>(P, L);
  // bound on |P - linear interpolant| over [0, L]: L^2/8 max|P''|
  float b2 = 0.f, Lp = 1.f;
#pragma unroll
  for (int d = 2; d <= D; ++d) {
    b2 += d * (d - 1) * fabsf(P[d]) * Lp;
    Lp *= L;
  }
  float dev = 0.125f * L * L * b2;
  int ca = tf_cell(t, fminf(f0, f1) - dev), cb = tf_cell(t, fmaxf(f0, f1) + dev);
  if (ca == cb) {
    composite_cell<D>(P, L, ca, t, tau_l, C);
    return;
  }
  composite_piece_slow<D>(P, L, f0, t, tau_l, C);
}

// Pieces that may cross transfer-function nodes: 8 sub-intervals, node
// crossings by bisection inside each (kept out of line: rare on dense data).
template <int D>
__device__ __noinline__ void composite_piece_slow(const float* P, float L, float f0, const TfCtx& t, float& tau_l,
                                                   float* C) {
  const int NS = 8;
  float step = L / NS, ya = 0.f, fa = f0;
#pragma unroll 1
  for (int s = 1; s <= NS; ++s) {
    float yb = (s == NS) ? L : s * step;
    float fb = horner<D>(P, yb);
    int c0 = tf_cell(t, fa), c1 = tf_cell(t, fb);
    float ycur = ya;
    int ccur = c0;
    while (ccur != c1) {
      int cn = c1 > ccur ? ccur + 1 : ccur - 1;
      float v = t.lo + (c1 > ccur ? cn : ccur) * t.dv;  // boundary between ccur and cn
      float lo_y = ycur, hi_y = yb;
      bool up = c1 > ccur;
      for (int it = 0; it < 24; ++it) {
        float mid = 0.5f * (lo_y + hi_y);
        float fm = horner<D>(P, mid);
        if ((fm < v) == up) lo_y = mid; else hi_y = mid;
      }
      float yc = 0.5f * (lo_y + hi_y);
      float Q[D + 1];
#pragma unroll
      for (int d = 0; d <= D; ++d) Q[d] = P[d];
      taylor_shift<D, float>(Q, ycur);
      composite_cell<D>(Q, yc - ycur, ccur, t, tau_l, C);
      ycur = yc;
      ccur = cn;
    }
    float Q[D + 1];
#pragma unroll
    for (int d = 0; d <= D; ++d) Q[d] = P[d];
    taylor_shift<D, float>(Q, ycur);
    composite_cell<D>(Q, yb - ycur, ccur, t, tau_l, C);
    ya = yb;
    fa = fb;
  }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

struct WarpTable {
  float* tc_hi;
  float* tc_lo;
  float* hh;
  float* cc;
  float* tnext;
  float* fst;  // lower bound on the particle's first knot when it was staged;
               // non-decreasing along the table (batches arrive in bound order)
  int* meta;  // j | kn << 16 (kn = knots of this particle already passed)
  float* wk;  // emission buffer: position
  int* wv;    //                  entry | knot << 16
  float* sk;  // sorted buffer
  int* sv;
  int* hist;  // kNb bucket counts, then kNb offsets
  int* misc;  // [0] emission counter
};

__device__ __forceinline__ int meta_j(int m) { return m & 0xffff; }
__device__ __forceinline__ int meta_kn(int m) { return (m >> 16) & 0xff; }

// normalised knot offset of sorted knot k of an entry with knots (theta_1, theta_2)
__device__ __forceinline__ float knot_sigma(int K, int m, float2 th, int k) {
  if (K & 1) {
    if (k < m) { int s = m - k; return -(s == 1 ? th.x : th.y); }
    int s = k - m + 1;
    return s == 1 ? th.x : th.y;
  }
  if (k < m) { int s = m - k; return -(s == 1 ? th.x : th.y); }
  if (k == m) return 0.f;
  int s = k - m;
  return s == 1 ? th.x : th.y;
}

// slot (0 middle, s >= 1 theta_s) and mirror flag of sorted knot k
__device__ __forceinline__ int knot_slot(int K, int m, int k, bool& mirror) {
  mirror = k < m;
  if (k < m) return m - k;
  if (K & 1) return k - m + 1;
  return k - m;  // 0 for the middle knot
}

template <int D>
__device__ __forceinline__ void knot_delta(const RenderParams& p, const WarpTable& T, int e, int k, float* dl) {
  int j = meta_j(T.meta[e]);
  bool mir;
  int slot = knot_slot(p.K, p.m, k, mir);
  const float* jr = p.jump + (size_t)j * 3 * D + slot * D;
  float ih = 1.f / T.hh[e], s = T.cc[e];
  dl[0] = 0.f;
#pragma unroll
  for (int d = 1; d <= D; ++d) {
    s *= ih;
    float v = __ldg(jr + d - 1) * s;
    dl[d] = (mir && !(d & 1)) ? -v : v;
  }
}

// Exact coefficients at Ta of entry e's current piece (the one after its kn-1-th knot).
template <int D>
__device__ __forceinline__ void entry_piece_at(const RenderParams& p, const WarpTable& T, int e, df Ta, float* A) {
  int mt = T.meta[e], j = meta_j(mt), kn = meta_kn(mt), pc = kn - 1;
  int K = p.K, m = p.m, kp;
  float sg;
  if (!(K & 1)) {
    if (pc < m) { kp = m - pc; sg = -1.f; } else { kp = pc - m + 1; sg = 1.f; }
  } else {
    if (pc < m - 1) { kp = m - pc; sg = -1.f; }
    else if (pc == m - 1) { kp = 1; sg = 1.f; }
    else { kp = pc - m + 2; sg = 1.f; }
  }
  float2 th = __ldg(p.theta + j);
  float th0 = kp == 1 ? 0.f : th.x;
  float h = T.hh[e];
  float rel = (Ta.hi - T.tc_hi[e]) + (Ta.lo - T.tc_lo[e]);
  float z = sg * rel / h - th0;
  const float* pr = p.piece + (size_t)j * 2 * (D + 1) + (kp - 1) * (D + 1);
  float q[D + 1];
#pragma unroll
  for (int d = 0; d <= D; ++d) q[d] = __ldg(pr + d);
  taylor_shift<D, float>(q, z);
  float s = T.cc[e], f = sg / h;
#pragma unroll
  for (int d = 0; d <= D; ++d) {
    A[d] = q[d] * s;
    s *= f;
  }
}

// Per-warp window buffers live in shared memory; the candidate table of the
// ray lives in global scratch (L1-cached) so that dense regions never run out
// of room.
template <int D, typename S, int NW, bool DBG>
__global__ void __launch_bounds__(NW * 32, (NW == 4 ? 4 : 1)) k_render(RenderParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // ---- shared memory carve-up
  float4* s_tf = (float4*)smem;
  unsigned char* ptr = smem + sizeof(float4) * p.tf_n;
  float4* s_pos = (float4*)ptr;
  ptr += sizeof(float4) * kStage;
  float4* s_sph = (float4*)ptr;  // bounding sphere (centre, radius + q h_max) per staged chunk
  ptr += sizeof(float4) * kStageChunks;
  float* s_amp = (float*)ptr;
  ptr += sizeof(float) * kStage;
  int* s_idx = (int*)ptr;
  ptr += sizeof(int) * kStage;
  int* s_plan = (int*)ptr;  // [0..kStageChunks-1] chunk ids, [kStageChunks] count, [+1] work item
  ptr += sizeof(int) * (kStageChunks + 4);
  float* s_F = (float*)ptr;
  ptr += sizeof(float) * 4;
  const size_t per_warp = (sizeof(float) + sizeof(int)) * 2 * kW + sizeof(int) * (2 * kNb + 4);
  WarpTable T;
  {
    unsigned char* b = ptr + per_warp * wid;
    T.wk = (float*)b; b += sizeof(float) * kW;
    T.wv = (int*)b; b += sizeof(int) * kW;
    T.sk = (float*)b; b += sizeof(float) * kW;
    T.sv = (int*)b; b += sizeof(int) * kW;
    T.hist = (int*)b; b += sizeof(int) * 2 * kNb;
    T.misc = (int*)b;
    float* g = p.scratch + (size_t)(blockIdx.x * NW + wid) * kTableWords;
    T.tc_hi = g;
    T.tc_lo = g + kCap;
    T.hh = g + 2 * kCap;
    T.cc = g + 3 * kCap;
    T.tnext = g + 4 * kCap;
    T.fst = g + 5 * kCap;
    T.meta = (int*)(g + 6 * kCap);
  }
  for (int i = threadIdx.x; i < p.tf_n; i += blockDim.x) s_tf[i] = p.tf[i];
  TfCtx tfc{s_tf, p.tf_n, p.tf_lo, p.tf_inv_dv, p.tf_dv};
  unsigned long long st_cand = 0, st_tests = 0, st_knots = 0, st_win = 0, st_rays = 0, st_ert = 0, st_capped = 0;
  int st_maxtab = 0, st_flags = 0, st_maxact = 0;
  PT_DECL
  const int K = p.K, m = p.m;
  const float q = p.q;
  const float t_near = (float)p.cam.t_near;
  const df t_near_df = df_from_double(p.cam.t_near);

  for (int it = 0;; ++it) {
    // ------------------------------------------------------------ work item
    int item;
    if (DBG) {
      item = blockIdx.x + it * gridDim.x;
    } else if (p.dynamic) {
      __syncthreads();
      if (threadIdx.x == 0) s_plan[kStageChunks + 1] = (int)atomicAdd(p.work, 1u);
      __syncthreads();
      item = s_plan[kStageChunks + 1];
    } else {
      item = blockIdx.x + it * gridDim.x;
    }
    if (item >= (DBG ? p.n_dbg : p.n_items)) break;

    // ---- which rays
    int tile, px, py, sx0, sy0, sx1, sy1;
    long long dbg_row = -1;
    if (DBG) {
      dbg_row = item;
      int pix = p.dbg_pix[item];
      px = pix % p.cam.width;
      py = pix / p.cam.width;
      tile = (py / kTile) * p.tiles_x + px / kTile;
      sx0 = sx1 = px;
      sy0 = sy1 = py;
    } else {
      constexpr int SW = NW == 8 ? 4 : (NW == 4 ? 2 : 1);
      constexpr int SH = NW / SW;
      constexpr int SUB = (kTile / SW) * (kTile / SH);
      tile = item / SUB;
      int sub = item % SUB;
      int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
      sx0 = tx * kTile + (sub % (kTile / SW)) * SW;
      sy0 = ty * kTile + (sub / (kTile / SW)) * SH;
      sx1 = sx0 + SW - 1;
      sy1 = sy0 + SH - 1;
      px = sx0 + wid % SW;
      py = sy0 + wid / SW;
    }
    const bool in_img = px < p.cam.width && py < p.cam.height;

    // ---- the ray, FP64 -> double-float
    df o[3], v[3];
    {
      const DevCamera& c = p.cam;
      double sx = 2.0 * (px + 0.5) / c.width - 1.0, sy = 1.0 - 2.0 * (py + 0.5) / c.height;
      double oo[3], vv[3];
      if (c.proj == 0) {
        double ax = sx * c.tan_half * c.aspect, ay = sy * c.tan_half;
        double nrm = 0;
        for (int i = 0; i < 3; ++i) {
          vv[i] = c.f[i] + ax * c.r[i] + ay * c.u[i];
          nrm += vv[i] * vv[i];
        }
        nrm = sqrt(nrm);
        for (int i = 0; i < 3; ++i) {
          vv[i] /= nrm;
          oo[i] = c.eye[i];
        }
      } else {
        for (int i = 0; i < 3; ++i) {
          oo[i] = c.eye[i] + sx * c.half_w * c.r[i] + sy * c.half_h * c.u[i];
          vv[i] = c.f[i];
        }
      }
      for (int i = 0; i < 3; ++i) {
        o[i] = df_from_double(oo[i]);
        v[i] = df_from_double(vv[i]);
      }
    }

    // ---- per-ray state
    bool done = !in_img;
    bool started = false;
    df Ta = {0.f, 0.f}, t_start = {0.f, 0.f};
    float tau_ray = 0.f, col[3] = {0.f, 0.f, 0.f};
    int n_tab = 0, win_count = 0, new_cands = 0;
    S carry[D + 1];
#pragma unroll
    for (int d = 0; d <= D; ++d) carry[d] = (S)0;
    long long dbg_np = 0;  // field pieces written
    long long dbg_nc = 0;  // candidate ids written
    unsigned long long my_knots = 0;

    const int2 tr = p.tile_range[tile];
    int ci = tr.x;
    const int ce = tr.y;
    float Fprev = -__int_as_float(0x7f800000);  // bound that held before the current batch

    for (;;) {
      // ------------------------------------------------------------------ plan
      PT_BEGIN
      __syncthreads();
      if (wid == 0) {
        int taken = 0;
        float Fnext = __int_as_float(0x7f800000);  // +inf
        bool fset = false;
        while (ci < ce && taken < kStageChunks) {
          int idx = ci + lane;
          bool valid = idx < ce;
          int cid = valid ? (int)p.pair_val[idx] : -1;
          bool ok = false;
          if (valid) {
            float4 r = __ldg(p.chunk_rect + cid);
            ok = r.x <= (float)sx1 + 0.5f && r.z >= (float)sx0 - 0.5f && r.y <= (float)sy1 + 0.5f &&
                 r.w >= (float)sy0 - 0.5f;
          }
          unsigned mk = __ballot_sync(kFull, ok);
          int need = kStageChunks - taken;
          int avail = __popc(mk);
          int rank = __popc(mk & lanemask_lt());
          if (ok && rank < need) s_plan[taken + rank] = cid;
          if (avail >= need) {
            // last taken lane, then the next overlapping one in this batch
            unsigned mm = mk;
            for (int i = 0; i < need - 1; ++i) mm &= mm - 1;
            int last = __ffs(mm) - 1;
            unsigned rest = mk & ~((2u << last) - 1u);
            if (rest) {
              int nl = __ffs(rest) - 1;
              uint64_t key = p.pair_key[ci + nl];
              unsigned ob = (unsigned)(key & 0xffffffffu);
              unsigned b = (ob & 0x80000000u) ? (ob & 0x7fffffffu) : ~ob;
              Fnext = __uint_as_float(b);
              fset = true;
              ci += nl;  // resume at the next overlapping chunk
            } else {
              ci += last + 1;
            }
            taken = kStageChunks;
          } else {
            taken += avail;
            ci += min(32, ce - ci);
          }
        }
        if (!fset && ci < ce) {
          uint64_t key = p.pair_key[ci];
          unsigned ob = (unsigned)(key & 0xffffffffu);
          unsigned b = (ob & 0x80000000u) ? (ob & 0x7fffffffu) : ~ob;
          Fnext = __uint_as_float(b);
        }
        if (lane == 0) {
          s_plan[kStageChunks] = taken;
          s_F[0] = Fnext;
        }
      }
      __syncthreads();
      const int nplan = s_plan[kStageChunks];
      const float F = s_F[0];
      const float Fbatch = Fprev;  // every knot of this batch's particles lies at or beyond it
      Fprev = F;
      // ---------------------------------------------------------------- stage
      for (int i = threadIdx.x; i < nplan * kChunk; i += blockDim.x) {
        int c = s_plan[i / kChunk], r = i % kChunk;
        int2 ch = __ldg(p.chunk + c);
        if (r < ch.y) {
          s_pos[i] = __ldg(p.pos + ch.x + r);
          s_amp[i] = __ldg(p.amp + ch.x + r);
          s_idx[i] = ch.x + r;
        } else {
          s_pos[i] = make_float4(0.f, 0.f, 0.f, 0.f);
          s_amp[i] = 0.f;
          s_idx[i] = -1;
        }
      }
      for (int c = threadIdx.x; c < nplan; c += blockDim.x) {
        int cid = s_plan[c];
        float4 lo = __ldg(p.chunk_lo + cid), hi = __ldg(p.chunk_hi + cid);
        float hx = 0.5f * (hi.x - lo.x), hy = 0.5f * (hi.y - lo.y), hz = 0.5f * (hi.z - lo.z);
        s_sph[c] = make_float4(lo.x + hx, lo.y + hy, lo.z + hz, sqrtf(hx * hx + hy * hy + hz * hz) + q * lo.w);
      }
      __syncthreads();
      if (__syncthreads_and(done ? 1 : 0)) break;
      PT_END(0)

      if (!done) {
        PT_BEGIN
        // ---------------------------------------- chunks this ray can meet
        unsigned cmask = 0;
        {
          bool hit = false;
          if (lane < nplan) {
            float4 sp = s_sph[lane];
            float cx = sp.x - o[0].hi, cy = sp.y - o[1].hi, cz = sp.z - o[2].hi;
            float t = cx * v[0].hi + cy * v[1].hi + cz * v[2].hi;
            float wx = cx - t * v[0].hi, wy = cy - t * v[1].hi, wz = cz - t * v[2].hi;
            float rr = sp.w + 1e-5f * (fabsf(t) + fabsf(cx) + fabsf(cy) + fabsf(cz) + 1e-2f);
            hit = wx * wx + wy * wy + wz * wz <= rr * rr;
          }
          cmask = __ballot_sync(kFull, hit);
        }
        // ------------------------------------------------------ candidates
        while (cmask) {
          const int cidx = __ffs(cmask) - 1;
          cmask &= cmask - 1;
          const int i = cidx * kChunk + lane;
          bool cand = false;
          df tc = {0.f, 0.f};
          float h = 0.f, d2 = 0.f, a = 0.f;
          df wv[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
          {
            float4 P = s_pos[i];
            h = P.w;
            if (h > 0.f) {
              ++st_tests;
              float R = q * h;
              float px_ = P.x - o[0].hi, py_ = P.y - o[1].hi, pz_ = P.z - o[2].hi;
              float t = px_ * v[0].hi + py_ * v[1].hi + pz_ * v[2].hi;
              float wx = px_ - t * v[0].hi, wy = py_ - t * v[1].hi, wz = pz_ - t * v[2].hi;
              float d2f = wx * wx + wy * wy + wz * wz;
              float tol = 4e-6f * (fabsf(t) + fabsf(px_) + fabsf(py_) + fabsf(pz_) + 1e-3f);
              float Rt = R + tol;
              if (d2f < Rt * Rt) {
                // double-float: p = chi - o, t = p.v, w = p - t v
                df pp[3];
                float pc3[3] = {P.x, P.y, P.z};
#pragma unroll
                for (int k = 0; k < 3; ++k) pp[k] = df_add(df{pc3[k], 0.f}, df_neg(o[k]));
                df tt = df_add(df_add(df_mul(pp[0], v[0]), df_mul(pp[1], v[1])), df_mul(pp[2], v[2]));
                float dd = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                  df w = df_add(pp[k], df_neg(df_mul(tt, v[k])));
                  dd = fmaf(w.hi, w.hi, fmaf(2.f * w.hi, w.lo, dd));
                  wv[k] = w;
                }
                float R2 = R * R;
                if (dd < R2) {
                  float ex = tt.hi + sqrtf(fmaxf(R2 - dd, 0.f));
                  if (ex > t_near) {
                    cand = true;
                    tc = tt;
                    d2 = dd;
                    a = s_amp[i];
                  }
                }
              }
            }
          }
          unsigned mk = __ballot_sync(kFull, cand);
          if (!mk) continue;
          int rank = __popc(mk & lanemask_lt());
          int slot = n_tab + rank;
          if (cand) {
            if (slot < kCap) {
              // table entry: nearest L entry (FP64 re-check near a midpoint)
              float x = sqrtf(d2) / h * p.lam_scale;
              int j = (int)floorf(x + 0.5f);
              float fr = x - floorf(x);
              if (fabsf(fr - 0.5f) < 2e-3f) {
                // near a midpoint: decide in FP64 from the double-float components
                double d2d = 0.0;
                for (int k = 0; k < 3; ++k) {
                  double wk = (double)wv[k].hi + (double)wv[k].lo;
                  d2d += wk * wk;
                }
                double xd = sqrt(d2d) / (double)h * ((double)(p.n_lambda - 1) / (double)q);
                j = (int)floor(xd + 0.5);
              }
              j = min(max(j, 0), p.n_lambda - 1);
              T.tc_hi[slot] = tc.hi;
              T.tc_lo[slot] = tc.lo;
              T.hh[slot] = h;
              T.cc[slot] = a / (h * h * h);
              T.meta[slot] = j;
              float2 th = __ldg(p.theta + j);
              float tn = tc.hi + knot_sigma(K, m, th, 0) * h;
              T.tnext[slot] = tn;
              T.fst[slot] = Fbatch;
              // a first knot before the processed part of the ray would mean the
              // ordering bound was violated: report it
              if (started && tn < Ta.hi - 1e-6f * fabsf(Ta.hi)) st_flags |= 8;
              if (DBG && p.dbg_cands) {
                long long ci2 = dbg_nc + rank;
                if (ci2 < p.cand_cap) p.dbg_cands[dbg_row * p.cand_cap + ci2] = p.orig[s_idx[i]];
              }
            } else {
              st_flags |= 1;
            }
          }
          int added = __popc(mk);
          st_cand += added;
          dbg_nc += added;
          new_cands += added;
          n_tab = min(kCap, n_tab + added);
        }
        st_maxtab = max(st_maxtab, n_tab);
        __syncwarp();
        PT_END(1)

        // ------------------------------------------------------ windows
        // process once enough knots are final, at the end of the stream, or
        // when the table fills up
        const bool go = !(F < __int_as_float(0x7f800000)) || new_cands >= kDefer || n_tab > kCap - 2 * kStage;
        if (go) new_cands = 0;
        while (go && !done) {
          PT_BEGIN
          // lcap: longest window for which FP32 round-off stays small relative to
          // every particle with a knot in it -- gamma h for an active particle; for
          // a pending one, the window may run up to its first knot or gamma h
          // beyond Ta, whichever is farther
          int n_act = 0, n_fin = 0;
          float tmin = __int_as_float(0x7f800000), lcap = __int_as_float(0x7f800000);
          for (int e = lane; e < n_tab; e += 32) {
            int kn = meta_kn(T.meta[e]);
            if (kn > K) {
              ++n_fin;
              continue;
            }
            float tn = T.tnext[e], gh = p.window_h * T.hh[e];
            tmin = fminf(tmin, tn);
            if (kn >= 1) {
              ++n_act;
              lcap = fminf(lcap, gh);
            } else {
              lcap = fminf(lcap, fmaxf(tn - Ta.hi, gh));
            }
          }
          n_act = warp_sum_i(n_act);
          n_fin = warp_sum_i(n_fin);
          st_maxact = max(st_maxact, n_act);
          tmin = warp_min(tmin);
          lcap = warp_min(lcap);
          PT_END(2)
          PT_BEGIN
          if (tmin == __int_as_float(0x7f800000)) {
            n_tab = 0;
            break;
          }
          bool fresh = false;
          if (n_act == 0) {
            if (!(tmin < F)) break;
            // exact position of the first pending knot
            int ebest = -1;
            for (int e0 = 0; e0 < n_tab; e0 += 32) {
              int e = e0 + lane;
              bool hitm = e < n_tab && meta_kn(T.meta[e]) <= K && T.tnext[e] == tmin;
              unsigned who = __ballot_sync(kFull, hitm);
              if (who) {
                ebest = e0 + __ffs(who) - 1;
                break;
              }
            }
            if (ebest < 0) {  // cannot happen: tmin is one of the entries' values
              st_flags |= 4;
              done = true;
              n_tab = 0;
              break;
            }
            int mt = T.meta[ebest];
            float2 th = __ldg(p.theta + meta_j(mt));
            float sgm = knot_sigma(K, m, th, meta_kn(mt));
            df kp = df{T.tc_hi[ebest], T.tc_lo[ebest]};
            {
              float pr = sgm * T.hh[ebest];
              float pe = fmaf(sgm, T.hh[ebest], -pr);
              kp = df_add(kp, df{pr, pe});
            }
            if (started) {
              // gap: field identically 0 on [Ta, kp)
              df a0 = df_add(Ta, df_neg(t_start));
              float from = a0.hi + a0.lo > 0.f ? 0.f : -(a0.hi + a0.lo);
              df gl = df_add(kp, df_neg(Ta));
              float L = gl.hi + gl.lo - from;
              if (L > 0.f) {
                float z0[D + 1];
#pragma unroll
                for (int d = 0; d <= D; ++d) z0[d] = 0.f;
                float tl = 0.f, Cg[3] = {0.f, 0.f, 0.f};
                composite_cell<D>(z0, L, tf_cell(tfc, 0.f), tfc, tl, Cg);
                float w = __expf(-tau_ray);
                col[0] += w * Cg[0];
                col[1] += w * Cg[1];
                col[2] += w * Cg[2];
                tau_ray += tl;
              }
              if (DBG && p.dbg_field && lane == 0 && dbg_np < p.field_cap) {
                double* fo = p.dbg_field + ((size_t)dbg_row * p.field_cap + dbg_np) * (D + 3);
                fo[0] = df_to_double(Ta);
                fo[1] = df_to_double(kp);
                for (int d = 0; d <= D; ++d) fo[2 + d] = 0.0;
              }
              if (DBG && df_to_double(kp) > df_to_double(Ta)) ++dbg_np;
            } else {
              started = true;
              t_start = (df_to_double(kp) > (double)p.cam.t_near) ? kp : t_near_df;
            }
            Ta = kp;
            fresh = true;
#pragma unroll
            for (int d = 0; d <= D; ++d) carry[d] = (S)0;
          }
          // a window ends at the bound F, and spans at most lcap (above); at a
          // fresh start the pending particle at Ta bounds it by its own gamma h
          float Uh_lim = lcap;
          if (fresh) {
            float l2 = __int_as_float(0x7f800000);
            for (int e = lane; e < n_tab; e += 32) {
              int kn = meta_kn(T.meta[e]);
              if (kn > K) continue;
              float tn = T.tnext[e], gh = p.window_h * T.hh[e];
              l2 = fminf(l2, fmaxf(tn - Ta.hi, gh));
            }
            Uh_lim = warp_min(l2);
          }
          const bool finF = F < __int_as_float(0x7f800000);
          float Ulim = finF ? ((F - Ta.hi) - Ta.lo) : __int_as_float(0x7f800000);
          const bool capped = Uh_lim < Ulim;
          if (capped) {
            Ulim = Uh_lim;
            ++st_capped;
          }
          // prefilter on the approximate next-knot position (absolute FP32)
          const float Wend = fminf(F, Ta.hi + Ulim);
          const float Fpre = Wend + 1e-3f * fabsf(Wend) + 1e-30f;
          int cnt = 0;
          float umax = 0.f;
          for (int e = lane; e < n_tab; e += 32) {
            if (!(T.fst[e] < Fpre)) break;  // this and all later entries start beyond the window
            int mt = T.meta[e], kn = meta_kn(mt);
            if (kn > K || !(T.tnext[e] < Fpre)) continue;
            float2 th = __ldg(p.theta + meta_j(mt));
            float base = (T.tc_hi[e] - Ta.hi) + (T.tc_lo[e] - Ta.lo), hh = T.hh[e];
            for (int k = kn; k <= K; ++k) {
              float u = fmaf(knot_sigma(K, m, th, k), hh, base);
              if (!(u < Ulim)) break;
              ++cnt;
              umax = fmaxf(umax, u);
            }
          }
          cnt = warp_sum_i(cnt);
          umax = warp_max(umax);
          // no knot below the bound: wait for more particles, unless the window
          // was capped -- then the current polynomial alone spans it
          if (cnt == 0 && !capped) break;
          // choose the window: all knots below Ulim, or a bucket prefix of them
          float Ub = Ulim, Uh = 0.f;
          int bstar = kNb;
          bool by_bucket = false;
          if (cnt > kW) {
            by_bucket = true;
            Uh = umax > 0.f ? umax : 1e-30f;
            bool fixed = false;
            for (int zoom = 0; zoom < 6 && !fixed; ++zoom) {
              for (int b = lane; b < kNb; b += 32) T.hist[b] = 0;
              __syncwarp();
              float sc = kNb / Uh;
              for (int e = lane; e < n_tab; e += 32) {
                if (!(T.fst[e] < Fpre)) break;
                int mt = T.meta[e], kn = meta_kn(mt);
                if (kn > K || !(T.tnext[e] < Fpre)) continue;
                float2 th = __ldg(p.theta + meta_j(mt));
                float base = (T.tc_hi[e] - Ta.hi) + (T.tc_lo[e] - Ta.lo), hh = T.hh[e];
                for (int k = kn; k <= K; ++k) {
                  float u = fmaf(knot_sigma(K, m, th, k), hh, base);
                  if (!(u < Ulim)) break;
                  int b = min(kNb - 1, max(0, (int)fminf(u * sc, (float)kNb)));
                  if (u <= Uh) atomicAdd(&T.hist[b], 1);
                }
              }
              __syncwarp();
              // inclusive scan over the 64 buckets (2 per lane)
              int h0 = T.hist[2 * lane], h1 = T.hist[2 * lane + 1];
              int s2 = h0 + h1, x = s2;
#pragma unroll
              for (int o2 = 1; o2 < 32; o2 <<= 1) {
                int y = __shfl_up_sync(kFull, x, o2);
                if (lane >= o2) x += y;
              }
              int ex = x - s2;  // count in buckets < 2 lane
              // largest b with count(bucket < b) <= kW
              int bl = -1;
              if (ex + h0 <= kW) bl = 2 * lane + 1;
              if (ex + h0 + h1 <= kW) bl = 2 * lane + 2;
              if (ex > kW) bl = -1;
              int bbest = bl;
#pragma unroll
              for (int o2 = 16; o2; o2 >>= 1) bbest = max(bbest, __shfl_xor_sync(kFull, bbest, o2));
              if (bbest >= 1) {
                bstar = bbest;
                fixed = true;
              } else {
                Uh = Uh / kNb;  // first bucket too full: zoom into it
              }
              __syncwarp();
            }
            if (!fixed) {
              st_flags |= 2;
              bstar = 1;
            }
            Ub = (bstar >= kNb) ? Uh : Uh * ((float)bstar / kNb);
          }

          PT_END(3)
          PT_BEGIN
          // anchor: exact coefficients of the field at Ta
          S A[D + 1];
          bool do_anchor = p.anchor_every > 0 && (fresh || (win_count % p.anchor_every) == 0);
          if (fresh) {
#pragma unroll
            for (int d = 0; d <= D; ++d) A[d] = (S)0;
          } else if (do_anchor) {
            float acc[D + 1];
#pragma unroll
            for (int d = 0; d <= D; ++d) acc[d] = 0.f;
            for (int e = lane; e < n_tab; e += 32) {
              if (!(T.fst[e] < Ta.hi + 1e-6f * fabsf(Ta.hi))) break;  // later entries have not started
              int kn = meta_kn(T.meta[e]);
              if (kn < 1 || kn > K) continue;
              float Ae[D + 1];
              entry_piece_at<D>(p, T, e, Ta, Ae);
#pragma unroll
              for (int d = 0; d <= D; ++d) acc[d] += Ae[d];
            }
#pragma unroll
            for (int d = 0; d <= D; ++d) A[d] = (S)warp_sum(acc[d]);
          } else {
#pragma unroll
            for (int d = 0; d <= D; ++d) A[d] = carry[d];
          }
          PT_END(4)
          PT_BEGIN
          // emission of the window's knots
          if (lane == 0) T.misc[0] = 0;
          __syncwarp();
          const float scb = by_bucket ? kNb / Uh : 0.f;
          int act_after = 0;  // particles still active after this window's knots
          for (int e = lane; e < n_tab; e += 32) {
            if (!(T.fst[e] < Fpre)) break;
            int mt = T.meta[e], kn = meta_kn(mt);
            if (kn > K) continue;
            if (!(T.tnext[e] < Fpre)) {
              act_after += kn >= 1;
              continue;
            }
            float2 th = __ldg(p.theta + meta_j(mt));
            float base = (T.tc_hi[e] - Ta.hi) + (T.tc_lo[e] - Ta.lo), hh = T.hh[e];
            int k = kn;
            for (; k <= K; ++k) {
              float u = fmaf(knot_sigma(K, m, th, k), hh, base);
              bool take;
              if (by_bucket) take = u < Ulim && u <= Uh && min(kNb - 1, max(0, (int)fminf(u * scb, (float)kNb))) < bstar;
              else take = u < Ulim;
              if (!take) break;
              int pos = atomicAdd(&T.misc[0], 1);
              if (pos < kW) {
                T.wk[pos] = fmaxf(u, 0.f);
                T.wv[pos] = e | (k << 16);
              }
            }
            if (k != kn) {
              T.meta[e] = meta_j(mt) | (k << 16);
              T.tnext[e] = k <= K ? T.tc_hi[e] + knot_sigma(K, m, th, k) * hh : __int_as_float(0x7f800000);
            }
            act_after += (k >= 1 && k <= K);
          }
          act_after = warp_sum_i(act_after);
          __syncwarp();
          int nwin = min(T.misc[0], kW);
          if (T.misc[0] > kW) st_flags |= 2;
          // no particle is active after the window's last knot: the field is
          // identically zero from there on, so the window ends at that knot (a
          // later knot starts a new segment; the gap is composited only then)
          const bool final_w = nwin > 0 && act_after == 0;
          my_knots += nwin;
          ++st_win;
          ++win_count;
          PT_END(5)
          PT_BEGIN
          // bucket sort of the window by position
          {
            float wmax = 0.f;
            for (int i = lane; i < nwin; i += 32) wmax = fmaxf(wmax, T.wk[i]);
            wmax = warp_max(wmax);
            float sc = wmax > 0.f ? kNb / wmax : 0.f;
            for (int b = lane; b < kNb; b += 32) T.hist[b] = 0;
            __syncwarp();
            int bk[kKpl], rk[kKpl];
#pragma unroll
            for (int r = 0; r < kKpl; ++r) {
              int i = lane + 32 * r;
              if (i < nwin) {
                bk[r] = min(kNb - 1, max(0, (int)fminf(T.wk[i] * sc, (float)kNb)));
                rk[r] = atomicAdd(&T.hist[bk[r]], 1);
              }
            }
            __syncwarp();
            int h0 = T.hist[2 * lane], h1 = T.hist[2 * lane + 1];
            int s2 = h0 + h1, x = s2;
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
              int y = __shfl_up_sync(kFull, x, o2);
              if (lane >= o2) x += y;
            }
            int ex = x - s2;
            T.hist[kNb + 2 * lane] = ex;
            T.hist[kNb + 2 * lane + 1] = ex + h0;
            __syncwarp();
#pragma unroll
            for (int r = 0; r < kKpl; ++r) {
              int i = lane + 32 * r;
              if (i < nwin) {
                int dst = T.hist[kNb + bk[r]] + rk[r];
                T.sk[dst] = T.wk[i];
                T.sv[dst] = T.wv[i];
              }
            }
            __syncwarp();
            // insertion sort inside the two buckets of this lane
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
              int b = 2 * lane + bb;
              int lo = T.hist[kNb + b], n = T.hist[b];
              for (int i = lo + 1; i < lo + n; ++i) {
                float kk = T.sk[i];
                int vv = T.sv[i];
                int jj = i - 1;
                while (jj >= lo && T.sk[jj] > kk) {
                  T.sk[jj + 1] = T.sk[jj];
                  T.sv[jj + 1] = T.sv[jj];
                  --jj;
                }
                T.sk[jj + 1] = kk;
                T.sv[jj + 1] = vv;
              }
            }
            __syncwarp();
          }
          PT_END(6)
          PT_BEGIN
          // ---- segmented scan of the difference coefficients (Sec. 2)
          const float Uend = final_w ? (nwin > 0 ? T.sk[nwin - 1] : 0.f) : Ub;
          float ul[kKpl];
          int pl[kKpl];
#pragma unroll
          for (int r = 0; r < kKpl; ++r) {
            int g = lane * kKpl + r;
            ul[r] = g < nwin ? T.sk[g] : Uend;
            pl[r] = g < nwin ? T.sv[g] : -1;
          }
          S agg[D + 1];
#pragma unroll
          for (int d = 0; d <= D; ++d) agg[d] = (S)0;
          bool has = false;
          float ufirst = ul[0], ulast = ul[0];
#pragma unroll
          for (int r = 0; r < kKpl; ++r) {
            if (pl[r] >= 0) {
              float dl[D + 1];
              knot_delta<D>(p, T, pl[r] & 0xffff, pl[r] >> 16, dl);
              if (has) taylor_shift<D, S>(agg, (S)(ul[r] - ulast));
#pragma unroll
              for (int d = 1; d <= D; ++d) agg[d] += (S)dl[d];
              ulast = ul[r];
              has = true;
            }
          }
          // inclusive warp scan of (agg, ulast, has)
          S sa[D + 1];
#pragma unroll
          for (int d = 0; d <= D; ++d) sa[d] = agg[d];
          float se = ulast;
          int sh = has ? 1 : 0;
#pragma unroll
          for (int o2 = 1; o2 < 32; o2 <<= 1) {
            S oa[D + 1];
#pragma unroll
            for (int d = 0; d <= D; ++d) oa[d] = __shfl_up_sync(kFull, sa[d], o2);
            float oe = __shfl_up_sync(kFull, se, o2);
            int oh = __shfl_up_sync(kFull, sh, o2);
            if (lane >= o2 && oh) {
              if (sh) {
                // (other, oe) (+) (mine, se) = (Shift(other, se - oe) + mine, se)
                taylor_shift<D, S>(oa, (S)(se - oe));
#pragma unroll
                for (int d = 0; d <= D; ++d) sa[d] += oa[d];
              } else {
#pragma unroll
                for (int d = 0; d <= D; ++d) sa[d] = oa[d];
                se = oe;
                sh = 1;
              }
            }
          }
          // exclusive prefix
          S pa[D + 1];
#pragma unroll
          for (int d = 0; d <= D; ++d) pa[d] = __shfl_up_sync(kFull, sa[d], 1);
          float pe = __shfl_up_sync(kFull, se, 1);
          int ph = __shfl_up_sync(kFull, sh, 1);
          if (lane == 0) ph = 0;
          // incoming polynomial at this lane's first knot
          S P[D + 1];
#pragma unroll
          for (int d = 0; d <= D; ++d) P[d] = A[d];
          taylor_shift<D, S>(P, (S)ufirst);
          if (ph) {
            taylor_shift<D, S>(pa, (S)(ufirst - pe));
#pragma unroll
            for (int d = 0; d <= D; ++d) P[d] += pa[d];
          }
          // next lane's first knot (piece end for this lane's last knot)
          float unext = __shfl_down_sync(kFull, ul[0], 1);
          if (lane == 31) unext = Uend;
          // ---- composite this lane's pieces
          float tau_l = 0.f, Cl[3] = {0.f, 0.f, 0.f};
          const df rs = df_add(t_start, df_neg(Ta));
          const float ystart = rs.hi + rs.lo;  // window-relative start of compositing
          if (lane == 0) {
            // leading piece [0, u_0] (or the whole window if it has no knot) with the anchor polynomial
            float Pf[D + 1];
#pragma unroll
            for (int d = 0; d <= D; ++d) Pf[d] = (float)A[d];
            float a0 = fmaxf(0.f, ystart), b0 = ul[0];
            if (b0 > a0) {
              if (a0 > 0.f) taylor_shift<D, float>(Pf, a0);
              composite_piece<D>(Pf, b0 - a0, tfc, tau_l, Cl);
            }
            if (DBG && p.dbg_field && ul[0] > 0.f && dbg_np < p.field_cap) {
              double* fo = p.dbg_field + ((size_t)dbg_row * p.field_cap + dbg_np) * (D + 3);
              fo[0] = df_to_double(Ta);
              fo[1] = df_to_double(Ta) + (double)ul[0];
              for (int d = 0; d <= D; ++d) fo[2 + d] = (double)A[d];
            }
          }
          // count pieces per lane for debug output ordering
          long long dbg_base = 0, npieces = 0;
          if (DBG) {
            int cntp = 0;
#pragma unroll
            for (int r = 0; r < kKpl; ++r) {
              if (pl[r] < 0) continue;
              float en = (r + 1 < kKpl && pl[r + 1] >= 0) ? ul[r + 1] : (r + 1 < kKpl ? Uend : unext);
              if (en > ul[r]) ++cntp;
            }
            int lead = (lane == 0 && ul[0] > 0.f) ? 1 : 0;
            int tot = cntp + lead, xx = tot;
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
              int y = __shfl_up_sync(kFull, xx, o2);
              if (lane >= o2) xx += y;
            }
            dbg_base = dbg_np + (xx - tot) + lead;
            npieces = __shfl_sync(kFull, xx, 31);
          }
          float lastu = ufirst;
          bool any = false;
#pragma unroll
          for (int r = 0; r < kKpl; ++r) {
            if (pl[r] < 0) continue;
            if (any) taylor_shift<D, S>(P, (S)(ul[r] - lastu));
            float dl[D + 1];
            knot_delta<D>(p, T, pl[r] & 0xffff, pl[r] >> 16, dl);
#pragma unroll
            for (int d = 1; d <= D; ++d) P[d] += (S)dl[d];
            any = true;
            lastu = ul[r];
            float en = (r + 1 < kKpl && pl[r + 1] >= 0) ? ul[r + 1] : (r + 1 < kKpl ? Uend : unext);
            float Pf[D + 1];
#pragma unroll
            for (int d = 0; d <= D; ++d) Pf[d] = (float)P[d];
            float a0 = fmaxf(ul[r], ystart);
            if (en > a0) {
              float Q[D + 1];
#pragma unroll
              for (int d = 0; d <= D; ++d) Q[d] = Pf[d];
              if (a0 > ul[r]) taylor_shift<D, float>(Q, a0 - ul[r]);
              composite_piece<D>(Q, en - a0, tfc, tau_l, Cl);
            }
            if (DBG && p.dbg_field && en > ul[r]) {
              if (dbg_base < p.field_cap) {
                double* fo = p.dbg_field + ((size_t)dbg_row * p.field_cap + dbg_base) * (D + 3);
                fo[0] = df_to_double(Ta) + (double)ul[r];
                fo[1] = df_to_double(Ta) + (double)en;
                for (int d = 0; d <= D; ++d) fo[2 + d] = (double)Pf[d];
              }
              ++dbg_base;
            }
          }
          if (DBG) dbg_np += npieces;
          // carry the polynomial to the window end (plain recurrence / next window)
          {
            S cpy[D + 1];
#pragma unroll
            for (int d = 0; d <= D; ++d) cpy[d] = P[d];
            if (any) taylor_shift<D, S>(cpy, (S)(Uend - lastu));
            unsigned anym = __ballot_sync(kFull, any);
            int lastlane = anym ? 31 - __clz(anym) : 0;
#pragma unroll
            for (int d = 0; d <= D; ++d) carry[d] = __shfl_sync(kFull, cpy[d], lastlane);
          }
          // combine lanes: transmittance as accumulated optical depth
          float tx = tau_l;
#pragma unroll
          for (int o2 = 1; o2 < 32; o2 <<= 1) {
            float y = __shfl_up_sync(kFull, tx, o2);
            if (lane >= o2) tx += y;
          }
          float tex = tx - tau_l;
          float w = __expf(-(tau_ray + tex));
          float c0 = warp_sum(w * Cl[0]), c1 = warp_sum(w * Cl[1]), c2 = warp_sum(w * Cl[2]);
          col[0] += c0;
          col[1] += c1;
          col[2] += c2;
          tau_ray += __shfl_sync(kFull, tx, 31);
          // advance
          Ta = df_add(Ta, df{Uend, 0.f});
          if (p.tau_ert > 0.f && tau_ray > p.tau_ert) {
            done = true;
            n_tab = 0;
            break;
          }
          PT_END(7)
          PT_BEGIN
          // compact the table when a quarter was finished at the window start
          {
            if (n_fin * 4 >= n_tab || final_w) {
              int wr = 0;
              for (int b0 = 0; b0 < n_tab; b0 += 32) {
                int e = b0 + lane;
                bool keep = e < n_tab && meta_kn(T.meta[e]) <= K;
                float a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0, a7 = 0;
                int a6 = 0;
                if (keep) {
                  a1 = T.tc_hi[e];
                  a2 = T.tc_lo[e];
                  a3 = T.hh[e];
                  a4 = T.cc[e];
                  a5 = T.tnext[e];
                  a6 = T.meta[e];
                  a7 = T.fst[e];
                }
                unsigned km = __ballot_sync(kFull, keep);
                __syncwarp();
                if (keep) {
                  int d = wr + __popc(km & lanemask_lt());
                  T.tc_hi[d] = a1;
                  T.tc_lo[d] = a2;
                  T.hh[d] = a3;
                  T.cc[d] = a4;
                  T.tnext[d] = a5;
                  T.meta[d] = a6;
                  T.fst[d] = a7;
                }
                wr += __popc(km);
                __syncwarp();
              }
              n_tab = wr;
            }
          }
          PT_END(8)
          if (final_w && n_tab == 0) break;
        }
      }
      if (nplan == 0) break;
    }

    // ---- output
    if (in_img) {
      ++st_rays;
      if (p.tau_ert > 0.f && tau_ray > p.tau_ert) ++st_ert;
    }
    st_knots += my_knots;
    if (in_img && lane == 0) {
      float alpha = -expm1f(-tau_ray);
      if (DBG) {
        p.dbg_rgba[4 * dbg_row + 0] = col[0];
        p.dbg_rgba[4 * dbg_row + 1] = col[1];
        p.dbg_rgba[4 * dbg_row + 2] = col[2];
        p.dbg_rgba[4 * dbg_row + 3] = alpha;
        p.dbg_counts[4 * dbg_row + 0] = dbg_nc;
        p.dbg_counts[4 * dbg_row + 1] = (long long)my_knots;
        p.dbg_counts[4 * dbg_row + 2] = dbg_np;
        p.dbg_counts[4 * dbg_row + 3] = st_flags;
      } else {
        float4* o4 = (float4*)p.out;
        o4[(size_t)py * p.cam.width + px] = make_float4(col[0], col[1], col[2], alpha);
      }
    }
  }
  // ---- statistics (one set of atomics per warp)
  unsigned long long tests = st_tests;
#pragma unroll
  for (int o2 = 16; o2; o2 >>= 1) tests += __shfl_xor_sync(kFull, tests, o2);
  if (lane == 0 && p.stats) {
    atomicAdd(p.stats + 0, st_rays);
    atomicAdd(p.stats + 1, st_cand);
    atomicAdd(p.stats + 2, st_knots);
    atomicAdd(p.stats + 3, st_win);
    atomicAdd(p.stats + 5, tests);
    atomicMax(p.stats + 6, (unsigned long long)st_maxtab);
    atomicOr(p.stats + 7, (unsigned long long)st_flags);
    atomicAdd(p.stats + 8, st_ert);
    atomicMax(p.stats + 11, (unsigned long long)st_maxact);
    atomicAdd(p.stats + 12, st_capped);
#ifdef SPHDVR_PHASE_TIMING
    for (int ph = 0; ph < 10; ++ph) atomicAdd(p.stats + 16 + ph, (unsigned long long)pt_acc[ph]);
#endif
  }
}

inline size_t render_smem_bytes(int tf_n, int nw) {
  size_t per_warp = (sizeof(float) + sizeof(int)) * 2 * kW + sizeof(int) * (2 * kNb + 4);
  return sizeof(float4) * tf_n + (sizeof(float4) + sizeof(float) + sizeof(int)) * kStage +
         sizeof(float4) * kStageChunks + sizeof(int) * (kStageChunks + 4) + sizeof(float) * 4 + per_warp * nw;
}

}  // namespace sphdvr
