// Per-ray field reconstruction and compositing kernel.
//
// Every warp is an independent persistent worker that owns one viewing ray at
// a time (no block-wide barriers).  The ray's 16x16 binning tile lists its
// chunks sorted by a lower bound F of every knot position a chunk's particles
// can produce.  Per ray:
//   1. candidate gathering: the warp walks the tile's chunk list, keeps the
//      chunks whose screen rectangle covers the pixel and whose bounding
//      sphere (grown by q h_max) meets the ray, and tests their particles
//      (one per lane) in FP32, and in double-float (hi + lo FP32 pairs) near
//      the decision; a candidate has d < q h and its support ends after
//      t_near (Sec. 3.1);
//   2. per-particle approximation: L = d/h picks the nearest table entry; the
//      particle's K+1 knots are t_chi + h * sigma_k with localized difference
//      coefficients a h^-3 * s_kd / h^d (Sec. 2, Sec. 3.1); the particle gets a
//      slot in the ray's particle table;
//   3. waiting list: new particles are sorted by their first knot (warp bucket
//      sort in shared memory) and merged into the ray's list of particles that
//      have not started yet; every knot below the bound F of the next chunk is
//      final;
//   4. windows: the knots of a window are generated from the active particles
//      (their next knots) and the waiting particles that start inside it, all
//      below the window end, and sorted in shared memory; a window holds at most
//      W knots and is shortened so that FP32 round-off stays small for the
//      particles it touches;
//   5. segmented prefix sum: the coefficient-update recurrence of Sec. 2 as an
//      associative scan over the warp -- (A, e_A) (+) (B, e_B) =
//      (Shift(A, e_B - e_A) + B, e_B) -- seeded with the field's exact
//      coefficients at the window start, summed over the active particles'
//      own pieces (re-anchoring bounds the FP32 drift that Sec. 4.1
//      describes);
//   6. classification + compositing per piece: pieces are split where the
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

constexpr int kCap = 4096;          // particle entries per ray
constexpr int kMaxRayWindows = 1 << 16;  // windows one ray may take in k_render
constexpr int kFlagWindowLimit = 64;     // frame flag: a ray reached kMaxRayWindows (pixel wrong)
constexpr int kNK = 512;            // new knots awaiting a merge (shared memory)
constexpr int kLevels = 128;        // smoothing-length bins (quarter octaves) for the window limit
constexpr int kLevelBase = (127 - 28) << 2;  // bin 0 starts at h = 2^-28
constexpr int kRenderWarps = 4;     // rays (warps) per CTA in normal rendering
// which render kernel a frame runs (by precision mode)
constexpr int kKernRay = 0;     // FP32_ANCHORED, FP32_NAIVE: the lean window kernel k_ray (ray.cuh)
constexpr int kKernF64 = 1;     // FP64_NAIVE: k_render with FP64 running coefficients
constexpr int kKernReinit = 2;  // FP32_REINIT: k_render with reinitialisation knots
constexpr int kKernQuant = 3;   // INT64_QUANT: k_render's quantised integer path
constexpr int kKernRayFB = 4;   // k_ray's fallback pass over the rays its frame pass abandoned
constexpr int kKernRaySh = 5;   // shaded rendering: k_ray with the across-ray gradient (FP32 modes)
constexpr int kKernRayShFB = 6; // its fallback pass
constexpr int kKernRayCp = 7;   // FP32_KAHAN: k_ray with compensated running sums
constexpr int kKernRayCpFB = 8; // its fallback pass
// per-ray global scratch (32-bit words): particle records (4 words), table
// entries, active list, free stack, two buffers of the waiting list (key, value)
constexpr int kTableWords = 11 * kCap;
// per-warp shared memory (bytes): radix histogram, smoothing-length histogram,
// processed-knot counts (4 bits per entry), and a work area shared in time by the new-knot buffers (two key/value
// buffers, the second also stages pending knots during a merge) and the
// window's difference coefficients
constexpr int kWorkBytes = 4 * kNK * 4;
constexpr int kWarpSmem = 256 * 4 + kLevels * 4 + kCap / 2 + kWorkBytes;

// One frame of a batch rendered by a single launch.  The frames' binning
// outputs are concatenated: frame f's tile ranges start at tile_base (and
// index the common pair arrays), its chunk rectangles at f * rect_stride.
struct RenderFrame {
  DevCamera cam;
  int tiles_x, tiles_y, tile_base;
  int item_end;  // work items of this and the preceding frames
  float* out;
};

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
  // gradient tables (shaded rendering): difference coefficients and pieces of
  // G_L = w'(rho)/rho on the same knots, and the shading ka + kd |F'| / sqrt(|grad F|^2 + g0^2)
  const float* gjump;
  const float* gpiece;
  float shade_ka, shade_kd, shade_g2;  // shading: ka, kd and the squared softening gradient g0^2
  // transfer function
  int tf_n;
  float tf_lo, tf_inv_dv, tf_dv;
  const float4* tf;
  // options
  int anchor_every;  // 0: never (naive recurrence)
  float reinit_dt;   // > 0: re-anchor at the reinitialisation knots t = j reinit_dt (naive in between)
  // quantised path (QT instantiation): length quantum tau and value quantum sigma
  double q_tau, q_inv_tau, q_sigma;
  float window_h;    // window length limit in units of the smallest h it touches
  float window_fill; // k_ray: windows aim at this fraction of their capacity from the previous density (>= 1: off)
  float tau_ert;     // stop when accumulated optical depth exceeds this
  float* out;
  unsigned long long* stats;
  float* scratch;       // per-ray scratch: (grid * NW) * kTableWords words
  unsigned* work;       // work-queue counter (dynamic scheduling), zeroed per frame
  int n_items;          // rays (tile-major, 256 per tile); of all frames in a batch
  const RenderFrame* frames;  // batch (BT instantiation): per-frame fields, device memory
  int n_frames;
  int rect_stride;            // batch: chunk rectangles per frame
  int dynamic;          // 1: atomic work queue, 0: static stride
  // k_ray: per-ray capacities of the frame pass (> 0: smaller than the default,
  // to exercise the fallback); the list of abandoned rays ([0] count, then up
  // to ovf_cap work items; nullptr: no fallback, a full buffer only sets a flag)
  int ray_cap;
  unsigned* ovf;
  int ovf_cap;
  // debug
  int n_dbg;
  const int* dbg_pix;
  float* dbg_rgba;
  long long* dbg_counts;
  long long* dbg_cands;
  int cand_cap;
  double* dbg_field;
  int field_cap;
  double* dbg_grad;  // shaded rendering: per field row the across-ray gradient's coefficients [3][D+1]
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

__host__ __device__ constexpr int binom_i(int n, int k) {
  int r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
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
// Shading factor ka + kd |F'(y)| / sqrt(|grad F|^2 + g0^2) at y of a piece (gradient
// extension): the gradient is F'(y) v + (GQ_x, GQ_y, GQ_z)(y), the across-ray part
// being perpendicular to v; g2 = g0^2 softens the cosine where the gradient is small
// (with g0 = 0, a vanishing gradient gives ka + kd).
template <int D>
__device__ __forceinline__ float shade_factor(const float* Q, const float* GQ, float y, float ka, float kd, float g2) {
  float dF = D * Q[D];
#pragma unroll
  for (int d = D - 1; d >= 1; --d) dF = fmaf(dF, y, d * Q[d]);
  const float gx = horner<D>(GQ, y), gy = horner<D>(GQ + D + 1, y), gz = horner<D>(GQ + 2 * (D + 1), y);
  const float n2 = fmaf(dF, dF, fmaf(gx, gx, fmaf(gy, gy, fmaf(gz, gz, g2))));
  return n2 > 0.f ? fmaf(kd, fabsf(dF) * rsqrtf(n2), ka) : ka + kd;
}

// SH: the emission is shaded (shade_factor) with the across-ray gradient
// polynomials GQ[3][D+1] expanded at the same point as Q.
template <int D, bool SH = false>
__device__ __forceinline__ void composite_cell(const float* Q, float L, int c, const TfCtx& t, float& tau_l,
                                               float* C, const float* GQ = nullptr, float ka = 1.f, float kd = 0.f,
                                               float g2 = 0.f) {
  if (!(L > 0.f)) return;
  if (!SH && (c < 0 || c >= t.n - 1)) {
    float4 k = t.tf[c < 0 ? 0 : t.n - 1];
    float tau = k.w * L;
    float w = __expf(-tau_l) * (-expm1f(-tau));
    C[0] += k.x * w;
    C[1] += k.y * w;
    C[2] += k.z * w;
    tau_l += tau;
    return;
  }
  // clamped ends (shaded path): a constant transfer function, integrated like a cell
  const bool clamp = c < 0 || c >= t.n - 1;
  float4 a = t.tf[clamp ? (c < 0 ? 0 : t.n - 1) : c], b = clamp ? a : t.tf[c + 1];
  float vc = clamp ? 0.f : t.lo + c * t.dv;
  float g[D + 1], gi[D + 1];  // g - v_c, and its antiderivative's coefficients over y (gi_d = g_d / (d + 1))
#pragma unroll
  for (int d = 0; d <= D; ++d) g[d] = Q[d];
  g[0] -= vc;
#pragma unroll
  for (int d = 0; d <= D; ++d) gi[d] = g[d] * (1.f / (d + 1));
  float s1 = (b.w - a.w) * t.inv_dv;
  float cr = (b.x - a.x) * t.inv_dv, cg = (b.y - a.y) * t.inv_dv, cb = (b.z - a.z) * t.inv_dv;
  // sub-divide when the sub-piece is optically thick, so that 2-point
  // Gauss-Legendre stays accurate
  float tauL = a.w * L + s1 * (L * horner<D>(gi, L));
  int ns = 1;
  if (tauL > 0.25f) ns = min(32, (int)ceilf(tauL * 4.f));
  const float h = ns == 1 ? L : L / ns;
  const float x0 = 0.21132486540518713f, x1 = 0.78867513459481287f;
  float Gprev = 0.f;
#pragma unroll 1
  for (int s = 0; s < ns; ++s) {
    float ya = s * h;
    float y0 = ya + x0 * h, y1 = ya + x1 * h;
    float G0 = y0 * horner<D>(gi, y0), G1 = y1 * horner<D>(gi, y1);
    float g0 = horner<D>(g, y0), g1 = horner<D>(g, y1);
    float e0 = __expf(-(tau_l + a.w * y0 + s1 * G0));
    float e1 = __expf(-(tau_l + a.w * y1 + s1 * G1));
    float sg0 = fmaxf(a.w + s1 * g0, 0.f) * e0, sg1 = fmaxf(a.w + s1 * g1, 0.f) * e1;
    if (SH) {
      sg0 *= shade_factor<D>(Q, GQ, y0, ka, kd, g2);
      sg1 *= shade_factor<D>(Q, GQ, y1, ka, kd, g2);
    }
    float hw = 0.5f * h;
    C[0] += hw * ((a.x + cr * g0) * sg0 + (a.x + cr * g1) * sg1);
    C[1] += hw * ((a.y + cg * g0) * sg0 + (a.y + cg * g1) * sg1);
    C[2] += hw * ((a.z + cb * g0) * sg0 + (a.z + cb * g1) * sg1);
    (void)Gprev;
  }
  tau_l += tauL;
}

template <int D, bool SH = false>
__device__ __forceinline__ void composite_piece_slow_body(const float* P, float L, float f0, const TfCtx& t,
                                                          float& tau_l, float* C, const float* GP = nullptr,
                                                          float ka = 1.f, float kd = 0.f, float g2 = 0.f);
template <int D>
__device__ __noinline__ void composite_piece_slow(const float* P, float L, float f0, const TfCtx& t, float& tau_l,
                                                   float* C) {
  composite_piece_slow_body<D>(P, L, f0, t, tau_l, C);
}

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
// crossings found inside each by a bracketed root search (kept out of line).
template <int D, bool SH>
__device__ __forceinline__ void composite_piece_slow_body(const float* P, float L, float f0, const TfCtx& t,
                                                          float& tau_l, float* C, const float* GP, float ka,
                                                          float kd, float g2) {
  const int NS = 8;
  const float step = L / NS;
  float ya = 0.f, fa = f0;
#pragma unroll 1
  for (int s = 1; s <= NS; ++s) {
    const float yb = (s == NS) ? L : s * step;
    const float fb = horner<D>(P, yb);
    const int c1 = tf_cell(t, fb);
    float ycur = ya, fcur = fa;
    int ccur = tf_cell(t, fa);
#pragma unroll 1
    for (;;) {
      float yend = yb;
      int cnext = ccur;
      if (ccur != c1) {
        // crossing of the node between ccur and the next cell towards c1:
        // Illinois (modified regula falsi) on P(y) - v, bracketed in [ycur, yb]
        cnext = c1 > ccur ? ccur + 1 : ccur - 1;
        const float v = t.lo + (c1 > ccur ? cnext : ccur) * t.dv;
        float a = ycur, b = yb, ga = fcur - v, gb = fb - v, c = 0.5f * (a + b);
        int side = 0;
#pragma unroll 1
        for (int it = 0; it < 20 && b - a > 1e-7f * L; ++it) {
          c = (gb != ga) ? (a * gb - b * ga) / (gb - ga) : 0.5f * (a + b);
          if (!(c > a && c < b)) c = 0.5f * (a + b);
          const float gc = horner<D>(P, c) - v;
          if (gc == 0.f) break;
          if ((gc > 0.f) == (gb > 0.f)) {
            b = c;
            gb = gc;
            if (side == -1) ga *= 0.5f;
            side = -1;
          } else {
            a = c;
            ga = gc;
            if (side == 1) gb *= 0.5f;
            side = 1;
          }
        }
        yend = c;
      }
      float Q[D + 1];
#pragma unroll
      for (int d = 0; d <= D; ++d) Q[d] = P[d];
      taylor_shift<D, float>(Q, ycur);
      if (SH) {
        float GQ[3 * (D + 1)];
#pragma unroll
        for (int i = 0; i < 3 * (D + 1); ++i) GQ[i] = GP[i];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) taylor_shift<D, float>(GQ + ch * (D + 1), ycur);
        composite_cell<D, true>(Q, yend - ycur, ccur, t, tau_l, C, GQ, ka, kd, g2);
      } else {
        composite_cell<D>(Q, yend - ycur, ccur, t, tau_l, C);
      }
      if (cnext == ccur) break;
      ycur = yend;
      fcur = t.lo + (c1 > ccur ? cnext : ccur) * t.dv;
      ccur = cnext;
    }
    ya = yb;
    fa = fb;
  }
}

template <int D>
struct Poly {
  float c[D + 1];
};
// optical depth and un-attenuated colour accumulated by one lane
struct Acc {
  float tau, r, g, b;
};

// Out of line, with value arguments, so that the render kernel holds a
// single copy of the compositing code.
template <int D>
__device__ __noinline__ Acc composite_piece_v(Poly<D> P, float L, TfCtx t, Acc a) {
  float C[3] = {a.r, a.g, a.b};
  float tau = a.tau;
  composite_piece<D>(P.c, L, t, tau, C);
  return Acc{tau, C[0], C[1], C[2]};
}

// The transfer-function-crossing path with value arguments: a caller's arrays
// stay in registers (a pointer argument of an out-of-line call would put them
// in local memory on every use).
template <int D>
__device__ __noinline__ Acc composite_piece_slow_v(Poly<D> P, float L, float f0, TfCtx t, Acc a) {
  float C[3] = {a.r, a.g, a.b};
  float tau = a.tau;
  composite_piece_slow_body<D>(P.c, L, f0, t, tau, C);
  return Acc{tau, C[0], C[1], C[2]};
}

// Across-ray gradient polynomials of a piece, by value (shaded compositing).
template <int D>
struct Poly3 {
  float c[3 * (D + 1)];
};

template <int D>
__device__ __noinline__ Acc composite_piece_slow_sh_v(Poly<D> P, Poly3<D> G, float L, float f0, TfCtx t, Acc a,
                                                      float ka, float kd, float g2) {
  float C[3] = {a.r, a.g, a.b};
  float tau = a.tau;
  composite_piece_slow_body<D, true>(P.c, L, f0, t, tau, C, G.c, ka, kd, g2);
  return Acc{tau, C[0], C[1], C[2]};
}

// Shaded compositing of [0, L] of a piece P with across-ray gradient GP[3][D+1]:
// one transfer-function cell inline, crossings out of line.
template <int D>
__device__ __forceinline__ void composite_piece_sh_inl(const float* P, const float* GP, float L, const TfCtx& t,
                                                       float& tau_l, float* C, float ka, float kd, float g2) {
  if (!(L > 0.f)) return;
  const float f0 = P[0], f1 = horner<D>(P, L);
  float b2 = 0.f, Lp = 1.f;
#pragma unroll
  for (int d = 2; d <= D; ++d) {
    b2 += d * (d - 1) * fabsf(P[d]) * Lp;
    Lp *= L;
  }
  const float dev = 0.125f * L * L * b2;
  const int ca = tf_cell(t, fminf(f0, f1) - dev), cb = tf_cell(t, fmaxf(f0, f1) + dev);
  if (ca == cb) {
    composite_cell<D, true>(P, L, ca, t, tau_l, C, GP, ka, kd, g2);
    return;
  }
  Poly<D> pp;
  Poly3<D> gg;
#pragma unroll
  for (int d = 0; d <= D; ++d) pp.c[d] = P[d];
#pragma unroll
  for (int i = 0; i < 3 * (D + 1); ++i) gg.c[i] = GP[i];
  const Acc r = composite_piece_slow_sh_v<D>(pp, gg, L, f0, t, Acc{tau_l, C[0], C[1], C[2]}, ka, kd, g2);
  tau_l = r.tau;
  C[0] = r.r;
  C[1] = r.g;
  C[2] = r.b;
}

// Composite [0, L] of piece polynomial P, inline: the common case (the piece
// stays in one transfer-function cell) here, crossings out of line.
template <int D>
__device__ __forceinline__ void composite_piece_inl(const float* P, float L, const TfCtx& t, float& tau_l, float* C) {
  if (!(L > 0.f)) return;
  const float f0 = P[0], f1 = horner<D>(P, L);
  float b2 = 0.f, Lp = 1.f;
#pragma unroll
  for (int d = 2; d <= D; ++d) {
    b2 += d * (d - 1) * fabsf(P[d]) * Lp;
    Lp *= L;
  }
  const float dev = 0.125f * L * L * b2;
  const int ca = tf_cell(t, fminf(f0, f1) - dev), cb = tf_cell(t, fmaxf(f0, f1) + dev);
  if (ca == cb) {
    composite_cell<D>(P, L, ca, t, tau_l, C);
    return;
  }
  Poly<D> pp;
#pragma unroll
  for (int d = 0; d <= D; ++d) pp.c[d] = P[d];
  const Acc r = composite_piece_slow_v<D>(pp, L, f0, t, Acc{tau_l, C[0], C[1], C[2]});
  tau_l = r.tau;
  C[0] = r.r;
  C[1] = r.g;
  C[2] = r.b;
}
// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

// Per-ray scratch: entry arrays, lists and knot buffers in global memory
// (L1/L2-resident while the ray is live); masks and histograms in shared memory.
struct RayScratch {
  float4* ent;   // (t_chi hi, t_chi lo, h, a / h^3)
  int* jj;       // table entry (Lambda index)
  int* act;      // active list: entries whose first knot has been processed
  int* fre;      // free stack of entry slots
  float* wk0;    // waiting particles (first knot not yet composited), sorted by
  int* wv0;      // the FP32 position of their first knot: key, slot (two buffers)
  float* wk1;
  int* wv1;
  int* rh;       // shared: radix histogram (256 bins)
  int* lvl;      // shared: active particles per smoothing-length bin
  unsigned* knc; // shared: knots processed so far per entry (4-bit counts, 8 per word)
  float* nk0;    // shared: new knots (unsorted, then radix ping-pong)
  int* nv0;
  float* nk1;
  int* nv1;
  float* wdl;    // shared: the window's difference coefficients (aliases the new-knot buffers)
};

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

// localized difference coefficients of knot k of a particle with table entry
// j, smoothing length h and amplitude c = a / h^3 (Sec. 2, Sec. 3.1)
template <int D>
__device__ __forceinline__ void knot_delta(const RenderParams& p, int j, float h, float c, int k, float* dl) {
  bool mir;
  int slot = knot_slot(p.K, p.m, k, mir);
  const float* jr = p.jump + (size_t)j * 3 * D + slot * D;
  float ih = __fdividef(1.f, h), s = c;
#pragma unroll
  for (int d = 1; d <= D; ++d) {
    s *= ih;
    float v = __ldg(jr + d - 1) * s;
    dl[d - 1] = (mir && !(d & 1)) ? -v : v;
  }
}

// ---- quantised fixed-point knots (Sec. 4.2-4.4): positions are integer
// multiples of the length quantum tau, difference coefficients of order d
// integer multiples of sigma / tau^d, and the coefficient update is exact
// integer arithmetic.  The int64 operations wrap modulo 2^64; every value the
// rendering reads back (a knot's localized coefficients) is a true integer of
// magnitude below 2^63 when sigma bounds the field as Sec. 4.4 prescribes, and
// wrapping sums and products are exact modulo 2^64, so intermediate overflow
// cannot change it.

// Integers of the quantised path are kept as uint64 (two's complement bit
// patterns): wrapping arithmetic is defined for unsigned types.
typedef unsigned long long u64;

// integer position of sorted knot k (0..K) of a particle: tbar_0 = [t_chi / tau],
// tbar_{+-s} = tbar_0 +- [h theta_s / tau]
__device__ __forceinline__ u64 qknot_pos(const RenderParams& p, float4 E, float2 th, int k) {
  const u64 t0 = (u64)__double2ll_rn(((double)E.x + (double)E.y) * p.q_inv_tau);
  bool mir;
  const int s = knot_slot(p.K, p.m, k, mir);
  if (s == 0) return t0;  // the middle knot (even K)
  const u64 off = (u64)__double2ll_rn((double)E.z * (double)(s == 1 ? th.x : th.y) * p.q_inv_tau);
  return mir ? t0 - off : t0 + off;
}

// Quantised localized difference coefficients, orders 1..D, of sorted knot k of
// a particle (order 0 is zero: the approximations are continuous).  Knots
// +-theta_s take [tau^d c s^_sd / (sigma h^d)], mirrored with (-1)^(d+1); the
// odd orders of the middle knot (even K), resp. of the knots +-theta_1 (odd K,
// in decreasing order), follow from exact shifted evenness about tbar_0.
// Returns false if a rounded coefficient, or the integer knot offset
// [h theta_s / tau] or centre [t_chi / tau], is beyond 2^62 (the quanta are too
// fine for this particle: its integers may wrap).  This is a per-particle
// bound: it does not prove that the sums over many particles stay below 2^63
// (that needs sigma to bound the field, Sec. 4.4).
template <int D>
__device__ __noinline__ bool qknot_coef(const RenderParams& p, float4 E, float2 th, int j, int k, u64* out) {
  const int K = p.K, m = p.m;
  u64 fr[2][D + 1], off[2];
  const double r = p.q_tau / (double)E.z, f = (double)E.w / p.q_sigma;
  bool ok = fabs(((double)E.x + (double)E.y) * p.q_inv_tau) < 4.6116860184273879e18;  // 2^62
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const double offd = (double)E.z * (double)(s == 0 ? th.x : th.y) * p.q_inv_tau;
    ok = ok && fabs(offd) < 4.6116860184273879e18;
    off[s] = (u64)__double2ll_rn(offd);
    const float* jr = p.jump + (size_t)j * 3 * D + (s + 1) * D;
    double g = f;
#pragma unroll
    for (int d = 1; d <= D; ++d) {
      g *= r;
      const double v = s < m ? g * (double)__ldg(jr + d - 1) : 0.0;
      ok = ok && fabs(v) < 4.6116860184273879e18;  // 2^62
      fr[s][d] = (u64)__double2ll_rn(v);
    }
    fr[s][0] = 0;
  }
  // coefficients of the mirrored knot -theta_s: (-1)^(d+1) times those of +theta_s
  auto neg = [&](int s, int d) -> u64 { return (d & 1) ? fr[s][d] : 0ull - fr[s][d]; };
  u64 mid[D + 1];
#pragma unroll
  for (int d = 0; d <= D; ++d) mid[d] = 0;
  if (!(K & 1)) {
#pragma unroll
    for (int d = 1; d <= D; d += 2) {
      u64 acc = 0;
      for (int s = 0; s < m; ++s) {
        u64 pw = 1;
#pragma unroll
        for (int jx = d; jx <= D; ++jx) {
          acc += (u64)binom_i(jx, d) * neg(s, jx) * pw;
          pw *= off[s];
        }
      }
      mid[d] = 0ull - 2ull * acc;
    }
  } else {
#pragma unroll
    for (int d = (D & 1) ? D : D - 1; d >= 1; d -= 2) {
      u64 v = 0;
      for (int s = 1; s < m; ++s) v -= neg(s, d);
      for (int s = 0; s < m; ++s) {
        u64 pw = off[s];
#pragma unroll
        for (int jx = d + 1; jx <= D; ++jx) {
          v -= (u64)binom_i(jx, d) * neg(s, jx) * pw;
          pw *= off[s];
        }
      }
      fr[0][d] = v;  // odd d: the same for +theta_1 and -theta_1
    }
  }
  bool mir;
  const int s = knot_slot(K, m, k, mir);
#pragma unroll
  for (int d = 1; d <= D; ++d) out[d] = s == 0 ? mid[d] : (mir ? neg(s - 1, d) : fr[s - 1][d]);
  return ok;
}

__device__ __forceinline__ int knots_done(const RayScratch& T, int e) { return (T.knc[e >> 3] >> (4 * (e & 7))) & 15; }

// Exact coefficients at Ta of the piece after the first kn knots of a particle
// (entry record E, table entry j).
template <int D>
__device__ __forceinline__ void entry_piece_at(const RenderParams& p, float4 E, int j, int kn, df Ta, float* A) {
  int pc = kn - 1;
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
  const float h = E.z, ih = __fdividef(1.f, h);
  float rel = (Ta.hi - E.x) + (Ta.lo - E.y);
  float z = sg * rel * ih - th0;
  const float* pr = p.piece + (size_t)j * 2 * (D + 1) + (kp - 1) * (D + 1);
  float q[D + 1];
#pragma unroll
  for (int d = 0; d <= D; ++d) q[d] = __ldg(pr + d);
  taylor_shift<D, float>(q, z);
  float s = E.w, f = sg * ih;
#pragma unroll
  for (int d = 0; d <= D; ++d) {
    A[d] = q[d] * s;
    s *= f;
  }
}

// bin of h > 0: exponent and the two leading mantissa bits (quarter octaves)
__device__ __forceinline__ int h_level(float h) {
  return min(kLevels - 1, max(0, (__float_as_int(h) >> 21) - kLevelBase));
}
// lower edge of bin l
__device__ __forceinline__ float level_lo(int l) { return __int_as_float((l + kLevelBase) << 21); }

// order-preserving map of an FP32 value to an unsigned key
__device__ __forceinline__ unsigned f2key(float x) {
  unsigned b = __float_as_uint(x);
  return b ^ ((unsigned)((int)b >> 31) | 0x80000000u);
}

// Stable LSD radix sort (8-bit digits) of n (key, value) pairs by FP32 key,
// one warp; digits that every key shares are skipped.  Returns which buffer
// (0 or 1) holds the result.
__device__ __forceinline__ int warp_radix_sort(float* k0, int* v0, float* k1, int* v1, int n, int* rh) {
  const int lane = threadIdx.x & 31;
  int cur = 0;
  // digits above the highest bit in which the keys differ are shared by all
  unsigned kmin = 0xffffffffu, kmax = 0u;
#pragma unroll 1
  for (int i = lane; i < n; i += 32) {
    const unsigned kk = f2key(k0[i]);
    kmin = min(kmin, kk);
    kmax = max(kmax, kk);
  }
  const unsigned diff = __reduce_min_sync(kFull, kmin) ^ __reduce_max_sync(kFull, kmax);
#pragma unroll 1
  for (int pass = 0; pass < 4; ++pass) {
    const int sh = 8 * pass;
    if ((diff >> sh) == 0u) break;
    const float* kc = cur ? k1 : k0;
    const int* vc = cur ? v1 : v0;
    float* kd = cur ? k0 : k1;
    int* vd = cur ? v0 : v1;
    for (int b = lane; b < 256; b += 32) rh[b] = 0;
    __syncwarp();
#pragma unroll 1
    for (int base = 0; base < n; base += 32) {
      const int i = base + lane;
      const int d = i < n ? (int)((f2key(kc[i]) >> sh) & 255) : 256 + lane;
      const unsigned peers = __match_any_sync(kFull, d);
      if (i < n && (peers & lanemask_lt()) == 0u) atomicAdd(&rh[d], __popc(peers));
    }
    __syncwarp();
    int c[8], s = 0;
    bool all_one = false;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      c[r] = rh[lane * 8 + r];
      s += c[r];
      all_one |= c[r] == n;
    }
    if (__any_sync(kFull, all_one)) continue;  // every key has this digit
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    int ex = x - s;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      rh[lane * 8 + r] = ex;
      ex += c[r];
    }
    __syncwarp();
#pragma unroll 1
    for (int base = 0; base < n; base += 32) {
      const int i = base + lane;
      const bool valid = i < n;
      const float kk = valid ? kc[i] : 0.f;
      const int vv = valid ? vc[i] : 0;
      const int d = valid ? (int)((f2key(kk) >> sh) & 255) : 256 + lane;
      const unsigned peers = __match_any_sync(kFull, d);
      const int rank = __popc(peers & lanemask_lt());
      const int pos = valid ? rh[d] + rank : 0;
      __syncwarp();
      if (valid && rank == 0) rh[d] += __popc(peers);
      __syncwarp();
      if (valid) {
        kd[pos] = kk;
        vd[pos] = vv;
      }
    }
    __syncwarp();
    cur ^= 1;
  }
  return cur;
}

// Sort n <= 512 (key, value) pairs by FP32 key, one warp: 256 buckets over
// [min, max] of the keys (bucket index monotone in the key), a counting pass,
// a scatter (order inside a bucket arbitrary), then insertion sort inside each
// bucket (8 buckets per lane; equal keys by value).  Falls back to the radix sort when a bucket
// holds more than 32 keys.  Returns which buffer (0 or 1) holds the result.
__device__ __forceinline__ int warp_bucket_sort(float* k0, int* v0, float* k1, int* v1, int n, int* rh) {
  const int lane = threadIdx.x & 31;
  float lo = __int_as_float(0x7f800000), hi = -lo;
#pragma unroll 1
  for (int i = lane; i < n; i += 32) {
    lo = fminf(lo, k0[i]);
    hi = fmaxf(hi, k0[i]);
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  if (!(hi > lo)) return 0;  // all keys equal (or n <= 1)
  const float sc = 256.f / (hi - lo);
  if (!(sc < 1e30f)) return warp_radix_sort(k0, v0, k1, v1, n, rh);  // keys closer than FP32 resolves here
  for (int b = lane; b < 256; b += 32) rh[b] = 0;
  __syncwarp();
#pragma unroll 1
  for (int i = lane; i < n; i += 32) atomicAdd(&rh[min(255, (int)((k0[i] - lo) * sc))], 1);
  __syncwarp();
  int c[8], s = 0, cmax = 0;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    c[r] = rh[lane * 8 + r];
    s += c[r];
    cmax = max(cmax, c[r]);
  }
  if (__any_sync(kFull, cmax > 32)) return warp_radix_sort(k0, v0, k1, v1, n, rh);
  int x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  const int base = x - s;
  __syncwarp();
  {
    int ex = base;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      rh[lane * 8 + r] = ex;
      ex += c[r];
    }
  }
  __syncwarp();
#pragma unroll 1
  for (int i = lane; i < n; i += 32) {
    const float kk = k0[i];
    const int pos = atomicAdd(&rh[min(255, (int)((kk - lo) * sc))], 1);
    k1[pos] = kk;
    v1[pos] = v0[i];
  }
  __syncwarp();
  // insertion sort inside this lane's 8 buckets [base, base + s); after the
  // scatter rh[b] holds the end of bucket b (read from shared memory, so that
  // no per-lane array is indexed in the rolled loop)
  {
    int b0 = base;
#pragma unroll 1
    for (int r = 0; r < 8; ++r) {
      const int b1 = rh[lane * 8 + r];
#pragma unroll 1
      for (int i = b0 + 1; i < b1; ++i) {
        const float kk = k1[i];
        const int vv = v1[i];
        int j = i - 1;
        while (j >= b0 && (k1[j] > kk || (k1[j] == kk && v1[j] > vv))) {
          k1[j + 1] = k1[j];
          v1[j + 1] = v1[j];
          --j;
        }
        k1[j + 1] = kk;
        v1[j + 1] = vv;
      }
      b0 = b1;
    }
  }
  __syncwarp();
  return 1;
}

// Merge the sorted pending knots a[0, na) (global) with the sorted new knots
// b[0, nb) (shared) into o[0, nout), nout <= na + nb (the largest keys are
// dropped when it is smaller); equal keys take a first.  The output is made
// in tiles of 32 * 8: the next 256 elements of a are staged in shared memory
// (stk, stv; loaded into registers while the previous tile is merged), each
// lane finds its 8-element slice by a merge-path search and merges it
// sequentially.
__device__ __forceinline__ void warp_tile_merge(const float* ak, const int* av, int na, const float* bk,
                                                const int* bv, int nb, float* ok, int* ov, int nout, float* stk,
                                                int* stv) {
  constexpr int kPer = 8, kTileOut = 32 * kPer;
  const int lane = threadIdx.x & 31;
  float pk_[kPer];
  int pv_[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int i = u * 32 + lane;
    pk_[u] = i < na ? ak[i] : 0.f;
    pv_[u] = i < na ? av[i] : 0;
  }
  int ia0 = 0, ib0 = 0;  // consumed so far
#pragma unroll 1
  for (int o0 = 0; o0 < nout; o0 += kTileOut) {
    const int ta = min(kTileOut, na - ia0);  // staged part of a
    const int tb = nb - ib0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int i = u * 32 + lane;
      if (i < ta) {
        stk[i] = pk_[u];
        stv[i] = pv_[u];
      }
    }
    __syncwarp();
    const int tout = min(kTileOut, nout - o0);
    const float* bt = bk + ib0;
    const int* bvt = bv + ib0;
    // merge path: a elements among the first d outputs of this tile
    auto path = [&](int d) -> int {
      int lo = max(0, d - tb), hi = min(d, ta);
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (!(bt[d - 1 - mid] < stk[mid])) lo = mid + 1;
        else hi = mid;
      }
      return lo;
    };
    const int used_a = path(tout);
    // next tile of a, in flight while this one is merged
    const int nx = ia0 + used_a;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int i = nx + u * 32 + lane;
      pk_[u] = i < na ? ak[i] : 0.f;
      pv_[u] = i < na ? av[i] : 0;
    }
    const int d0 = min(lane * kPer, tout), d1 = min(d0 + kPer, tout);
    int ia = path(d0), ib = d0 - ia;
#pragma unroll 1
    for (int d = d0; d < d1; ++d) {
      const bool take_a = ib >= tb || (ia < ta && stk[ia] <= bt[ib]);
      if (take_a) {
        ok[o0 + d] = stk[ia];
        ov[o0 + d] = stv[ia];
        ++ia;
      } else {
        ok[o0 + d] = bt[ib];
        ov[o0 + d] = bvt[ib];
        ++ib;
      }
    }
    __syncwarp();
    ia0 += used_a;
    ib0 += tout - used_a;
  }
  __syncwarp();
}

// Number of keys below w in the sorted range k[lo, hi) (32-ary search).
__device__ __forceinline__ int warp_count_below(const float* k, int lo, int hi, float w) {
  const int lane = threadIdx.x & 31;
  int n = hi - lo, base = lo;
  if (n <= 0) return 0;
  while (n > 32) {
    const int step = (n + 31) / 32;
    const int idx = base + lane * step;
    const unsigned mb = __ballot_sync(kFull, idx < hi && k[idx] < w);
    const int c = __popc(mb);
    if (c == 0) return base - lo;
    base += (c - 1) * step;
    n = min(step, hi - base);
  }
  const unsigned mb = __ballot_sync(kFull, lane < n && k[base + lane] < w);
  return base + __popc(mb) - lo;
}

// One pass over the active list: drops particles whose last knot has been
// processed (their slots go to the free stack) and, if `sum`, adds every
// remaining particle's own piece at Ta (the anchor).  Two entries per lane
// per step so that their loads overlap.
template <int D>
__device__ __forceinline__ void active_pass(const RenderParams& p, const RayScratch& T, int& nal, int& nfree, df Ta,
                                            bool sum, float* acc) {
  const int lane = threadIdx.x & 31;
  const int K = p.K;
  int wr = 0;
#pragma unroll 1
  for (int b0 = 0; b0 < nal; b0 += 64) {
    int e[2], kn[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = b0 + 32 * u + lane;
      e[u] = i < nal ? T.act[i] : -1;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) kn[u] = e[u] >= 0 ? knots_done(T, e[u]) : 0;
    bool keep[2], fin[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      fin[u] = e[u] >= 0 && kn[u] > K;
      keep[u] = e[u] >= 0 && !fin[u];
    }
    if (sum) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (keep[u]) {
          float Ae[D + 1];
          entry_piece_at<D>(p, T.ent[e[u]], T.jj[e[u]], kn[u], Ta, Ae);
#pragma unroll
          for (int d = 0; d <= D; ++d) acc[d] += Ae[d];
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const unsigned km = __ballot_sync(kFull, keep[u]), fm = __ballot_sync(kFull, fin[u]);
      if (keep[u]) T.act[wr + __popc(km & lanemask_lt())] = e[u];
      if (fin[u]) T.fre[nfree + __popc(fm & lanemask_lt())] = e[u];
      wr += __popc(km);
      nfree += __popc(fm);
    }
  }
  __syncwarp();
  nal = wr;
}

// Nearest Lambda entry decided in FP64 from the double-float components of the
// ray-to-particle vector (used near a midpoint between entries).
static __device__ __noinline__ int nearest_entry_fp64(df w0, df w1, df w2, float h, int n_lambda, float q) {
  const double x0 = (double)w0.hi + (double)w0.lo, x1 = (double)w1.hi + (double)w1.lo,
               x2 = (double)w2.hi + (double)w2.lo;
  const double d2d = x0 * x0 + x1 * x1 + x2 * x2;
  const double xd = sqrt(d2d) / (double)h * ((double)(n_lambda - 1) / (double)q);
  return (int)floor(xd + 0.5);
}

// Each warp is an independent worker; the only shared state of a CTA is the
// transfer function.
// RE: reinitialisation knots (precision mode FP32_REINIT), a separate
// instantiation so that the other modes carry none of its code.
// BT: a batch of frames sharing data, table, transfer function and options;
// the work queue spans the rays of all of them.
// QT: the quantised fixed-point path (Sec. 4.2-4.4): knots at integer multiples
// of tau, exact integer coefficient update, no anchoring (nothing drifts).
template <int D, typename S, int NW, bool DBG, bool RE, bool BT = false, bool QT = false>
__global__ void __launch_bounds__(NW * 32, (NW == 4 ? 4 : 1)) k_render(RenderParams p) {
  // knots per lane in a window: as many as the shared work area holds with the
  // window's D difference coefficients, its positions and its knot ids
  // (quantised path: D int64 coefficients, an int64 position, the FP32 position
  // and the id per knot)
  constexpr int KPLQ = kWorkBytes / (32 * (2 * D + 4) * 4) < 16 ? kWorkBytes / (32 * (2 * D + 4) * 4) : 16;
  constexpr int KPL = QT ? KPLQ : (D <= 2 ? 16 : (D == 3 ? 12 : 8));
  constexpr int WCAP = 32 * KPL;
  static_assert(!QT || WCAP * (2 * D + 4) * 4 <= kWorkBytes, "quantised window does not fit the work area");
  static_assert(WCAP * (D + 2) * 4 <= kWorkBytes && WCAP <= kNK, "window does not fit the work area");
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float4* s_tf = (float4*)smem;
  RayScratch T;
  {
    unsigned char* b = smem + sizeof(float4) * p.tf_n + (size_t)kWarpSmem * wid;
    T.rh = (int*)b;
    T.lvl = (int*)(b + 256 * 4);
    T.knc = (unsigned*)(b + 256 * 4 + kLevels * 4);
    float* w = (float*)(b + 256 * 4 + kLevels * 4 + kCap / 2);
    T.nk0 = w;
    T.nv0 = (int*)(w + kNK);
    T.nk1 = w + 2 * kNK;
    T.nv1 = (int*)(w + 3 * kNK);
    T.wdl = w;
    float* g = p.scratch + (size_t)(blockIdx.x * NW + wid) * kTableWords;
    T.ent = (float4*)g;
    T.jj = (int*)(g + 4 * kCap);
    T.act = (int*)(g + 5 * kCap);
    T.fre = (int*)(g + 6 * kCap);
    float* q0 = g + 7 * kCap;
    T.wk0 = q0;
    T.wv0 = (int*)(q0 + kCap);
    T.wk1 = q0 + 2 * kCap;
    T.wv1 = (int*)(q0 + 3 * kCap);
  }
  for (int i = threadIdx.x; i < p.tf_n; i += blockDim.x) s_tf[i] = p.tf[i];
  __syncthreads();
  const TfCtx tfc{s_tf, p.tf_n, p.tf_lo, p.tf_inv_dv, p.tf_dv};
  unsigned long long st_cand = 0, st_tests = 0, st_knots = 0, st_win = 0, st_rays = 0, st_ert = 0, st_capped = 0;
  int st_maxtab = 0, st_flags = 0, st_maxact = 0;
  PT_DECL
  const int K = p.K, m = p.m;
  const float q = p.q, gam = p.window_h;
  const float kInf = __int_as_float(0x7f800000);

  for (int it = 0;; ++it) {
    // ------------------------------------------------------------ work item
    int item;
    if (DBG) {
      item = blockIdx.x + it * gridDim.x;
    } else if (p.dynamic) {
      unsigned v = 0;
      if (lane == 0) v = atomicAdd(p.work, 1u);
      item = (int)__shfl_sync(kFull, v, 0);
    } else {
      item = (blockIdx.x * NW + wid) + it * gridDim.x * NW;
    }
    if (item >= (DBG ? p.n_dbg : p.n_items)) break;
    int fb = 0;  // frame of the ray (batch)
    if (BT) {
      while (fb + 1 < p.n_frames && item >= p.frames[fb].item_end) ++fb;
      if (fb > 0) item -= p.frames[fb - 1].item_end;
    }
    const DevCamera& cam = BT ? p.frames[fb].cam : p.cam;
    const int tiles_x = BT ? p.frames[fb].tiles_x : p.tiles_x;
    const float t_near = (float)cam.t_near;
    const df t_near_df = df_from_double(cam.t_near);
    int tile, px, py;
    long long dbg_row = -1;
    if (DBG) {
      dbg_row = item;
      const int pix = p.dbg_pix[item];
      px = pix % cam.width;
      py = pix / cam.width;
      tile = (py / kTile) * tiles_x + px / kTile;
    } else {
      tile = item >> 8;
      const int sub = item & 255;
      px = (tile % tiles_x) * kTile + (sub & 15);
      py = (tile / tiles_x) * kTile + (sub >> 4);
    }
    if (px >= cam.width || py >= cam.height) continue;
    const float pxf = (float)px, pyf = (float)py;

    // ---- the ray, FP64 -> double-float
    df o[3], v[3];
    {
      const DevCamera& c = cam;
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
    bool done = false, started = false;
    df Ta = {0.f, 0.f}, t_start = {0.f, 0.f};
    float tau_ray = 0.f, col[3] = {0.f, 0.f, 0.f};
    S carry[D + 1];
#pragma unroll
    for (int d = 0; d <= D; ++d) carry[d] = (S)0;
    // quantised path: exact coefficients qc at the integer position qct of the
    // last knot processed
    u64 qc[D + 1], qct = 0;
#pragma unroll
    for (int d = 0; d <= D; ++d) qc[d] = 0;
    int hwm = 0, nfree = 0, nal = 0, n_act = 0, whead = 0, nwait = 0, wb = 0, nnk = 0, win_count = 0;
    bool at_reinit = false;  // the next window starts at a reinitialisation knot
    long long dbg_np = 0, dbg_nc = 0;
    int lane_tan = 0;  // particles within 1e-6 h of tangency (this lane's tests)
    unsigned long long my_knots = 0;
    for (int b = lane; b < kLevels; b += 32) T.lvl[b] = 0;
    __syncwarp();

    const int2 tr = p.tile_range[(BT ? p.frames[fb].tile_base : 0) + tile];
    const int ce = tr.y;
    // the tile list is read 32 entries at a time; each lane keeps its
    // entry's chunk, particle range and bound F for when the chunk is processed
    int gcur = -64, g_cid = 0, g_first = 0, g_cnt = 0;
    unsigned gmask = 0;
    float g_F = 0.f;
    const float oxh = o[0].hi, oyh = o[1].hi, ozh = o[2].hi, vxh = v[0].hi, vyh = v[1].hi, vzh = v[2].hi;
    // next chunk of the tile list at or after `from` that can reach this ray
    auto next_hit = [&](int from) -> int {
      for (;;) {
        if (from >= ce) return ce;
        if (from < gcur || from >= gcur + 32) {
          gcur = from;
          const int idx = from + lane;
          bool hit = false;
          if (idx < ce) {
            g_cid = (int)__ldg(p.pair_val + idx);
            const unsigned ob = (unsigned)(__ldg(p.pair_key + idx) & 0xffffffffu);
            g_F = __uint_as_float((ob & 0x80000000u) ? (ob & 0x7fffffffu) : ~ob);
            const float4 r = __ldg(p.chunk_rect + (BT ? fb * p.rect_stride : 0) + g_cid);
            if (r.x <= pxf + 0.5f && r.z >= pxf - 0.5f && r.y <= pyf + 0.5f && r.w >= pyf - 0.5f) {
              const float4 lo = __ldg(p.chunk_lo + g_cid), hi = __ldg(p.chunk_hi + g_cid);
              const int2 chk = __ldg(p.chunk + g_cid);
              g_first = chk.x;
              g_cnt = chk.y;
              const float hx = 0.5f * (hi.x - lo.x), hy = 0.5f * (hi.y - lo.y), hz = 0.5f * (hi.z - lo.z);
              const float rad = sqrtf(hx * hx + hy * hy + hz * hz) + q * lo.w;
              const float cx = lo.x + hx - oxh, cy = lo.y + hy - oyh, cz = lo.z + hz - ozh;
              const float t = cx * vxh + cy * vyh + cz * vzh;
              const float wx = cx - t * vxh, wy = cy - t * vyh, wz = cz - t * vzh;
              const float rr = rad + 1e-5f * (fabsf(t) + fabsf(cx) + fabsf(cy) + fabsf(cz) + 1e-2f);
              hit = wx * wx + wy * wy + wz * wz <= rr * rr;
            }
          }
          gmask = __ballot_sync(kFull, hit);
        }
        const unsigned mk = gmask & (0xffffffffu << (from - gcur));
        if (mk) return gcur + __ffs(mk) - 1;
        from = gcur + 32;
      }
    };

    PT_BEGIN
    int cur = next_hit(tr.x);
    PT_END(0)
    for (;;) {
      const bool last = cur >= ce;
      const int src = cur - gcur;  // this lane group holds entry `cur`
      const float F = last ? kInf : __shfl_sync(kFull, g_F, src & 31);
      const int room = nfree + (kCap - hwm);
      if (last || nnk + 32 > kNK || room < 32) {
        PT_BEGIN
        // ---- sort the new particles by first knot and merge them into the waiting list
        if (nnk > 0) {
          const int rb = warp_bucket_sort(T.nk0, T.nv0, T.nk1, T.nv1, nnk, T.rh);
          const int na = nwait - whead;
          const int nout = min(na + nnk, kCap);
          warp_tile_merge((wb ? T.wk1 : T.wk0) + whead, (wb ? T.wv1 : T.wv0) + whead, na, rb ? T.nk1 : T.nk0,
                          rb ? T.nv1 : T.nv0, nnk, wb ? T.wk0 : T.wk1, wb ? T.wv0 : T.wv1, nout, rb ? T.nk0 : T.nk1,
                          rb ? T.nv0 : T.nv1);
          wb ^= 1;
          whead = 0;
          nwait = nout;
          nnk = 0;
        }
        PT_END(2)

        // ---- windows: every knot below F is final
        while (!done) {
          if (win_count >= kMaxRayWindows) {
            // a ray this long (two orders of magnitude beyond the windows of
            // any ray measured) is ended here and flagged: its pixel is wrong
            st_flags |= kFlagWindowLimit;
            done = true;
            break;
          }
          PT_BEGIN
          const float* WK = wb ? T.wk1 : T.wk0;
          const int* WV = wb ? T.wv1 : T.wv0;
          // waiting particles that have already started (FP32 ties) leave the list
          while (whead < nwait) {
            const int i = whead + lane;
            const unsigned st_ = __ballot_sync(kFull, i < nwait && knots_done(T, WV[i]) > 0);
            const int run = __ffs(~st_) - 1;  // leading started entries
            whead += run < 0 ? 32 : run;
            if (run >= 0) break;
          }
          whead = min(whead, nwait);
          bool fresh = false;
          float h_fresh = kInf;
          if (n_act == 0) {
            // the field is zero at Ta: restart at the first waiting particle's first knot
            if (whead >= nwait) break;
            if (!(WK[whead] < F)) break;
            const int e0 = WV[whead];
            const float sg = knot_sigma(K, m, __ldg(p.theta + T.jj[e0]), 0);
            const float4 E0 = T.ent[e0];
            df kp = df{E0.x, E0.y};
            {
              const float pr = sg * E0.z;
              const float pe = fmaf(sg, E0.z, -pr);
              kp = df_add(kp, df{pr, pe});
            }
            if (started) {
              // gap: field identically 0 on [Ta, kp)
              df a0 = df_add(Ta, df_neg(t_start));
              float from = a0.hi + a0.lo > 0.f ? 0.f : -(a0.hi + a0.lo);
              df gl = df_add(kp, df_neg(Ta));
              float L = gl.hi + gl.lo - from;
              if (L > 0.f) {
                Poly<D> z0;
#pragma unroll
                for (int d = 0; d <= D; ++d) z0.c[d] = 0.f;
                const Acc g = composite_piece_v<D>(z0, L, tfc, Acc{0.f, 0.f, 0.f, 0.f});
                float w = __expf(-tau_ray);
                col[0] += w * g.r;
                col[1] += w * g.g;
                col[2] += w * g.b;
                tau_ray += g.tau;
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
              t_start = (df_to_double(kp) > (double)cam.t_near) ? kp : t_near_df;
            }
            Ta = kp;
            fresh = true;
            h_fresh = E0.z;
#pragma unroll
            for (int d = 0; d <= D; ++d) carry[d] = (S)0;
            if (QT) {
#pragma unroll
              for (int d = 0; d <= D; ++d) qc[d] = 0;
              qct = 0;
            }
          }
          // window end (relative to Ta): the bound F, and gamma times the
          // lower edge of the smallest bin of h among the active particles
          // (at a restart: gamma h of the particle restarted at)
          float U = kInf;
          if (F < kInf) U = (F - Ta.hi) - Ta.lo;
          // a quantised knot lies within tau of the FP32 knot F bounds
          if (QT && F < kInf) U -= 2.f * (float)p.q_tau;
          bool capped = false;
          if (gam * h_fresh < U) {
            U = gam * h_fresh;
            capped = true;
          }
          // reinitialisation knots: the window ends at the next one
          float ureinit = -1.f;
          if (RE) {
            const double ta = (double)Ta.hi + (double)Ta.lo, dt = (double)p.reinit_dt;
            const float ur = (float)((floor(ta / dt + 1e-6) + 1.0) * dt - ta);
            if (ur < U) {
              U = ur;
              capped = true;
              ureinit = ur;
            }
          }
          if (n_act > 0) {
            // smallest occupied bin (4 per lane)
            const int4 c4 = *(const int4*)(T.lvl + 4 * lane);
            const int mine = c4.x > 0 ? 0 : (c4.y > 0 ? 1 : (c4.z > 0 ? 2 : (c4.w > 0 ? 3 : 4)));
            const unsigned mb = __ballot_sync(kFull, mine < 4);
            const int l0 = mb ? __ffs(mb) - 1 : 31;
            const int lv = mb ? 4 * l0 + __shfl_sync(kFull, mine, l0) : kLevels - 1;
            const float lim = gam * level_lo(lv);
            if (lim < U) {
              U = lim;
              capped = true;
            }
          }
          PT_END(3)
          PT_BEGIN
          // ---- the window's knots: every active particle's next knots and the
          // knots of the waiting particles that start inside the window, all
          // below U, into the generation buffer (shared); in the same pass the
          // anchor (exact field coefficients at Ta, every 2nd window) and the
          // removal of finished particles from the active list
          S A[D + 1];
          const bool do_anchor =
              !fresh && ((p.anchor_every > 0 && (win_count % p.anchor_every) == 0) || (RE && at_reinit));
          float acc[D + 1];
#pragma unroll
          for (int d = 0; d <= D; ++d) acc[d] = 0.f;
          float cap2 = kInf;
          int T_all = 0;
          int* hist = T.rh;  // hist[64]: the emission counter
#pragma unroll 1
          for (int gen = 0;; ++gen) {
            if (lane == 0) hist[64] = 0;
            __syncwarp();
            // active particles (lanes [0, nal)) and the waiting particles whose
            // first knot lies below U (lanes [nal, nal + ns))
            const int ns = warp_count_below(WK, whead, nwait, Ta.hi + U);
            int wr = 0;
#pragma unroll 1
            for (int b0 = 0; b0 < nal + ns; b0 += 32) {
              const int i = b0 + lane;
              int e = -1, kstart = 0;
              bool keep = false, fin = false;
              if (i < nal) {
                e = T.act[i];
                kstart = knots_done(T, e);
                fin = kstart > K;
                keep = !fin;
              } else if (i < nal + ns) {
                e = WV[whead + i - nal];
                if (knots_done(T, e) != 0) e = -1;  // started already (FP32 ties)
              }
              if (e >= 0 && !fin) {
                const float4 E = T.ent[e];
                const int j = T.jj[e];
                if (gen == 0 && do_anchor && keep) {
                  float Ae[D + 1];
                  entry_piece_at<D>(p, E, j, kstart, Ta, Ae);
#pragma unroll
                  for (int d = 0; d <= D; ++d) acc[d] += Ae[d];
                }
                const float2 th = __ldg(p.theta + j);
                const float base = (E.x - Ta.hi) + (E.y - Ta.lo);
                const double ta_d = (double)Ta.hi + (double)Ta.lo;
#pragma unroll 1
                for (int k = kstart; k <= K; ++k) {
                  const float u = QT ? (float)((double)(long long)qknot_pos(p, E, th, k) * p.q_tau - ta_d)
                                     : fmaf(knot_sigma(K, m, th, k), E.z, base);
                  if (!(u < U)) break;
                  // a particle starting inside the window bounds it by its own
                  // gamma h, or by its first knot when that lies farther
                  if (k == 0) cap2 = fminf(cap2, fmaxf(u, gam * E.z));
                  const int pos = atomicAdd(&hist[64], 1);
                  if (pos < kNK) {
                    T.nk0[pos] = u;
                    T.nv0[pos] = e | (k << 16);
                  }
                }
              }
              if (gen == 0 && b0 < nal) {
                // drop finished particles (their slots go to the free stack)
                const unsigned km = __ballot_sync(kFull, keep), fm = __ballot_sync(kFull, fin);
                __syncwarp();
                if (keep) T.act[wr + __popc(km & lanemask_lt())] = e;
                if (fin) T.fre[nfree + __popc(fm & lanemask_lt())] = e;
                wr += __popc(km);
                nfree += __popc(fm);
              }
            }
            if (gen == 0) nal = wr;
            __syncwarp();
            T_all = hist[64];
            if (T_all <= kNK || gen >= 16) break;
            // too many knots below U for the buffer: shrink U in proportion
            // (to about WCAP of them at uniform density) and generate again
            U *= 0.9f * (float)WCAP / (float)T_all;
            capped = false;
            cap2 = kInf;
            __syncwarp();
          }
          if (T_all > kNK) {
            st_flags |= 2;
            T_all = kNK;
          }
          cap2 = warp_min(cap2);
          if (do_anchor) {
#pragma unroll
            for (int d = 0; d <= D; ++d) A[d] = (S)warp_sum(acc[d]);
          } else {
#pragma unroll
            for (int d = 0; d <= D; ++d) A[d] = fresh ? (S)0 : carry[d];
          }
          if (QT) {
            // the exact polynomial at the last knot, expanded at the window start
            double ca[D + 1], sc = p.q_sigma;
#pragma unroll
            for (int d = 0; d <= D; ++d) {
              ca[d] = (double)(long long)qc[d] * sc;
              sc *= p.q_inv_tau;
            }
            taylor_shift<D, double>(ca, ((double)Ta.hi + (double)Ta.lo) - (double)(long long)qct * p.q_tau);
#pragma unroll
            for (int d = 0; d <= D; ++d) A[d] = (S)ca[d];
          }
          // sort by position (ties: slot, then knot index)
          const int rb = warp_bucket_sort(T.nk0, T.nv0, T.nk1, T.nv1, T_all, T.rh);
          const float* GK = rb ? T.nk1 : T.nk0;
          const int* GV = rb ? T.nv1 : T.nv0;
          if (cap2 < U) {
            U = cap2;
            capped = true;
          }
          int nc = warp_count_below(GK, 0, T_all, U);
          if (nc > WCAP) {  // full: it ends at the first knot left out
            nc = WCAP;
            U = GK[WCAP];
            capped = false;
          }
          PT_END(4)
          PT_BEGIN
          if (nc == 0 && !capped) {
            PT_END(5)
            break;  // nothing final below F: wait for more particles
          }
          // load the window lane-major (lane l holds knots l*KPL ... l*KPL+KPL-1),
          // then stage it in shared memory at r * 32 + l with its difference coefficients
          float uu[KPL];
          int pl[KPL];
#pragma unroll
          for (int r = 0; r < KPL; ++r) {
            const int i = lane * KPL + r;
            uu[r] = i < nc ? GK[i] : 0.f;
            pl[r] = i < nc ? GV[i] : -1;
          }
          __syncwarp();
          // quantised path: [WCAP * D] int64 coefficients, [WCAP] int64 positions
          u64* const qd = (u64*)T.wdl;
          u64* const qt = qd + WCAP * D;
          float* su = QT ? (float*)(qt + WCAP) : T.wdl + WCAP * D;
          int* sv = (int*)(su + WCAP);
#pragma unroll 2
          for (int r = 0; r < KPL; ++r) {
            if (pl[r] >= 0) {
              const int e = pl[r] & 0xffff, k = pl[r] >> 16;
              const float4 E = T.ent[e];
              if (QT) {
                const float2 th = __ldg(p.theta + T.jj[e]);
                u64 qa[D + 1];
                if (!qknot_coef<D>(p, E, th, T.jj[e], k, qa)) st_flags |= 16;
#pragma unroll
                for (int d = 0; d < D; ++d) qd[(r * D + d) * 32 + lane] = qa[d + 1];
                qt[r * 32 + lane] = qknot_pos(p, E, th, k);
              } else {
                float dl[D];
                knot_delta<D>(p, T.jj[e], E.z, E.w, k, dl);
#pragma unroll
                for (int d = 0; d < D; ++d) T.wdl[(r * D + d) * 32 + lane] = dl[d];
              }
            }
            su[r * 32 + lane] = uu[r];
            sv[r * 32 + lane] = pl[r];
          }
          const int cnt_l = min(max(nc - lane * KPL, 0), KPL);  // this lane's knots (a prefix)
          int nf = 0, nl = 0;
          float umax = 0.f;
#pragma unroll 1
          for (int r = 0; r < cnt_l; ++r) {
            const int k = sv[r * 32 + lane] >> 16;
            nf += k == 0;
            nl += k == K;
            umax = fmaxf(umax, su[r * 32 + lane]);
          }
          nf = warp_sum_i(nf);
          nl = warp_sum_i(nl);
          umax = warp_max(umax);
          const int act_after = n_act + nf - nl;
          // no particle is active after the window's last knot: the field is
          // identically zero from there on, so the window ends at that knot
          const bool final_w = nc > 0 && act_after == 0;
          float Uend = final_w ? fminf(umax, U) : U;
          if (!(Uend < kInf)) {
            st_flags |= 4;
            Uend = umax;
          }
          Uend = fmaxf(Uend, 0.f);
          if (RE) at_reinit = ureinit >= 0.f && !final_w && Uend == ureinit;  // the next window starts on one
#pragma unroll 1
          for (int r = 0; r < KPL; ++r)
            su[r * 32 + lane] = r < cnt_l ? fminf(fmaxf(su[r * 32 + lane], 0.f), Uend) : Uend;
          PT_END(5)

          PT_BEGIN
          // mark the window's knots processed; active list and bin counts
#pragma unroll 1
          for (int r = 0; r < KPL; ++r) {
            const bool valid = r < cnt_l;
            const int vv = sv[r * 32 + lane];
            const int e = vv & 0xffff, k = vv >> 16;
            if (valid) atomicAdd(T.knc + (e >> 3), 1u << (4 * (e & 7)));
            const bool first = valid && k == 0;
            const unsigned mm = __ballot_sync(kFull, first);
            if (first) T.act[nal + __popc(mm & lanemask_lt())] = e;
            nal += __popc(mm);
            if (valid && (k == 0 || k == K)) atomicAdd(&T.lvl[h_level(T.ent[e].z)], k == 0 ? 1 : -1);
          }
          __syncwarp();
          n_act = act_after;
          st_maxact = max(st_maxact, n_act);
          my_knots += nc;
          ++st_win;
          ++win_count;
          if (capped) ++st_capped;
          PT_END(6)

          PT_BEGIN
          const float ufirst = su[lane];
          const bool has = cnt_l > 0;
          // incoming polynomial at this lane's first knot: P (FP32/FP64 paths),
          // qP at integer position qtp (quantised path)
          S P[D + 1];
          u64 qP[D + 1], qtp = 0;
          if (!QT) {
            // ---- segmented scan of the difference coefficients (Sec. 2)
            S agg[D + 1];
#pragma unroll
            for (int d = 0; d <= D; ++d) agg[d] = (S)0;
            float ulast = ufirst;
#pragma unroll 1
            for (int r = 0; r < cnt_l; ++r) {
              const float ur = su[r * 32 + lane];
              if (r > 0) taylor_shift<D, S>(agg, (S)(ur - ulast));
#pragma unroll
              for (int d = 1; d <= D; ++d) agg[d] += (S)T.wdl[(r * D + d - 1) * 32 + lane];
              ulast = ur;
            }
            // inclusive warp scan of (agg, ulast, has)
            S sa[D + 1];
#pragma unroll
            for (int d = 0; d <= D; ++d) sa[d] = agg[d];
            float se = ulast;
            int sh = has ? 1 : 0;
#pragma unroll 1
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
#pragma unroll
            for (int d = 0; d <= D; ++d) P[d] = A[d];
            taylor_shift<D, S>(P, (S)ufirst);
            if (ph) {
              taylor_shift<D, S>(pa, (S)(ufirst - pe));
#pragma unroll
              for (int d = 0; d <= D; ++d) P[d] += pa[d];
            }
          } else {
            // ---- the same scan in exact integers (Sec. 4.2): knot positions
            // and coefficient sums are uint64 bit patterns of int64 values
            u64 agg[D + 1];
#pragma unroll
            for (int d = 0; d <= D; ++d) agg[d] = 0;
            const u64 qfirst = has ? qt[lane] : 0ull;
            u64 qlast = qfirst;
#pragma unroll 1
            for (int r = 0; r < cnt_l; ++r) {
              const u64 tr = qt[r * 32 + lane];
              if (r > 0) taylor_shift<D, u64>(agg, tr - qlast);
#pragma unroll
              for (int d = 1; d <= D; ++d) agg[d] += qd[(r * D + d - 1) * 32 + lane];
              qlast = tr;
            }
            u64 sa[D + 1], se = qlast;
#pragma unroll
            for (int d = 0; d <= D; ++d) sa[d] = agg[d];
            int sh = has ? 1 : 0;
#pragma unroll 1
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
              u64 oa[D + 1];
#pragma unroll
              for (int d = 0; d <= D; ++d) oa[d] = __shfl_up_sync(kFull, sa[d], o2);
              const u64 oe = __shfl_up_sync(kFull, se, o2);
              const int oh = __shfl_up_sync(kFull, sh, o2);
              if (lane >= o2 && oh) {
                if (sh) {
                  taylor_shift<D, u64>(oa, se - oe);
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
            u64 pa[D + 1];
#pragma unroll
            for (int d = 0; d <= D; ++d) pa[d] = __shfl_up_sync(kFull, sa[d], 1);
            const u64 pe = __shfl_up_sync(kFull, se, 1);
            int ph = __shfl_up_sync(kFull, sh, 1);
            if (lane == 0) ph = 0;
#pragma unroll
            for (int d = 0; d <= D; ++d) qP[d] = qc[d];
            taylor_shift<D, u64>(qP, qfirst - qct);
            if (ph) {
              taylor_shift<D, u64>(pa, qfirst - pe);
#pragma unroll
              for (int d = 0; d <= D; ++d) qP[d] += pa[d];
            }
            qtp = qfirst;
          }
          // next lane's first knot (piece end for this lane's last knot)
          float unext = __shfl_down_sync(kFull, ufirst, 1);
          if (lane == 31) unext = Uend;
          const float ulane_end = cnt_l == KPL ? unext : Uend;
          // ---- composite this lane's pieces: lane 0 first takes the leading
          // piece [0, u_0] (the whole window if it has no knot) with the
          // window's incoming polynomial, then every lane one piece per knot
          Acc acc_l{0.f, 0.f, 0.f, 0.f};
          const df rs = df_add(t_start, df_neg(Ta));
          const float ystart = rs.hi + rs.lo;  // window-relative start of compositing
          long long dbg_base = 0, npieces = 0;
          if (DBG) {
            int cntp = 0;
#pragma unroll 1
            for (int r = 0; r < cnt_l; ++r) {
              const float en = r + 1 < cnt_l ? su[(r + 1) * 32 + lane] : ulane_end;
              if (en > su[r * 32 + lane]) ++cntp;
            }
            int lead = (lane == 0 && ufirst > 0.f) ? 1 : 0;
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
#pragma unroll 1
          for (int sp = lane == 0 ? -1 : 0; sp < cnt_l; ++sp) {
            Poly<D> Pf;
            float ua, ub;
            if (sp < 0) {
#pragma unroll
              for (int d = 0; d <= D; ++d) Pf.c[d] = (float)A[d];
              ua = 0.f;
              ub = ufirst;
            } else {
              ua = su[sp * 32 + lane];
              if (QT) {
                // exact update at the knot's integer position, then the piece's
                // polynomial in ray units: coefficient d is qP_d sigma / tau^d
                const u64 tcur = qt[sp * 32 + lane];
                if (sp > 0) taylor_shift<D, u64>(qP, tcur - qtp);
#pragma unroll
                for (int d = 1; d <= D; ++d) qP[d] += qd[(sp * D + d - 1) * 32 + lane];
                qtp = tcur;
                double sc = p.q_sigma;
#pragma unroll
                for (int d = 0; d <= D; ++d) {
                  Pf.c[d] = (float)((double)(long long)qP[d] * sc);
                  sc *= p.q_inv_tau;
                }
              } else {
                if (sp > 0) taylor_shift<D, S>(P, (S)(ua - lastu));
#pragma unroll
                for (int d = 1; d <= D; ++d) P[d] += (S)T.wdl[(sp * D + d - 1) * 32 + lane];
#pragma unroll
                for (int d = 0; d <= D; ++d) Pf.c[d] = (float)P[d];
              }
              lastu = ua;
              ub = sp + 1 < cnt_l ? su[(sp + 1) * 32 + lane] : ulane_end;
            }
            const float a0 = fmaxf(ua, ystart);
            if (ub > a0) {
              if (a0 > ua) taylor_shift<D, float>(Pf.c, a0 - ua);
              acc_l = composite_piece_v<D>(Pf, ub - a0, tfc, acc_l);
            }
            if (DBG && p.dbg_field && ub > ua) {
              const long long row = sp < 0 ? dbg_np : dbg_base++;
              if (row < p.field_cap) {
                double* fo = p.dbg_field + ((size_t)dbg_row * p.field_cap + row) * (D + 3);
                fo[0] = df_to_double(Ta) + (double)ua;
                fo[1] = df_to_double(Ta) + (double)ub;
                double sc = p.q_sigma;
                for (int d = 0; d <= D; ++d) {
                  fo[2 + d] = sp < 0 ? (double)A[d] : (QT ? (double)(long long)qP[d] * sc : (double)P[d]);
                  sc *= p.q_inv_tau;
                }
              }
            }
          }
          if (DBG) dbg_np += npieces;
          // carry the polynomial to the window end (plain recurrence / next window)
          if (QT) {
            // exact: the last lane's coefficients at its last knot
            const unsigned anym = __ballot_sync(kFull, has);
            if (anym) {
              const int lastlane = 31 - __clz(anym);
#pragma unroll
              for (int d = 0; d <= D; ++d) qc[d] = __shfl_sync(kFull, qP[d], lastlane);
              qct = __shfl_sync(kFull, qtp, lastlane);
            }
          } else {
            S cpy[D + 1];
#pragma unroll
            for (int d = 0; d <= D; ++d) cpy[d] = P[d];
            if (has) taylor_shift<D, S>(cpy, (S)(Uend - lastu));
            unsigned anym = __ballot_sync(kFull, has);
            if (anym) {
              int lastlane = 31 - __clz(anym);
#pragma unroll
              for (int d = 0; d <= D; ++d) carry[d] = __shfl_sync(kFull, cpy[d], lastlane);
            } else {
              // no knot in the window: the anchor polynomial spans it
#pragma unroll
              for (int d = 0; d <= D; ++d) carry[d] = A[d];
              taylor_shift<D, S>(carry, (S)Uend);
            }
          }
          // combine lanes: transmittance as accumulated optical depth
          float tx = acc_l.tau;
#pragma unroll
          for (int o2 = 1; o2 < 32; o2 <<= 1) {
            float y = __shfl_up_sync(kFull, tx, o2);
            if (lane >= o2) tx += y;
          }
          float tex = tx - acc_l.tau;
          float w = __expf(-(tau_ray + tex));
          float c0 = warp_sum(w * acc_l.r), c1 = warp_sum(w * acc_l.g), c2 = warp_sum(w * acc_l.b);
          col[0] += c0;
          col[1] += c1;
          col[2] += c2;
          tau_ray += __shfl_sync(kFull, tx, 31);
          // advance
          Ta = df_add(Ta, df{Uend, 0.f});
          PT_END(7)
          if (p.tau_ert > 0.f && tau_ray > p.tau_ert) {
            done = true;
            break;
          }
        }
        if (done) break;
        if (nfree + (kCap - hwm) < 32) {
          // reclaim the slots of finished particles
          float dummy[D + 1];
          active_pass<D>(p, T, nal, nfree, Ta, false, dummy);
        }
      }
      if (last) break;

      // ------------------------------------------------ candidates of one chunk
      PT_BEGIN
      {
        const int ch_first = __shfl_sync(kFull, g_first, src & 31);
        const int ch_cnt = __shfl_sync(kFull, g_cnt, src & 31);
        bool cand = false;
        df tc = {0.f, 0.f};
        float h = 0.f, d2 = 0.f, a = 0.f;
        df wv[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        const int pidx = ch_first + lane;
        if (lane < ch_cnt) {
          const float4 P = __ldg(p.pos + pidx);
          h = P.w;
          if (h > 0.f) {
            ++st_tests;
            const float R = q * h;
            const float px_ = P.x - o[0].hi, py_ = P.y - o[1].hi, pz_ = P.z - o[2].hi;
            const float t = px_ * v[0].hi + py_ * v[1].hi + pz_ * v[2].hi;
            const float wx = px_ - t * v[0].hi, wy = py_ - t * v[1].hi, wz = pz_ - t * v[2].hi;
            const float d2f = wx * wx + wy * wy + wz * wz;
            const float tol = 4e-6f * (fabsf(t) + fabsf(px_) + fabsf(py_) + fabsf(pz_) + 1e-3f);
            const float Rt = R + tol;
            if (d2f < Rt * Rt) {
              // double-float: p = chi - o, t = p.v, w = p - t v
              df pp[3];
              const float pc3[3] = {P.x, P.y, P.z};
#pragma unroll
              for (int k = 0; k < 3; ++k) pp[k] = df_add(df{pc3[k], 0.f}, df_neg(o[k]));
              const df tt = df_add(df_add(df_mul(pp[0], v[0]), df_mul(pp[1], v[1])), df_mul(pp[2], v[2]));
              float dd = 0.f;
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                df w = df_add(pp[k], df_neg(df_mul(tt, v[k])));
                dd = fmaf(w.hi, w.hi, fmaf(2.f * w.hi, w.lo, dd));
                wv[k] = w;
              }
              const float R2 = R * R;
              if (DBG && fabsf(dd - R2) <= 2e-6f * q * h * h) ++lane_tan;
              if (dd < R2) {
                const float ex = tt.hi + sqrtf(fmaxf(R2 - dd, 0.f));
                if (ex > t_near) {
                  cand = true;
                  tc = tt;
                  d2 = dd;
                  a = __ldg(p.amp + pidx);
                }
              }
            }
          }
        }
        const unsigned mk = __ballot_sync(kFull, cand);
        if (mk) {
          const int n_new = __popc(mk);
          const int rank = __popc(mk & lanemask_lt());
          const int from_free = min(n_new, nfree);
          const int n_store = min(n_new, from_free + (kCap - hwm));
          if (n_store < n_new) st_flags |= 1;
          if (cand && rank < n_store) {
            const int e = rank < from_free ? T.fre[nfree - 1 - rank] : hwm + (rank - from_free);
            // nearest Lambda entry (FP64 re-check near a midpoint)
            const float x = (d2 > 0.f ? d2 * rsqrtf(d2) : 0.f) * __fdividef(p.lam_scale, h);
            int j = (int)floorf(x + 0.5f);
            const float fr = x - floorf(x);
            if (fabsf(fr - 0.5f) < 2e-3f) j = nearest_entry_fp64(wv[0], wv[1], wv[2], h, p.n_lambda, q);
            j = min(max(j, 0), p.n_lambda - 1);
            T.ent[e] = make_float4(tc.hi, tc.lo, h, __fdividef(a, h * h * h));
            T.jj[e] = j;
            atomicAnd(T.knc + (e >> 3), ~(15u << (4 * (e & 7))));
            const float2 th = __ldg(p.theta + j);
            const float k0 = tc.hi + fmaf(knot_sigma(K, m, th, 0), h, tc.lo);  // first knot
            T.nk0[nnk + rank] = k0;
            T.nv0[nnk + rank] = e;
            // a first knot behind the processed part of the ray would mean the
            // ordering bound was violated: report it
            if (started && k0 < Ta.hi - 1e-6f * fabsf(Ta.hi)) st_flags |= 8;
            if (DBG && p.dbg_cands) {
              const long long ci2 = dbg_nc + rank;
              if (ci2 < p.cand_cap) p.dbg_cands[dbg_row * p.cand_cap + ci2] = p.orig[pidx];
            }
          }
          nfree -= from_free;
          hwm += n_store - from_free;
          nnk += n_store;
          st_cand += n_new;
          dbg_nc += n_new;
          st_maxtab = max(st_maxtab, hwm - nfree);
        }
        __syncwarp();
      }
      PT_END(1)
      PT_BEGIN
      cur = next_hit(cur + 1);
      PT_END(0)
    }

    // ---- output
    ++st_rays;
    if (p.tau_ert > 0.f && tau_ray > p.tau_ert) ++st_ert;
    st_knots += my_knots;
    const int ray_tan = DBG ? warp_sum_i(lane_tan) : 0;
    if (lane == 0) {
      float alpha = -expm1f(-tau_ray);
      if (DBG) {
        p.dbg_rgba[4 * dbg_row + 0] = col[0];
        p.dbg_rgba[4 * dbg_row + 1] = col[1];
        p.dbg_rgba[4 * dbg_row + 2] = col[2];
        p.dbg_rgba[4 * dbg_row + 3] = alpha;
        long long* cnt = p.dbg_counts + 8 * dbg_row;
        cnt[0] = dbg_nc;
        cnt[1] = (long long)my_knots;
        cnt[2] = dbg_np;
        cnt[3] = st_flags;
        cnt[4] = ray_tan;
        cnt[5] = 0;
        cnt[6] = 0;
        cnt[7] = 0;
      } else {
        float4* o4 = (float4*)(BT ? p.frames[fb].out : p.out);
        o4[(size_t)py * cam.width + px] = make_float4(col[0], col[1], col[2], alpha);
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

inline size_t render_smem_bytes(int tf_n, int nw) { return sizeof(float4) * tf_n + (size_t)kWarpSmem * nw; }

}  // namespace sphdvr
