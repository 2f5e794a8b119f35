// Lean window kernel for the FP32 modes (FP32_ANCHORED, FP32_NAIVE).
//
// Same method and the same window rules as k_render (render.cuh): one warp per
// viewing ray, the ray's 16x16 tile list of chunks consumed in order of the
// bound F, new particles sorted by first knot into a waiting list, windows of
// knots generated from the active particles and the starters, sorted, scanned
// with the coefficient-update recurrence of Sec. 2 (seeded every
// anchor_every-th window with the exact sum of the active particles' own
// pieces, Sec. 4.1 "direct localized coefficients"), and composited per piece
// (Sec. 1, pass 3 of Sec. 2).  What differs is where the state lives and how
// the warp moves it:
//   * the active particles (those whose first knot has been composited and
//     whose last has not) are kept as records in shared memory (structure of
//     arrays; beyond kRayAS of them in a global-memory extension), compacted in
//     the generation pass of every window -- no slot indirection, no per-entry
//     knot counters outside the record;
//   * a window's knots are emitted at offsets from a warp prefix sum of the
//     lanes' knot counts, not by one shared atomic per knot;
//   * the window's knots are split evenly over the lanes for the scan and the
//     compositing, and each knot's difference coefficients are formed where
//     they are used instead of being staged;
//   * a window's end also follows the knot density of the previous window, so
//     that a window seldom generates more knots than it can hold.
// Only particles that have not started yet live in global slots (their
// records, found through the sorted waiting list).
#pragma once

#include "render.cuh"

namespace sphdvr {

#ifndef SPHDVR_RAY_AS
#define SPHDVR_RAY_AS 384
#endif
#ifndef SPHDVR_RAY_MINB
#define SPHDVR_RAY_MINB 3
#endif
#ifndef SPHDVR_RAY_NK
#define SPHDVR_RAY_NK 512
#endif
#ifndef SPHDVR_RAY_U1
#define SPHDVR_RAY_U1 1
#endif
#ifndef SPHDVR_RAY_U2
#define SPHDVR_RAY_U2 1
#endif
constexpr int kRayUnrollScan = SPHDVR_RAY_U1;  // unrolling of the lanes' scan loop
constexpr int kRayUnrollComp = SPHDVR_RAY_U2;  // unrolling of the lanes' compositing loop
constexpr int kRayAS = SPHDVR_RAY_AS;    // active particles held in shared memory (per warp)
constexpr int kRayWarps = 4;             // warps (rays in flight) per CTA
constexpr int kRayMinBlocks = SPHDVR_RAY_MINB;  // CTAs per SM the register budget is set for
constexpr int kRayNK = SPHDVR_RAY_NK;    // window / new-particle buffer (knots)
constexpr int kRayWcap = kRayNK - 64;  // knots composited per window
constexpr int kRayStats = 12;          // the warp's statistics, summed over its rays (shared memory)

// Per-ray capacities.  The frame pass holds up to 4096 waiting particles
// (gathered, not started) and 4096 active ones per ray; a ray that needs more
// is abandoned there, listed, and rendered again by the fallback pass, whose
// warps hold four times as many (the parity hook uses the larger capacities
// too).  Capacity changes no arithmetic of a ray that fits it.
// GR: the shaded (gradient) variant, whose records also hold the vector d
// from the ray to the particle (3 more words per active and waiting particle).
template <bool BIG, bool GR = false>
struct RayCaps {
  static constexpr int WC = BIG ? 16384 : 4096;   // waiting slots
  static constexpr int ACT = BIG ? 16384 : 4096;  // active particles in all (beyond kRayAS in global memory)
  // per-warp shared memory: active records (t_chi hi, t_chi lo, h, c, j | done << 16
  // [, d_x, d_y, d_z]), the window / new-particle buffers (two key/value pairs of
  // kRayNK entries), the sort histogram (+ scratch words), the started bits of the waiting slots, the
  // warp's frame statistics
  static constexpr int SMEM = kRayAS * (GR ? 32 : 20) + 4 * kRayNK * 4 + (256 + 32) * 4 + (WC / 32) * 4 + kRayStats * 8;
  // per-warp global scratch (32-bit words): slot records (float4), slot table
  // entries, free stack, slot -> active index map, two waiting-list buffers
  // (key, slot), the active extension (5 arrays) [, slot d (float4), the
  // active extension's d (3 arrays)]
  static constexpr int WORDS =
      4 * WC + 3 * WC + 4 * WC + 5 * (ACT - kRayAS) + (GR ? 4 * WC + 3 * (ACT - kRayAS) : 0);
  static_assert(WORDS % 4 == 0, "per-warp scratch keeps float4 alignment");
};
static_assert(kRayAS % 32 == 0, "the shared part of the active set is a whole number of lane groups");
static_assert(kRayNK >= 256 && kRayNK <= 512 && kRayNK % 32 == 0, "the window sort and merge take 256..512 entries");
constexpr int kRayWords = RayCaps<false>::WORDS;     // per warp of the frame pass
constexpr int kRayWordsBig = RayCaps<true>::WORDS;   // per warp of the fallback pass and the parity hook
constexpr int kRayWordsGR = RayCaps<false, true>::WORDS;    // the same, shaded variant
constexpr int kRayWordsBigGR = RayCaps<true, true>::WORDS;
constexpr int kRayFlagRefit = 32;  // frame flag: a ray overflowed the fallback's capacities too (image wrong)

inline size_t ray_smem_bytes(int tf_n, int nw, bool big, bool gr = false) {
  const int per = gr ? (big ? RayCaps<true, true>::SMEM : RayCaps<false, true>::SMEM)
                     : (big ? RayCaps<true>::SMEM : RayCaps<false>::SMEM);
  return sizeof(float4) * tf_n + (size_t)per * nw;
}

// Active set: index i < kRayAS in shared memory, else at i - kRayAS in global memory.
struct ActSet {
  float *th, *tl, *h, *c;
  int* jk;  // table entry (bits 0..15) | knots processed (bits 16..19)
  float *gth, *gtl, *gh, *gc;
  int* gjk;
  float *dx, *dy, *dz, *gdx, *gdy, *gdz;  // shaded variant: the vector from the ray to the particle
};

__device__ __forceinline__ void act_get(const ActSet& A, int i, float4& r, int& jk) {
  if (i < kRayAS) {
    r = make_float4(A.th[i], A.tl[i], A.h[i], A.c[i]);
    jk = A.jk[i];
  } else {
    const int g = i - kRayAS;
    r = make_float4(A.gth[g], A.gtl[g], A.gh[g], A.gc[g]);
    jk = A.gjk[g];
  }
}
__device__ __forceinline__ float4 act_getE(const ActSet& A, int i) {
  if (i < kRayAS) return make_float4(A.th[i], A.tl[i], A.h[i], A.c[i]);
  const int g = i - kRayAS;
  return make_float4(A.gth[g], A.gtl[g], A.gh[g], A.gc[g]);
}
__device__ __forceinline__ void act_put(const ActSet& A, int i, float4 r, int jk) {
  if (i < kRayAS) {
    A.th[i] = r.x;
    A.tl[i] = r.y;
    A.h[i] = r.z;
    A.c[i] = r.w;
    A.jk[i] = jk;
  } else {
    const int g = i - kRayAS;
    A.gth[g] = r.x;
    A.gtl[g] = r.y;
    A.gh[g] = r.z;
    A.gc[g] = r.w;
    A.gjk[g] = jk;
  }
}
__device__ __forceinline__ int* act_jk_ptr(const ActSet& A, int i) { return i < kRayAS ? A.jk + i : A.gjk + (i - kRayAS); }
__device__ __forceinline__ float3 act_getd(const ActSet& A, int i) {
  if (i < kRayAS) return make_float3(A.dx[i], A.dy[i], A.dz[i]);
  const int g = i - kRayAS;
  return make_float3(A.gdx[g], A.gdy[g], A.gdz[g]);
}
__device__ __forceinline__ void act_putd(const ActSet& A, int i, float3 d) {
  if (i < kRayAS) {
    A.dx[i] = d.x;
    A.dy[i] = d.y;
    A.dz[i] = d.z;
  } else {
    const int g = i - kRayAS;
    A.gdx[g] = d.x;
    A.gdy[g] = d.y;
    A.gdz[g] = d.z;
  }
}

// Localized difference coefficients, orders 1..D, of sorted knot k of a
// particle with table entry j, smoothing length h and amplitude c, from table
// `tab` (the field's difference coefficients, or the gradient's; Sec. 2,
// Sec. 3.1); mirrored knots take (-1)^(d+1).
template <int D>
__device__ __forceinline__ void knot_delta_tab(const float* tab, int K, int m, int j, float h, float c, int k,
                                               float* dl) {
  bool mir;
  const int slot = knot_slot(K, m, k, mir);
  const float* jr = tab + (size_t)j * 3 * D + slot * D;
  const float ih = __fdividef(1.f, h);
  float s = c;
#pragma unroll
  for (int d = 1; d <= D; ++d) {
    s *= ih;
    const float v = __ldg(jr + d - 1) * s;
    dl[d - 1] = (mir && !(d & 1)) ? -v : v;
  }
}

// Exact coefficients at Ta of a particle's own piece after its first kn knots,
// from piece table `tab` with amplitude c (the anchor of a window).
template <int D>
__device__ __forceinline__ void entry_piece_at_tab(const float* tab, int K, int m, float4 E, float c, float2 th,
                                                   int j, int kn, df Ta, float* A) {
  const int pc = kn - 1;
  int kp;
  float sg;
  if (!(K & 1)) {
    if (pc < m) { kp = m - pc; sg = -1.f; } else { kp = pc - m + 1; sg = 1.f; }
  } else {
    if (pc < m - 1) { kp = m - pc; sg = -1.f; }
    else if (pc == m - 1) { kp = 1; sg = 1.f; }
    else { kp = pc - m + 2; sg = 1.f; }
  }
  const float th0 = kp == 1 ? 0.f : th.x;
  const float h = E.z, ih = __fdividef(1.f, h);
  const float rel = (Ta.hi - E.x) + (Ta.lo - E.y);
  const float z = sg * rel * ih - th0;
  const float* pr = tab + (size_t)j * 2 * (D + 1) + (kp - 1) * (D + 1);
  float q[D + 1];
#pragma unroll
  for (int d = 0; d <= D; ++d) q[d] = __ldg(pr + d);
  taylor_shift<D, float>(q, z);
  float s = c;
  const float f = sg * ih;
#pragma unroll
  for (int d = 0; d <= D; ++d) {
    A[d] = q[d] * s;
    s *= f;
  }
}

// Normalised offsets of a particle's knots 0..K in sorted order (Sec. 3.1: the
// table's positive knots theta_1, theta_2 mirrored, with a middle knot at 0
// when K is even); entries beyond K are unused.  K is the same on every lane.
__device__ __forceinline__ void knot_sigmas(int K, float2 th, float (&sg)[5]) {
  const float a = th.x, b = th.y;
  if (K == 4) {
    sg[0] = -b; sg[1] = -a; sg[2] = 0.f; sg[3] = a; sg[4] = b;
  } else if (K == 3) {
    sg[0] = -b; sg[1] = -a; sg[2] = a; sg[3] = b; sg[4] = b;
  } else if (K == 2) {
    sg[0] = -a; sg[1] = 0.f; sg[2] = a; sg[3] = a; sg[4] = a;
  } else {
    sg[0] = -a; sg[1] = a; sg[2] = a; sg[3] = a; sg[4] = a;
  }
}

// exclusive prefix sum over the warp; *total gets the sum of all lanes
__device__ __forceinline__ int warp_excl_scan(int v, int* total) {
  const int lane = threadIdx.x & 31;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  *total = __shfl_sync(kFull, x, 31);
  return x - v;
}

// FB: the fallback pass -- its rays are those the frame pass listed in
// p.ovf; it and the parity hook (DBG) hold the larger capacities.
// GR: shaded rendering -- besides the field, the across-ray gradient's three
// components are carried through the same knots (channels 1..3 of every
// polynomial), and the emission is shaded (Conclusion: additive features).
// CP: compensated running sums (FP32_KAHAN) -- channel 1 holds the rounding
// error of every addition of difference coefficients and of lane prefixes
// (TwoSum), shifted alongside the sum; the field is the sum of both channels.
template <int D, int NW, bool DBG, bool BT, bool FB = false, bool GR = false, bool CP = false>
__global__ void __launch_bounds__(NW * 32, (NW == kRayWarps ? ((GR || CP) ? (GR ? 1 : 2) : kRayMinBlocks) : 1))
    k_ray(RenderParams p) {
  static_assert(!(GR && CP), "shading runs on the anchored and plain FP32 recurrences only");
  constexpr bool BIG = DBG || FB;
  // polynomial channels: the field [, the across-ray gradient x, y, z | the compensation]
  constexpr int NC = GR ? 4 : (CP ? 2 : 1);
  constexpr int NP = NC * (D + 1);
  constexpr int WCX = RayCaps<BIG, GR>::WC, ACTX = RayCaps<BIG, GR>::ACT;
  // capacities in force (the frame pass may be given smaller ones, to test the fallback)
  const int cap_wc = (!BIG && p.ray_cap > 0) ? min(p.ray_cap, WCX) : WCX;
  const int cap_act = (!BIG && p.ray_cap > 0) ? min(p.ray_cap, ACTX) : ACTX;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float4* s_tf = (float4*)smem;
  ActSet A;
  float *nk0, *nk1, *wk0, *wk1;
  int *nv0, *nv1, *wv0, *wv1, *rh, *s_j, *s_fre, *s_map;
  unsigned* stb;
  unsigned long long* wst;  // the warp's statistics: rays, candidates, knots, windows, tests, largest waiting
                            // table, flags, terminated rays, most active, capped windows, tangency tests
  float4* s_rec;
  float4* s_dp = nullptr;  // shaded variant: slot d (the vector from the ray to the particle)
  {
    unsigned char* b = smem + sizeof(float4) * p.tf_n + (size_t)RayCaps<BIG, GR>::SMEM * wid;
    A.th = (float*)b;
    A.tl = A.th + kRayAS;
    A.h = A.tl + kRayAS;
    A.c = A.h + kRayAS;
    A.jk = (int*)(A.c + kRayAS);
    float* w = (float*)(A.jk + kRayAS);
    if (GR) {
      A.dx = w;
      A.dy = w + kRayAS;
      A.dz = w + 2 * kRayAS;
      w += 3 * kRayAS;
    }
    nk0 = w;
    nv0 = (int*)(w + kRayNK);
    nk1 = w + 2 * kRayNK;
    nv1 = (int*)(w + 3 * kRayNK);
    rh = (int*)(w + 4 * kRayNK);
    stb = (unsigned*)(rh + 256 + 32);
    wst = (unsigned long long*)(stb + WCX / 32);
    float* g = p.scratch + (size_t)(blockIdx.x * NW + wid) * RayCaps<BIG, GR>::WORDS;
    s_rec = (float4*)g;
    s_j = (int*)(g + 4 * WCX);
    s_fre = s_j + WCX;
    s_map = s_fre + WCX;
    float* q0 = (float*)(s_map + WCX);
    wk0 = q0;
    wv0 = (int*)(q0 + WCX);
    wk1 = q0 + 2 * WCX;
    wv1 = (int*)(q0 + 3 * WCX);
    float* o = q0 + 4 * WCX;
    constexpr int OC = ACTX - kRayAS;
    A.gth = o;
    A.gtl = o + OC;
    A.gh = o + 2 * OC;
    A.gc = o + 3 * OC;
    A.gjk = (int*)(o + 4 * OC);
    if (GR) {
      s_dp = (float4*)(o + 5 * OC);
      float* gd = o + 5 * OC + 4 * WCX;
      A.gdx = gd;
      A.gdy = gd + OC;
      A.gdz = gd + 2 * OC;
    }
  }
  for (int i = threadIdx.x; i < p.tf_n; i += blockDim.x) s_tf[i] = p.tf[i];
  __syncthreads();
  const TfCtx tfc{s_tf, p.tf_n, p.tf_lo, p.tf_inv_dv, p.tf_dv};
  if (lane < kRayStats) wst[lane] = 0ull;
  __syncwarp();
  PT_DECL
#ifdef SPHDVR_PHASE_TIMING
  unsigned long long why_n[6] = {0, 0, 0, 0, 0, 0};  // what ended each window (instrumented builds)
#define WHY(k) why = (k)
#else
#define WHY(k)
#endif
  const int K = p.K, m = p.m;
  const float q = p.q, gam = p.window_h;
  const float kInf = __int_as_float(0x7f800000);
  // aim a window at this many knots from the knot density of the previous one
  constexpr int kWcap = kRayWcap;
  const float kTarget = p.window_fill < 1.f ? p.window_fill * (float)kWcap : __int_as_float(0x7f800000);

  for (int it = 0;; ++it) {
    // ------------------------------------------------------------ work item
    int item;
    if (FB) {
      const int k = blockIdx.x * NW + wid + it * gridDim.x * NW;
      if (k >= min((int)p.ovf[0], p.ovf_cap)) break;
      item = (int)p.ovf[1 + k];
    } else if (DBG) {
      item = blockIdx.x + it * gridDim.x;
    } else if (p.dynamic) {
      unsigned v = 0;
      if (lane == 0) v = atomicAdd(p.work, 1u);
      item = (int)__shfl_sync(kFull, v, 0);
    } else {
      item = (blockIdx.x * NW + wid) + it * gridDim.x * NW;
    }
    if (item >= (DBG ? p.n_dbg : p.n_items)) break;
    const int item_all = item;  // the work item before the batch's frame offset
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
    float carry[NP];  // the polynomials at the end of the previous window (channel c at c * (D + 1))
#pragma unroll
    for (int i = 0; i < NP; ++i) carry[i] = 0.f;
    // slots: hwm used so far, nfree on the free stack; active set [0, nal),
    // n_act of them not finished; waiting list [whead, nwait) of buffer wb;
    // nnk new particles in the batch
    int hwm = 0, nfree = 0, nal = 0, n_act = 0, whead = 0, nwait = 0, wb = 0, nnk = 0, win_count = 0;
    float hmin = kInf;  // smallest h in the active set (it may include particles finished since)
    float dens = 0.f;   // knots per unit length of the previous window (0: none)
    long long dbg_np = 0, dbg_nc = 0, dbg_win = 0;
    int rf = 0, ray_tan = 0, ray_maxact = 0;  // this ray's flags, tangency-band tests, most active particles
    unsigned r_tests = 0, r_cand = 0, r_win = 0, r_capped = 0, my_knots = 0;  // this ray's counters
    int ray_maxtab = 0;  // most waiting slots in use

    const int2 tr = p.tile_range[(BT ? p.frames[fb].tile_base : 0) + tile];
    const int ce = tr.y;
    int gcur = -64, g_cid = 0, g_first = 0, g_cnt = 0;
    unsigned gmask = 0;
    float g_F = 0.f;
    const float oxh = o[0].hi, oyh = o[1].hi, ozh = o[2].hi, vxh = v[0].hi, vyh = v[1].hi, vzh = v[2].hi;
    // reciprocal direction for the slab test (a zero component becomes a huge finite one of either sign)
    const float ivx = 1.f / (fabsf(vxh) > 1e-30f ? vxh : 1e-30f), ivy = 1.f / (fabsf(vyh) > 1e-30f ? vyh : 1e-30f),
                ivz = 1.f / (fabsf(vzh) > 1e-30f ? vzh : 1e-30f);
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
              const float slack = 1e-5f * (fabsf(t) + fabsf(cx) + fabsf(cy) + fabsf(cz) + 1e-2f);
              const float rr = rad + slack;
              hit = wx * wx + wy * wy + wz * wz <= rr * rr;
              if (hit) {
                // and the box grown by q h_max (plus the slack) must meet the ray's line
                const float g = q * lo.w + slack;
                const float ax = (lo.x - g - oxh) * ivx, bx = (hi.x + g - oxh) * ivx;
                const float ay = (lo.y - g - oyh) * ivy, by = (hi.y + g - oyh) * ivy;
                const float az = (lo.z - g - ozh) * ivz, bz = (hi.z + g - ozh) * ivz;
                const float tmin = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fminf(az, bz));
                const float tmax = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fmaxf(az, bz));
                hit = tmin <= tmax + slack * (fabsf(tmax) + 1.f);
              }
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
      const int src = cur - gcur;
      const float F = last ? kInf : __shfl_sync(kFull, g_F, src & 31);
      if (done) break;  // abandoned (capacity): the fallback pass renders it
      const int room = nfree + (cap_wc - hwm);
      if (last || nnk + 32 > kRayNK || room < 32) {
        // ---- sort the new particles by first knot and merge them into the waiting list
        PT_BEGIN
        if (nnk > 0) {
          const int rb = warp_bucket_sort(nk0, nv0, nk1, nv1, nnk, rh);
          const int na = nwait - whead;
          const int nout = min(na + nnk, cap_wc);
          warp_tile_merge((wb ? wk1 : wk0) + whead, (wb ? wv1 : wv0) + whead, na, rb ? nk1 : nk0, rb ? nv1 : nv0,
                          nnk, wb ? wk0 : wk1, wb ? wv0 : wv1, nout, rb ? nk0 : nk1, rb ? nv0 : nv1);
          wb ^= 1;
          whead = 0;
          nwait = nout;
          nnk = 0;
        }
        PT_END(2)

        // ---- windows: every knot below F is final
        while (!done) {
          if (!BIG && p.ovf && (rf & 3)) {  // a capacity overflowed: abandon the ray to the fallback pass
            done = true;
            break;
          }
          PT_BEGIN
          const float* WK = wb ? wk1 : wk0;
          const int* WV = wb ? wv1 : wv0;
          // waiting particles that have started leave the head of the list; their slots are freed
          while (whead < nwait) {
            const int i = whead + lane;
            const int sl = i < nwait ? WV[i] : 0;
            const bool stt = i < nwait && ((stb[sl >> 5] >> (sl & 31)) & 1u);
            const unsigned sm = __ballot_sync(kFull, stt);
            const int run = __ffs(~sm) - 1;  // leading started entries (-1: all 32)
            const int nl = run < 0 ? 32 : run;
            if (lane < nl) s_fre[nfree + lane] = sl;
            nfree += nl;
            whead += nl;
            if (run >= 0) break;
          }
          bool fresh = false;
          float h_fresh = kInf;
          if (n_act == 0) {
            // the field is zero at Ta: restart at the first waiting particle's first knot
            if (whead >= nwait || !(WK[whead] < F)) {
              PT_END(3)
              break;
            }
            const int e0 = WV[whead];
            const float4 E0 = s_rec[e0];
            const float sg = knot_sigma(K, m, __ldg(p.theta + s_j[e0]), 0);
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
                // a zero field has a zero gradient: the shading factor is ka with a
                // softening gradient g0 > 0, ka + kd without one
                float w = __expf(-tau_ray) * (GR ? (p.shade_g2 > 0.f ? p.shade_ka : p.shade_ka + p.shade_kd) : 1.f);
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
            for (int i = 0; i < NP; ++i) carry[i] = 0.f;
          }
          // window end U (relative to Ta): the bound F; gamma times the
          // smallest h of the active set (at a restart: of the particle
          // restarted at); the knot density of the previous window
          float U = kInf;
          if (F < kInf) U = (F - Ta.hi) - Ta.lo;
          bool capped = false;
#ifdef SPHDVR_PHASE_TIMING
          int why = 0;
#endif
          if (gam * h_fresh < U) {
            U = gam * h_fresh;
            capped = true;
            WHY(1);
          }
          if (n_act > 0 && gam * hmin < U) {
            U = gam * hmin;
            capped = true;
            WHY(1);
          }
          if (dens > 0.f && kTarget < U * dens) {
            U = kTarget / dens;
            capped = true;
            WHY(2);
          }
          PT_END(3)
          PT_BEGIN

          // ---- generation: the active particles' next knots and the knots of
          // the waiting particles that start inside the window, all below U;
          // in the same pass the anchor (every anchor_every-th window) and the
          // compaction of the active set (finished particles leave)
          const bool do_anchor = !fresh && p.anchor_every > 0 && (win_count % p.anchor_every) == 0;
          float acc[NP];
#pragma unroll
          for (int i = 0; i < NP; ++i) acc[i] = 0.f;
          float cap2 = kInf, hmin_new = kInf;
          int T_all = 0, ns = 0, ns_as = 0;
#pragma unroll 1
          for (int gen = 0;; ++gen) {
            T_all = 0;
            int wr = 0;
#pragma unroll 1
            for (int b0 = 0; b0 < nal; b0 += 32) {
              const int i = b0 + lane;
              const bool valid = i < nal;
              float4 E = make_float4(0.f, 0.f, 1.f, 0.f);
              int jk = 0;
              float3 dp = make_float3(0.f, 0.f, 0.f);
              if (valid) {
                act_get(A, i, E, jk);
                if (GR) dp = act_getd(A, i);
              }
              const int kd = (jk >> 16) & 15, j = jk & 0xffff;
              const bool keep = valid && kd <= K;
              int ne = 0;
              float uk[5];  // the particle's knots relative to Ta (branch-free, fully unrolled)
              if (keep) {
                const float2 th = __ldg(p.theta + j);
                if (gen == 0 && do_anchor) {
                  float Ae[D + 1];
                  entry_piece_at<D>(p, E, j, kd, Ta, Ae);
#pragma unroll
                  for (int d = 0; d <= D; ++d) acc[d] += Ae[d];
                  if (GR) {
                    // the across-ray gradient's own pieces: amplitude -c d / h^2
                    const float gsc = -__fdividef(E.w, E.z * E.z);
                    const float dc[3] = {dp.x, dp.y, dp.z};
#pragma unroll
                    for (int ch = 1; ch < NC; ++ch) {
                      entry_piece_at_tab<D>(p.gpiece, K, m, E, gsc * dc[ch - 1], th, j, kd, Ta, Ae);
#pragma unroll
                      for (int d = 0; d <= D; ++d) acc[ch * (D + 1) + d] += Ae[d];
                    }
                  }
                }
                float sg[5];
                knot_sigmas(K, th, sg);
                const float base = (E.x - Ta.hi) + (E.y - Ta.lo);
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                  uk[k] = fmaf(sg[k], E.z, base);
                  ne += (k >= kd && k <= K && uk[k] < U) ? 1 : 0;  // the knots below U are a prefix
                }
              }
              const unsigned km = __ballot_sync(kFull, keep);
              const int ni = gen == 0 ? wr + __popc(km & lanemask_lt()) : i;
              int tot;
              const int off = T_all + warp_excl_scan(ne, &tot) - kd;
#pragma unroll
              for (int k = 0; k < 5; ++k) {
                const int pos = off + k;
                if (k >= kd && k < kd + ne && pos < kRayNK) {
                  nk0[pos] = uk[k];
                  nv0[pos] = (ni << 4) | k;
                }
              }
              T_all += tot;
              if (gen == 0) {
                __syncwarp();
                if (keep) {
                  if (ni != i) {
                    act_put(A, ni, E, jk);
                    if (GR) act_putd(A, ni, dp);
                  }
                  hmin_new = fminf(hmin_new, E.z);
                }
                wr += __popc(km);
              }
            }
            if (gen == 0) nal = wr;
            __syncwarp();
            // the starters: waiting particles whose first knot lies below U;
            // each gets an entry of the active set now (knots processed 0), so
            // that its knots index the active set like every other knot; the
            // entry is kept if its first knot turns out to be processed
            ns = warp_count_below(WK, whead, nwait, Ta.hi + U);
            ns_as = 0;
#pragma unroll 1
            for (int b0 = 0; b0 < ns; b0 += 32) {
              const int ii = b0 + lane;
              int e = ii < ns ? WV[whead + ii] : -1;
              if (e >= 0 && ((stb[e >> 5] >> (e & 31)) & 1u)) e = -1;  // started already (FP32 ties)
              int ne = 0;
              float uk[5];
              float4 E = make_float4(0.f, 0.f, 1.f, 0.f);
              int je = 0;
              if (e >= 0) {
                E = s_rec[e];
                je = s_j[e];
                float sg[5];
                knot_sigmas(K, __ldg(p.theta + je), sg);
                const float base = (E.x - Ta.hi) + (E.y - Ta.lo);
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                  uk[k] = fmaf(sg[k], E.z, base);
                  ne += (k <= K && uk[k] < U) ? 1 : 0;
                }
                // a particle starting inside the window bounds it by its own
                // gamma h, or by its first knot when that lies farther
                if (ne > 0) cap2 = fminf(cap2, fmaxf(uk[0], gam * E.z));
              }
              const unsigned sm = __ballot_sync(kFull, ne > 0);
              const int ni = nal + ns_as + __popc(sm & lanemask_lt());
              ns_as += __popc(sm);
              if (ne > 0) {
                if (ni < cap_act) {
                  act_put(A, ni, E, je);
                  if (GR) {
                    const float4 d4 = s_dp[e];
                    act_putd(A, ni, make_float3(d4.x, d4.y, d4.z));
                  }
                } else {
                  rf |= 1;  // the active set is full
                  ne = 0;
                }
              }
              // every starter of the range records its entry, -1 for none: the
              // range comes from the waiting list's absolute FP32 keys, the knots
              // from positions relative to Ta, so a starter may have no knot below U
              if (e >= 0) s_map[e] = ne > 0 ? ni : -1;
              int tot;
              const int off = T_all + warp_excl_scan(ne, &tot);
#pragma unroll
              for (int k = 0; k < 5; ++k) {
                const int pos = off + k;
                if (k < ne && pos < kRayNK) {
                  nk0[pos] = uk[k];
                  nv0[pos] = (ni << 4) | k;
                }
              }
              T_all += tot;
            }
            if (T_all <= kRayNK || gen >= 16) break;
            // too many knots below U for the buffer: shrink U in proportion
            // (to about the window capacity at uniform density) and generate again
            U *= 0.9f * (float)kWcap / (float)T_all;
            capped = false;
            cap2 = kInf;
            __syncwarp();
          }
          if (T_all > kRayNK) {
            rf |= 2;
            T_all = kRayNK;
          }
          PT_END(4)
          PT_BEGIN
          cap2 = warp_min(cap2);
          float Aw[NP];  // the polynomials' coefficients at the window start
#pragma unroll
          for (int i = 0; i < NP; ++i) Aw[i] = do_anchor ? warp_sum(acc[i]) : (fresh ? 0.f : carry[i]);
          __syncwarp();
          // sort by position (ties: by id)
          const int rb = warp_bucket_sort(nk0, nv0, nk1, nv1, T_all, rh);
          const float* GK = rb ? nk1 : nk0;
          const int* GV = rb ? nv1 : nv0;
          // the first pass keeps each knot's difference coefficients for the
          // second (D <= 3, unshaded): in the free key/value buffers and in
          // the knot's own value word, which the second pass no longer needs
          constexpr bool kStash = !GR && D <= 3;
          // (the value words hold the bits of a float: written and read as int,
          // so that no access of the value array goes through another type)
          float* const stash0 = rb ? nk0 : nk1;
          int* const stash1 = rb ? nv0 : nv1;
          int* const stash2 = rb ? nv1 : nv0;
          if (cap2 < U) {
            U = cap2;
            capped = true;
            WHY(3);
          }
          int nc = warp_count_below(GK, 0, T_all, U);
          if (nc > kWcap) {  // full: it ends at the first knot left out
            nc = kWcap;
            U = GK[kWcap];
            capped = false;
            WHY(4);
          }
          if (nc == 0 && !capped) {
            PT_END(5)
            break;  // nothing final below F: wait for more particles
          }

          // (the knots are marked processed in the scan's first pass below; the
          // starters given entries in the generation pass are part of the set)
          const int nal_w = nal + ns_as;
          PT_END(5)
          PT_BEGIN

          // ---- segmented scan of the difference coefficients (Sec. 2) and
          // compositing; lane l takes the knots [i0, i1) of the window
          // (balanced: the lanes' sequential loops below are the critical path)
          const int i0 = (lane * nc) >> 5, i1 = ((lane + 1) * nc) >> 5;
          const bool has = i1 > i0;
          // every window knot lies below U (and below the window end), so only
          // the start needs clamping
          auto uat = [&](int i) -> float { return fmaxf(GK[i], 0.f); };
          // difference coefficients of window knot i (Sec. 2, Sec. 3.1), orders
          // 1..D of every channel: dl[ch * D + d - 1]
          auto deltas = [&](int i, float* dl) {
            const int vv = GV[i];
            const int k = vv & 7;
            float h, c;
            int j;
            float3 dp = make_float3(0.f, 0.f, 0.f);
            {
              const int idx = vv >> 4;
              float4 E;
              int jk;
              act_get(A, idx, E, jk);
              h = E.z;
              c = E.w;
              j = jk & 0xffff;
              if (GR) dp = act_getd(A, idx);
            }
            knot_delta<D>(p, j, h, c, k, dl);
            if (GR) {
              // the across-ray gradient: amplitude -c d / h^2 on the gradient table
              const float gsc = -__fdividef(c, h * h);
              const float dc[3] = {dp.x, dp.y, dp.z};
#pragma unroll
              for (int ch = 1; ch < NC; ++ch) knot_delta_tab<D>(p.gjump, K, m, j, h, gsc * dc[ch - 1], k, dl + ch * D);
            }
          };
          // every channel of a polynomial array shifted by s
          auto shift_all = [&](float* q, float sft) {
#pragma unroll
            for (int ch = 0; ch < NC; ++ch) taylor_shift<D, float>(q + ch * (D + 1), sft);
          };
          // X += the difference coefficients dl of one knot (compensated: TwoSum into channel 1)
          auto add_deltas = [&](float* X, const float* dl) {
            if (CP) {
#pragma unroll
              for (int d = 1; d <= D; ++d) {
                const float a = X[d], b = dl[d - 1];
                const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
                X[d] = s;
                X[D + 1 + d] += __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
              }
            } else {
#pragma unroll
              for (int ch = 0; ch < NC; ++ch)
#pragma unroll
                for (int d = 1; d <= D; ++d) X[ch * (D + 1) + d] += dl[ch * D + d - 1];
            }
          };
          // X += Y, polynomials of every channel (compensated: TwoSum of the sums, errors added)
          auto add_poly = [&](float* X, const float* Y) {
            if (CP) {
#pragma unroll
              for (int d = 0; d <= D; ++d) {
                const float a = X[d], b = Y[d];
                const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
                X[d] = s;
                X[D + 1 + d] += Y[D + 1 + d] + __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
              }
            } else {
#pragma unroll
              for (int q = 0; q < NP; ++q) X[q] += Y[q];
            }
          };
          const float ufirst = has ? uat(i0) : 0.f;
          float P[NP];
          float Uend;
          {
            float agg[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) agg[q] = 0.f;
            float ulast = ufirst;
            int nf = 0, nl = 0;  // the window's first and last knots of particles
#pragma unroll kRayUnrollScan
            for (int i = i0; i < i1; ++i) {
              const float ur = uat(i);
              if (i > i0) shift_all(agg, ur - ulast);
              float dl[NC * D];
              deltas(i, dl);
              const int vv = GV[i];
              if (kStash) {
                stash0[i] = dl[0];
                if (D >= 2) stash1[i] = __float_as_int(dl[1 % D]);
                if (D >= 3) stash2[i] = __float_as_int(dl[2 % D]);
              }
              add_deltas(agg, dl);
              ulast = ur;
              // mark the knot processed (a starter's first knot starts it)
              const int k = vv & 7;
              nf += k == 0;
              nl += k == K;
              atomicAdd(act_jk_ptr(A, vv >> 4), 1 << 16);
            }
            __syncwarp();
            // the starters whose first knot was processed leave the waiting
            // list (started bit); the entries of the others become holes
            // (dropped by the next window's compaction)
#pragma unroll 1
            for (int b0 = 0; b0 < ns; b0 += 32) {
              const int ii = b0 + lane;
              const int e = ii < ns ? WV[whead + ii] : -1;
              if (e >= 0 && !((stb[e >> 5] >> (e & 31)) & 1u)) {
                const int ni = s_map[e];
                if (ni >= 0 && ni < cap_act) {
                  int* jp = act_jk_ptr(A, ni);
                  const int jk = *jp;
                  if ((jk >> 16) & 15) {
                    atomicOr(stb + (e >> 5), 1u << (e & 31));
                    hmin_new = fminf(hmin_new, act_getE(A, ni).z);
                  } else {
                    *jp = jk | (15 << 16);
                  }
                }
              }
            }
            nf = warp_sum_i(nf);
            nl = warp_sum_i(nl);
            const int act_after = n_act + nf - nl;
            // no particle is active after the window's last knot: the field is
            // identically zero from there on, so the window ends at that knot
            const float umax = nc > 0 ? GK[nc - 1] : 0.f;
            const bool final_w = nc > 0 && act_after == 0;
            Uend = final_w ? fminf(umax, U) : U;
            if (!(Uend < kInf)) {
              rf |= 4;
              Uend = umax;
            }
            Uend = fmaxf(Uend, 0.f);
#ifdef SPHDVR_PHASE_TIMING
            if (final_w && Uend < U) why = 5;
            ++why_n[why];
#endif
            __syncwarp();
            nal = nal_w;
            if (nal > cap_act) {
              rf |= 1;
              nal = cap_act;
            }
            n_act = act_after;
            hmin = warp_min(hmin_new);
            ray_maxact = max(ray_maxact, n_act);
            my_knots += nc;
            ++r_win;
            ++win_count;
            if (DBG) ++dbg_win;
            if (capped) ++r_capped;
            // inclusive warp scan of (agg, ulast, has):
            // (other, oe) (+) (mine, se) = (Shift(other, se - oe) + mine, se)
            float sa[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) sa[q] = agg[q];
            float se = ulast;
            int sh = has ? 1 : 0;
#pragma unroll 1
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
              float oa[NP];
#pragma unroll
              for (int q = 0; q < NP; ++q) oa[q] = __shfl_up_sync(kFull, sa[q], o2);
              const float oe = __shfl_up_sync(kFull, se, o2);
              const int oh = __shfl_up_sync(kFull, sh, o2);
              if (lane >= o2 && oh) {
                if (sh) {
                  shift_all(oa, se - oe);
                  add_poly(sa, oa);
                } else {
#pragma unroll
                  for (int q = 0; q < NP; ++q) sa[q] = oa[q];
                  se = oe;
                  sh = 1;
                }
              }
            }
            // exclusive prefix: the polynomials just before this lane's first knot
            float pa[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) pa[q] = __shfl_up_sync(kFull, sa[q], 1);
            const float pe = __shfl_up_sync(kFull, se, 1);
            int ph = __shfl_up_sync(kFull, sh, 1);
            if (lane == 0) ph = 0;
#pragma unroll
            for (int q = 0; q < NP; ++q) P[q] = Aw[q];
            shift_all(P, ufirst);
            if (ph) {
              shift_all(pa, ufirst - pe);
              add_poly(P, pa);
            }
          }
          PT_END(7)
          PT_BEGIN
          // ---- composite: lane 0 first takes the leading piece [0, u_0] of the
          // window (all of it if the window has no knot) with the incoming
          // polynomial, then every lane one piece per knot
          float tau_l = 0.f, col_l[3] = {0.f, 0.f, 0.f};  // this lane's optical depth and colour
          const df rs = df_add(t_start, df_neg(Ta));
          const float ystart = rs.hi + rs.lo;  // window-relative start of compositing
          long long dbg_base = 0, npieces = 0;
          if (DBG) {
            int cntp = 0;
#pragma unroll 1
            for (int i = i0; i < i1; ++i) {
              const float en = i + 1 < nc ? uat(i + 1) : Uend;
              if (en > uat(i)) ++cntp;
            }
            const float u0w = nc > 0 ? uat(0) : Uend;
            const int lead = (lane == 0 && u0w > 0.f) ? 1 : 0;
            const int tot = cntp + lead;
            int xx = tot;
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
              const int y = __shfl_up_sync(kFull, xx, o2);
              if (lane >= o2) xx += y;
            }
            dbg_base = dbg_np + (xx - tot) + lead;
            npieces = __shfl_sync(kFull, xx, 31);
          }
          float lastu = ufirst;
          // lane 0's first iteration (i = -1) is the leading piece [0, u_0] of
          // the window with the incoming polynomial; the compositing code is
          // inlined once, here (a call would save the live registers to local
          // memory around every piece)
#pragma unroll kRayUnrollComp
          for (int i = (lane == 0 ? -1 : i0); i < i1; ++i) {
            float Pc[NP], ua, ub;
            if (i < 0) {
#pragma unroll
              for (int q = 0; q < NP; ++q) Pc[q] = Aw[q];
              ua = 0.f;
              ub = nc > 0 ? uat(0) : Uend;
            } else {
              ua = uat(i);
              if (i > i0) shift_all(P, ua - lastu);
              float dl[NC * D];
              if (kStash) {
                dl[0] = stash0[i];
                if (D >= 2) dl[1 % D] = __int_as_float(stash1[i]);
                if (D >= 3) dl[2 % D] = __int_as_float(stash2[i]);
              } else {
                deltas(i, dl);
              }
              add_deltas(P, dl);
              lastu = ua;
#pragma unroll
              for (int q = 0; q < NP; ++q) Pc[q] = P[q];
              ub = i + 1 < nc ? uat(i + 1) : Uend;
            }
            if (CP) {  // the field: sum and compensation
#pragma unroll
              for (int d = 0; d <= D; ++d) Pc[d] += Pc[D + 1 + d];
            }
            if (DBG && p.dbg_field && ub > ua) {
              const long long row = i < 0 ? dbg_np : dbg_base++;
              if (row < p.field_cap) {
                double* fo = p.dbg_field + ((size_t)dbg_row * p.field_cap + row) * (D + 3);
                fo[0] = df_to_double(Ta) + (double)ua;
                fo[1] = df_to_double(Ta) + (double)ub;
                for (int d = 0; d <= D; ++d) fo[2 + d] = (double)Pc[d];
                if (GR && p.dbg_grad) {
                  double* go = p.dbg_grad + ((size_t)dbg_row * p.field_cap + row) * 3 * (D + 1);
                  for (int q = 0; q < 3 * (D + 1); ++q) go[q] = (double)Pc[D + 1 + q];
                }
              }
            }
            const float a0 = fmaxf(ua, ystart);
            if (ub > a0) {
              if (a0 > ua) shift_all(Pc, a0 - ua);
              if (GR)
                composite_piece_sh_inl<D>(Pc, Pc + D + 1, ub - a0, tfc, tau_l, col_l, p.shade_ka, p.shade_kd,
                                          p.shade_g2);
              else
                composite_piece_inl<D>(Pc, ub - a0, tfc, tau_l, col_l);
            }
          }
          if (DBG) dbg_np += npieces;
          PT_END(8)
          PT_BEGIN
          // carry the polynomial to the window end (plain recurrence / next window)
          {
            float cpy[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) cpy[q] = P[q];
            if (has) shift_all(cpy, Uend - lastu);
            const unsigned anym = __ballot_sync(kFull, has);
            if (anym) {
              const int lastlane = 31 - __clz(anym);
#pragma unroll
              for (int q = 0; q < NP; ++q) carry[q] = __shfl_sync(kFull, cpy[q], lastlane);
            } else {
              // no knot in the window: the incoming polynomial spans it
#pragma unroll
              for (int q = 0; q < NP; ++q) carry[q] = Aw[q];
              shift_all(carry, Uend);
            }
          }
          // combine lanes: transmittance as accumulated optical depth
          float tx = tau_l;
#pragma unroll
          for (int o2 = 1; o2 < 32; o2 <<= 1) {
            const float y = __shfl_up_sync(kFull, tx, o2);
            if (lane >= o2) tx += y;
          }
          const float tex = tx - tau_l;
          const float w = __expf(-(tau_ray + tex));
          col[0] += warp_sum(w * col_l[0]);
          col[1] += warp_sum(w * col_l[1]);
          col[2] += warp_sum(w * col_l[2]);
          tau_ray += __shfl_sync(kFull, tx, 31);
          dens = (nc > 0 && Uend > 0.f) ? (float)nc / Uend : 0.f;
          Ta = df_add(Ta, df{Uend, 0.f});
          __syncwarp();
          PT_END(9)
          if (p.tau_ert > 0.f && tau_ray > p.tau_ert) {
            done = true;
            break;
          }
        }
        if (done) break;
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
            ++r_tests;
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
              // within 1e-6 h of tangency: |d - q h| <= 1e-6 h (counted and reported)
              if (fabsf(dd - R2) <= 2e-6f * q * h * h) ++ray_tan;
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
          const int n_store = min(n_new, from_free + (cap_wc - hwm));
          if (n_store < n_new) {
            rf |= 1;
            if (!BIG && p.ovf) done = true;  // abandoned: the fallback pass renders the ray
          }
          if (cand && rank < n_store) {
            const int e = rank < from_free ? s_fre[nfree - 1 - rank] : hwm + (rank - from_free);
            // nearest Lambda entry (FP64 re-check near a midpoint)
            const float x = (d2 > 0.f ? d2 * rsqrtf(d2) : 0.f) * __fdividef(p.lam_scale, h);
            int j = (int)floorf(x + 0.5f);
            const float fr = x - floorf(x);
            if (fabsf(fr - 0.5f) < 2e-3f) j = nearest_entry_fp64(wv[0], wv[1], wv[2], h, p.n_lambda, q);
            j = min(max(j, 0), p.n_lambda - 1);
            s_rec[e] = make_float4(tc.hi, tc.lo, h, __fdividef(a, h * h * h));
            // shaded variant: the vector from the ray's closest point to the particle
            if (GR) s_dp[e] = make_float4(wv[0].hi + wv[0].lo, wv[1].hi + wv[1].lo, wv[2].hi + wv[2].lo, 0.f);
            s_j[e] = j;
            atomicAnd(stb + (e >> 5), ~(1u << (e & 31)));
            const float2 th = __ldg(p.theta + j);
            const float k0 = tc.hi + fmaf(knot_sigma(K, m, th, 0), h, tc.lo);  // first knot
            nk0[nnk + rank] = k0;
            nv0[nnk + rank] = e;
            // a first knot behind the processed part of the ray would mean the
            // ordering bound was violated: report it
            if (started && k0 < Ta.hi - 1e-6f * fabsf(Ta.hi)) rf |= 8;
            if (DBG && p.dbg_cands) {
              const long long ci2 = dbg_nc + rank;
              if (ci2 < p.cand_cap) p.dbg_cands[dbg_row * p.cand_cap + ci2] = p.orig[pidx];
            }
          }
          nfree -= from_free;
          hwm += n_store - from_free;
          nnk += n_store;
          r_cand += n_new;
          dbg_nc += n_new;
          ray_maxtab = max(ray_maxtab, hwm - nfree);
        }
        __syncwarp();
      }
      PT_END(1)
      PT_BEGIN
      cur = next_hit(cur + 1);
      PT_END(0)
    }

    // ---- output
    if (!BIG && p.ovf && (rf & 3)) {
      // abandoned: listed for the fallback pass, which writes the pixel and counts the ray
      if (lane == 0) {
        const unsigned k = atomicAdd(p.ovf, 1u);
        if (k < (unsigned)p.ovf_cap) {
          p.ovf[1 + k] = (unsigned)item_all;
        } else {
          wst[6] |= (unsigned long long)(kRayFlagRefit | (rf & 3));  // the list is full: this pixel stays unwritten
        }
      }
      continue;
    }
    if (FB && (rf & 3)) rf |= kRayFlagRefit;
    {
      // the ray's counters into the warp's statistics (tests and tangency-band
      // tests are counted per lane)
      const int tn = warp_sum_i(ray_tan), rt = warp_sum_i((int)r_tests);
      if (lane == 0) {
        wst[0] += 1ull;
        wst[1] += r_cand;
        wst[2] += my_knots;
        wst[3] += r_win;
        wst[4] += (unsigned)rt;
        wst[5] = max(wst[5], (unsigned long long)ray_maxtab);
        wst[6] |= (unsigned long long)rf;
        if (p.tau_ert > 0.f && tau_ray > p.tau_ert) wst[7] += 1ull;
        wst[8] = max(wst[8], (unsigned long long)ray_maxact);
        wst[9] += r_capped;
        wst[10] += (unsigned)tn;
      }
      __syncwarp();
    }
    if (DBG) {
      const int tn = warp_sum_i(ray_tan);
      if (lane == 0) {
        const float alpha = -expm1f(-tau_ray);
        p.dbg_rgba[4 * dbg_row + 0] = col[0];
        p.dbg_rgba[4 * dbg_row + 1] = col[1];
        p.dbg_rgba[4 * dbg_row + 2] = col[2];
        p.dbg_rgba[4 * dbg_row + 3] = alpha;
        long long* cnt = p.dbg_counts + 8 * dbg_row;
        cnt[0] = dbg_nc;
        cnt[1] = (long long)my_knots;
        cnt[2] = dbg_np;
        cnt[3] = rf;
        cnt[4] = tn;
        cnt[5] = dbg_win;
        cnt[6] = ray_maxact;
        cnt[7] = 0;
      }
    } else if (lane == 0) {
      const float alpha = -expm1f(-tau_ray);
      float4* o4 = (float4*)(BT ? p.frames[fb].out : p.out);
      o4[(size_t)py * cam.width + px] = make_float4(col[0], col[1], col[2], alpha);
    }
  }
  // ---- statistics (one set of atomics per warp)
  __syncwarp();
  if (lane == 0 && p.stats) {
    atomicAdd(p.stats + 0, wst[0]);
    atomicAdd(p.stats + 1, wst[1]);
    atomicAdd(p.stats + 2, wst[2]);
    atomicAdd(p.stats + 3, wst[3]);
    atomicAdd(p.stats + 5, wst[4]);
    atomicMax(p.stats + 6, wst[5]);
    atomicOr(p.stats + 7, wst[6]);
    atomicAdd(p.stats + 8, wst[7]);
    atomicMax(p.stats + 11, wst[8]);
    atomicAdd(p.stats + 12, wst[9]);
    atomicAdd(p.stats + 13, wst[10]);
#ifdef SPHDVR_PHASE_TIMING
    for (int ph = 0; ph < 10; ++ph) atomicAdd(p.stats + 16 + ph, (unsigned long long)pt_acc[ph]);
    for (int k = 0; k < 6; ++k) atomicAdd(p.stats + 26 + k, why_n[k]);
#endif
  }
}

}  // namespace sphdvr
