// Internal declarations of the sphdvr library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "sphdvr.h"

namespace sphdvr {

// Host look-up-table builder (lutgen.cpp).  Returns 0 on success.
int build_lut_host(int kernel, int K, int D, int n_lambda, double* theta, double* pieces, double* err);
// Gradient table for given knots (the across-ray gradient's G_L).  Returns 0 on success.
int build_grad_host(int kernel, int K, int D, int n_lambda, const double* theta, double* gpieces, double* gerr);
// Per-particle relative approximation error of a table from its per-entry errors.  Returns 0 on success.
int lut_error_measure_host(int kernel, int n_lambda, const double* err, double* E);
// Quantisation error estimate Q_E(tau, sigma) (Sec. 4.4) and the quantum values
// for a bit length and data variance ratio.  Return 0 on success.
int quant_error_host(int kernel, int D, double tau, double sigma, double* qe);
int quant_params_host(int kernel, int D, int int_bits, double ratio, double* tau, double* sigma, double* qe);
// w(0), the kernel's peak value
double kernel_peak_host(int kernel);

constexpr int kChunk = 32;       // particles per chunk of the acceleration structure
constexpr int kTile = 16;        // binning tile edge in pixels
constexpr int kMaxTf = 4096;     // transfer-function nodes

// Device copy of a look-up table.  For entry j:
//   theta[j]             = (theta_1, theta_2)            (theta_2 unused when m = 1)
//   jump[j*3*D + s*D + d-1]: localized difference coefficient of order d at
//                          knot slot s (0: middle knot at 0, s>=1: knot +theta_s),
//                          normalised units (Sec. 2); knot -theta_s mirrors
//                          slot s with sign (-1)^(d+1).
//   piece[j*2*(D+1) + (k-1)*(D+1) + d]: P_k local coefficients at theta_{k-1}.
struct DevLut {
  int kernel = 0, K = 0, D = 0, n_lambda = 0, m = 0;
  float q = 2.f;
  float reach = 2.f;  // largest theta_m of the table: knots lie within t_chi +- reach h
  float2* theta = nullptr;
  float* jump = nullptr;
  float* piece = nullptr;
  // gradient tables (sphdvr_lut_set_gradient), same layouts as jump / piece,
  // for G_L = w'(rho) / rho on the same knots; nullptr when absent
  float* gjump = nullptr;
  float* gpiece = nullptr;
};

// Per-frame camera, precomputed on the host in FP64.
struct DevCamera {
  int proj;  // 0 perspective, 1 orthographic
  int width, height;
  double eye[3], f[3], r[3], u[3];
  double tan_half, aspect, half_w, half_h, t_near;
};

struct DevTf {
  int n;
  float lo, hi, inv_dv;
  const float4* rgba;  // (r, g, b, sigma_scale * A)
};

// Grow-only device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace sphdvr

struct sphdvr_ctx {
  int device = 0;
  std::string last_error;
  // frame work buffers (grow-only)
  sphdvr::DevBuf chunk_rect, chunk_front, chunk_ntile, chunk_off, pair_key, pair_val, pair_key2, pair_val2,
      tile_range, scan_tmp, sort_tmp, stats, tf, img, dbg_pix, dbg_rgba, dbg_counts, dbg_cands, dbg_field, dbg_grad, table,
      work, fb_table, fb_list;
  sphdvr::DevBuf frames;  // frame records of a batch
  int num_sms = 0;
  std::vector<int64_t> last_stats = std::vector<int64_t>(16, 0);
  cudaStream_t last_stream = nullptr;
  bool stats_pending = false;
  // device counters of the last frame (the context's stats buffer, or the
  // static scratch array for sphdvr_render_static_scratch)
  const unsigned long long* stats_src = nullptr;
  int64_t last_pairs = 0;
  int64_t launches = 0;        // kernel launches since the context was created
  int64_t frame_launch0 = 0;   // value of `launches` when the last frame started
  cudaEvent_t ev_render0 = nullptr, ev_render1 = nullptr;  // around the last render kernel
  bool ev_ready = false;
};

struct sphdvr_lut {
  sphdvr_ctx* ctx = nullptr;
  sphdvr::DevLut d;
};

struct sphdvr_dataset {
  sphdvr_ctx* ctx = nullptr;
  int64_t n = 0;
  int n_chunks = 0;
  int n_levels = 0;
  float4* pos = nullptr;    // (x, y, z, h) in chunk order
  float* amp = nullptr;     // mass * value / density
  int* orig = nullptr;      // original particle index
  int2* chunk = nullptr;    // (start, count)
  float4* chunk_lo = nullptr;  // tight bbox min, w = max h
  float4* chunk_hi = nullptr;  // tight bbox max
  size_t bytes = 0;
};

namespace sphdvr {

// helpers implemented in api.cpp
sphdvr_status set_err(sphdvr_ctx* ctx, sphdvr_status st, const std::string& msg);
// EINVAL when opts ask for shading (entry points whose buffers are sized for unshaded rendering).
sphdvr_status reject_shading(sphdvr_ctx* ctx, const sphdvr_render_opts* o, const char* where);
sphdvr_status cuda_err(sphdvr_ctx* ctx, cudaError_t e, const char* where);
sphdvr_status ensure(sphdvr_ctx* ctx, DevBuf& b, size_t bytes);
sphdvr_status dev_alloc(sphdvr_ctx* ctx, void** p, size_t bytes);
// Argument checks shared by the render entry points (api.cu).
sphdvr_status check_camera(sphdvr_ctx* ctx, const sphdvr_camera* c, DevCamera* out);
sphdvr_status check_opts(sphdvr_ctx* ctx, const sphdvr_render_opts* o);
sphdvr_status check_common(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut);
// Validate a transfer function and pack it as (r, g, b, sigma_scale * A).
sphdvr_status pack_tf(sphdvr_ctx* ctx, const sphdvr_tf* tf, std::vector<float4>& out);

// sort.cu
// Exclusive prefix sum of n uint32 values (in may equal out).  If total is
// non-null the grand total is written there (device pointer).  tmp: device
// scratch of scan_tmp_words(n) words.
size_t scan_tmp_words(int64_t n);
sphdvr_status scan_exclusive_u32(sphdvr_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                                 uint32_t* tmp, cudaStream_t st);
// Stable LSD radix sort of (key, value) pairs on key bits [0, nbits).
// Result ends in keys/vals; keys2/vals2 are scratch of the same size; tmp:
// device scratch of sort_tmp_words(n) words.
size_t sort_tmp_words(int64_t n);
sphdvr_status radix_sort_u64(sphdvr_ctx* ctx, uint64_t* keys, uint32_t* vals, uint64_t* keys2, uint32_t* vals2,
                             int64_t n, int nbits, uint32_t* tmp, cudaStream_t st);

// dataset.cu
sphdvr_status build_dataset(sphdvr_ctx* ctx, sphdvr_dataset* ds, const float* pos, const float* h,
                            const float* mass, const float* density, const float* value, cudaStream_t st);

// frame.cu
struct RenderArgs {
  const sphdvr_dataset* ds;
  const DevLut* lut;
  DevCamera cam;
  int tf_n;
  float tf_lo, tf_hi;
  const float4* tf_host;  // validated table (r, g, b, sigma_scale * A), host memory
  const sphdvr_render_opts* opts;
  float* out;           // device image (normal mode)
  // debug mode (parity hook): listed pixels, device outputs
  int n_dbg = 0;
  const int* dbg_pix = nullptr;
  float* dbg_rgba = nullptr;
  long long* dbg_counts = nullptr;
  long long* dbg_cands = nullptr;
  int cand_cap = 0;
  double* dbg_field = nullptr;
  int field_cap = 0;
  double* dbg_grad = nullptr;  // shaded rendering: across-ray gradient rows beside the field rows
};
// Device scratch of one frame: every buffer the binning and the render
// kernel write besides the caller's image.
struct FrameWork {
  float4* chunk_rect = nullptr;       // [chunks]
  unsigned* chunk_front = nullptr;    // [chunks]
  uint32_t* chunk_ntile = nullptr;    // [chunks]
  uint32_t* chunk_off = nullptr;      // [chunks + 4] (total at [chunks])
  uint64_t* pair_key = nullptr;       // [pair_cap] x 2 buffers
  uint64_t* pair_key2 = nullptr;
  uint32_t* pair_val = nullptr;
  uint32_t* pair_val2 = nullptr;
  size_t pair_cap = 0;
  int2* tile_range = nullptr;         // [tiles]
  uint32_t* tmp = nullptr;            // scan / sort scratch
  size_t tmp_words = 0;
  unsigned long long* stats = nullptr;  // [16]
  float4* tf = nullptr;               // transfer function (r, g, b, sigma)
  float* table = nullptr;             // per-ray candidate tables of the persistent render grid
  int table_ctas = 0;                 // CTAs the table scratch covers
  unsigned* work = nullptr;           // work-queue counter
  // fallback pass of k_ray: per-warp scratch of fb_warps one-warp CTAs with the
  // larger per-ray capacities, and the list of abandoned rays ([0] count)
  float* fb_table = nullptr;
  int fb_warps = 0;
  unsigned* fb_list = nullptr;
  int fb_cap = 0;
};
// Rays one frame (or batch) can hand to the fallback pass.
constexpr int kFallbackList = 1 << 16;
// Scratch floats of the fallback pass for `warps` warps.
size_t fallback_floats(int warps, bool shaded = false);
// Persistent render grid for this frame and the table scratch it needs (floats).
int render_grid(sphdvr_ctx* ctx, const RenderArgs& a);
// The same for a batch of frames sharing data set, table and options.
int render_grid_batch(sphdvr_ctx* ctx, const RenderArgs* a, int n);
size_t render_table_floats(int grid, bool dbg, bool shaded = false);
// Render with scratch from the context's grow-only buffers.
sphdvr_status render_frame(sphdvr_ctx* ctx, const RenderArgs& a, cudaStream_t st);
// Render with caller-provided scratch; `sizer` (if non-null) is called with
// the pair count once it is known and must make room (return non-OK to stop).
typedef sphdvr_status (*PairSizer)(sphdvr_ctx* ctx, FrameWork& w, size_t pairs, void* user);
sphdvr_status render_frame_ws(sphdvr_ctx* ctx, const RenderArgs& a, FrameWork& w, PairSizer sizer, void* user,
                              cudaStream_t st);
// As render_frame, with the pair buffers sized by `sizer`.
sphdvr_status render_frame_sized(sphdvr_ctx* ctx, const RenderArgs& a, cudaStream_t st, PairSizer sizer, void* user);
// Render n (1..SPHDVR_MAX_BATCH) frames that share data set, table, transfer
// function and options with one launch of the render kernel, whose work
// queue spans the rays of all of them; scratch from the context's buffers.
// The frames' chunk rectangles, pairs and tile ranges are concatenated; the
// pair buffers are sized by `sizer` for the pairs of all frames.
sphdvr_status render_batch_sized(sphdvr_ctx* ctx, const RenderArgs* a, int n, cudaStream_t st, PairSizer sizer,
                                 void* user);
// Pixel rectangles of the chunks (rect[c] = x0, y0, x1, y1: the ray of pixel
// (px, py) can meet a particle of chunk c only if x0 - 0.5 <= px <= x1 + 0.5
// and y0 - 0.5 <= py <= y1 + 0.5).
sphdvr_status project_chunk_rects(sphdvr_ctx* ctx, const RenderArgs& a, float4* rect, unsigned* front, uint32_t* ntile,
                                  cudaStream_t st);
// The particle-centric pass order of Sec. 2 (scatter.cu).
sphdvr_status render_scatter(sphdvr_ctx* ctx, const RenderArgs& a, cudaStream_t st);
// Capacity-bound frame (no host synchronisation, allocation or host copy, so
// it can be captured into a CUDA graph): bins into w's pair buffers of
// w.pair_cap entries (pairs beyond are dropped and *ovf is set), sorts all
// w.pair_cap entries, and renders with `grid` CTAs.  w.tf must already hold
// the transfer function.
sphdvr_status render_frame_planned(sphdvr_ctx* ctx, const RenderArgs& a, const FrameWork& w, int grid, unsigned* ovf,
                                   cudaStream_t st);
// The sizer of render_frame: grows the context's pair buffers.
sphdvr_status ctx_pair_sizer(sphdvr_ctx* ctx, FrameWork& w, size_t pairs, void* user);
// Device bytes a frame needs besides its pair buffers, and the pair buffers'
// bytes for a given pair count (both without the grow-only headroom).
size_t frame_fixed_bytes(sphdvr_ctx* ctx, const RenderArgs& a);
size_t batch_fixed_bytes(sphdvr_ctx* ctx, const RenderArgs* a, int n);
size_t pair_bytes(size_t pairs);
// Device bytes the context holds after ctx_pair_sizer grew its pair buffers
// for `pairs` pairs.
size_t held_after_pair_sizer(const sphdvr_ctx* ctx, size_t pairs);
// api.cu: frame buffers a context holds; release them all.
size_t ctx_held_bytes(const sphdvr_ctx* ctx);
void ctx_release_buffers(sphdvr_ctx* ctx);

}  // namespace sphdvr
