// C-ABI entry points of libsphdvr (see include/sphdvr.h for the contract).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sphdvr_internal.h"

namespace sphdvr {

sphdvr_status set_err(sphdvr_ctx* ctx, sphdvr_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

sphdvr_status cuda_err(sphdvr_ctx* ctx, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return SPHDVR_OK;
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return set_err(ctx, SPHDVR_ENOMEM, m);
  return set_err(ctx, SPHDVR_ECUDA, m);
}

sphdvr_status dev_alloc(sphdvr_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_err(ctx, e == cudaErrorMemoryAllocation ? SPHDVR_ENOMEM : SPHDVR_ECUDA,
                   "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  return SPHDVR_OK;
}

sphdvr_status ensure(sphdvr_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return SPHDVR_OK;
  if (b.p) {
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t want = bytes + bytes / 4 + 256;
  sphdvr_status s = dev_alloc(ctx, &b.p, want);
  if (s == SPHDVR_OK) b.bytes = want;
  return s;
}

namespace {

void free_buf(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

}  // namespace

sphdvr_status check_camera(sphdvr_ctx* ctx, const sphdvr_camera* c, DevCamera* out) {
  if (!c) return set_err(ctx, SPHDVR_EINVAL, "camera is NULL");
  if (c->width < 1 || c->height < 1 || c->width > 32768 || c->height > 32768)
    return set_err(ctx, SPHDVR_EINVAL, "camera: width/height out of [1, 32768]");
  if (c->projection != 0 && c->projection != 1) return set_err(ctx, SPHDVR_EINVAL, "camera: projection must be 0 or 1");
  double f[3], r[3], u[3];
  for (int i = 0; i < 3; ++i) f[i] = c->target[i] - c->eye[i];
  double nf = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  if (!(nf > 0) || !std::isfinite(nf)) return set_err(ctx, SPHDVR_EINVAL, "camera: eye == target or not finite");
  for (int i = 0; i < 3; ++i) f[i] /= nf;
  r[0] = f[1] * c->up[2] - f[2] * c->up[1];
  r[1] = f[2] * c->up[0] - f[0] * c->up[2];
  r[2] = f[0] * c->up[1] - f[1] * c->up[0];
  double nr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (!(nr > 1e-12) || !std::isfinite(nr)) return set_err(ctx, SPHDVR_EINVAL, "camera: up is parallel to the view direction");
  for (int i = 0; i < 3; ++i) r[i] /= nr;
  u[0] = r[1] * f[2] - r[2] * f[1];
  u[1] = r[2] * f[0] - r[0] * f[2];
  u[2] = r[0] * f[1] - r[1] * f[0];
  if (c->projection == 0 && !(c->fovy_deg > 0 && c->fovy_deg < 179))
    return set_err(ctx, SPHDVR_EINVAL, "camera: fovy_deg must be in (0, 179)");
  if (c->projection == 1 && !(c->half_w > 0 && c->half_h > 0))
    return set_err(ctx, SPHDVR_EINVAL, "camera: half_w and half_h must be > 0");
  if (!std::isfinite(c->t_near)) return set_err(ctx, SPHDVR_EINVAL, "camera: t_near not finite");
  DevCamera d;
  d.proj = c->projection;
  d.width = c->width;
  d.height = c->height;
  for (int i = 0; i < 3; ++i) {
    d.eye[i] = c->eye[i];
    d.f[i] = f[i];
    d.r[i] = r[i];
    d.u[i] = u[i];
  }
  d.tan_half = std::tan(c->fovy_deg * M_PI / 360.0);
  d.aspect = (double)c->width / c->height;
  d.half_w = c->half_w;
  d.half_h = c->half_h;
  d.t_near = c->t_near;
  *out = d;
  return SPHDVR_OK;
}

// Validate the transfer function and pack it as (r, g, b, sigma_scale * A).
sphdvr_status pack_tf(sphdvr_ctx* ctx, const sphdvr_tf* tf, std::vector<float4>& out) {
  if (!tf || !tf->rgba) return set_err(ctx, SPHDVR_EINVAL, "transfer function is NULL");
  if (tf->n < 2 || tf->n > kMaxTf) return set_err(ctx, SPHDVR_EINVAL, "transfer function: n out of [2, 4096]");
  if (!(tf->lo < tf->hi) || !std::isfinite(tf->lo) || !std::isfinite(tf->hi))
    return set_err(ctx, SPHDVR_EINVAL, "transfer function: need finite lo < hi");
  if (!(tf->sigma_scale >= 0) || !std::isfinite(tf->sigma_scale))
    return set_err(ctx, SPHDVR_EINVAL, "transfer function: sigma_scale must be finite and >= 0");
  out.resize(tf->n);
  for (int i = 0; i < tf->n; ++i) {
    float v[4];
    for (int k = 0; k < 4; ++k) {
      v[k] = tf->rgba[4 * i + k];
      if (!std::isfinite(v[k]) || v[k] < 0)
        return set_err(ctx, SPHDVR_EINVAL, "transfer function: entries must be finite and >= 0");
    }
    out[i] = make_float4(v[0], v[1], v[2], (float)(v[3] * tf->sigma_scale));
  }
  return SPHDVR_OK;
}

sphdvr_status check_opts(sphdvr_ctx* ctx, const sphdvr_render_opts* o) {
  if (!o) return SPHDVR_OK;
  if (o->precision < 0 || o->precision > 5) return set_err(ctx, SPHDVR_EINVAL, "opts: precision out of range");
  if (o->precision == SPHDVR_PREC_INT64_QUANT &&
      !(o->quant_tau > 0 && std::isfinite(o->quant_tau) && o->quant_sigma > 0 && std::isfinite(o->quant_sigma)))
    return set_err(ctx, SPHDVR_EINVAL, "opts: INT64_QUANT needs finite quant_tau > 0 and quant_sigma > 0");
  if (!(o->reinit_dt >= 0.f) || !std::isfinite(o->reinit_dt))
    return set_err(ctx, SPHDVR_EINVAL, "opts: reinit_dt must be finite and >= 0");
  if (o->precision == 3 && !(o->reinit_dt > 0.f))
    return set_err(ctx, SPHDVR_EINVAL, "opts: FP32_REINIT needs reinit_dt > 0");
  if (o->precision == 0 && o->anchor_every < 1) return set_err(ctx, SPHDVR_EINVAL, "opts: anchor_every must be >= 1");
  if (!(o->ert_eps >= 0.f && o->ert_eps < 1.f)) return set_err(ctx, SPHDVR_EINVAL, "opts: ert_eps must be in [0, 1)");
  if (!(o->window_h >= 0.f) || !std::isfinite(o->window_h)) return set_err(ctx, SPHDVR_EINVAL, "opts: window_h must be >= 0");
  if (o->ray_capacity != 0 && (o->ray_capacity < 64 || o->ray_capacity > 4096))
    return set_err(ctx, SPHDVR_EINVAL, "opts: ray_capacity must be 0 or in [64, 4096]");
  if (o->reserved) return set_err(ctx, SPHDVR_EINVAL, "opts: reserved field must be 0");
  if (!(o->window_fill >= 0.f) || !std::isfinite(o->window_fill))
    return set_err(ctx, SPHDVR_EINVAL, "opts: window_fill must be finite and >= 0");
  if (o->ctas_per_sm < 0 || o->ctas_per_sm > 32) return set_err(ctx, SPHDVR_EINVAL, "opts: ctas_per_sm out of [0, 32]");
  if (o->shading != 0 && o->shading != 1) return set_err(ctx, SPHDVR_EINVAL, "opts: shading must be 0 or 1");
  if (o->shading) {
    if (o->precision != SPHDVR_PREC_FP32_ANCHORED && o->precision != SPHDVR_PREC_FP32_NAIVE)
      return set_err(ctx, SPHDVR_EINVAL, "opts: shading needs FP32_ANCHORED or FP32_NAIVE");
    if (!(o->shade_ka >= 0.f) || !std::isfinite(o->shade_ka) || !(o->shade_kd >= 0.f) || !std::isfinite(o->shade_kd) ||
        !(o->shade_g0 >= 0.f) || !std::isfinite(o->shade_g0 * o->shade_g0))
      return set_err(ctx, SPHDVR_EINVAL, "opts: shade_ka, shade_kd and shade_g0 must be finite and >= 0");
  }
  return SPHDVR_OK;
}

sphdvr_status reject_shading(sphdvr_ctx* ctx, const sphdvr_render_opts* o, const char* where) {
  if (o && o->shading) return set_err(ctx, SPHDVR_EINVAL, std::string(where) + ": shading is available through sphdvr_render and sphdvr_debug_rays only");
  return SPHDVR_OK;
}

sphdvr_status check_common(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut) {
  if (!ctx) return SPHDVR_EINVAL;
  if (!ds || !lut) return set_err(ctx, SPHDVR_EINVAL, "dataset or table is NULL");
  if (ds->ctx != ctx || lut->ctx != ctx) return set_err(ctx, SPHDVR_EINVAL, "object belongs to another context");
  cudaError_t e = cudaSetDevice(ctx->device);
  return cuda_err(ctx, e, "cudaSetDevice");
}

}  // namespace sphdvr

namespace sphdvr {

size_t ctx_held_bytes(const sphdvr_ctx* c) {
  const DevBuf* bufs[] = {&c->chunk_rect, &c->chunk_front, &c->chunk_ntile, &c->chunk_off, &c->pair_key,
                          &c->pair_val, &c->pair_key2, &c->pair_val2, &c->tile_range, &c->scan_tmp, &c->sort_tmp,
                          &c->stats, &c->tf, &c->img, &c->dbg_pix, &c->dbg_rgba, &c->dbg_counts, &c->dbg_cands,
                          &c->dbg_field, &c->dbg_grad, &c->table, &c->work, &c->frames, &c->fb_table, &c->fb_list};
  size_t t = 0;
  for (const DevBuf* b : bufs) t += b->bytes;
  return t;
}

void ctx_release_buffers(sphdvr_ctx* c) {
  DevBuf* bufs[] = {&c->chunk_rect, &c->chunk_front, &c->chunk_ntile, &c->chunk_off, &c->pair_key, &c->pair_val,
                    &c->pair_key2, &c->pair_val2, &c->tile_range, &c->scan_tmp, &c->sort_tmp, &c->stats,
                    &c->tf, &c->img, &c->dbg_pix, &c->dbg_rgba, &c->dbg_counts, &c->dbg_cands, &c->dbg_field,
                    &c->dbg_grad, &c->table, &c->work, &c->frames, &c->fb_table, &c->fb_list};
  for (DevBuf* b : bufs) free_buf(*b);
  c->stats_pending = false;
}

}  // namespace sphdvr

using namespace sphdvr;

extern "C" {

const char* sphdvr_status_string(int s) {
  switch (s) {
    case SPHDVR_OK: return "ok";
    case SPHDVR_EINVAL: return "invalid argument";
    case SPHDVR_ENOMEM: return "out of memory";
    case SPHDVR_ECUDA: return "CUDA error";
    case SPHDVR_ETIMEOUT: return "timed out";
    case SPHDVR_EBUSY: return "does not fit the memory budget";
    case SPHDVR_EOVERFLOW: return "buffer capacity exceeded";
    case SPHDVR_EDEVICE: return "no usable sm_103 device";
    case SPHDVR_ENOTFOUND: return "not found";
  }
  return "unknown status";
}

const char* sphdvr_version(void) { return "sphdvr 0.1 (sm_103a)"; }

sphdvr_status sphdvr_create(int device, sphdvr_ctx** out) {
  if (!out) return SPHDVR_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return SPHDVR_EDEVICE;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return SPHDVR_EDEVICE;
  if (!(prop.major == 10 && prop.minor == 3)) return SPHDVR_EDEVICE;
  if (cudaSetDevice(device) != cudaSuccess) return SPHDVR_EDEVICE;
  sphdvr_ctx* c = new (std::nothrow) sphdvr_ctx();
  if (!c) return SPHDVR_ENOMEM;
  c->device = device;
  // the events around every render kernel, created here so that no render
  // call has to create them
  if (cudaEventCreate(&c->ev_render0) != cudaSuccess || cudaEventCreate(&c->ev_render1) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return SPHDVR_ECUDA;
  }
  c->ev_ready = true;
  *out = c;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_destroy(sphdvr_ctx* c) {
  if (!c) return SPHDVR_EINVAL;
  cudaSetDevice(c->device);
  ctx_release_buffers(c);
  if (c->ev_ready) {
    cudaEventDestroy(c->ev_render0);
    cudaEventDestroy(c->ev_render1);
  }
  delete c;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_last_error(const sphdvr_ctx* c, char* buf, size_t len) {
  if (!c || !buf || len == 0) return SPHDVR_EINVAL;
  std::snprintf(buf, len, "%s", c->last_error.c_str());
  return SPHDVR_OK;
}

// ---- table files ---------------------------------------------------------
namespace {
struct LutFileHeader {
  char magic[8];
  uint32_t version;
  int32_t kernel, K, D, n_lambda;
  int32_t reserved;  // 0
  double q;
};
static_assert(sizeof(LutFileHeader) == 40, "table file header layout");
constexpr char kLutMagic[8] = {'S', 'P', 'H', 'D', 'V', 'R', 'L', 'T'};

bool lut_dims_ok(int kernel, int K, int D, int n_lambda) {
  return kernel >= 0 && kernel <= 3 && K >= 1 && K <= 4 && D >= 1 && D <= 6 && n_lambda >= 2 && n_lambda <= 65536;
}

// open a table file and read and check its header; *f is left after the header
sphdvr_status lut_open(const char* path, LutFileHeader& h, std::FILE** f) {
  if (!path) return SPHDVR_EINVAL;
  *f = std::fopen(path, "rb");
  if (!*f) return SPHDVR_ENOTFOUND;
  if (std::fread(&h, sizeof(h), 1, *f) != 1 || std::memcmp(h.magic, kLutMagic, 8) != 0 || h.version != 1 ||
      !lut_dims_ok(h.kernel, h.K, h.D, h.n_lambda)) {
    std::fclose(*f);
    *f = nullptr;
    return SPHDVR_EINVAL;
  }
  return SPHDVR_OK;
}
}  // namespace

sphdvr_status sphdvr_lut_save(const char* path, int kernel, int K, int D, int n_lambda, const double* theta,
                              const double* pieces, const double* err) {
  if (!path || !theta || !pieces || !lut_dims_ok(kernel, K, D, n_lambda)) return SPHDVR_EINVAL;
  const size_t n = (size_t)n_lambda, m = (size_t)(K + 1) / 2;
  LutFileHeader h;
  std::memcpy(h.magic, kLutMagic, 8);
  h.version = 1;
  h.kernel = kernel;
  h.K = K;
  h.D = D;
  h.n_lambda = n_lambda;
  h.reserved = 0;
  h.q = kernel == 3 ? 1.0 : 2.0;
  std::FILE* f = std::fopen(path, "wb");
  if (!f) return SPHDVR_ENOTFOUND;
  std::vector<double> zeros(err ? 0 : n, 0.0);
  bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(theta, sizeof(double), n * m, f) == n * m &&
            std::fwrite(pieces, sizeof(double), n * m * (D + 1), f) == n * m * (D + 1) &&
            std::fwrite(err ? err : zeros.data(), sizeof(double), n, f) == n;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? SPHDVR_OK : SPHDVR_EINVAL;
}

sphdvr_status sphdvr_lut_read_header(const char* path, int* kernel, int* K, int* D, int* n_lambda) {
  if (!kernel || !K || !D || !n_lambda) return SPHDVR_EINVAL;
  LutFileHeader h;
  std::FILE* f = nullptr;
  sphdvr_status s = lut_open(path, h, &f);
  if (s != SPHDVR_OK) return s;
  std::fclose(f);
  *kernel = h.kernel;
  *K = h.K;
  *D = h.D;
  *n_lambda = h.n_lambda;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_lut_read(const char* path, double* theta, double* pieces, double* err) {
  if (!theta || !pieces) return SPHDVR_EINVAL;
  LutFileHeader h;
  std::FILE* f = nullptr;
  sphdvr_status s = lut_open(path, h, &f);
  if (s != SPHDVR_OK) return s;
  const size_t n = (size_t)h.n_lambda, m = (size_t)(h.K + 1) / 2, np = n * m * (h.D + 1);
  std::vector<double> e(n);
  bool ok = std::fread(theta, sizeof(double), n * m, f) == n * m && std::fread(pieces, sizeof(double), np, f) == np &&
            std::fread(e.data(), sizeof(double), n, f) == n;
  char extra;
  ok = ok && std::fread(&extra, 1, 1, f) == 0;  // nothing after the table
  std::fclose(f);
  if (!ok) return SPHDVR_EINVAL;
  if (err) std::memcpy(err, e.data(), n * sizeof(double));
  return SPHDVR_OK;
}

sphdvr_status sphdvr_lut_load(sphdvr_ctx* ctx, const char* path, sphdvr_lut** out) {
  if (!ctx || !out) return SPHDVR_EINVAL;
  *out = nullptr;
  int kernel, K, D, n;
  sphdvr_status s = sphdvr_lut_read_header(path, &kernel, &K, &D, &n);
  if (s != SPHDVR_OK) return set_err(ctx, s, "lut_load: cannot read the table file header");
  const size_t m = (size_t)(K + 1) / 2;
  std::vector<double> th((size_t)n * m), pc((size_t)n * m * (D + 1));
  if ((s = sphdvr_lut_read(path, th.data(), pc.data(), nullptr)) != SPHDVR_OK)
    return set_err(ctx, s, "lut_load: short or malformed table file");
  return sphdvr_lut_create(ctx, kernel, K, D, n, th.data(), pc.data(), out);
}

sphdvr_status sphdvr_quant_error(int kernel, int D, double tau, double sigma, double* qe) {
  return quant_error_host(kernel, D, tau, sigma, qe) == 0 ? SPHDVR_OK : SPHDVR_EINVAL;
}

sphdvr_status sphdvr_quant_params(int kernel, int D, int int_bits, double variance_ratio, double* tau_rel,
                                  double* sigma_rel, double* qe) {
  return quant_params_host(kernel, D, int_bits, variance_ratio, tau_rel, sigma_rel, qe) == 0 ? SPHDVR_OK
                                                                                              : SPHDVR_EINVAL;
}

sphdvr_status sphdvr_lut_error_measure(int kernel, int n_lambda, const double* err, double* E) {
  return lut_error_measure_host(kernel, n_lambda, err, E) == 0 ? SPHDVR_OK : SPHDVR_EINVAL;
}

sphdvr_status sphdvr_lut_build(int kernel, int K, int D, int n_lambda, double* theta, double* pieces, double* err) {
  if (kernel < 0 || kernel > 3 || K < 1 || K > 4 || D < 1 || D > 6 || n_lambda < 2 || n_lambda > 65536 || !theta ||
      !pieces)
    return SPHDVR_EINVAL;
  return build_lut_host(kernel, K, D, n_lambda, theta, pieces, err) ? SPHDVR_EINVAL : SPHDVR_OK;
}

// Device layouts of one table's pieces (for the field, or for the gradient's
// G_L on the same knots): per entry the localized difference coefficients
// (Sec. 2) at the knot slots -- jump[j*3*D + s*D + d-1], slot 0 the middle knot
// (even K), slot s >= 1 the knot +theta_s -- and the pieces' local
// coefficients piece[j*2*(D+1) + (k-1)*(D+1) + d].  False on a non-finite
// coefficient.
static bool difference_tables(int K, int D, int n_lambda, const double* theta, const double* pieces,
                              std::vector<float>& jump, std::vector<float>& pc) {
  const int m = (K + 1) / 2;
  jump.assign((size_t)n_lambda * 3 * D, 0.f);
  pc.assign((size_t)n_lambda * 2 * (D + 1), 0.f);
  for (int j = 0; j < n_lambda; ++j) {
    const double* T = theta + (size_t)j * m;
    const double* P = pieces + (size_t)j * m * (D + 1);
    for (int i = 0; i < m * (D + 1); ++i)
      if (!std::isfinite(P[i])) return false;
    for (int k = 0; k < m; ++k)
      for (int d = 0; d <= D; ++d) pc[(size_t)j * 2 * (D + 1) + k * (D + 1) + d] = (float)P[k * (D + 1) + d];
    // localized difference coefficients (Sec. 2) at +theta_r: P_{r+1} - P_r expanded at theta_r
    for (int r = 1; r <= m; ++r) {
      double q[8] = {0};
      for (int d = 0; d <= D; ++d) q[d] = P[(r - 1) * (D + 1) + d];
      double s = T[r - 1] - (r > 1 ? T[r - 2] : 0.0);
      for (int i = 0; i < D; ++i)
        for (int k = D - 1; k >= i; --k) q[k] += s * q[k + 1];
      for (int d = 1; d <= D; ++d) {
        double nxt = r < m ? P[r * (D + 1) + d] : 0.0;
        jump[(size_t)j * 3 * D + r * D + d - 1] = (float)(nxt - q[d]);
      }
    }
    // middle knot (even K): P_1(s) - P_1(-s) = 2 * odd part
    if (!(K & 1))
      for (int d = 1; d <= D; d += 2) jump[(size_t)j * 3 * D + 0 * D + d - 1] = (float)(2.0 * P[d]);
  }
  return true;
}

sphdvr_status sphdvr_lut_create(sphdvr_ctx* ctx, int kernel, int K, int D, int n_lambda, const double* theta,
                                const double* pieces, sphdvr_lut** out) {
  if (!ctx || !out) return SPHDVR_EINVAL;
  *out = nullptr;
  if (kernel < 0 || kernel > 3 || K < 1 || K > 4 || D < 1 || D > 6 || n_lambda < 2 || n_lambda > 65536 || !theta ||
      !pieces)
    return set_err(ctx, SPHDVR_EINVAL, "lut_create: bad arguments (K in [1,4], D in [1,6], n_lambda in [2,65536])");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  const int m = (K + 1) / 2;
  std::vector<float> th(2 * (size_t)n_lambda, 0.f), jump, pc;
  for (int j = 0; j < n_lambda; ++j) {
    const double* T = theta + (size_t)j * m;
    for (int k = 0; k < m; ++k) {
      if (!std::isfinite(T[k]) || T[k] < 0 || (k && T[k] < T[k - 1]))
        return set_err(ctx, SPHDVR_EINVAL, "lut_create: knots must be finite, >= 0 and non-decreasing");
    }
    th[2 * j] = (float)T[0];
    th[2 * j + 1] = (float)(m > 1 ? T[1] : T[0]);
  }
  if (!difference_tables(K, D, n_lambda, theta, pieces, jump, pc))
    return set_err(ctx, SPHDVR_EINVAL, "lut_create: non-finite piece coefficient");
  sphdvr_lut* L = new (std::nothrow) sphdvr_lut();
  if (!L) return set_err(ctx, SPHDVR_ENOMEM, "lut_create: host allocation");
  L->ctx = ctx;
  L->d.kernel = kernel;
  L->d.K = K;
  L->d.D = D;
  L->d.n_lambda = n_lambda;
  L->d.m = m;
  L->d.q = kernel == SPHDVR_KERNEL_POLY6 ? 1.f : 2.f;
  {
    // largest outer knot of the table (optimal outer knots may sit slightly
    // beyond the support): every knot lies within reach * h of its t_chi
    double reach = 0.0;
    for (int j = 0; j < n_lambda; ++j) reach = std::max(reach, theta[(size_t)j * m + m - 1]);
    L->d.reach = (float)(reach * (1.0 + 1e-6));
  }
  sphdvr_status s;
  if ((s = dev_alloc(ctx, (void**)&L->d.theta, th.size() * sizeof(float))) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&L->d.jump, jump.size() * sizeof(float))) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&L->d.piece, pc.size() * sizeof(float))) != SPHDVR_OK) {
    sphdvr_lut_free(L);
    return s;
  }
  if ((e = cudaMemcpy(L->d.theta, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(L->d.jump, jump.data(), jump.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(L->d.piece, pc.data(), pc.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) {
    sphdvr_lut_free(L);
    return cuda_err(ctx, e, "lut upload");
  }
  *out = L;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_lut_build_grad(int kernel, int K, int D, int n_lambda, const double* theta, double* gpieces,
                                    double* gerr) {
  if (kernel < 0 || kernel > 3 || K < 1 || K > 4 || D < 1 || D > 6 || n_lambda < 2 || n_lambda > 65536 || !theta ||
      !gpieces)
    return SPHDVR_EINVAL;
  const int m = (K + 1) / 2;
  for (int64_t i = 0; i < (int64_t)n_lambda * m; ++i)
    if (!std::isfinite(theta[i]) || theta[i] < 0) return SPHDVR_EINVAL;
  return build_grad_host(kernel, K, D, n_lambda, theta, gpieces, gerr) == 0 ? SPHDVR_OK : SPHDVR_EINVAL;
}

sphdvr_status sphdvr_lut_set_gradient(sphdvr_lut* L, const double* theta, const double* gpieces) {
  if (!L || !theta || !gpieces) return SPHDVR_EINVAL;
  sphdvr_ctx* ctx = L->ctx;
  const DevLut& d = L->d;
  std::vector<float> jump, pc;
  if (!difference_tables(d.K, d.D, d.n_lambda, theta, gpieces, jump, pc))
    return set_err(ctx, SPHDVR_EINVAL, "lut_set_gradient: non-finite piece coefficient");
  // the knots must be the table's own (the gradient shares them)
  std::vector<float> th(2 * (size_t)d.n_lambda);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaMemcpy(th.data(), d.theta, th.size() * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "lut_set_gradient: table knots");
  const int m = d.m;
  for (int j = 0; j < d.n_lambda; ++j)
    if (th[2 * j] != (float)theta[(size_t)j * m] || (m > 1 && th[2 * j + 1] != (float)theta[(size_t)j * m + 1]))
      return set_err(ctx, SPHDVR_EINVAL, "lut_set_gradient: knots differ from the table's");
  float *gj = nullptr, *gp = nullptr;
  sphdvr_status s;
  if ((s = dev_alloc(ctx, (void**)&gj, jump.size() * sizeof(float))) != SPHDVR_OK) return s;
  if ((s = dev_alloc(ctx, (void**)&gp, pc.size() * sizeof(float))) != SPHDVR_OK) {
    cudaFree(gj);
    return s;
  }
  if ((e = cudaMemcpy(gj, jump.data(), jump.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(gp, pc.data(), pc.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(gj);
    cudaFree(gp);
    return cuda_err(ctx, e, "lut_set_gradient: upload");
  }
  cudaFree(L->d.gjump);
  cudaFree(L->d.gpiece);
  L->d.gjump = gj;
  L->d.gpiece = gp;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_lut_free(sphdvr_lut* L) {
  if (!L) return SPHDVR_EINVAL;
  if (L->ctx) cudaSetDevice(L->ctx->device);
  cudaFree(L->d.theta);
  cudaFree(L->d.jump);
  cudaFree(L->d.piece);
  cudaFree(L->d.gjump);
  cudaFree(L->d.gpiece);
  delete L;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_dataset_create(sphdvr_ctx* ctx, int64_t n, const float* pos, const float* h, const float* mass,
                                    const float* density, const float* value, int inputs_on_device, void* stream,
                                    sphdvr_dataset** out) {
  if (!ctx || !out) return SPHDVR_EINVAL;
  *out = nullptr;
  if (n < 1 || n > ((int64_t)1 << 30)) return set_err(ctx, SPHDVR_EINVAL, "dataset: n out of [1, 2^30]");
  if (!pos || !h) return set_err(ctx, SPHDVR_EINVAL, "dataset: pos and h are required");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const float* src[5] = {pos, h, mass, density, value};
  const size_t cnt[5] = {3 * (size_t)n, (size_t)n, (size_t)n, (size_t)n, (size_t)n};
  float* dv[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  sphdvr_status s = SPHDVR_OK;
  if (!inputs_on_device) {
    for (int i = 0; i < 5 && s == SPHDVR_OK; ++i) {
      if (!src[i]) continue;
      s = dev_alloc(ctx, (void**)&dv[i], cnt[i] * sizeof(float));
      if (s == SPHDVR_OK) {
        e = cudaMemcpyAsync(dv[i], src[i], cnt[i] * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = cuda_err(ctx, e, "dataset upload");
      }
    }
  } else {
    for (int i = 0; i < 5; ++i) dv[i] = const_cast<float*>(src[i]);
  }
  sphdvr_dataset* ds = nullptr;
  if (s == SPHDVR_OK) {
    ds = new (std::nothrow) sphdvr_dataset();
    if (!ds) s = set_err(ctx, SPHDVR_ENOMEM, "dataset: host allocation");
  }
  if (s == SPHDVR_OK) {
    ds->ctx = ctx;
    ds->n = n;
    s = build_dataset(ctx, ds, dv[0], dv[1], dv[2], dv[3], dv[4], st);
  }
  if (!inputs_on_device) {
    cudaStreamSynchronize(st);
    for (int i = 0; i < 5; ++i) cudaFree(dv[i]);
  }
  if (s != SPHDVR_OK) {
    if (ds) sphdvr_dataset_free(ds);
    return s;
  }
  *out = ds;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_dataset_free(sphdvr_dataset* ds) {
  if (!ds) return SPHDVR_EINVAL;
  if (ds->ctx) cudaSetDevice(ds->ctx->device);
  cudaFree(ds->pos);
  cudaFree(ds->amp);
  cudaFree(ds->orig);
  cudaFree(ds->chunk);
  cudaFree(ds->chunk_lo);
  cudaFree(ds->chunk_hi);
  delete ds;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_ctx_info(const sphdvr_ctx* ctx, int64_t info[4]) {
  if (!ctx || !info) return SPHDVR_EINVAL;
  info[0] = (int64_t)ctx_held_bytes(ctx);
  info[1] = ctx->launches;
  info[2] = ctx->device;
  info[3] = 0;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_dataset_info(const sphdvr_dataset* ds, int64_t info[8]) {
  if (!ds || !info) return SPHDVR_EINVAL;
  info[0] = ds->n;
  info[1] = ds->n_chunks;
  info[2] = ds->n_levels;
  info[3] = (int64_t)ds->bytes;
  for (int i = 4; i < 8; ++i) info[i] = 0;
  return SPHDVR_OK;
}

static sphdvr_status do_render(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                               const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                               float* rgba_out, cudaStream_t st, RenderArgs* base) {
  sphdvr_status s = check_common(ctx, ds, lut);
  if (s != SPHDVR_OK) return s;
  if ((s = check_opts(ctx, opts)) != SPHDVR_OK) return s;
  if (opts && opts->shading && !(lut->d.gjump && lut->d.gpiece))
    return set_err(ctx, SPHDVR_EINVAL, "render: shading needs a table with a gradient (sphdvr_lut_set_gradient)");
  RenderArgs a = base ? *base : RenderArgs();
  a.ds = ds;
  a.lut = &lut->d;
  if ((s = check_camera(ctx, cam, &a.cam)) != SPHDVR_OK) return s;
  std::vector<float4> tfh;
  if ((s = pack_tf(ctx, tf, tfh)) != SPHDVR_OK) return s;
  a.tf_n = tf->n;
  a.tf_lo = (float)tf->lo;
  a.tf_hi = (float)tf->hi;
  a.tf_host = tfh.data();
  a.opts = opts;
  a.out = rgba_out;
  ctx->frame_launch0 = ctx->launches;
  s = render_frame(ctx, a, st);
  if (s != SPHDVR_OK) return s;
  ctx->last_stream = st;
  ctx->stats_src = nullptr;
  ctx->stats_pending = true;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_render(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                            const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                            float* rgba_out, void* stream) {
  if (!ctx) return SPHDVR_EINVAL;
  if (!rgba_out) return set_err(ctx, SPHDVR_EINVAL, "render: rgba_out is NULL");
  return do_render(ctx, ds, lut, cam, tf, opts, rgba_out, (cudaStream_t)stream, nullptr);
}

sphdvr_status sphdvr_render_batch(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut, int n_frames,
                                  const sphdvr_camera* cams, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                  float* const* rgba_out, void* stream) {
  if (!ctx) return SPHDVR_EINVAL;
  if (n_frames < 1 || n_frames > SPHDVR_MAX_BATCH)
    return set_err(ctx, SPHDVR_EINVAL, "render_batch: n_frames out of [1, SPHDVR_MAX_BATCH]");
  if (!cams || !rgba_out) return set_err(ctx, SPHDVR_EINVAL, "render_batch: NULL argument");
  sphdvr_status s = check_common(ctx, ds, lut);
  if (s != SPHDVR_OK) return s;
  if ((s = check_opts(ctx, opts)) != SPHDVR_OK || (s = reject_shading(ctx, opts, "render_batch")) != SPHDVR_OK)
    return s;
  std::vector<float4> tfh;
  if ((s = pack_tf(ctx, tf, tfh)) != SPHDVR_OK) return s;
  RenderArgs a[SPHDVR_MAX_BATCH];
  for (int f = 0; f < n_frames; ++f) {
    if (!rgba_out[f]) return set_err(ctx, SPHDVR_EINVAL, "render_batch: rgba_out[f] is NULL");
    a[f].ds = ds;
    a[f].lut = &lut->d;
    if ((s = check_camera(ctx, &cams[f], &a[f].cam)) != SPHDVR_OK) return s;
    a[f].tf_n = tf->n;
    a[f].tf_lo = (float)tf->lo;
    a[f].tf_hi = (float)tf->hi;
    a[f].tf_host = tfh.data();
    a[f].opts = opts;
    a[f].out = rgba_out[f];
  }
  ctx->frame_launch0 = ctx->launches;
  const cudaStream_t st = (cudaStream_t)stream;
  s = render_batch_sized(ctx, a, n_frames, st, ctx_pair_sizer, nullptr);
  if (s != SPHDVR_OK) return s;
  ctx->last_stream = st;
  ctx->stats_src = nullptr;
  ctx->stats_pending = true;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_render_scatter(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                    const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                    float* rgba_out, void* stream) {
  if (!ctx) return SPHDVR_EINVAL;
  if (!rgba_out) return set_err(ctx, SPHDVR_EINVAL, "render_scatter: rgba_out is NULL");
  sphdvr_status s = check_common(ctx, ds, lut);
  if (s != SPHDVR_OK) return s;
  if ((s = check_opts(ctx, opts)) != SPHDVR_OK || (s = reject_shading(ctx, opts, "render_scatter")) != SPHDVR_OK)
    return s;
  RenderArgs a{};
  a.ds = ds;
  a.lut = &lut->d;
  if ((s = check_camera(ctx, cam, &a.cam)) != SPHDVR_OK) return s;
  std::vector<float4> tfh;
  if ((s = pack_tf(ctx, tf, tfh)) != SPHDVR_OK) return s;
  a.tf_n = tf->n;
  a.tf_lo = (float)tf->lo;
  a.tf_hi = (float)tf->hi;
  a.tf_host = tfh.data();
  a.opts = opts;
  a.out = rgba_out;
  ctx->frame_launch0 = ctx->launches;
  const cudaStream_t st = (cudaStream_t)stream;
  if ((s = render_scatter(ctx, a, st)) != SPHDVR_OK) return s;
  ctx->last_stream = st;
  ctx->stats_src = nullptr;
  ctx->stats_pending = true;
  return SPHDVR_OK;
}

sphdvr_status sphdvr_render_host(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                 const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                 float* rgba_host, void* stream) {
  if (!ctx) return SPHDVR_EINVAL;
  if (!rgba_host || !cam) return set_err(ctx, SPHDVR_EINVAL, "render_host: NULL argument");
  if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
    return set_err(ctx, SPHDVR_EINVAL, "camera: width/height out of [1, 32768]");
  size_t bytes = (size_t)cam->width * cam->height * 4 * sizeof(float);
  sphdvr_status s = ensure(ctx, ctx->img, bytes);
  if (s != SPHDVR_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  s = do_render(ctx, ds, lut, cam, tf, opts, (float*)ctx->img.p, st, nullptr);
  if (s != SPHDVR_OK) return s;
  cudaError_t e = cudaMemcpyAsync(rgba_host, ctx->img.p, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_err(ctx, e, "render_host copy");
}

sphdvr_status sphdvr_frame_stats(sphdvr_ctx* ctx, int64_t out[16]) {
  if (!ctx || !out) return SPHDVR_EINVAL;
  const unsigned long long* src = ctx->stats_src ? ctx->stats_src : (const unsigned long long*)ctx->stats.p;
  if (ctx->stats_pending && src) {
    unsigned long long h[16];
    cudaError_t e = cudaMemcpyAsync(h, src, sizeof(h), cudaMemcpyDeviceToHost, ctx->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->last_stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "frame stats");
    for (int i = 0; i < 16; ++i) ctx->last_stats[i] = (int64_t)h[i];
    ctx->stats_pending = false;
  }
  for (int i = 0; i < 16; ++i) out[i] = ctx->last_stats[i];
  out[4] = ctx->last_pairs;
  out[9] = 0;
  if (ctx->ev_ready) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev_render0, ctx->ev_render1) == cudaSuccess) out[9] = (int64_t)(ms * 1e6);
    cudaGetLastError();
  }
  out[10] = ctx->launches - ctx->frame_launch0;
  out[11] = ctx->last_stats[11];
  out[12] = ctx->last_stats[12];
  out[13] = ctx->last_stats[13];
  out[14] = 0;
  out[15] = 0;
  return SPHDVR_OK;
}

#ifdef SPHDVR_PHASE_TIMING
// Instrumented builds only: per-phase clock64 totals of the last frame's render kernel.
// out[0..9] phase clocks, out[10..15] windows by what ended them (k_ray).
sphdvr_status sphdvr_phase_times(sphdvr_ctx* ctx, int64_t out[16]) {
  if (!ctx || !out || !ctx->stats.p) return SPHDVR_EINVAL;
  unsigned long long h[16];
  cudaError_t e = cudaMemcpy(h, (unsigned long long*)ctx->stats.p + 16, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "phase times");
  for (int i = 0; i < 16; ++i) out[i] = (int64_t)h[i];
  return SPHDVR_OK;
}
#endif

static sphdvr_status debug_rays(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                int n_pix, const int* pix, float* rgba, int64_t* counts, int64_t* cand_ids,
                                int cand_cap, double* field, double* grad, int field_cap) {
  if (!ctx) return SPHDVR_EINVAL;
  if (n_pix < 1 || !pix || !rgba || !counts || !cam) return set_err(ctx, SPHDVR_EINVAL, "debug_rays: bad arguments");
  if ((cand_ids && cand_cap < 1) || (field && field_cap < 1)) return set_err(ctx, SPHDVR_EINVAL, "debug_rays: capacity < 1");
  for (int i = 0; i < n_pix; ++i)
    if (pix[i] < 0 || (int64_t)pix[i] >= (int64_t)cam->width * cam->height)
      return set_err(ctx, SPHDVR_EINVAL, "debug_rays: pixel index out of range");
  sphdvr_status s = check_common(ctx, ds, lut);
  if (s != SPHDVR_OK) return s;
  const int D = lut->d.D;
  if ((s = ensure(ctx, ctx->dbg_pix, n_pix * sizeof(int))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->dbg_rgba, n_pix * 4 * sizeof(float))) != SPHDVR_OK ||
      (s = ensure(ctx, ctx->dbg_counts, n_pix * 8 * sizeof(int64_t))) != SPHDVR_OK)
    return s;
  if (cand_ids && (s = ensure(ctx, ctx->dbg_cands, (size_t)n_pix * cand_cap * sizeof(int64_t))) != SPHDVR_OK) return s;
  if (field && (s = ensure(ctx, ctx->dbg_field, (size_t)n_pix * field_cap * (D + 3) * sizeof(double))) != SPHDVR_OK)
    return s;
  const size_t grad_doubles = (size_t)n_pix * field_cap * 3 * (D + 1);
  if (grad && (s = ensure(ctx, ctx->dbg_grad, grad_doubles * sizeof(double))) != SPHDVR_OK) return s;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaMemcpy(ctx->dbg_pix.p, pix, n_pix * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_err(ctx, e, "debug upload");
  RenderArgs a;
  a.n_dbg = n_pix;
  a.dbg_pix = (const int*)ctx->dbg_pix.p;
  a.dbg_rgba = (float*)ctx->dbg_rgba.p;
  a.dbg_counts = (long long*)ctx->dbg_counts.p;
  a.dbg_cands = cand_ids ? (long long*)ctx->dbg_cands.p : nullptr;
  a.cand_cap = cand_ids ? cand_cap : 0;
  a.dbg_field = field ? (double*)ctx->dbg_field.p : nullptr;
  a.field_cap = (field || grad) ? field_cap : 0;
  a.dbg_grad = grad ? (double*)ctx->dbg_grad.p : nullptr;
  if (grad && !field) {  // the kernel writes gradient rows beside field rows
    if ((s = ensure(ctx, ctx->dbg_field, (size_t)n_pix * field_cap * (D + 3) * sizeof(double))) != SPHDVR_OK) return s;
    a.dbg_field = (double*)ctx->dbg_field.p;
  }
  s = do_render(ctx, ds, lut, cam, tf, opts, nullptr, st, &a);
  if (s != SPHDVR_OK) return s;
  if ((e = cudaMemcpy(rgba, ctx->dbg_rgba.p, n_pix * 4 * sizeof(float), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(counts, ctx->dbg_counts.p, n_pix * 8 * sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_err(ctx, e, "debug download");
  if (cand_ids &&
      (e = cudaMemcpy(cand_ids, ctx->dbg_cands.p, (size_t)n_pix * cand_cap * sizeof(int64_t), cudaMemcpyDeviceToHost)) !=
          cudaSuccess)
    return cuda_err(ctx, e, "debug download");
  if (field && (e = cudaMemcpy(field, ctx->dbg_field.p, (size_t)n_pix * field_cap * (D + 3) * sizeof(double),
                               cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_err(ctx, e, "debug download");
  if (grad && (e = cudaMemcpy(grad, ctx->dbg_grad.p, grad_doubles * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_err(ctx, e, "debug download");
  bool over = false;
  for (int i = 0; i < n_pix; ++i) {
    if (cand_ids && counts[8 * i] > cand_cap) over = true;
    if ((field || grad) && counts[8 * i + 2] > field_cap) over = true;
    if (counts[8 * i + 3]) over = true;
  }
  return over ? set_err(ctx, SPHDVR_EOVERFLOW, "debug_rays: a capacity or per-ray buffer was exceeded") : SPHDVR_OK;
}

sphdvr_status sphdvr_debug_rays(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                int n_pix, const int* pix, float* rgba, int64_t* counts, int64_t* cand_ids,
                                int cand_cap, double* field, int field_cap) {
  return debug_rays(ctx, ds, lut, cam, tf, opts, n_pix, pix, rgba, counts, cand_ids, cand_cap, field, nullptr,
                    field_cap);
}

sphdvr_status sphdvr_debug_rays_grad(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                     const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                     int n_pix, const int* pix, float* rgba, int64_t* counts, double* field,
                                     double* grad, int field_cap) {
  if (!ctx) return SPHDVR_EINVAL;
  if (!opts || !opts->shading) return set_err(ctx, SPHDVR_EINVAL, "debug_rays_grad: opts->shading must be 1");
  if (grad && field_cap < 1) return set_err(ctx, SPHDVR_EINVAL, "debug_rays: capacity < 1");
  return debug_rays(ctx, ds, lut, cam, tf, opts, n_pix, pix, rgba, counts, nullptr, 0, field, grad, field_cap);
}

}  // extern "C"
