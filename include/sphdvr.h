/*
 * sphdvr -- per-ray higher-order SPH field reconstruction and direct volume
 * rendering on one NVIDIA B300 (sm_103a), after arXiv 2401.02896
 * ("Particle-Wise Higher-Order SPH Field Approximation for DVR").
 *
 * C ABI.  Every call returns an sphdvr_status and never throws.  Objects are
 * opaque and owned by the library until their _free/_destroy call.  Output
 * buffers are owned by the caller.  Pointers documented as "device" must be
 * CUDA device pointers on the context's device; "host" pointers are ordinary
 * host memory (pinned memory makes the copies faster but is not required).
 * Calls on one context are not thread-safe; use one context per host thread.
 * Frames rendered through one context share its work buffers: on one stream
 * they are ordered; on different streams they must not overlap in time (use
 * a context per stream, as the frame server's workers do).
 *
 * Method (paper sections):
 *   Sec. 1     SPH field f(x) = sum_i a_i / l_i^3 w(|x - chi_i| / l_i), with
 *              a_i = mass_i * value_i / density_i and l_i the smoothing length;
 *              kernel w with compact support [0, q).
 *   Sec. 3.1   on a ray x(t) = o + t v a particle contributes
 *              a_i / l_i^3 B_L((t - t_chi) / l_i), B_L(s) = w(sqrt(L^2 + s^2)),
 *              L = dist(chi_i, ray) / l_i; B_L is replaced by its optimal even
 *              piecewise polynomial S_L (K pieces, degree <= D) taken from a
 *              look-up table over equidistant L (nearest entry).
 *   Sec. 2     each S_L is stored as knots with localized difference
 *              coefficients; summing all particles amounts to sorting their
 *              knots and running the coefficient-update recurrence (eq.
 *              Piecewise-Coefficients-Update).
 *   Sec. 1/2   the resulting piecewise polynomial of the field is classified by
 *              a transfer function and composited front to back.
 */
#ifndef SPHDVR_H
#define SPHDVR_H

#include <stddef.h>
#include <stdint.h>

/* Most frames one sphdvr_render_batch call (or one server launch) renders. */
#define SPHDVR_MAX_BATCH 8

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPHDVR_OK = 0,
  SPHDVR_EINVAL = 1,    /* invalid argument (null pointer, bad size, NaN, h <= 0, ...) */
  SPHDVR_ENOMEM = 2,    /* a device or host allocation failed */
  SPHDVR_ECUDA = 3,     /* a CUDA runtime call failed; see sphdvr_last_error */
  SPHDVR_ETIMEOUT = 4,  /* a bounded wait ran out (serving) */
  SPHDVR_EBUSY = 5,     /* a request can never fit the server's memory budget */
  SPHDVR_EOVERFLOW = 6, /* a fixed-capacity buffer was too small; results are incomplete */
  SPHDVR_EDEVICE = 7,   /* no usable CUDA device, or not a compute capability 10.3 device */
  SPHDVR_ENOTFOUND = 8  /* unknown ticket or object */
} sphdvr_status;

typedef enum {
  SPHDVR_KERNEL_M4 = 0,          /* cubic B-spline, Sec. 1 eq. (cubic-kernel), q = 2 */
  SPHDVR_KERNEL_WENDLAND_C2 = 1, /* (21/16pi)(1-r/2)^4(2r+1), q = 2 */
  SPHDVR_KERNEL_WENDLAND_C4 = 2, /* (495/256pi)(1-r/2)^6(35r^2/12+3r+1), q = 2 */
  SPHDVR_KERNEL_POLY6 = 3        /* (315/64pi)(1-r^2)^3, q = 1 (test kernel) */
} sphdvr_kernel;

typedef enum {
  /* FP32 knots, difference coefficients and compositing; the recurrence of
   * Sec. 2 runs inside windows of sorted knots and every `anchor_every`-th
   * window re-starts from the exact sum of the active particles' own pieces. */
  SPHDVR_PREC_FP32_ANCHORED = 0,
  /* FP32 recurrence run front to back along the whole ray with no re-start:
   * the paper's plain scheme, which exhibits the drift of Sec. 4.1. */
  SPHDVR_PREC_FP32_NAIVE = 1,
  /* as NAIVE, but the recurrence's running coefficients are FP64. */
  SPHDVR_PREC_FP64_NAIVE = 2,
  /* FP32 recurrence run front to back with reinitialisation knots at
   * t = j * reinit_dt (j integer) on every ray: there the running
   * coefficients are replaced by the exact sum of the active particles' own
   * pieces -- the paper's first mitigation of the drift (Sec. 4.1). */
  SPHDVR_PREC_FP32_REINIT = 3,
  /* the quantised fixed-point path (Sec. 4.2-4.4): knot positions are
   * integer multiples of quant_tau, difference coefficients of order d
   * integer multiples of quant_sigma / quant_tau^d (rounded as Sec. 4.3
   * prescribes, with each particle's approximation exactly compactly
   * supported and shifted-even), and the coefficient update is exact
   * 64-bit integer arithmetic -- no drift, no re-anchoring; the error is the
   * quantisation error of Sec. 4.4 (sphdvr_quant_params gives quanta and
   * estimate).  quant_sigma must bound the field as Sec. 4.4 prescribes
   * (A_max / 2^63) so that every coefficient fits 64 bits; compositing is
   * FP32 as in the other modes. */
  SPHDVR_PREC_INT64_QUANT = 4,
  /* as FP32_NAIVE, with compensated running sums: every addition of
   * difference coefficients to the running coefficients, and of one lane's
   * prefix to the next, keeps its rounding error (TwoSum) in a second set of
   * coefficients that is Taylor-shifted alongside; the field is the sum of
   * both.  The shifts themselves and the FP32 difference coefficients are not
   * compensated: a particle's FP32 difference coefficients do not sum to zero,
   * and that residue of Sec. 4.1's drift remains. */
  SPHDVR_PREC_FP32_KAHAN = 5
} sphdvr_precision;

/* Viewing rays.  Basis: f = normalize(target - eye), r = normalize(f x up),
 * u = r x f.  Pixel (px, py), row 0 on top, index p = py * width + px:
 *   sx = 2 (px + 0.5) / width - 1,  sy = 1 - 2 (py + 0.5) / height.
 * Perspective: o = eye, v = normalize(f + sx tan(fovy/2) width/height r
 *                                       + sy tan(fovy/2) u).
 * Orthographic: o = eye + sx half_w r + sy half_h u, v = f.
 * The ray is x(t) = o + t v for t >= t_near. */
typedef struct {
  int projection; /* 0 perspective, 1 orthographic */
  double eye[3];
  double target[3];
  double up[3];
  double fovy_deg; /* perspective: full vertical field of view in degrees */
  double half_w;   /* orthographic: half width of the view rectangle */
  double half_h;   /* orthographic: half height */
  double t_near;
  int width;
  int height;
} sphdvr_camera;

/* Piecewise-linear RGBA transfer function (classification, Sec. 1).
 * Node i sits at value lo + i (hi - lo)/(n - 1); values outside [lo, hi]
 * clamp to the end nodes.  RGB is the emitted colour in [0,1]; the
 * extinction coefficient per unit length is sigma(f) = sigma_scale * A(f). */
typedef struct {
  int n;             /* 2 <= n <= 4096 */
  double lo, hi;     /* lo < hi */
  const float* rgba; /* host pointer, n*4 floats */
  double sigma_scale;
} sphdvr_tf;

/* Compositing (emission-absorption, front to back, black transparent
 * background), over [max(first knot, t_near), last knot] of the ray:
 *   RGB = int c(F(t)) sigma(F(t)) exp(-int_t0^t sigma(F)) dt,
 *   A   = 1 - exp(-int sigma(F) dt),
 * written as premultiplied float RGBA, 4 floats per pixel, row-major. */
typedef struct {
  int precision;     /* sphdvr_precision */
  int anchor_every;  /* FP32_ANCHORED: re-anchor every n-th window (>= 1) */
  float ert_eps;     /* stop a ray once its transmittance drops below this; 0 = never */
  int persistent;    /* 1: render warps pull rays from a device work queue; 0: static stride */
  float window_h;    /* a window of knots spans at most window_h times the smallest
                        smoothing length among the ray's pending particles (> 0);
                        0 selects the default 1.0 */
  float reinit_dt;   /* FP32_REINIT: spacing of the reinitialisation knots along t (> 0); else 0 */
  int ray_capacity;  /* FP32_ANCHORED / FP32_NAIVE: particles a ray may hold waiting and
                        active in the frame pass; 0 selects 4096, else in [64, 4096].  A
                        ray that needs more is abandoned by the frame pass and rendered
                        again by a fallback pass with 16384 of each (same image); only a
                        ray beyond that too, or beyond the fallback's list of 65,536 rays
                        per frame, is wrong (left unwritten when the list is full), and
                        sets frame flag bit 5.  Smaller values exist to exercise the
                        fallback. */
  int reserved;      /* must be 0 */
  double quant_tau;   /* INT64_QUANT: length quantum (ray-parameter units, > 0) */
  double quant_sigma; /* INT64_QUANT: field value quantum (> 0) */
  float window_fill;  /* FP32_ANCHORED / FP32_NAIVE: a window also ends where the knot density
                         of the previous window puts window_fill times its capacity of knots
                         (0 selects 0.85; values >= 1 turn the rule off) */
  int ctas_per_sm;    /* render-grid CTAs per SM (0: as many as fit; else 1 .. that) */
  int shading;        /* 1: shaded rendering -- the emission of every point is scaled by
                           ka + kd |dF/dt| / sqrt(|grad F|^2 + g0^2): the cosine between the
                           field's gradient and the ray (a light at the eye), softened where the
                           gradient is small against g0 (there the shading tends to ka, and the
                           rounding noise of a vanishing gradient changes nothing).  The
                           gradient is reconstructed along the ray like the field (see
                           sphdvr_lut_set_gradient), which the table must carry.  FP32_ANCHORED
                           / FP32_NAIVE, through sphdvr_render and sphdvr_debug_rays only.
                           0: off (the shade_* fields are ignored) */
  float shade_ka;     /* shading: ambient weight, finite and >= 0 */
  float shade_kd;     /* shading: diffuse weight, finite and >= 0 */
  float shade_g0;     /* shading: softening gradient magnitude g0 (field units per length),
                         finite and >= 0; 0 gives the plain cosine, which is ill-conditioned
                         where the gradient vanishes */
} sphdvr_render_opts;

typedef struct sphdvr_ctx sphdvr_ctx;
typedef struct sphdvr_lut sphdvr_lut;
typedef struct sphdvr_dataset sphdvr_dataset;

/* Human-readable name of a status code (static storage). */
const char* sphdvr_status_string(int status);

/* Library build string (static storage). */
const char* sphdvr_version(void);

/* Create a context on CUDA device `device`.  EDEVICE if the device does not
 * exist or is not compute capability 10.3. */
sphdvr_status sphdvr_create(int device, sphdvr_ctx** out);
sphdvr_status sphdvr_destroy(sphdvr_ctx* ctx);

/* Copy the context's last error message (NUL-terminated, truncated to len). */
sphdvr_status sphdvr_last_error(const sphdvr_ctx* ctx, char* buf, size_t len);

/* ---------------------------------------------------------------------------
 * Look-up table (Sec. 3.1-3.4): for L_j = j q / (n_lambda - 1),
 * j = 0..n_lambda-1, the optimal approximation S_{L_j} of B_{L_j}.  m =
 * ceil(K/2) positive knots theta_1 < ... < theta_m (plus a middle knot at 0
 * when K is even); on [theta_{k-1}, theta_k] (theta_0 = 0) S(s) equals
 *   P_k(s) = sum_d pieces[j][k-1][d] (s - theta_{k-1})^d,  S(-s) = S(s),
 * and S = 0 for |s| >= theta_m.  The last entry (L = q) is the zero function
 * with all knots at 0.
 * ------------------------------------------------------------------------- */

/* Compute the table on the host in FP64 (CPU threads).  K in [1,4], D in
 * [1,6], n_lambda in [2, 65536].  Host outputs, caller-allocated:
 *   theta [n_lambda * m], pieces [n_lambda * m * (D+1)], err [n_lambda]
 *   (err = ||S_L - B_L||_2, may be NULL).  EINVAL on bad arguments. */
sphdvr_status sphdvr_lut_build(int kernel, int K, int D, int n_lambda, double* theta, double* pieces, double* err);

/* Per-particle relative approximation error E of a table, from its per-entry
 * errors err[j] = ||S_{L_j} - B_{L_j}||_2 (host array, n_lambda >= 3 entries on
 * the uniform grid above, e.g. from sphdvr_lut_build): the error along the rays
 * of one direction integrated over all of them and divided by the L2 norm of a
 * normalised particle's contribution -- the approximation part of the paper's
 * combined accuracy measure (Sec. "Combined Accuracy Measure"; its
 * quantisation part is zero on this library's floating-point path).  A
 * readout for users choosing (kernel, K, D), e.g. M4 with K = 4, D = 3 gives
 * about 9.3e-4.  EINVAL on a bad kernel, n_lambda < 3, NULL pointers or
 * negative / non-finite errors. */
sphdvr_status sphdvr_lut_error_measure(int kernel, int n_lambda, const double* err, double* E);

/* Quantisation error estimate Q_E(tau, sigma) of Sec. 4.4 (derivation App. A.4)
 * for a normalised particle (unit mass, density, smoothing length and
 * attribute): the expected relative L2 error from rounding knot positions to
 * multiples of the length quantum `tau` (> 0) and difference coefficients of
 * order d to multiples of sigma / tau^d (`sigma` >= 0), for degree D (0..16).
 * For a particle with smoothing length h and m v / (rho h^3) = pc, pass
 * tau / h and sigma / pc.  EINVAL on a bad kernel, D or quantum. */
sphdvr_status sphdvr_quant_error(int kernel, int D, double tau, double sigma, double* qe);

/* Quantum values of Sec. 4.4 for an integer bit length `int_bits` (8..1024;
 * int_max = 2^(int_bits-1)) and a data variance ratio A_max / (w(0) pc_rep)
 * (> 0; A_max bounds the field, w(0) pc_rep is the representative particle's
 * peak value): sigma_rel = ratio * w(0) / int_max and the length quantum
 * tau_rel minimising Q_E(tau_rel, sigma_rel) (Q_E is convex in tau), both
 * relative to the representative particle (multiply by pc_rep and h_rep), and
 * that Q_E.  The combined per-particle error of Sec. 5.2 is sqrt(E^2 + qe^2)
 * with E from sphdvr_lut_error_measure; e.g. M4, 64 bits, ratio 1e5, D = 3
 * gives qe = 8.56e-5, and with K = 4 a combined 9.29e-4.  EINVAL on bad
 * arguments. */
sphdvr_status sphdvr_quant_params(int kernel, int D, int int_bits, double variance_ratio, double* tau_rel,
                                  double* sigma_rel, double* qe);

/* Quantum values for a resident data set (Sec. 4.4's "short analysis of the
 * data set"): a_max, a rigorous upper bound of |field| (every particle's peak
 * |c| w(0), c = m v / (rho h^3), summed over the cells its support meets of a
 * grid of cells about q times the median h wide (at most 128 per axis); the
 * largest sum, plus 1 %), sigma = a_max / 2^(int_bits-1),
 * and tau minimising Q_E for the representative particle (median h, median
 * c), with that Q_E.  One tau serves every particle: particles far smaller
 * than the median get coarse knots, and where h << tau the local
 * coefficients may not fit int_bits (data with h over decades).  Copies the
 * data set's particles to the host once (synchronising).  EINVAL on bad
 * arguments or an empty data set. */
sphdvr_status sphdvr_dataset_quant_params(sphdvr_ctx* ctx, const sphdvr_dataset* ds, int kernel, int D, int int_bits,
                                          double* tau, double* sigma, double* qe, double* a_max);

/* Upload a table (host arrays in the layout above, e.g. from
 * sphdvr_lut_build) to the context's device as FP32 knots, difference
 * coefficients (Sec. 2) and pieces.  The library keeps no reference to the
 * host arrays. */
sphdvr_status sphdvr_lut_create(sphdvr_ctx* ctx, int kernel, int K, int D, int n_lambda, const double* theta,
                                const double* pieces, sphdvr_lut** out);
sphdvr_status sphdvr_lut_free(sphdvr_lut* lut);

/* Gradient table (the Conclusion: quantities generated additively from the
 * particles' contributions, gradients among them, are approximated the same
 * way as the field).  A particle's field contribution c w(|x - chi| / h) has
 * the gradient c (x - chi) w'(r) / (r h^2): its part across a ray is, at ray
 * parameter s from the closest point, (closest point - chi) c / h^2 times
 * G_L(s) = w'(rho) / rho with rho = sqrt(L^2 + s^2) (along the ray it is the
 * derivative of the field piece itself).  For every entry j of a table with
 * knots theta (layout of sphdvr_lut_build) this computes in FP64 the optimal
 * even piecewise polynomial approximation of G_{L_j} on the entry's OWN
 * knots (the projection of Sec. 3.3 with G in place of B): gpieces in the
 * layout of `pieces`, [n_lambda * m * (D+1)], and gerr[j] its L2 error (gerr
 * may be NULL).  Host arrays, caller-allocated.  EINVAL on bad arguments. */
sphdvr_status sphdvr_lut_build_grad(int kernel, int K, int D, int n_lambda, const double* theta, double* gpieces,
                                    double* gerr);

/* Attach a gradient table (from sphdvr_lut_build_grad with this table's
 * knots) to a device table, replacing any earlier one; shaded rendering needs
 * it.  `theta` must be the knots the table was created with (compared in
 * FP32; EINVAL otherwise).  Host arrays; synchronous upload. */
sphdvr_status sphdvr_lut_set_gradient(sphdvr_lut* lut, const double* theta, const double* gpieces);

/* Table files (the table is built once, offline, Sec. 3.1).  Layout, little
 * endian: 8 bytes "SPHDVRLT", uint32 version 1, int32 kernel, K, D, n_lambda,
 * int32 0, float64 q, then float64 theta[n_lambda][m], pieces[n_lambda][m][D+1] and
 * err[n_lambda] in the layouts of sphdvr_lut_build (m = ceil(K/2)).
 * sphdvr_lut_save writes one (err may be NULL: zeros); sphdvr_lut_read_header
 * reads kernel, K, D and n_lambda; sphdvr_lut_read fills caller arrays of
 * those sizes (err may be NULL); sphdvr_lut_load reads a file and makes it a
 * device table as sphdvr_lut_create does.  ENOTFOUND if the file cannot be
 * opened, EINVAL for a short or malformed file or bad arguments. */
sphdvr_status sphdvr_lut_save(const char* path, int kernel, int K, int D, int n_lambda, const double* theta,
                              const double* pieces, const double* err);
sphdvr_status sphdvr_lut_read_header(const char* path, int* kernel, int* K, int* D, int* n_lambda);
sphdvr_status sphdvr_lut_read(const char* path, double* theta, double* pieces, double* err);
sphdvr_status sphdvr_lut_load(sphdvr_ctx* ctx, const char* path, sphdvr_lut** out);

/* ---------------------------------------------------------------------------
 * Particle data sets, resident on the device.
 * ------------------------------------------------------------------------- */

/* Copy n particles into the library and build the acceleration structure:
 * particles are grouped in h-levels (factor 2 in smoothing length), sorted in
 * Morton order within a level and cut into chunks of at most 32 particles,
 * each chunk with its tight bounding box and maximum smoothing length.
 * Inputs (all FP32, n entries; pos is n*3 xyz): host pointers, or device
 * pointers when inputs_on_device != 0.  mass, density may be NULL (then 1).
 * value may be NULL (then 1).  EINVAL when n < 1, a pointer is NULL, or any
 * h is not finite and > 0 or any position is not finite.  `stream` is a
 * cudaStream_t (NULL = legacy default stream); the call returns after the
 * build has completed.  The caller keeps ownership of the inputs. */
sphdvr_status sphdvr_dataset_create(sphdvr_ctx* ctx, int64_t n, const float* pos, const float* h, const float* mass,
                                    const float* density, const float* value, int inputs_on_device, void* stream,
                                    sphdvr_dataset** out);
sphdvr_status sphdvr_dataset_free(sphdvr_dataset* ds);

/* info[0] particles, [1] chunks, [2] h-levels, [3] device bytes held,
 * [4..7] 0. */
sphdvr_status sphdvr_dataset_info(const sphdvr_dataset* ds, int64_t info[8]);

/* Context figures: info[0] device bytes the context holds in its grow-only
 * frame buffers (binning, per-ray scratch, counters, debug buffers; data sets
 * and tables are counted by their own objects), info[1] kernel launches so
 * far, info[2] device ordinal, info[3] 0. */
sphdvr_status sphdvr_ctx_info(const sphdvr_ctx* ctx, int64_t info[4]);

/* ---------------------------------------------------------------------------
 * Rendering.
 * ------------------------------------------------------------------------- */

/* Render one frame into `rgba_out` (DEVICE pointer, width*height*4 floats,
 * caller-owned), enqueued on `stream` (cudaStream_t, NULL = legacy default).
 * The call returns when the frame has been enqueued and its work buffers
 * are in place; it synchronises the stream only to size those buffers.
 * `opts` may be NULL (defaults: FP32_ANCHORED, anchor_every 2, ert_eps 1e-5,
 * work queue).  The kernel w (and its support q) is the one the table
 * was built for.  Returns EOVERFLOW
 * (image still written, possibly wrong) if a per-ray buffer overflowed. */
sphdvr_status sphdvr_render(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                            const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                            float* rgba_out, void* stream);

/* As sphdvr_render, but `rgba_host` is a HOST pointer: the call renders into
 * a library-owned device buffer, copies the image to the host and returns
 * after the copy has completed (end-to-end form). */
sphdvr_status sphdvr_render_host(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                 const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                 float* rgba_host, void* stream);

/* Render `n_frames` (1..SPHDVR_MAX_BATCH) frames of the same data set with
 * the same table, transfer function and options in ONE launch of the render
 * kernel (no counterpart in the paper: a serving service).  cams[f] is frame
 * f's camera (sizes may differ); rgba_out[f] its DEVICE image (width*height*4
 * floats, caller-owned).  Each frame is binned as in sphdvr_render; the
 * kernel's warps then take rays from one work queue that runs through all
 * frames in order, so the long rays at the end of one frame overlap with
 * the next frame's rays instead of leaving SMs idle.  Images equal those of
 * n separate sphdvr_render calls.  Enqueued on `stream`; the call
 * synchronises the stream once per frame to size its pair buffers.  Frame
 * statistics (sphdvr_frame_stats) are summed over the batch.  EINVAL for
 * n_frames out of range or a NULL pointer, before any work is enqueued. */
sphdvr_status sphdvr_render_batch(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut, int n_frames,
                                  const sphdvr_camera* cams, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                  float* const* rgba_out, void* stream);

/* The pass order the paper states (Sec. 2, "Method Overview"), as an
 * alternative to sphdvr_render's ray gathering: (1) every particle computes
 * its knots on every ray it meets and scatters them into one frame-wide list,
 * (2) the list is sorted by (ray, position), (3) every ray runs the
 * coefficient update over its sorted knots and composites.  The update is the
 * plain recurrence in FP64, with each knot's difference coefficients taken in
 * FP64 as the difference of the particle's adjacent pieces, so that every
 * particle's differences cancel to FP64 rounding and the recurrence keeps no
 * FP32 residue (the drift of Sec. 4.1 stays at FP64 level).  Same arguments and image layout as sphdvr_render; opts: only
 * ert_eps is used.  The frame's knots are held at once (24 bytes each with
 * the sort's second buffer): EOVERFLOW (nothing rendered) beyond 2^31 - 1
 * knots; at most 2^29 particles. */
sphdvr_status sphdvr_render_scatter(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                    const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                    float* rgba_out, void* stream);

/* Frame plans (no counterpart in the paper: a serving service).  A plan holds
 * every device buffer of a frame of at most max_width x max_height pixels and
 * the uploaded transfer function, so that sphdvr_frame_plan_render neither
 * allocates, synchronises with the host nor copies from the host: it only
 * enqueues kernels, device copies and memsets on `stream`, and can be
 * captured into a CUDA graph (stream capture) and replayed; a replay renders
 * the captured camera into the captured image.  The chunk-tile pairs of a
 * frame go into buffers of `pair_cap` entries (the count is never read back;
 * the unused entries are sorted along, so a frame costs the sort of pair_cap
 * entries): size it from sphdvr_frame_stats()[4] of a representative frame
 * with a margin.  A frame with more pairs drops the excess (its image is then
 * wrong) and sets a flag that sphdvr_frame_plan_overflowed reads and clears
 * (synchronising).  Data set, table, options and transfer function are fixed
 * at creation; the data set and table must outlive the plan, the plan its
 * context.  Renders of one plan must not overlap (they share its buffers).
 * EINVAL for sizes out of [1, 32768], pair_cap out of [2, 2^31 - 1], a NULL
 * argument, or a camera larger than the plan. */
typedef struct sphdvr_frame_plan sphdvr_frame_plan;
sphdvr_status sphdvr_frame_plan_create(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                       const sphdvr_tf* tf, const sphdvr_render_opts* opts, int max_width,
                                       int max_height, int64_t pair_cap, sphdvr_frame_plan** plan);
sphdvr_status sphdvr_frame_plan_render(sphdvr_frame_plan* plan, const sphdvr_camera* cam, float* rgba_out,
                                       void* stream);
sphdvr_status sphdvr_frame_plan_overflowed(sphdvr_frame_plan* plan, int* overflowed);
sphdvr_status sphdvr_frame_plan_destroy(sphdvr_frame_plan* plan);

/* Allocation-free form of sphdvr_render (no counterpart in the paper: a
 * library service for callers that must not allocate device memory while
 * they render, e.g. a server whose device memory is all handed to its own
 * pool, a process at its memory limit, or a latency-bound caller that cannot
 * take the device-wide synchronisation cudaMalloc/cudaFree may bring).
 *
 * Same arguments, kernels and image as sphdvr_render; `rgba_out` is a DEVICE
 * pointer (width*height*4 floats, caller-owned).  Every scratch buffer of the
 * frame is carved from one file-scope device array of 192 MiB inside the
 * library, so the call allocates no device or host memory.  Limits (EINVAL
 * before any work is enqueued): at most 65536 tiles of 16x16 pixels (e.g.
 * 4096 x 4096) and at most 1048576 dataset chunks (sphdvr_dataset_info
 * info[1]); EOVERFLOW when the frame has more than 2097152 chunk-tile pairs
 * (nothing is rendered then).  The render grid is capped at 64 CTAs.
 *
 * The first call on a device looks up the array's device address (set-up,
 * once per device).  The call cannot be captured into a CUDA graph: it
 * synchronises `stream` once to read the frame's pair count, as
 * sphdvr_render does (callers that need graphs use the frame plans,
 * sphdvr_frame_plan_*).  All calls in the process share the one array: calls
 * that can overlap in time (different streams, threads or contexts on the
 * same device) race on it and must be ordered by the caller.  Every buffer
 * that must start at zero is cleared on the stream by the call itself.  The
 * frame's counters and flags (sphdvr_frame_stats, e.g. out[7] bit 0 for a
 * per-ray buffer that overflowed, bit 4 for quanta too fine) stay in the
 * array: sphdvr_frame_stats reads them from there, until the next call on
 * the array overwrites them. */
sphdvr_status sphdvr_render_static_scratch(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                           const sphdvr_camera* cam, const sphdvr_tf* tf,
                                           const sphdvr_render_opts* opts, float* rgba_out, void* stream);

/* Autotuner (no counterpart in the paper: a serving service).  Picks the
 * runtime parameters of the FP32 window kernel -- ctas_per_sm (render-grid
 * occupancy, 1..3), window_h (1, 1.5, 2) and window_fill (0.6, 0.85, off) --
 * for this data set, table, transfer function and camera by timing real frames
 * (CUDA events around the render kernels on `stream`, best of two after a
 * warm-up), one parameter at a time from `base` (NULL: the defaults), on the
 * camera's view at no more than 512 x 512 pixels; a change is kept only for a
 * gain above 1 %.  None of the parameters changes what is computed beyond
 * FP32 rounding (window_h <= 2 keeps the field within its tolerance).
 * *tuned gets `base` with the chosen values; ms (may be NULL) the frame times
 * before and after, in ms.  cache_path (may be NULL): a JSON-lines file keyed
 * by device name, kernel, K, D, table size, log2 of the particle, chunk and
 * pixel counts, the data set's smoothing-length levels, precision and
 * anchor_every -- a hit returns the cached choice without timing, a miss
 * appends its result.  Allocates one frame image for the duration of the call;
 * changes no device setting.  EINVAL for bad arguments or a precision other
 * than FP32_ANCHORED / FP32_NAIVE. */
sphdvr_status sphdvr_autotune(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                              const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* base,
                              const char* cache_path, void* stream, sphdvr_render_opts* tuned, double ms[2]);

/* FP32 FMA throughput of the context's device in TFLOP/s (no counterpart in
 * the paper: the roofline denominator of the render kernel, which is bound by
 * FP32/ALU issue).  Eight independent FMA chains per thread on every resident
 * thread, best of three timed launches after a warm-up (CUDA events on
 * `stream`; about 0.1 s in all).  Changes no clock or other device setting.
 * Synchronises `stream`. */
sphdvr_status sphdvr_measure_fp32_peak(sphdvr_ctx* ctx, void* stream, double* tflops);

/* Statistics of the context's last completed frame (synchronises its
 * stream): out[0] rays, [1] candidate particle-ray segments, [2] knots,
 * [3] windows, [4] chunk-tile pairs, [5] particle tests, [6] max table
 * occupancy, [7] flags (bit 0 table overflow, bit 1 window overflow, bit 3 a
 * knot arrived behind the processed part of its ray, bit 4 INT64_QUANT: a
 * particle's rounded coefficient, integer knot offset or centre beyond 2^62,
 * the quanta too fine for it -- a per-particle bound, not a proof that the
 * summed integers fit: that needs quant_sigma to bound the field; bit 6 a
 * ray of the FP64, reinitialisation or quantised modes reached 65,536 windows
 * and was ended there, its pixel wrong),
 * [8] rays stopped
 * by early termination, [9] device time of the render kernel in ns (CUDA
 * events on the render stream), [10] kernel launches of the frame,
 * [11] largest number of particles active at one point of a ray, [12] windows
 * that ended before the bound of the next chunk (window_h limit, knot density
 * or a particle starting inside them), [13] particle tests within 1e-6 h of
 * tangency (|dist(chi, ray) - q h| <= 1e-6 h: the candidate decision there
 * rests on rounding; FP32_ANCHORED / FP32_NAIVE only), [14..15] 0. */
sphdvr_status sphdvr_frame_stats(sphdvr_ctx* ctx, int64_t out[16]);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of frames (a library service; the paper
 * renders single frames).
 *
 * A server owns `max_inflight` (1..8) worker threads, each with its own CUDA
 * stream and frame buffers; submitted requests are rendered in submission
 * order by whichever worker is free, so frames overlap on the GPU.  A free
 * worker takes the oldest queued request together with later queued requests
 * of the same data set, table, transfer function and options, up to
 * max_batch frames and max_batch_rays rays in all (sphdvr_server_set_batch;
 * defaults SPHDVR_MAX_BATCH and 512*512), and renders them with one launch
 * (sphdvr_render_batch); a batch completes as a whole.  Small frames gain
 * most: their rays are too few to keep every SM busy until the frame ends.  The
 * device memory all workers hold for frame buffers stays within `hbm_budget`
 * bytes (datasets and tables are not counted: they belong to the caller's
 * context): a worker whose frame does not fit beside the others' holdings
 * frees what it holds and waits until they release enough.
 * ------------------------------------------------------------------------- */
typedef struct sphdvr_server sphdvr_server;

sphdvr_status sphdvr_server_create(sphdvr_ctx* ctx, size_t hbm_budget, int max_inflight, sphdvr_server** out);

/* Queue one frame: arguments as sphdvr_render (`rgba_out` a DEVICE pointer
 * that must stay valid, and `ds`, `lut` alive, until the request completes).
 * The camera, transfer function and options are copied.  Returns at once
 * with a ticket; SPHDVR_EBUSY if the frame's fixed buffers alone exceed the
 * budget.  A frame whose pair buffers make it exceed the budget fails later
 * with SPHDVR_EBUSY (reported by sphdvr_server_wait). */
sphdvr_status sphdvr_server_submit(sphdvr_server* srv, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                   const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                   float* rgba_out, uint64_t* ticket);

/* Wait for a ticket: returns the frame's status once it has completed (its
 * image is then in rgba_out and the ticket is retired), SPHDVR_ETIMEOUT if
 * it has not completed within timeout_ms (the ticket stays valid; a negative
 * timeout waits until completion), SPHDVR_ENOTFOUND for an unknown or
 * retired ticket. */
sphdvr_status sphdvr_server_wait(sphdvr_server* srv, uint64_t ticket, int timeout_ms);

/* out[0] p50 and out[1] p99 latency (ms, submission to completion) of the
 * completed frames, out[2] rays per second over the time from the first
 * submission to the last completion, out[3] frames completed, out[4] frames
 * failed, out[5] device bytes the workers hold, out[6] largest latency (ms),
 * out[7] frames queued and not yet started. */
sphdvr_status sphdvr_server_stats(sphdvr_server* srv, double out[8]);

/* Batch limits: at most `max_batch` frames (1..SPHDVR_MAX_BATCH; 1 turns
 * batching off) with at most `max_batch_rays` rays (width*height summed over
 * the frames; >= 0) per launch; the oldest queued request is always taken,
 * whatever its size.  Apply to batches formed after the call. */
sphdvr_status sphdvr_server_set_batch(sphdvr_server* srv, int max_batch, int64_t max_batch_rays);

/* out[0] render launches the workers made, out[1] frames those launches
 * rendered (out[1] / out[0] is the mean batch size), out[2] largest batch,
 * out[3] 0. */
sphdvr_status sphdvr_server_batch_stats(sphdvr_server* srv, int64_t out[4]);

/* Finish every queued frame, then stop the workers and free their buffers.
 * Tickets not waited for are retired. */
sphdvr_status sphdvr_server_destroy(sphdvr_server* srv);

/* Parity hook: render the listed pixels with the same kernels and return,
 * per pixel r (all HOST pointers):
 *   rgba[4r..4r+3]
 *   counts[8r..8r+7]: candidates, knots, field pieces written, flags (as in
 *     sphdvr_frame_stats out[7]), particles tested within 1e-6 h of tangency
 *     (|dist(chi, ray) - q h| <= 1e-6 h, counted and reported: their candidate
 *     decision rests on rounding), windows (FP32_ANCHORED / FP32_NAIVE; else
 *     0), most particles active at one point of the ray (idem), 0
 *   cand_ids[r*cand_cap ...]: original indices of the candidate particles
 *   field[(r*field_cap + i)*(D+3) ...]: FP64 rows (t_a, t_b, A_0..A_D), one per
 *     field piece of positive length, front to back, A the field's localized
 *     coefficients at t_a (Sec. 2) as the kernel computed them.
 * cand_ids / field may be NULL.  EOVERFLOW if a capacity was too small (the
 * first entries are still written). */
sphdvr_status sphdvr_debug_rays(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                int n_pix, const int* pix, float* rgba, int64_t* counts, int64_t* cand_ids,
                                int cand_cap, double* field, int field_cap);

/* As sphdvr_debug_rays with opts->shading = 1 (required), and beside every
 * field row i of pixel r the across-ray gradient of the field on that piece:
 *   grad[((r*field_cap + i)*3 + c)*(D+1) + d], c = x, y, z: its localized
 * coefficients at t_a (the gradient there is sum_d grad[..d] (t - t_a)^d; the
 * along-ray part is the derivative of the field row).  grad (HOST, may be NULL)
 * holds n_pix * field_cap * 3 * (D+1) doubles. */
sphdvr_status sphdvr_debug_rays_grad(sphdvr_ctx* ctx, const sphdvr_dataset* ds, const sphdvr_lut* lut,
                                     const sphdvr_camera* cam, const sphdvr_tf* tf, const sphdvr_render_opts* opts,
                                     int n_pix, const int* pix, float* rgba, int64_t* counts, double* field,
                                     double* grad, int field_cap);

#ifdef __cplusplus
}
#endif

#endif /* SPHDVR_H */
