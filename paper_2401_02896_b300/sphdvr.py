"""Python binding of libsphdvr, the B300-native per-ray higher-order SPH DVR
library (arXiv 2401.02896).

Argument marshalling only: every function calls the C-ABI entry point of the
same name in ``lib/libsphdvr.so`` (see ``include/sphdvr.h``).  Device memory
and streams may come from PyTorch (``tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``); nothing is computed here.
The library must have been built (``python -m paper_2401_02896_b300._build``);
importing the binding without it raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))  # the package directory
LIB_PATH = os.path.join(_HERE, "lib", "libsphdvr.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, EOVERFLOW, EDEVICE, ENOTFOUND = range(9)
KERNELS = {"m4": 0, "wendland_c2": 1, "wendland_c4": 2, "poly6": 3}
PRECISIONS = {"fp32_anchored": 0, "fp32_naive": 1, "fp64_naive": 2, "fp32_reinit": 3, "int64_quant": 4,
              "fp32_kahan": 5}


class SphdvrError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("sphdvr status %d (%s): %s" % (status, status_string(status), message))
        self.status = status


class Camera(ctypes.Structure):
    _fields_ = [
        ("projection", ctypes.c_int),
        ("eye", ctypes.c_double * 3),
        ("target", ctypes.c_double * 3),
        ("up", ctypes.c_double * 3),
        ("fovy_deg", ctypes.c_double),
        ("half_w", ctypes.c_double),
        ("half_h", ctypes.c_double),
        ("t_near", ctypes.c_double),
        ("width", ctypes.c_int),
        ("height", ctypes.c_int),
    ]


class Tf(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("lo", ctypes.c_double),
        ("hi", ctypes.c_double),
        ("rgba", ctypes.c_void_p),
        ("sigma_scale", ctypes.c_double),
    ]


class RenderOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("anchor_every", ctypes.c_int),
        ("ert_eps", ctypes.c_float),
        ("persistent", ctypes.c_int),
        ("window_h", ctypes.c_float),
        ("reinit_dt", ctypes.c_float),
        ("ray_capacity", ctypes.c_int),
        ("reserved", ctypes.c_int),
        ("quant_tau", ctypes.c_double),
        ("quant_sigma", ctypes.c_double),
        ("window_fill", ctypes.c_float),
        ("ctas_per_sm", ctypes.c_int),
        ("shading", ctypes.c_int),
        ("shade_ka", ctypes.c_float),
        ("shade_kd", ctypes.c_float),
        ("shade_g0", ctypes.c_float),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsphdvr.so is not built (expected at %s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    sig = {
        "sphdvr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "sphdvr_version": (ctypes.c_char_p, []),
        "sphdvr_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vp)]),
        "sphdvr_destroy": (ctypes.c_int, [vp]),
        "sphdvr_last_error": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_size_t]),
        "sphdvr_lut_build": (ctypes.c_int, [ctypes.c_int] * 4 + [vp, vp, vp]),
        "sphdvr_lut_create": (ctypes.c_int, [vp] + [ctypes.c_int] * 4 + [vp, vp, ctypes.POINTER(vp)]),
        "sphdvr_lut_free": (ctypes.c_int, [vp]),
        "sphdvr_lut_save": (ctypes.c_int, [ctypes.c_char_p] + [ctypes.c_int] * 4 + [vp, vp, vp]),
        "sphdvr_lut_read_header": (ctypes.c_int, [ctypes.c_char_p] + [ctypes.POINTER(ctypes.c_int)] * 4),
        "sphdvr_lut_read": (ctypes.c_int, [ctypes.c_char_p, vp, vp, vp]),
        "sphdvr_lut_load": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.POINTER(vp)]),
        "sphdvr_dataset_create": (ctypes.c_int, [vp, ctypes.c_int64, vp, vp, vp, vp, vp, ctypes.c_int, vp,
                                                 ctypes.POINTER(vp)]),
        "sphdvr_dataset_free": (ctypes.c_int, [vp]),
        "sphdvr_dataset_info": (ctypes.c_int, [vp, i64p]),
        "sphdvr_ctx_info": (ctypes.c_int, [vp, i64p]),
        "sphdvr_measure_fp32_peak": (ctypes.c_int, [vp, vp, ctypes.POINTER(ctypes.c_double)]),
        "sphdvr_autotune": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(Camera), ctypes.POINTER(Tf),
                                           ctypes.POINTER(RenderOpts), ctypes.c_char_p, vp, ctypes.POINTER(RenderOpts),
                                           ctypes.POINTER(ctypes.c_double)]),
        "sphdvr_render": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(Camera), ctypes.POINTER(Tf),
                                         ctypes.POINTER(RenderOpts), vp, vp]),
        "sphdvr_render_batch": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.POINTER(Camera), ctypes.POINTER(Tf),
                                               ctypes.POINTER(RenderOpts), ctypes.POINTER(vp), vp]),
        "sphdvr_frame_plan_create": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(Tf), ctypes.POINTER(RenderOpts),
                                                    ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(vp)]),
        "sphdvr_frame_plan_render": (ctypes.c_int, [vp, ctypes.POINTER(Camera), vp, vp]),
        "sphdvr_frame_plan_overflowed": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int)]),
        "sphdvr_frame_plan_destroy": (ctypes.c_int, [vp]),
        "sphdvr_render_scatter": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(Camera), ctypes.POINTER(Tf),
                                                 ctypes.POINTER(RenderOpts), vp, vp]),
        "sphdvr_render_host": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(Camera), ctypes.POINTER(Tf),
                                              ctypes.POINTER(RenderOpts), vp, vp]),
        "sphdvr_render_static_scratch": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(Camera), ctypes.POINTER(Tf),
                                                       ctypes.POINTER(RenderOpts), vp, vp]),
        "sphdvr_lut_error_measure": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                    ctypes.POINTER(ctypes.c_double)]),
        "sphdvr_quant_error": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.POINTER(ctypes.c_double)]),
        "sphdvr_quant_params": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
                                + [ctypes.POINTER(ctypes.c_double)] * 3),
        "sphdvr_frame_stats": (ctypes.c_int, [vp, i64p]),
        "sphdvr_dataset_quant_params": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
                                        + [ctypes.POINTER(ctypes.c_double)] * 4),
        "sphdvr_server_create": (ctypes.c_int, [vp, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)]),
        "sphdvr_server_submit": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(Camera), ctypes.POINTER(Tf),
                                                ctypes.POINTER(RenderOpts), vp, ctypes.POINTER(ctypes.c_uint64)]),
        "sphdvr_server_wait": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_int]),
        "sphdvr_server_stats": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double)]),
        "sphdvr_server_destroy": (ctypes.c_int, [vp]),
        "sphdvr_server_set_batch": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int64]),
        "sphdvr_server_batch_stats": (ctypes.c_int, [vp, i64p]),
        "sphdvr_debug_rays": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(Camera), ctypes.POINTER(Tf),
                                             ctypes.POINTER(RenderOpts), ctypes.c_int, vp, vp, vp, vp, ctypes.c_int,
                                             vp, ctypes.c_int]),
        "sphdvr_debug_rays_grad": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(Camera), ctypes.POINTER(Tf),
                                                  ctypes.POINTER(RenderOpts), ctypes.c_int, vp, vp, vp, vp, vp,
                                                  ctypes.c_int]),
        "sphdvr_lut_build_grad": (ctypes.c_int, [ctypes.c_int] * 4 + [vp, vp, vp]),
        "sphdvr_lut_set_gradient": (ctypes.c_int, [vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def status_string(s):
    return _lib.sphdvr_status_string(int(s)).decode()


def version():
    return _lib.sphdvr_version().decode()


def last_error(ctx):
    buf = ctypes.create_string_buffer(1024)
    _lib.sphdvr_last_error(ctx, buf, 1024)
    return buf.value.decode(errors="replace")


def _check(st, ctx=None, allow=()):
    if st != OK and st not in allow:
        raise SphdvrError(st, last_error(ctx) if ctx else "")
    return st


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _kid(k):
    return KERNELS[k] if isinstance(k, str) else int(k)


# ---------------------------------------------------------------------------
# plain-data conversions (camera / TF / options dicts as produced by
# paper_2401_02896_b300.synthetic)
# ---------------------------------------------------------------------------

def camera_struct(cam):
    c = Camera()
    c.projection = 0 if cam["projection"] == "perspective" else 1
    for i in range(3):
        c.eye[i] = cam["eye"][i]
        c.target[i] = cam["target"][i]
        c.up[i] = cam["up"][i]
    c.fovy_deg = cam.get("fovy_deg", 0.0)
    c.half_w = cam.get("half_w", 0.0)
    c.half_h = cam.get("half_h", 0.0)
    c.t_near = cam.get("t_near", 0.0)
    c.width = cam["width"]
    c.height = cam["height"]
    return c


def tf_struct(tf):
    rgba = np.ascontiguousarray(tf["rgba"], dtype=np.float32)
    t = Tf()
    t.n = rgba.shape[0]
    t.lo = tf["lo"]
    t.hi = tf["hi"]
    t.rgba = rgba.ctypes.data
    t.sigma_scale = tf.get("sigma_scale", 1.0)
    t._keep = rgba  # keep the host array alive with the struct
    return t


def opts_struct(opts=None):
    o = RenderOpts()
    opts = opts or {}
    o.precision = PRECISIONS[opts.get("precision", "fp32_anchored")] if isinstance(
        opts.get("precision", "fp32_anchored"), str) else int(opts["precision"])
    o.anchor_every = int(opts.get("anchor_every", 2))
    o.ert_eps = float(opts.get("ert_eps", 1e-5))
    o.persistent = int(opts.get("persistent", 1))
    o.window_h = float(opts.get("window_h", 0.0))
    o.reinit_dt = float(opts.get("reinit_dt", 0.0))
    o.quant_tau = float(opts.get("quant_tau", 0.0))
    o.quant_sigma = float(opts.get("quant_sigma", 0.0))
    o.ray_capacity = int(opts.get("ray_capacity", 0))
    o.window_fill = float(opts.get("window_fill", 0.0))
    o.ctas_per_sm = int(opts.get("ctas_per_sm", 0))
    o.shading = int(opts.get("shading", 0))
    o.shade_ka = float(opts.get("shade_ka", 0.0))
    o.shade_kd = float(opts.get("shade_kd", 0.0))
    o.shade_g0 = float(opts.get("shade_g0", 0.0))
    return o


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------

def sphdvr_create(device=0):
    h = ctypes.c_void_p()
    st = _lib.sphdvr_create(int(device), ctypes.byref(h))
    _check(st)
    return h


def sphdvr_destroy(ctx):
    return _check(_lib.sphdvr_destroy(ctx))


def sphdvr_lut_error_measure(kernel, err):
    """Per-particle relative approximation error of a table from its per-entry errors (host)."""
    e = np.ascontiguousarray(err, dtype=np.float64)
    out = ctypes.c_double()
    _check(_lib.sphdvr_lut_error_measure(_kid(kernel), int(e.shape[0]),
                                         e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(out)))
    return out.value


def sphdvr_quant_error(kernel, D, tau, sigma):
    """Q_E(tau, sigma) of a normalised particle (Sec. 4.4)."""
    q = ctypes.c_double()
    _check(_lib.sphdvr_quant_error(_kid(kernel), int(D), float(tau), float(sigma), ctypes.byref(q)))
    return q.value


def sphdvr_quant_params(kernel, D, int_bits, variance_ratio):
    """(tau_rel, sigma_rel, Q_E): quantum values for a bit length and data variance ratio (Sec. 4.4)."""
    t, s_, q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.sphdvr_quant_params(_kid(kernel), int(D), int(int_bits), float(variance_ratio), ctypes.byref(t),
                                    ctypes.byref(s_), ctypes.byref(q)))
    return t.value, s_.value, q.value


def sphdvr_lut_build(kernel, K, D, n_lambda):
    """FP64 table of optimal approximations (host): returns (theta [n,m], pieces [n,m,D+1], err [n])."""
    m = (K + 1) // 2
    th = np.zeros((n_lambda, m))
    pc = np.zeros((n_lambda, m, D + 1))
    err = np.zeros(n_lambda)
    _check(_lib.sphdvr_lut_build(_kid(kernel), K, D, n_lambda, _p(th), _p(pc), _p(err)))
    return th, pc, err


def sphdvr_lut_create(ctx, kernel, K, D, n_lambda, theta, pieces):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    pc = np.ascontiguousarray(pieces, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(_lib.sphdvr_lut_create(ctx, _kid(kernel), K, D, n_lambda, _p(th), _p(pc), ctypes.byref(h)), ctx)
    return h


def sphdvr_lut_build_grad(kernel, K, D, n_lambda, theta):
    """FP64 gradient table on a table's knots (host): returns (gpieces [n,m,D+1], gerr [n])."""
    m = (K + 1) // 2
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.shape != (n_lambda, m):
        raise ValueError("theta must have shape (n_lambda, m)")
    gp = np.zeros((n_lambda, m, D + 1))
    ge = np.zeros(n_lambda)
    _check(_lib.sphdvr_lut_build_grad(_kid(kernel), K, D, n_lambda, _p(th), _p(gp), _p(ge)))
    return gp, ge


def sphdvr_lut_set_gradient(lut, theta, gpieces):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    gp = np.ascontiguousarray(gpieces, dtype=np.float64)
    return _check(_lib.sphdvr_lut_set_gradient(lut, _p(th), _p(gp)))


def sphdvr_lut_save(path, kernel, K, D, n_lambda, theta, pieces, err=None):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    pc = np.ascontiguousarray(pieces, dtype=np.float64)
    e = np.ascontiguousarray(err, dtype=np.float64) if err is not None else None
    _check(_lib.sphdvr_lut_save(os.fsencode(path), _kid(kernel), int(K), int(D), int(n_lambda), _p(th), _p(pc),
                                _p(e) if e is not None else None))


def sphdvr_lut_read(path):
    """(kernel id, K, D, n_lambda, theta, pieces, err) of a table file."""
    k, K, D, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib.sphdvr_lut_read_header(os.fsencode(path), ctypes.byref(k), ctypes.byref(K), ctypes.byref(D),
                                       ctypes.byref(n)))
    m = (K.value + 1) // 2
    th = np.zeros((n.value, m))
    pc = np.zeros((n.value, m, D.value + 1))
    err = np.zeros(n.value)
    _check(_lib.sphdvr_lut_read(os.fsencode(path), _p(th), _p(pc), _p(err)))
    return k.value, K.value, D.value, n.value, th, pc, err


def sphdvr_lut_load(ctx, path):
    h = ctypes.c_void_p()
    _check(_lib.sphdvr_lut_load(ctx, os.fsencode(path), ctypes.byref(h)), ctx)
    return h


def sphdvr_lut_free(lut):
    return _check(_lib.sphdvr_lut_free(lut))


def sphdvr_dataset_create(ctx, pos, h, mass=None, density=None, value=None, stream=None):
    """pos (n,3), h, mass, density, value (n,) float32: numpy arrays (host) or CUDA torch tensors (device)."""
    on_dev = hasattr(pos, "data_ptr")
    if on_dev:
        ptrs = [None if a is None else ctypes.c_void_p(a.data_ptr()) for a in (pos, h, mass, density, value)]
        keep = None
        n = pos.shape[0]
    else:
        keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (pos, h, mass, density, value)]
        ptrs = [_p(a) for a in keep]
        n = keep[0].shape[0]
    out = ctypes.c_void_p()
    st = _lib.sphdvr_dataset_create(ctx, int(n), ptrs[0], ptrs[1], ptrs[2], ptrs[3], ptrs[4], 1 if on_dev else 0,
                                    ctypes.c_void_p(stream) if stream else None, ctypes.byref(out))
    del keep
    _check(st, ctx)
    return out


def sphdvr_dataset_free(ds):
    return _check(_lib.sphdvr_dataset_free(ds))


def sphdvr_dataset_quant_params(ctx, ds, kernel, D, int_bits=64):
    """dict(tau, sigma, qe, a_max): quantum values for a resident data set (Sec. 4.4)."""
    v = [ctypes.c_double() for _ in range(4)]
    _check(_lib.sphdvr_dataset_quant_params(ctx, ds, _kid(kernel), int(D), int(int_bits), *[ctypes.byref(x) for x in v]),
           ctx)
    return dict(zip(("tau", "sigma", "qe", "a_max"), (x.value for x in v)))


def sphdvr_autotune(ctx, ds, lut, camera, tf, opts=None, cache_path=None, stream=None):
    """Tuned render options (dict) and the frame times before and after (ms)."""
    c, t, o = camera_struct(camera), tf_struct(tf), opts_struct(opts)
    out = RenderOpts()
    ms = (ctypes.c_double * 2)()
    _check(_lib.sphdvr_autotune(ctx, ds, lut, ctypes.byref(c), ctypes.byref(t), ctypes.byref(o),
                                os.fsencode(cache_path) if cache_path else None, ctypes.c_void_p(stream or 0),
                                ctypes.byref(out), ms), ctx)
    tuned = dict(opts or {})
    tuned.update(ctas_per_sm=out.ctas_per_sm, window_h=out.window_h, window_fill=out.window_fill)
    return tuned, (ms[0], ms[1])


def sphdvr_measure_fp32_peak(ctx, stream=None):
    """Measured FP32 FMA throughput of the context's device, TFLOP/s."""
    t = ctypes.c_double()
    _check(_lib.sphdvr_measure_fp32_peak(ctx, ctypes.c_void_p(stream or 0), ctypes.byref(t)), ctx)
    return t.value


def sphdvr_ctx_info(ctx):
    info = (ctypes.c_int64 * 4)()
    _check(_lib.sphdvr_ctx_info(ctx, info), ctx)
    return dict(held_bytes=int(info[0]), launches=int(info[1]), device=int(info[2]))


def sphdvr_dataset_info(ds):
    info = (ctypes.c_int64 * 8)()
    _check(_lib.sphdvr_dataset_info(ds, info))
    return dict(particles=info[0], chunks=info[1], levels=info[2], bytes=info[3])


def sphdvr_render(ctx, ds, lut, camera, tf, opts, out_ptr, stream=None, allow_overflow=False):
    """Render into a device buffer (int pointer, e.g. torch tensor .data_ptr())."""
    c, t, o = camera_struct(camera), tf_struct(tf), opts_struct(opts)
    st = _lib.sphdvr_render(ctx, ds, lut, ctypes.byref(c), ctypes.byref(t), ctypes.byref(o),
                            ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream) if stream else None)
    return _check(st, ctx, (EOVERFLOW,) if allow_overflow else ())


MAX_BATCH = 8


def sphdvr_render_batch(ctx, ds, lut, cameras, tf, opts, out_ptrs, stream=None, allow_overflow=False):
    """Render several frames (same data, table, transfer function, options) with one kernel launch."""
    n = len(cameras)
    cams = (Camera * max(n, 1))(*[camera_struct(c) for c in cameras])
    outs = (ctypes.c_void_p * max(len(out_ptrs), 1))(*[ctypes.c_void_p(p) for p in out_ptrs])
    t, o = tf_struct(tf), opts_struct(opts)
    st = _lib.sphdvr_render_batch(ctx, ds, lut, n, cams, ctypes.byref(t), ctypes.byref(o), outs,
                                  ctypes.c_void_p(stream) if stream else None)
    return _check(st, ctx, (EOVERFLOW,) if allow_overflow else ())


def sphdvr_render_scatter(ctx, ds, lut, camera, tf, opts, out_ptr, stream=None):
    """The paper's pass order: scatter knots per particle, sort per ray, accumulate and composite."""
    c, t, o = camera_struct(camera), tf_struct(tf), opts_struct(opts)
    st = _lib.sphdvr_render_scatter(ctx, ds, lut, ctypes.byref(c), ctypes.byref(t), ctypes.byref(o),
                                    ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream) if stream else None)
    return _check(st, ctx)


def sphdvr_render_static_scratch(ctx, ds, lut, camera, tf, opts, out_ptr, stream=None):
    """As sphdvr_render, with all frame scratch in the library's fixed device array (no allocation)."""
    c, t, o = camera_struct(camera), tf_struct(tf), opts_struct(opts)
    st = _lib.sphdvr_render_static_scratch(ctx, ds, lut, ctypes.byref(c), ctypes.byref(t), ctypes.byref(o),
                                           ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream) if stream else None)
    return _check(st, ctx)


def sphdvr_render_host(ctx, ds, lut, camera, tf, opts, out=None, stream=None, allow_overflow=False):
    """Render into host memory (numpy float32 (H, W, 4)); copies happen inside the call."""
    c, t, o = camera_struct(camera), tf_struct(tf), opts_struct(opts)
    if out is None:
        out = np.empty((camera["height"], camera["width"], 4), np.float32)
    st = _lib.sphdvr_render_host(ctx, ds, lut, ctypes.byref(c), ctypes.byref(t), ctypes.byref(o), _p(out),
                                 ctypes.c_void_p(stream) if stream else None)
    _check(st, ctx, (EOVERFLOW,) if allow_overflow else ())
    return out


def sphdvr_frame_stats(ctx):
    s = (ctypes.c_int64 * 16)()
    _check(_lib.sphdvr_frame_stats(ctx, s), ctx)
    keys = ["rays", "segments", "knots", "windows", "pairs", "tests", "max_table", "overflow", "ert_rays",
            "render_ns", "launches", "max_active", "capped_windows", "tangency_tests"]
    return {k: int(s[i]) for i, k in enumerate(keys)}


def sphdvr_debug_rays(ctx, ds, lut, camera, tf, opts, pixels, cand_cap=0, field_cap=0, D=None):
    """Parity hook: per listed pixel, rgba, counts (candidates, knots, field pieces, flags, tangency-band
    tests, windows, most active particles, 0), candidate ids and field pieces (FP64 rows)."""
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    n = pix.shape[0]
    rgba = np.zeros((n, 4), np.float32)
    counts = np.zeros((n, 8), np.int64)
    cands = np.full((n, cand_cap), -1, np.int64) if cand_cap else None
    if field_cap and D is None:
        raise ValueError("debug_rays needs D to size the field buffer")
    field = np.zeros((n, field_cap, D + 3)) if field_cap else None
    c, t, o = camera_struct(camera), tf_struct(tf), opts_struct(opts)
    st = _lib.sphdvr_debug_rays(ctx, ds, lut, ctypes.byref(c), ctypes.byref(t), ctypes.byref(o), n, _p(pix),
                                _p(rgba), _p(counts), _p(cands), int(cand_cap), _p(field), int(field_cap))
    _check(st, ctx, (EOVERFLOW,))
    return dict(rgba=rgba, counts=counts, cand_ids=cands, field=field, overflow=st == EOVERFLOW)


def sphdvr_debug_rays_grad(ctx, ds, lut, camera, tf, opts, pixels, field_cap, D):
    """Shaded parity hook: rgba, counts, field rows [n, field_cap, D+3] and the across-ray gradient's rows
    [n, field_cap, 3, D+1] (localized coefficients at each row's t_a)."""
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    n = pix.shape[0]
    rgba = np.zeros((n, 4), np.float32)
    counts = np.zeros((n, 8), np.int64)
    field = np.zeros((n, field_cap, D + 3))
    grad = np.zeros((n, field_cap, 3, D + 1))
    c, t, o = camera_struct(camera), tf_struct(tf), opts_struct(opts)
    st = _lib.sphdvr_debug_rays_grad(ctx, ds, lut, ctypes.byref(c), ctypes.byref(t), ctypes.byref(o), n, _p(pix),
                                     _p(rgba), _p(counts), _p(field), _p(grad), int(field_cap))
    _check(st, ctx, (EOVERFLOW,))
    return dict(rgba=rgba, counts=counts, field=field, grad=grad, overflow=st == EOVERFLOW)


class FramePlan:
    """Preallocated frame (no allocation, host synchronisation or host copy per render: capturable)."""

    def __init__(self, ctx, ds, lut, tf, opts, max_width, max_height, pair_cap):
        self.ctx = ctx
        t, o = tf_struct(tf), opts_struct(opts)
        h = ctypes.c_void_p()
        _check(_lib.sphdvr_frame_plan_create(ctx, ds, lut, ctypes.byref(t), ctypes.byref(o), int(max_width),
                                             int(max_height), int(pair_cap), ctypes.byref(h)), ctx)
        self.h = h

    def render(self, camera, out_ptr, stream=None):
        c = camera_struct(camera)
        _check(_lib.sphdvr_frame_plan_render(self.h, ctypes.byref(c), ctypes.c_void_p(out_ptr),
                                             ctypes.c_void_p(stream) if stream else None), self.ctx)

    def overflowed(self):
        v = ctypes.c_int()
        _check(_lib.sphdvr_frame_plan_overflowed(self.h, ctypes.byref(v)), self.ctx)
        return bool(v.value)

    def destroy(self):
        if self.h is not None:
            _check(_lib.sphdvr_frame_plan_destroy(self.h))
            self.h = None


class Server:
    """Frame server (continuous batching over worker streams, device-memory budget)."""

    def __init__(self, ctx, hbm_budget, max_inflight=2):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(_lib.sphdvr_server_create(ctx, int(hbm_budget), int(max_inflight), ctypes.byref(h)), ctx)
        self.h = h

    def submit(self, ds, lut, camera, tf, opts, out_ptr):
        """Queue one frame into a device buffer; returns its ticket."""
        c, t, o = camera_struct(camera), tf_struct(tf), opts_struct(opts)
        tk = ctypes.c_uint64()
        _check(_lib.sphdvr_server_submit(self.h, ds, lut, ctypes.byref(c), ctypes.byref(t), ctypes.byref(o),
                                         ctypes.c_void_p(out_ptr), ctypes.byref(tk)), self.ctx)
        return tk.value

    def wait(self, ticket, timeout_ms=-1):
        """True once the frame completed, False on timeout; raises on a failed frame."""
        st = _lib.sphdvr_server_wait(self.h, ctypes.c_uint64(ticket), int(timeout_ms))
        if st == ETIMEOUT:
            return False
        _check(st, self.ctx)
        return True

    def stats(self):
        o = (ctypes.c_double * 8)()
        _check(_lib.sphdvr_server_stats(self.h, o), self.ctx)
        keys = ["p50_ms", "p99_ms", "rays_per_s", "completed", "failed", "held_bytes", "max_ms", "queued"]
        return dict(zip(keys, list(o)))

    def set_batch(self, max_batch, max_batch_rays=512 * 512):
        """Frames and rays one render launch may take (max_batch 1 turns batching off)."""
        _check(_lib.sphdvr_server_set_batch(self.h, int(max_batch), int(max_batch_rays)), self.ctx)

    def batch_stats(self):
        o = (ctypes.c_int64 * 4)()
        _check(_lib.sphdvr_server_batch_stats(self.h, o), self.ctx)
        return dict(launches=o[0], frames=o[1], largest=o[2])

    def destroy(self):
        if self.h is not None:
            _check(_lib.sphdvr_server_destroy(self.h))
            self.h = None


def header_functions():
    """Names of the functions ``include/sphdvr.h`` declares (used by the ABI tests)."""
    import re

    root = os.path.dirname(_HERE)
    txt = open(os.path.join(root, "include", "sphdvr.h")).read()
    return sorted(set(re.findall(r"^\S.*?\b(sphdvr_[a-z_0-9]+)\(", txt, re.M)))
