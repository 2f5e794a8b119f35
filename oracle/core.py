"""ctypes binding of the oracle's C core (test infrastructure only).

Every function here marshals numpy arrays into ``oracle.c`` and back; the
arithmetic is in the C file, which cites the paper section of each step.
"""
import ctypes
import os

import numpy as np

from . import build as _build

KERNELS = {"m4": 0, "wendland_c2": 1, "wendland_c4": 2, "poly6": 3}

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_kernel_support.restype = ctypes.c_double
        lib.orc_kernel_support.argtypes = [ctypes.c_int]
        lib.orc_kernel_w.restype = ctypes.c_double
        lib.orc_kernel_w.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_lut_build.restype = ctypes.c_int
        lib.orc_lut_build.argtypes = [ctypes.c_int] * 4 + [dp] * 5
        lib.orc_fixed_knots.restype = ctypes.c_double
        lib.orc_fixed_knots.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        lib.orc_ray_norm2.restype = ctypes.c_double
        lib.orc_ray_norm2.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_ray_integral.restype = ctypes.c_double
        lib.orc_ray_integral.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_camera_ray.restype = None
        lib.orc_camera_ray.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp]
        lib.orc_render.restype = ctypes.c_int
        lib.orc_render.argtypes = [
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,  # n, pos, h, amp
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,  # kernel K D n_lambda
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,  # theta pieces cam
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_double,  # tf
            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,  # n_rays pix rgba stats
            ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,  # gpieces ka kd g0 gfield
        ]
        lib.orc_kernel_dw_r.restype = ctypes.c_double
        lib.orc_kernel_dw_r.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_lut_build_grad.restype = ctypes.c_int
        lib.orc_lut_build_grad.argtypes = [ctypes.c_int] * 4 + [dp] * 4
        lib.orc_composite_piece_shaded.restype = None
        lib.orc_composite_piece_shaded.argtypes = [
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_double,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
        ]
        lib.orc_composite_piece.restype = None
        lib.orc_composite_piece.argtypes = [
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_double,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
        ]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _kid(kernel):
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def num_threads():
    return _load().orc_num_threads()


def set_threads(n):
    _load().orc_set_threads(int(n))


def kernel_support(kernel):
    """q: w(r) = 0 for r >= q (units of the smoothing length)."""
    return _load().orc_kernel_support(_kid(kernel))


def kernel_w(kernel, r):
    """The SPH kernel w(r) (Sec. 1), vectorised over r."""
    lib = _load()
    k = _kid(kernel)
    r = np.asarray(r, dtype=np.float64)
    return np.vectorize(lambda x: lib.orc_kernel_w(k, float(x)))(r) if r.ndim else lib.orc_kernel_w(k, float(r))


def kernel_dw_r(kernel, r):
    """w'(r) / r of the SPH kernel (finite at r = 0), vectorised over r (gradients, oracle part 5)."""
    lib = _load()
    k = _kid(kernel)
    r = np.asarray(r, dtype=np.float64)
    return np.vectorize(lambda x: lib.orc_kernel_dw_r(k, float(x)))(r) if r.ndim else lib.orc_kernel_dw_r(k, float(r))


def lut_build_grad(lut):
    """Gradient table for a table of lut_build: per entry the optimal approximation of
    G_L(s) = w'(sqrt(L^2+s^2)) / sqrt(L^2+s^2) on the entry's own knots (the projection of Sec. 3.3).
    Returns a dict with ``gpieces`` [n][m][D+1], ``gerr`` (||S_G - G_L||) and ``normG`` (||G_L||)."""
    n, m, D = lut["n_lambda"], (lut["K"] + 1) // 2, lut["D"]
    th = np.ascontiguousarray(lut["theta"], dtype=np.float64)
    gp = np.zeros((n, m, D + 1))
    ge = np.zeros(n)
    ng = np.zeros(n)
    rc = _load().orc_lut_build_grad(lut["kernel"], lut["K"], D, n, _dptr(th), _dptr(gp), _dptr(ge), _dptr(ng))
    if rc:
        raise ValueError("orc_lut_build_grad rejected the table")
    return dict(gpieces=gp, gerr=ge, normG=ng)


def lut_build(kernel, K, D, n_lambda):
    """Look-up table of optimal approximations of B_L, L_j = j q/(n_lambda-1) (Sec. 3.1-3.4).

    Returns a dict with ``theta`` [n][m] (positive knots), ``pieces`` [n][m][D+1]
    (piece P_k expanded at th_{k-1}), ``err`` (E_L), ``normB`` (||B_L||),
    ``integ`` (int S_L dt), ``lam`` and the parameters.
    """
    m = (K + 1) // 2
    th = np.zeros((n_lambda, m))
    pc = np.zeros((n_lambda, m, D + 1))
    err = np.zeros(n_lambda)
    nb = np.zeros(n_lambda)
    ig = np.zeros(n_lambda)
    rc = _load().orc_lut_build(_kid(kernel), K, D, n_lambda, _dptr(th), _dptr(pc), _dptr(err), _dptr(nb), _dptr(ig))
    if rc:
        raise ValueError("orc_lut_build rejected (K=%d, D=%d, n=%d)" % (K, D, n_lambda))
    q = kernel_support(kernel)
    return dict(kernel=_kid(kernel), K=K, D=D, n_lambda=n_lambda, q=q, theta=th, pieces=pc, err=err, normB=nb,
                integ=ig, lam=np.arange(n_lambda) * q / (n_lambda - 1))


def fixed_knots(kernel, K, D, lam, theta):
    """Optimal approximation for GIVEN positive knots (Sec. 3.3): (E_L, pieces)."""
    m = (K + 1) // 2
    th = np.ascontiguousarray(theta, dtype=np.float64)
    pc = np.zeros((m, D + 1))
    e = _load().orc_fixed_knots(_kid(kernel), K, D, float(lam), _dptr(th), _dptr(pc))
    return e, pc


def ray_norm2(kernel, lam):
    return _load().orc_ray_norm2(_kid(kernel), float(lam))


def ray_integral(kernel, lam):
    return _load().orc_ray_integral(_kid(kernel), float(lam))


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

    @classmethod
    def from_dict(cls, d):
        c = cls()
        c.projection = 0 if d["projection"] == "perspective" else 1
        for i in range(3):
            c.eye[i] = d["eye"][i]
            c.target[i] = d["target"][i]
            c.up[i] = d["up"][i]
        c.fovy_deg = d.get("fovy_deg", 0.0)
        c.half_w = d.get("half_w", 0.0)
        c.half_h = d.get("half_h", 0.0)
        c.t_near = d.get("t_near", 0.0)
        c.width = d["width"]
        c.height = d["height"]
        return c


def camera_ray(cam, p):
    c = Camera.from_dict(cam)
    o = np.zeros(3)
    v = np.zeros(3)
    _load().orc_camera_ray(ctypes.byref(c), int(p), _dptr(o), _dptr(v))
    return o, v


def entry_knots(lut, j):
    """Sorted normalised knot offsets of table entry j (Sec. 4.3: mirrored knots + middle knot for even K)."""
    th = lut["theta"][j]
    K = lut["K"]
    s = list(-th[::-1])
    if K % 2 == 0:
        s.append(0.0)
    s += list(th)
    return np.array(s)


def particle_amplitude(particles):
    """Amplitude a_i = mass_i * value_i / density_i of every particle, FP64 (Sec. 1: a particle contributes
    mass * value / (density * h^3) * w(|x - chi| / h) to the field).  ``particles`` carries ``mass``,
    ``value`` and ``density`` (n,) arrays, each optional: a missing one counts as 1, as in the C ABI."""
    n = np.asarray(particles["h"]).shape[0]
    a = np.ones(n, dtype=np.float64)
    for key in ("mass", "value"):
        if particles.get(key) is not None:
            a = a * np.asarray(particles[key], dtype=np.float64)
    if particles.get("density") is not None:
        a = a / np.asarray(particles["density"], dtype=np.float64)
    return a


def render(particles, lut, camera, tf, pixels, cand_cap=0, field_cap=0, grad=None, shade=(1.0, 0.0)):
    """Render the listed pixels (row-major indices) by direct summation, FP64.

    ``particles``: dict with ``pos`` (n,3) float32, ``h`` (n,) float32 and the
    FP32 ``mass``, ``value``, ``density`` (n,) of the C ABI (each optional, 1
    if missing); the amplitude is ``particle_amplitude``.
    ``grad``: a gradient table of lut_build_grad, or None; with it the emission is
    shaded by ka + kd |F'| / sqrt(|grad|^2 + g0^2) (``shade`` = (ka, kd) or (ka, kd, g0); g0 = 0 is the
    cosine |n . v|) and ``gfield`` holds per field
    row the perpendicular gradient's localized coefficients [3][D+1].
    Returns dict(rgba (r,4), stats (r,8) int64, cand_ids (r,cand_cap) or None,
    field (r, field_cap, D+3) or None, gfield (r, field_cap, 3, D+1) or None, truncated bool).
    """
    lib = _load()
    pos = np.ascontiguousarray(particles["pos"], dtype=np.float32)
    hs = np.ascontiguousarray(particles["h"], dtype=np.float32)
    amp = np.ascontiguousarray(particle_amplitude(particles), dtype=np.float64)
    n = pos.shape[0]
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    nr = pix.shape[0]
    D = lut["D"]
    th = np.ascontiguousarray(lut["theta"], dtype=np.float64)
    pc = np.ascontiguousarray(lut["pieces"], dtype=np.float64)
    cam = Camera.from_dict(camera)
    rgba_tf = np.ascontiguousarray(tf["rgba"], dtype=np.float64)
    out = np.zeros((nr, 4))
    stats = np.zeros((nr, 8), dtype=np.int64)
    cids = np.full((nr, cand_cap), -1, dtype=np.int64) if cand_cap else None
    fld = np.zeros((nr, field_cap, D + 3)) if field_cap else None
    gp = np.ascontiguousarray(grad["gpieces"], dtype=np.float64) if grad is not None else None
    gfld = np.zeros((nr, field_cap, 3, D + 1)) if (field_cap and grad is not None) else None
    rc = lib.orc_render(
        n, _ptr(pos), _ptr(hs), _ptr(amp), lut["kernel"], lut["K"], D, lut["n_lambda"], _ptr(th), _ptr(pc),
        ctypes.byref(cam), int(tf["rgba"].shape[0]), float(tf["lo"]), float(tf["hi"]), _ptr(rgba_tf),
        float(tf["sigma_scale"]), nr, _ptr(pix), _ptr(out), _ptr(stats),
        _ptr(cids) if cids is not None else None, int(cand_cap), _ptr(fld) if fld is not None else None,
        int(field_cap), _ptr(gp) if gp is not None else None, float(shade[0]), float(shade[1]),
        float(shade[2]) if len(shade) > 2 else 0.0,
        _ptr(gfld) if gfld is not None else None,
    )
    return dict(rgba=out, stats=stats, cand_ids=cids, field=fld, gfield=gfld, truncated=bool(rc & 2))


def composite_piece(tf, F, ya, yb, rgb=(0.0, 0.0, 0.0), T=1.0):
    """Composite one polynomial piece F(y) on [ya, yb] (exact; Sec. 1 DVR)."""
    lib = _load()
    F = np.ascontiguousarray(F, dtype=np.float64)
    rgba_tf = np.ascontiguousarray(tf["rgba"], dtype=np.float64)
    c = np.array(rgb, dtype=np.float64)
    t = np.array([T], dtype=np.float64)
    lib.orc_composite_piece(int(rgba_tf.shape[0]), float(tf["lo"]), float(tf["hi"]), _ptr(rgba_tf),
                            float(tf["sigma_scale"]), _ptr(F), len(F) - 1, float(ya), float(yb), _ptr(c), _ptr(t))
    return c, float(t[0])


def composite_piece_shaded(tf, F, GP, ka, kd, ya, yb, rgb=(0.0, 0.0, 0.0), T=1.0, g0=0.0):
    """Composite one piece with shading ka + kd |F'| / sqrt(|grad|^2 + g0^2) (oracle part 5); GP: [3][D+1]
    perpendicular gradient."""
    lib = _load()
    F = np.ascontiguousarray(F, dtype=np.float64)
    G = np.ascontiguousarray(GP, dtype=np.float64)
    rgba_tf = np.ascontiguousarray(tf["rgba"], dtype=np.float64)
    c = np.array(rgb, dtype=np.float64)
    t = np.array([T], dtype=np.float64)
    lib.orc_composite_piece_shaded(int(rgba_tf.shape[0]), float(tf["lo"]), float(tf["hi"]), _ptr(rgba_tf),
                                   float(tf["sigma_scale"]), _ptr(F), _ptr(G), len(F) - 1, float(ka), float(kd),
                                   float(g0), float(ya), float(yb), _ptr(c), _ptr(t))
    return c, float(t[0])


def field_eval(field_rows, t):
    """Evaluate a piecewise field (rows t_a, t_b, A_0..A_D) at points t (0 outside)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    out = np.zeros_like(t)
    rows = field_rows[field_rows[:, 1] > field_rows[:, 0]]
    if rows.size == 0:
        return out
    idx = np.searchsorted(rows[:, 0], t, side="right") - 1
    ok = (idx >= 0) & (t <= rows[np.clip(idx, 0, None), 1])
    for i in np.nonzero(ok)[0]:
        r = rows[idx[i]]
        y = t[i] - r[0]
        out[i] = np.polyval(r[2:][::-1], y)
    return out


if os.environ.get("ORACLE_EAGER_BUILD"):
    _load()
