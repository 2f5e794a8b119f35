"""ORACLE (test infrastructure, not part of the product): the quantised
fixed-point path of Sec. 4.2-4.4 and App. A.3-A.5, plain and exact.

* Kernel constants of the quantisation error estimate (App. A.4): kappa, the
  L2 norm of w over R^3, and kappa', whose defining double integral over the
  normalised distance s and the ray parameter t is taken in polar coordinates
  of the (s, t) half-plane: with s = r cos(phi), t = r sin(phi) the t-derivative
  of w(sqrt(s^2 + t^2)) is w'(r) sin(phi) and s ds dt = r^2 cos(phi) dr dphi, so
  kappa'^2 = int_0^q r^2 w'(r)^2 dr * int cos(phi) sin^2(phi) dphi
           = (2/3) int_0^q r^2 w'(r)^2 dr.
  Both integrals are evaluated exactly (sympy, polynomial pieces of w).
* Q_E(tau, sigma) (Sec. 4.4), its minimiser over tau (convex, App. A.5) and the
  quantum values for a bit length and data variance ratio (Sec. 4.4, 5.2).
* Quantised knots of one particle (Sec. 4.3, App. A.3): knot positions and
  localized difference coefficients as Python integers, with the middle knot
  (even K) or the innermost knots (odd K) set so that the particle's
  approximation is exactly shifted-even.
* The per-ray field of the quantised path as exact integers: on every interval
  between consecutive knot positions the localized coefficients are the sum,
  over the particles whose support covers the interval, of their own
  knots' difference coefficients shifted to the interval start -- the
  explicit form of the accumulation rule (Sec. 4.2), without the recurrence.
* Compositing of that field with the oracle's exact per-piece compositing.

Readings (where the paper leaves a choice):
* nearest-integer rounding rounds halves up (the paper leaves ties open);
* int_max for a bit length b is 2^(b-1);
* the "data variance ratio" of Sec. 5.2 is A_max over the representative
  particle's peak value w(0) * m v / (rho h^3): with it the printed Q_E
  values of the Sec. 5.2 figure (cubic B-spline, 64 bits, ratio 1e5) are
  reproduced to rounding (tests/test_oracle_quant.py).

Every function has a pin in tests/test_oracle_quant.py.
"""
import math
from functools import lru_cache

import numpy as np
import sympy as sp
from scipy.optimize import brentq

from .core import KERNELS, camera_ray, composite_piece, kernel_support, kernel_w, particle_amplitude, render

_r = sp.Symbol("r", nonnegative=True)


def _kid(kernel):
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def _kernel_pieces(kernel):
    """w(r) as polynomial pieces [(lo, hi, expr)] (Sec. 1 cubic B-spline; Wendland C2/C4; poly6)."""
    k, r, pi = _kid(kernel), _r, sp.pi
    R = sp.Rational
    if k == KERNELS["m4"]:
        return [(0, 1, ((2 - r) ** 3 - 4 * (1 - r) ** 3) / (4 * pi)), (1, 2, (2 - r) ** 3 / (4 * pi))]
    if k == KERNELS["wendland_c2"]:
        a = 1 - r / 2
        return [(0, 2, R(21, 16) / pi * a ** 4 * (2 * r + 1))]
    if k == KERNELS["wendland_c4"]:
        a = 1 - r / 2
        return [(0, 2, R(495, 256) / pi * a ** 6 * (R(35, 12) * r ** 2 + 3 * r + 1))]
    if k == KERNELS["poly6"]:
        return [(0, 1, R(315, 64) / pi * (1 - r ** 2) ** 3)]
    raise ValueError(kernel)


@lru_cache(maxsize=None)
def kernel_constants(kernel):
    """(kappa, kappa') of App. A.4 for the kernel, exact integrals evaluated to double."""
    k2 = sum(sp.integrate(_r ** 2 * e ** 2, (_r, lo, hi)) for lo, hi, e in _kernel_pieces(kernel))
    kp2 = sum(sp.integrate(_r ** 2 * sp.diff(e, _r) ** 2, (_r, lo, hi)) for lo, hi, e in _kernel_pieces(kernel))
    kappa = sp.sqrt(4 * sp.pi * k2)
    kappa_p = sp.sqrt(sp.Rational(2, 3) * kp2)
    return float(kappa.evalf(30)), float(kappa_p.evalf(30))


def _coef_weights(kernel, D):
    q = kernel_support(kernel)
    return [2.0 * q ** (2 * d + 3) / ((2 * d + 1) * (2 * d + 3)) for d in range(D + 1)]


def quant_error(kernel, D, tau, sigma):
    """Q_E(tau, sigma) of Sec. 4.4 for a normalised particle (unit mass, density, h, attribute)."""
    kap, kp = kernel_constants(kernel)
    c = _coef_weights(kernel, D)
    s = kp ** 2 * tau ** 2 + sum(c[d] * sigma ** 2 / tau ** (2 * d) for d in range(D + 1))
    return math.sqrt(s) / (4.0 * kap)


def optimal_tau(kernel, D, sigma):
    """The tau > 0 minimising Q_E(tau, sigma) (App. A.5): the radicand is convex in tau and its
    derivative, times tau, is increasing in log(tau); its root is bracketed and solved."""
    kap, kp = kernel_constants(kernel)
    c = _coef_weights(kernel, D)

    def g(x):  # tau * d/dtau of the radicand, tau = exp(x)
        t = math.exp(x)
        return 2 * kp ** 2 * t ** 2 - sum(2 * d * c[d] * sigma ** 2 / t ** (2 * d) for d in range(D + 1))

    lo, hi = -1.0, 1.0
    while g(lo) > 0:
        lo -= 4.0
    while g(hi) < 0:
        hi += 4.0
    return math.exp(brentq(g, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500))


def quant_params(kernel, D, int_bits, variance_ratio):
    """Relative quantum values (tau / h_rep, sigma / pc_rep) and Q_E for a bit length and a data
    variance ratio A_max / (w(0) pc_rep) (Sec. 4.4: sigma = A_max / int_max, tau minimising Q_E)."""
    int_max = 2.0 ** (int_bits - 1)
    sigma = variance_ratio * float(kernel_w(kernel, 0.0)) / int_max
    tau = optimal_tau(kernel, D, sigma)
    return tau, sigma, quant_error(kernel, D, tau, sigma)


# ---------------------------------------------------------------------------
# quantised knots (Sec. 4.3, App. A.3)
# ---------------------------------------------------------------------------

def _nearest(x):
    return int(math.floor(x + 0.5))


def _shift(a, delta):
    """Localized coefficients of sum_d a_d (t - t_a)^d re-expanded at t_a + delta (exact for ints)."""
    D = len(a) - 1
    return [sum(math.comb(d, e) * a[d] * delta ** (d - e) for d in range(e, D + 1)) for e in range(D + 1)]


def entry_jumps(lut, j):
    """Normalised localized difference coefficients of table entry j at its non-negative knots
    (Sec. 2): {k: (s_k, [s^_k0 .. s^_kD])}, k = 1..m at s_k = theta_k, and k = 0 at s = 0 for even K.
    From the table's pieces P_k(s) = sum_d p_kd (s - theta_{k-1})^d (theta_0 = 0): the jump at
    theta_k is P_{k+1} minus P_k re-expanded there (P_{m+1} = 0); the middle jump of the even
    function is 2 p_1d for odd d and 0 for even d."""
    K, D = lut["K"], lut["D"]
    m = (K + 1) // 2
    th = [0.0] + [float(x) for x in lut["theta"][j]]
    P = [[float(x) for x in lut["pieces"][j][k]] for k in range(m)]
    out = {}
    for k in range(1, m + 1):
        left = _shift(P[k - 1], th[k] - th[k - 1])
        right = P[k] if k < m else [0.0] * (D + 1)
        out[k] = (th[k], [right[d] - left[d] for d in range(D + 1)])
    if K % 2 == 0:
        out[0] = (0.0, [2.0 * P[0][d] if d % 2 == 1 else 0.0 for d in range(D + 1)])
    return out


def quantise_particle(lut, j, t_chi, h, c, tau, sigma):
    """Quantised knots [(tbar_k, [a^_k0 .. a^_kD])] for k = -m .. m (k = 0 only for even K), in
    order of k, of a particle at ray parameter t_chi with smoothing length h and amplitude
    c = m v / (rho h^3), table entry j (Sec. 4.3): tbar_0 = [t_chi / tau], tbar_{+-k} =
    tbar_0 +- [h theta_k / tau]; a^_kd = [tau^d c s^_kd / (sigma h^d)] for k >= 1 (not k = 1,
    odd d, odd K), a^_{-k,d} = (-1)^(d+1) a^_kd, a^_k0 = 0; the middle knot's odd-order
    coefficients (even K) or a^_{-1,d} for odd d in decreasing order (odd K) follow from exact
    shifted evenness."""
    K, D = lut["K"], lut["D"]
    m = (K + 1) // 2
    jumps = entry_jumps(lut, j)
    t0 = _nearest(t_chi / tau)
    tb = {0: t0}
    for k in range(1, m + 1):
        off = _nearest(h * jumps[k][0] / tau)
        tb[k] = t0 + off
        tb[-k] = 2 * t0 - tb[k]
    ah = {}
    for k in range(1, m + 1):
        s = jumps[k][1]
        ah[k] = [0] + [_nearest(tau ** d * c * s[d] / (sigma * h ** d)) for d in range(1, D + 1)]
        if K % 2 == 1 and k == 1:
            for d in range(1, D + 1, 2):
                ah[1][d] = 0  # set below from evenness
        ah[-k] = [(-1) ** (d + 1) * ah[k][d] for d in range(D + 1)]
    if K % 2 == 0:
        ah[0] = [0] * (D + 1)
        for d in range(1, D + 1, 2):
            ah[0][d] = -2 * sum(math.comb(jj, d) * ah[k][jj] * (t0 - tb[k]) ** (jj - d)
                                for k in range(-m, 0) for jj in range(d, D + 1))
    else:
        for d in sorted(range(1, D + 1, 2), reverse=True):
            v = -sum(ah[k][d] for k in range(-m, -1))
            v -= sum(math.comb(jj, d) * ah[k][jj] * (t0 - tb[k]) ** (jj - d)
                     for jj in range(d + 1, D + 1) for k in range(-m, 0))
            ah[-1][d] = v
            ah[1][d] = v  # (-1)^(d+1) = 1 for odd d
    ks = list(range(-m, m + 1)) if K % 2 == 0 else [k for k in range(-m, m + 1) if k != 0]
    return [(tb[k], ah[k]) for k in ks]


def particle_pieces(knots):
    """Exact localized coefficients of one quantised particle on each interval between its
    consecutive knots: [(tbar_a, tbar_b, [A_0 .. A_D])] (explicit sum over its preceding knots)."""
    out = []
    for i in range(len(knots) - 1):
        ta, tb_ = knots[i][0], knots[i + 1][0]
        D = len(knots[i][1]) - 1
        A = [0] * (D + 1)
        for tl, al in knots[: i + 1]:
            s = _shift(al, ta - tl)
            A = [A[e] + s[e] for e in range(D + 1)]
        out.append((ta, tb_, A))
    return out


def ray_candidates(particles, lut, camera, pixel, cand_cap=1 << 16):
    """The oracle's candidates of one ray with (t_chi, h, c, j) recomputed in FP64 (Sec. 2 pass 1)."""
    R = render(particles, lut, camera, dict(rgba=np.zeros((2, 4)), lo=0.0, hi=1.0, sigma_scale=0.0),
               np.array([pixel], dtype=np.int32), cand_cap=cand_cap)
    n = int(R["stats"][0, 0])
    ids = R["cand_ids"][0, :n]
    o, v = camera_ray(camera, int(pixel))
    q, nl = lut["q"], lut["n_lambda"]
    amp = particle_amplitude(particles)
    out = []
    for i in ids:
        p = np.asarray(particles["pos"][i], dtype=np.float64) - o
        h = float(particles["h"][i])
        tc = float(p @ v)
        d = float(np.linalg.norm(np.cross(p, v)))
        jj = min(int(math.floor(d / h * (nl - 1) / q + 0.5)), nl - 1)
        out.append((tc, h, float(amp[i]) / h ** 3, jj))
    return out


def quant_ray_int(lut, cands, tau, sigma):
    """Exact integer field of one ray: [(tbar_a, tbar_b, [A_0..A_D])] over every interval between
    consecutive distinct knot positions, A = sum over the particles covering the interval of their
    own exact coefficients there (each particle's knots from quantise_particle)."""
    parts = [quantise_particle(lut, j, tc, h, c, tau, sigma) for tc, h, c, j in cands]
    pos = sorted({t for kn in parts for t, _ in kn})
    D = lut["D"]
    rows = []
    for a, b in zip(pos[:-1], pos[1:]):
        A = [0] * (D + 1)
        for kn in parts:
            if not (kn[0][0] <= a < kn[-1][0]):
                continue
            for tl, al in kn:
                if tl > a:
                    break
                s = _shift(al, a - tl)
                A = [A[e] + s[e] for e in range(D + 1)]
        rows.append((a, b, A))
    return rows


def int_rows_to_field(rows, tau, sigma):
    """Float field rows (t_a, t_b, A_0..A_D) of integer rows: t = tbar tau, A_d = Abar_d sigma / tau^d."""
    if not rows:
        return np.zeros((0, 0))
    D = len(rows[0][2]) - 1
    out = np.zeros((len(rows), D + 3))
    for i, (a, b, A) in enumerate(rows):
        out[i, 0] = a * tau
        out[i, 1] = b * tau
        for d in range(D + 1):
            out[i, 2 + d] = float(A[d]) * (sigma / tau ** d)
    return out


def quant_render(particles, lut, camera, tf, pixels, tau, sigma, cand_cap=1 << 16):
    """Pixels of the quantised path: exact integer field per ray, composited front to back over
    [max(first knot, t_near), last knot] with the oracle's exact per-piece compositing (Sec. 1)."""
    t_near = float(camera.get("t_near", 0.0))
    rgba = np.zeros((len(pixels), 4))
    fields = []
    for r, p in enumerate(pixels):
        rows = quant_ray_int(lut, ray_candidates(particles, lut, camera, int(p), cand_cap), tau, sigma)
        F = int_rows_to_field(rows, tau, sigma)
        fields.append(F)
        rgb, T = (0.0, 0.0, 0.0), 1.0
        for row in F:
            ya = max(0.0, t_near - row[0])
            yb = row[1] - row[0]
            if yb > ya:
                rgb, T = composite_piece(tf, row[2:], ya, yb, rgb, T)
        rgba[r, :3] = rgb
        rgba[r, 3] = 1.0 - T
    return dict(rgba=rgba, field=fields)
