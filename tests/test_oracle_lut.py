"""Pins for the oracle's optimal approximations and look-up table (Sec. 3.2-3.4, Sec. 5.2).

* the printed error table E_{K,D} for the cubic B-spline (Sec. 5.2 figure),
* exactness for a kernel that is a polynomial in r^2 (poly6, D >= 6),
* the projection's residual is orthogonal to every basis function A~_kd (Sec. A.2),
* continuity, evenness and compact support of every tabulated approximation,
* local optimality of the knots, and the Cauchy-Schwarz bound on integrals.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad, simpson

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = json.load(open(os.path.join(HERE, "golden", "paper_error_table.json")))


def _kappa(k):
    q = oracle.kernel_support(k)
    pts = [1.0] if k == "m4" else None
    return math.sqrt(4 * math.pi * quad(lambda r: (r * oracle.kernel_w(k, r)) ** 2, 0, q, points=pts,
                                        epsabs=1e-16)[0])


def _E_KD(lut, kappa):
    # Sec. 5.2: E_{K,D} = (1/kappa) (2 pi int_0^q L E_L^2 dL)^(1/2)
    lam = lut["lam"]
    return math.sqrt(2 * math.pi * simpson(lam * lut["err"] ** 2, x=lam)) / kappa


@pytest.fixture(scope="module")
def kappa_m4():
    return _kappa("m4")


@pytest.mark.parametrize("key", sorted(TABLE["E"].keys()))
def test_printed_error_table(key, kappa_m4):
    K, D = map(int, key.split(","))
    # high-degree entries vary faster in L: integrate them on a finer grid
    lut = oracle.lut_build("m4", K, D, 513 if (D >= 5 and K >= 3) else 257)
    E = _E_KD(lut, kappa_m4)
    ref = TABLE["E"][key]
    # the paper's values are Riemann sums of unstated resolution; ours agree to ~2e-5 typically
    assert abs(E / ref - 1) < 1.5e-4, (K, D, E, ref)


@pytest.mark.parametrize("K", [1, 2])
def test_poly6_exact_for_degree_six(K):
    # B_L(t) = (315/64pi)(1 - L^2 - t^2)^3 is an even degree-6 polynomial on its support
    lut = oracle.lut_build("poly6", K, 6, 33)
    for j in range(32):
        lam = lut["lam"][j]
        assert lut["err"][j] <= 1e-11 * lut["normB"][j] + 1e-300
        if K == 1:
            assert abs(lut["theta"][j][0] - math.sqrt(1 - lam * lam)) < 1e-6
        ref = oracle.ray_integral("poly6", lam)
        assert abs(lut["integ"][j] - ref) <= 1e-10 * ref


def _basis(k, d, th, t):
    # A~_kd (Sec. 3.3)
    t = abs(t)
    a = th[k - 2] if k > 1 else 0.0
    b = th[k - 1]
    if t <= a:
        return 1.0
    if t >= b:
        return 0.0
    return 1.0 - ((t - a) / (b - a)) ** d


def _S(pieces, th, t):
    t = abs(t)
    lo = 0.0
    for k in range(len(th)):
        if t <= th[k]:
            return float(np.polyval(pieces[k][::-1], t - lo))
        lo = th[k]
    return 0.0


@pytest.mark.parametrize("kernel,K,D,lam,th", [
    ("m4", 4, 3, 0.37, [0.8, 1.7]),
    ("m4", 3, 4, 1.2, [0.5, 1.4]),
    ("wendland_c2", 2, 3, 0.6, [1.1]),
    ("wendland_c4", 4, 4, 1.5, [0.6, 1.2]),
    ("m4", 1, 4, 0.2, [1.6]),
])
def test_residual_orthogonal_to_basis(kernel, K, D, lam, th):
    e, pieces = oracle.fixed_knots(kernel, K, D, lam, th)
    assert e >= 0
    T = math.sqrt(oracle.kernel_support(kernel) ** 2 - lam * lam)
    B = lambda t: oracle.kernel_w(kernel, math.sqrt(lam * lam + t * t))  # noqa: E731
    pts = sorted(set([x for x in th] + ([math.sqrt(1 - lam * lam)] if kernel == "m4" and lam < 1 else [])))
    top = max(T, th[-1])
    nb = 0
    nB = math.sqrt(oracle.ray_norm2(kernel, lam))
    for k in range(1, len(th) + 1):
        for d in range(1, D + 1):
            if k == 1 and K % 2 == 1 and d % 2 == 1:
                continue
            nb += 1
            ip = 2 * quad(lambda t: (B(t) - _S(pieces, th, t)) * _basis(k, d, th, t), 0, top, points=pts,
                          epsabs=1e-15, limit=400)[0]
            assert abs(ip) < 1e-11 * nB, (k, d, ip)
    # dim S = floor(K D / 2) (Sec. 3.3)
    assert nb == (K * D) // 2
    # and the returned error is the residual norm
    r2 = 2 * quad(lambda t: (B(t) - _S(pieces, th, t)) ** 2, 0, top, points=pts, epsabs=1e-16, limit=400)[0]
    assert abs(math.sqrt(r2) - e) <= 1e-7 * nB


@pytest.mark.parametrize("kernel,K,D", [("m4", 4, 3), ("wendland_c2", 4, 3), ("m4", 3, 2), ("wendland_c4", 4, 4),
                                        ("m4", 2, 1)])
def test_table_continuity_evenness_support(kernel, K, D):
    lut = oracle.lut_build(kernel, K, D, 65)
    for j in range(64):
        th = lut["theta"][j]
        P = lut["pieces"][j]
        scale = max(1e-300, np.abs(P).max())
        lo = 0.0
        for k in range(len(th)):
            assert th[k] > lo
            end = np.polyval(P[k][::-1], th[k] - lo)
            nxt = P[k + 1][0] if k + 1 < len(th) else 0.0
            assert abs(end - nxt) <= 1e-10 * scale, (j, k)
            lo = th[k]
        if K % 2 == 1:
            assert np.all(np.abs(P[0][1::2]) <= 1e-12 * scale)
    # last entry: L = q, zero function with all knots at 0
    assert np.all(lut["theta"][-1] == 0) and np.all(lut["pieces"][-1] == 0)


@pytest.mark.parametrize("kernel,K,D", [("m4", 4, 3), ("wendland_c2", 4, 3), ("m4", 2, 2)])
def test_knots_locally_optimal(kernel, K, D):
    lut = oracle.lut_build(kernel, K, D, 17)
    rng = np.random.default_rng(7)
    for j in [1, 4, 8, 12, 15]:
        th = lut["theta"][j]
        e0 = lut["err"][j]
        for _ in range(6):
            d = rng.normal(size=th.shape)
            d *= 2e-3 / np.linalg.norm(d)
            e1, _p = oracle.fixed_knots(kernel, K, D, lut["lam"][j], th + d)
            assert e1 >= e0 * (1 - 1e-10), (j, e0, e1)


@pytest.mark.parametrize("kernel", ["m4", "wendland_c2", "wendland_c4"])
def test_integral_cauchy_schwarz_bound(kernel):
    lut = oracle.lut_build(kernel, 4, 3, 33)
    q = oracle.kernel_support(kernel)
    for j in range(32):
        lam = lut["lam"][j]
        IB = oracle.ray_integral(kernel, lam)
        T = math.sqrt(q * q - lam * lam)
        supp = 2 * max(T, lut["theta"][j][-1])
        assert abs(lut["integ"][j] - IB) <= math.sqrt(supp) * lut["err"][j] * (1 + 1e-9) + 1e-15
