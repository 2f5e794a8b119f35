"""Pins for the oracle's kernels and ray restrictions (Sec. 1, Sec. 3.1, Sec. A.4).

Each check compares the oracle with something other than itself: the kernel's
normalisation, constants the paper prints, closed-form line integrals derived
here, and scipy's adaptive quadrature.
"""
import math

import pytest
from scipy.integrate import quad

import oracle

KERNELS = ["m4", "wendland_c2", "wendland_c4", "poly6"]


def _pts(k):
    return [1.0] if k == "m4" else None


@pytest.mark.parametrize("k", KERNELS)
def test_kernel_normalised_in_3d(k):
    q = oracle.kernel_support(k)
    v = quad(lambda r: 4 * math.pi * r * r * oracle.kernel_w(k, r), 0, q, points=_pts(k), epsabs=1e-15,
             epsrel=1e-13)[0]
    assert abs(v - 1.0) < 1e-12
    assert oracle.kernel_w(k, q) == 0.0
    assert oracle.kernel_w(k, 1.01 * q) == 0.0
    assert oracle.kernel_w(k, 0.0) > 0.0


def test_m4_matches_cubic_kernel_definition():
    # Sec. 1 eq. (cubic-kernel), written out on a few radii
    for r in [0.0, 0.3, 0.999, 1.0, 1.5, 1.999, 2.0, 3.0]:
        if r < 1:
            ref = ((2 - r) ** 3 - 4 * (1 - r) ** 3) / (4 * math.pi)
        elif r < 2:
            ref = (2 - r) ** 3 / (4 * math.pi)
        else:
            ref = 0.0
        assert abs(oracle.kernel_w("m4", r) - ref) <= 1e-16


def test_m4_kappa_printed_value():
    # Sec. A.4: kappa = (4 pi int (t w(t))^2 dt)^(1/2) "roughly 0.352"
    kap = math.sqrt(4 * math.pi * quad(lambda r: (r * oracle.kernel_w("m4", r)) ** 2, 0, 2, points=[1.0],
                                       epsabs=1e-16)[0])
    assert abs(kap - 0.352) < 5e-4


def test_m4_kappa_prime_closed_form():
    # Sec. A.4: (int_0^q L int_R (dB_L/dt)^2 dt dL)^(1/2) = sqrt(14)/(7 pi) for the cubic B-spline.
    # dB/dt = w'(r) t / r with w' by central differences of the oracle's kernel.
    def wprime(r, h=1e-6):
        return (oracle.kernel_w("m4", r + h) - oracle.kernel_w("m4", max(r - h, 0.0))) / (r + h - max(r - h, 0.0))

    def inner(lam):
        T = math.sqrt(4 - lam * lam)
        pts = [math.sqrt(1 - lam * lam)] if lam < 1 else None

        def f(t):
            r = math.sqrt(lam * lam + t * t)
            return (wprime(r) * t / r) ** 2 if r > 0 else 0.0

        return 2 * quad(f, 0, T, points=pts, epsabs=1e-13, limit=200)[0]

    val = quad(lambda lam: lam * inner(lam), 0, 2, points=[1.0], epsabs=1e-12, limit=200)[0]
    assert abs(math.sqrt(val) - math.sqrt(14) / (7 * math.pi)) < 2e-7


def _m4_line_integral_closed_form(lam):
    """int_R w(sqrt(lam^2+t^2)) dt for the cubic B-spline, from antiderivatives in t of r^0..r^3."""
    L2 = lam * lam

    def ash(t):
        return math.asinh(t / lam) if lam > 0 else 0.0

    def R(t):  # antiderivatives of r^0, r^1, r^2, r^3 with r = sqrt(lam^2 + t^2)
        r = math.sqrt(L2 + t * t)
        return (t, 0.5 * (t * r + L2 * ash(t)), L2 * t + t ** 3 / 3,
                t * (2 * t * t + 5 * L2) * r / 8 + 3 * L2 * L2 * ash(t) / 8)

    def seg(a, b, coef):
        Ra, Rb = R(a), R(b)
        return sum(c * (Rb[i] - Ra[i]) for i, c in enumerate(coef))

    if lam >= 2:
        return 0.0
    t2 = math.sqrt(4 - L2)
    total = 0.0
    if lam < 1:
        t1 = math.sqrt(1 - L2)
        total += seg(0.0, t1, (4.0, 0.0, -6.0, 3.0))  # (2-r)^3 - 4(1-r)^3 = 4 - 6 r^2 + 3 r^3
        total += seg(t1, t2, (8.0, -12.0, 6.0, -1.0))  # (2-r)^3
    else:
        total += seg(0.0, t2, (8.0, -12.0, 6.0, -1.0))
    return 2 * total / (4 * math.pi)


@pytest.mark.parametrize("lam", [0.0, 1e-3, 0.1, 0.5, 0.99, 1.0, 1.3, 1.9, 1.999])
def test_ray_integral_m4_closed_form(lam):
    ref = _m4_line_integral_closed_form(lam)
    got = oracle.ray_integral("m4", lam)
    assert abs(got - ref) <= 1e-13 * max(1.0, abs(ref))


@pytest.mark.parametrize("k", KERNELS)
@pytest.mark.parametrize("frac", [0.0, 0.2, 0.6, 0.95])
def test_ray_integral_and_norm_vs_adaptive_quadrature(k, frac):
    q = oracle.kernel_support(k)
    lam = frac * q
    T = math.sqrt(q * q - lam * lam)
    pts = [math.sqrt(1 - lam * lam)] if (k == "m4" and lam < 1) else None
    f = lambda t: oracle.kernel_w(k, math.sqrt(lam * lam + t * t))  # noqa: E731
    I = 2 * quad(f, 0, T, points=pts, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    N2 = 2 * quad(lambda t: f(t) ** 2, 0, T, points=pts, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    assert abs(oracle.ray_integral(k, lam) - I) <= 1e-12 * I
    assert abs(oracle.ray_norm2(k, lam) - N2) <= 1e-12 * N2


@pytest.mark.parametrize("k", KERNELS)
def test_line_integrals_integrate_to_one(k):
    # 2 pi int_0^q L (int_R B_L dt) dL = int_{R^3} w dV = 1
    q = oracle.kernel_support(k)
    v = quad(lambda lam: 2 * math.pi * lam * oracle.ray_integral(k, lam), 0, q, points=_pts(k), epsabs=1e-13,
             limit=200)[0]
    assert abs(v - 1.0) < 1e-10
