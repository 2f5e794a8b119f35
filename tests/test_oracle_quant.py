"""Pins of the oracle's quantised fixed-point path (Sec. 4.2-4.4, App. A.3-A.5).

* kernel constants: kappa' of the cubic B-spline equals the closed form the
  paper prints (sqrt(14) / (7 pi)), kappa its printed value 0.352; for the
  other kernels both equal independent numerical quadratures of the paper's
  own definitions (the double integral for kappa');
* Q_E at the optimal length quantum reproduces every printed bar of the
  Sec. 5.2 figure, and sqrt(E^2 + Q_E^2) every printed combined mark;
* the optimal tau is a minimiser;
* every quantised particle is exactly compactly supported and exactly
  shifted-even (integer identities), for even and odd K;
* the quantised particle tends to the table's approximation as the quanta
  shrink, and a ray's quantised field tends to the oracle's unquantised field;
* the per-interval explicit sums equal the accumulation rule run as a
  recurrence (two computations of the same integers).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import dblquad, quad

import oracle
from oracle import quant as Q
from paper_2401_02896_b300 import synthetic as SY

from _helpers import oracle_lut

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_quant_error.json")))
GOLD_E = json.load(open(os.path.join(HERE, "golden", "paper_error_table.json")))


def test_kernel_constants_of_the_cubic_spline_match_the_paper():
    kap, kp = Q.kernel_constants("m4")
    assert abs(kp - math.sqrt(14) / (7 * math.pi)) < 1e-15
    assert abs(kap - GOLD_E["kappa"]["value"]) < 5e-4


@pytest.mark.parametrize("kernel", ["m4", "wendland_c2", "wendland_c4", "poly6"])
def test_kernel_constants_equal_numerical_quadrature_of_the_definitions(kernel):
    q = oracle.kernel_support(kernel)
    w = lambda r: oracle.kernel_w(kernel, r)  # noqa: E731  (the oracle's C kernel, not the sympy pieces)
    k2 = 4 * math.pi * quad(lambda r: (r * w(r)) ** 2, 0, q, points=[1.0] if q > 1 else None, epsabs=1e-15)[0]

    def dtw(t, s):  # t-derivative of w(sqrt(s^2 + t^2)) by a central difference
        e = 1e-5
        return (w(math.hypot(s, t + e)) - w(math.hypot(s, t - e))) / (2 * e)

    kp2 = dblquad(lambda t, s: 2 * s * dtw(t, s) ** 2, 0, q, 0, lambda s: math.sqrt(max(q * q - s * s, 0.0)),
                  epsabs=1e-10, epsrel=1e-8)[0]
    kap, kp = Q.kernel_constants(kernel)
    assert abs(kap / math.sqrt(k2) - 1) < 1e-10
    assert abs(kp / math.sqrt(kp2) - 1) < 2e-5


@pytest.mark.parametrize("D", [2, 3, 4, 5, 6])
def test_quant_error_reproduces_the_printed_bars(D):
    tau, sigma, qe = Q.quant_params(GOLD["kernel"], D, GOLD["int_bits"], GOLD["variance_ratio"])
    assert abs(qe / GOLD["QE"][str(D)] - 1) < 1e-12


def test_combined_error_reproduces_the_printed_marks():
    for key, val in GOLD["combined"].items():
        K, D = map(int, key.split(","))
        qe = Q.quant_params("m4", D, 64, 1e5)[2]
        assert abs(math.sqrt(GOLD_E["E"][key] ** 2 + qe ** 2) / val - 1) < 1e-12, key


@pytest.mark.parametrize("kernel,D", [("m4", 1), ("m4", 4), ("wendland_c2", 3), ("poly6", 6)])
def test_optimal_tau_minimises_the_estimate(kernel, D):
    sigma = 1e-9
    t = Q.optimal_tau(kernel, D, sigma)
    q0 = Q.quant_error(kernel, D, t, sigma)
    for f in (0.999, 1.001, 0.9, 1.1, 0.5, 2.0):
        assert Q.quant_error(kernel, D, t * f, sigma) > q0
    # Q_E grows with sigma at fixed tau, and at the optimum
    assert Q.quant_error(kernel, D, t, 2 * sigma) > q0
    assert Q.quant_params(kernel, D, 32, 1e5)[2] > Q.quant_params(kernel, D, 64, 1e5)[2]


def _recurrence(knots, D):
    """Eq. accumulation-rule run as a recurrence over knots sorted by position; returns the
    coefficients after each knot (exact integers)."""
    A, prev, out = [0] * (D + 1), None, []
    for t, a in knots:
        if prev is not None:
            A = Q._shift(A, t - prev)
        A = [A[d] + a[d] for d in range(D + 1)]
        prev = t
        out.append((t, list(A)))
    return out


@pytest.mark.parametrize("K,D", [(1, 2), (2, 1), (2, 3), (3, 2), (3, 3), (4, 3), (4, 4), (3, 5)])
def test_quantised_particles_are_compact_and_shifted_even(K, D):
    lut = oracle_lut("m4", K, D, 65)
    rng = np.random.default_rng(K * 10 + D)
    for _ in range(60):
        j = int(rng.integers(0, 64))
        h = float(10 ** rng.uniform(-2.5, -0.5))
        tau = h * float(10 ** rng.uniform(-4, -1.5))
        sigma = float(10 ** rng.uniform(-14, -6))
        kn = Q.quantise_particle(lut, j, float(rng.uniform(-3, 3)), h, float(10 ** rng.uniform(-1, 3)), tau, sigma)
        assert len(kn) == K + 1
        assert all(a[0] == 0 for _, a in kn)
        seq = _recurrence(sorted(kn, key=lambda x: x[0]), D)
        assert seq[-1][1] == [0] * (D + 1)  # compact support, exactly
        # shifted evenness: the accumulated polynomial just left of tbar_0 has no odd-order part
        # after the middle jump is applied (even K), resp. at tbar_0 (odd K)
        t0 = (kn[0][0] + kn[-1][0]) // 2
        left = [x for x in kn if x[0] < t0]
        A = [0] * (D + 1)
        for t, a in left:
            s = Q._shift(a, t0 - t)
            A = [A[d] + s[d] for d in range(D + 1)]
        if K % 2 == 0:
            mid = [a for t, a in kn if t == t0]
            A = [A[d] + sum(m_[d] for m_ in mid) for d in range(D + 1)]
            right_odd = [A[d] for d in range(1, D + 1, 2)]
            left_odd = [sum(Q._shift(a, t0 - t)[d] for t, a in left) for d in range(1, D + 1, 2)]
            assert right_odd == [-x for x in left_odd]
        else:
            assert all(A[d] == 0 for d in range(1, D + 1, 2))


@pytest.mark.parametrize("K,D", [(2, 3), (3, 2), (4, 3), (4, 4)])
def test_quantised_particle_tends_to_the_table_approximation(K, D):
    lut = oracle_lut("m4", K, D, 65)
    j, t_chi, h, c = 20, 0.37, 0.05, 2.0
    ts = np.linspace(t_chi - 2.1 * h, t_chi + 2.1 * h, 801)
    # the unquantised approximation c S((t - t_chi) / h) from the table's pieces
    m = (K + 1) // 2
    th = [0.0] + list(lut["theta"][j])

    def S(s):
        a = abs(s)
        for k in range(1, m + 1):
            if a <= th[k]:
                return sum(lut["pieces"][j][k - 1][d] * (a - th[k - 1]) ** d for d in range(D + 1))
        return 0.0

    ref = np.array([c * S((t - t_chi) / h) for t in ts])
    errs = []
    for scale in (1e-3, 1e-5, 1e-7):
        tau, sigma = scale * h, scale ** (D + 1) * c * 1e-3
        kn = Q.quantise_particle(lut, j, t_chi, h, c, tau, sigma)
        F = Q.int_rows_to_field(Q.particle_pieces(kn), tau, sigma)
        got = oracle.field_eval(F, ts)
        errs.append(np.abs(got - ref).max() / np.abs(ref).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5


@pytest.mark.parametrize("K,D,n_lambda", [(4, 3, 4096), (3, 2, 1025)])
def test_ray_field_recurrence_equals_explicit_sums_and_tends_to_the_unquantised_field(K, D, n_lambda):
    P = SY.uniform_cube()
    parts = dict(pos=P["pos"], h=P["h"], mass=P["mass"], value=P["value"], density=P["density"])
    lut = oracle_lut("m4", K, D, n_lambda)
    cam = SY.ortho_camera_z(32, 32)
    h_rep = float(np.median(P["h"]))
    pc_rep = float(np.median(oracle.particle_amplitude(parts) / P["h"].astype(np.float64) ** 3))
    for pix in (5 * 32 + 7, 16 * 32 + 16, 27 * 32 + 20):
        cands = Q.ray_candidates(parts, lut, cam, pix)
        assert len(cands) > 5
        R = oracle.render(parts, lut, cam, SY.tf_bumps(), np.array([pix], np.int32), field_cap=1 << 14)
        ref = R["field"][0][: int(R["stats"][0, 5])]
        ts = np.linspace(ref[0, 0], ref[-1, 1], 2001)
        fr = oracle.field_eval(ref, ts)
        prev = None
        for bits in (40, 64, 128):
            tau_rel, sig_rel, qe = Q.quant_params("m4", D, bits, 1e3)
            tau, sigma = tau_rel * h_rep, sig_rel * pc_rep
            rows = Q.quant_ray_int(lut, cands, tau, sigma)
            if bits == 64:
                # the recurrence over all knots of the ray gives the same integers at every interval start
                kn = sorted((x for tc, h, c, j in cands for x in Q.quantise_particle(lut, j, tc, h, c, tau, sigma)),
                            key=lambda x: x[0])
                rec = dict(_recurrence(kn, D))
                for a, b, A in rows:
                    assert rec[a] == A
                assert _recurrence(kn, D)[-1][1] == [0] * (D + 1)
            F = Q.int_rows_to_field(rows, tau, sigma)
            err = np.sqrt(np.mean((oracle.field_eval(F, ts) - fr) ** 2) / np.mean(fr ** 2))
            assert err < 50 * qe + 1e-12
            if prev is not None:
                assert err < prev
            prev = err
        assert prev < 1e-8
