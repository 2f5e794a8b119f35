"""Pins of the oracle's gradient part (the Conclusion's "gradients, analogous, as long as they are
additively generated from particle contributions") and of shaded compositing (a reading: emission
scaled by ka + kd |n . v|, a light along the viewing ray).

* w'(r)/r of every kernel equals central finite differences of w(r) divided by r;
* the perpendicular gradient's approximation G_L = w'(rho)/rho on the entry's knots is the projection of
  Sec. 3.3: exact for the poly6 kernel (G_L is a polynomial of degree 4 in s) on the exact B_L knots, and
  no worse than the field's own relative error bound class for M4;
* along a ray, F'(t) v + F_perp(t) matches the finite-difference gradient of the exact SPH sum within the
  approximation error, and F_perp is perpendicular to the ray;
* ka = 1, kd = 0 reproduces the unshaded image; a single shaded piece equals a fine midpoint sum, with and
  without the softening gradient g0; a huge g0 leaves ka times the unshaded emission.
"""
import numpy as np
import pytest

import oracle
from paper_2401_02896_b300 import synthetic as SY


@pytest.mark.parametrize("kernel", ["m4", "wendland_c2", "wendland_c4", "poly6"])
def test_kernel_derivative_matches_finite_differences(kernel):
    q = oracle.kernel_support(kernel)
    r = np.linspace(0.05, q - 0.05, 37)
    eps = 1e-6
    fd = (oracle.kernel_w(kernel, r + eps) - oracle.kernel_w(kernel, r - eps)) / (2 * eps) / r
    got = oracle.kernel_dw_r(kernel, r)
    assert np.abs(got - fd).max() <= 1e-6 * np.abs(fd).max()
    # the limit at r = 0 is the value just above it (w'(r)/r is smooth there)
    assert oracle.kernel_dw_r(kernel, 0.0) == pytest.approx(float(oracle.kernel_dw_r(kernel, 1e-7)), rel=1e-5)
    assert oracle.kernel_dw_r(kernel, q) == 0.0


def test_poly6_gradient_approximation_is_exact():
    """poly6: B_L is a polynomial of degree 6 in s on one piece (K = 1, D = 6 exact), G_L = w'/rho one of
    degree 4, so its projection on the same knots reproduces it."""
    L = oracle.lut_build("poly6", 1, 6, 65)
    G = oracle.lut_build_grad(L)
    rel = G["gerr"][:-1] / G["normG"][:-1]
    assert rel.max() < 1e-10
    # and the pieces are G itself: compare on a grid inside the support
    for j in (3, 20, 50):
        lam = L["lam"][j]
        T = np.sqrt(1 - lam ** 2)
        s = np.linspace(0, T, 17)
        exact = oracle.kernel_dw_r("poly6", np.sqrt(lam ** 2 + s ** 2))
        approx = np.polyval(G["gpieces"][j, 0][::-1], s)
        assert np.abs(approx - exact).max() <= 1e-9 * np.abs(exact).max()


def test_m4_gradient_approximation_error_is_small_and_decreases_with_degree():
    errs = []
    for D in (3, 5):
        L = oracle.lut_build("m4", 4, D, 33)
        G = oracle.lut_build_grad(L)
        errs.append(float((G["gerr"][:-1] / G["normG"][:-1]).max()))
    assert errs[0] < 2e-2 and errs[1] < errs[0], errs


def _exact_grad(P, x, kernel):
    """Finite-difference gradient of the exact SPH field sum c w(|x - chi| / h) at points x (n, 3)."""
    pos = P["pos"].astype(np.float64)
    h = P["h"].astype(np.float64)
    c = oracle.particle_amplitude(P) / h ** 3

    def f(y):
        r = np.linalg.norm(y[:, None, :] - pos[None, :, :], axis=2) / h[None, :]
        return (c[None, :] * oracle.kernel_w(kernel, r)).sum(axis=1)

    eps = 1e-6
    g = np.zeros_like(x)
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        g[:, k] = (f(x + e) - f(x - e)) / (2 * eps)
    return g


def _grad_on_ray(R, r, D, v, t):
    """F'(t) v + F_perp(t) from the oracle's field and gradient rows of ray r."""
    rows = R["field"][r, :R["stats"][r, 5]]
    grows = R["gfield"][r, :R["stats"][r, 5]]
    out = np.zeros((len(t), 3))
    for i, ti in enumerate(t):
        k = np.searchsorted(rows[:, 0], ti, side="right") - 1
        if k < 0 or ti > rows[k, 1]:
            continue
        y = ti - rows[k, 0]
        dF = sum(d * rows[k, 2 + d] * y ** (d - 1) for d in range(1, D + 1))
        gp = np.array([np.polyval(grows[k, comp][::-1], y) for comp in range(3)])
        out[i] = dF * v + gp
    return out


def test_ray_gradient_matches_finite_differences_of_the_exact_field():
    rng = np.random.default_rng(7)
    n = 40
    P = dict(pos=(0.35 + 0.3 * rng.random((n, 3))).astype(np.float32), h=np.full(n, 0.12, np.float32),
             mass=np.full(n, 1.0 / n, np.float32), density=np.ones(n, np.float32),
             value=rng.random(n).astype(np.float32))
    D = 6
    L = oracle.lut_build("m4", 4, D, 1025)
    G = oracle.lut_build_grad(L)
    cam = SY.ortho_camera_z(8, 8, lo=(0.4, 0.4), hi=(0.6, 0.6))
    tf = SY.tf_bumps()
    pix = np.array([9, 27, 36, 54], np.int32)
    R = oracle.render(P, L, cam, tf, pix, field_cap=4096, grad=G, shade=(0.3, 0.7))
    worst = 0.0
    for r, p in enumerate(pix):
        o, v = oracle.camera_ray(cam, int(p))
        rows = R["field"][r, :R["stats"][r, 5]]
        t = np.linspace(rows[0, 0], rows[-1, 1], 400)[1:-1]
        approx = _grad_on_ray(R, r, D, v, t)
        exact = _exact_grad(P, o[None, :] + t[:, None] * v[None, :], "m4")
        worst = max(worst, np.linalg.norm(approx - exact) / np.linalg.norm(exact))
        # the perpendicular part is perpendicular to the ray
        gr = R["gfield"][r, :R["stats"][r, 5]]
        dots = np.abs(np.einsum("kcd,c->kd", gr, v)).max()
        assert dots <= 1e-12 * max(1.0, np.abs(gr).max())
    assert worst < 2e-3, worst


def test_unit_shading_reproduces_the_unshaded_image_and_a_piece_matches_a_midpoint_sum():
    P = SY.uniform_cube(300, h=0.1)
    L = oracle.lut_build("m4", 4, 3, 129)
    G = oracle.lut_build_grad(L)
    cam = SY.ortho_camera_z(8, 8)
    tf = SY.tf_bumps()
    pix = np.arange(64, dtype=np.int32)
    a = oracle.render(P, L, cam, tf, pix)
    b = oracle.render(P, L, cam, tf, pix, grad=G, shade=(1.0, 0.0))
    assert np.abs(a["rgba"] - b["rgba"]).max() <= 1e-14
    # one shaded piece against a fine midpoint sum of its integrand
    F = np.array([0.9, 0.8, -1.5, 0.7])
    GP = np.array([[0.3, -0.2, 0.1, 0.0], [-0.4, 0.5, 0.2, -0.1], [0.0, 0.0, 0.0, 0.0]])
    ka, kd, yb = 0.25, 0.75, 0.9
    n = 200000
    y = (np.arange(n) + 0.5) * (yb / n)
    f = np.polyval(F[::-1], y)
    dF = np.polyval((F[1:] * np.arange(1, 4))[::-1], y)
    gp = np.stack([np.polyval(g[::-1], y) for g in GP])
    v = np.linspace(tf["lo"], tf["hi"], tf["rgba"].shape[0])
    rgba_f = np.stack([np.interp(f, v, tf["rgba"][:, k]) for k in range(4)], axis=1)
    sig = tf["sigma_scale"] * rgba_f[:, 3]
    tau = np.cumsum(sig) * (yb / n) - 0.5 * sig * (yb / n)
    for g0 in (0.0, 0.5):
        rgb, T = oracle.composite_piece_shaded(tf, F, GP, ka, kd, 0.0, yb, g0=g0)
        shade = ka + kd * np.abs(dF) / np.sqrt(dF ** 2 + (gp ** 2).sum(axis=0) + g0 ** 2)
        ref = (rgba_f[:, :3] * (sig * shade * np.exp(-tau))[:, None]).sum(axis=0) * (yb / n)
        assert np.abs(rgb - ref).max() <= 1e-6, g0
        assert T == pytest.approx(np.exp(-sig.sum() * (yb / n)), rel=1e-6)
    # a softening gradient far above |grad F| leaves the ambient part: ka times the unshaded emission
    rgb_inf, T_inf = oracle.composite_piece_shaded(tf, F, GP, ka, kd, 0.0, yb, g0=1e12)
    rgb_u, T_u = oracle.composite_piece(tf, F, 0.0, yb)
    assert np.abs(rgb_inf - ka * rgb_u).max() <= 1e-9 * np.abs(rgb_u).max() and T_inf == pytest.approx(T_u, rel=1e-12)
