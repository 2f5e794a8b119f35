"""Shaded rendering on the GPU against the oracle: the across-ray gradient reconstructed along every ray from
the particles' gradient contributions (the Conclusion: features generated additively from the particle
contributions, gradients among them, are approximated like the field), and emission shaded by
ka + kd |dF/dt| / sqrt(|grad F|^2 + g0^2) (a light at the eye, the cosine softened where the gradient is
small against g0; a reading).  g0 here is 1e-3 of the RMS across-ray gradient on the oracle's rays: above the
FP32 noise of a vanishing gradient, far below the gradients that shape the image.

* the field rows of the shaded kernel equal the oracle's within the field tolerance (the extra channels
  change nothing of the field);
* the gradient rows (localized coefficients of the three components) equal the oracle's: relative L2 of the
  vector over each ray within GRAD_REL_L2 (the sum cancels between particles on opposite sides of the ray:
  its FP32 rounding is relative to the sum of the magnitudes, not to the sum);
* shaded pixels within the pixel tolerance; ka = 1, kd = 0 gives the unshaded image;
* the full frame (render warps, fallback pass) gives the pixels of the parity hook;
* argument errors: shading without a gradient table, in a non-FP32 mode, in batched launches.
"""
import numpy as np
import pytest

import oracle
from paper_2401_02896_b300 import synthetic as SY

from _helpers import FIELD_REL_L2, PIXEL_ABS, field_rel_l2, oracle_lut

pytestmark = pytest.mark.gpu

GRAD_REL_L2 = 1e-4
KA, KD = 0.3, 0.7


@pytest.fixture(scope="module")
def S():
    from paper_2401_02896_b300 import sphdvr

    return sphdvr


def grad_rel_l2(field_a, grad_a, field_b, grad_b, D):
    """Relative L2 over the ray of the across-ray gradient vector: the three components as field rows."""
    num2 = den2 = 0.0
    for c in range(3):
        ra = np.concatenate([field_a[:, :2], grad_a[:, c, :]], axis=1)
        rb = np.concatenate([field_b[:, :2], grad_b[:, c, :]], axis=1)
        nb = _norm(rb, D)
        num2 += (field_rel_l2(ra, rb, D) * nb) ** 2
        den2 += nb ** 2
    return np.sqrt(num2 / den2) if den2 > 0 else np.sqrt(num2)


def _norm(rows, D):
    x, w = np.polynomial.legendre.leggauss(8)
    s = 0.0
    for r in rows:
        if r[1] <= r[0]:
            continue
        half = 0.5 * (r[1] - r[0])
        y = half * (x + 1)
        v = np.polyval(r[2:][::-1], y)
        s += half * np.sum(w * v * v)
    return np.sqrt(s)


@pytest.fixture(scope="module")
def setup(S):
    P = SY.halo_mixture(1_000_000, a_range=(5e-3, 0.05), seed=SY.BASE_SEED + 1, device="cuda")
    D = 3
    lut = oracle_lut("wendland_c2", 4, D, 4096)
    G = oracle.lut_build_grad(lut)
    ctx = S.sphdvr_create(0)
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    lt = S.sphdvr_lut_create(ctx, "wendland_c2", 4, D, 4096, lut["theta"], lut["pieces"])
    gp, _ = S.sphdvr_lut_build_grad("wendland_c2", 4, D, 4096, lut["theta"])
    S.sphdvr_lut_set_gradient(lt, lut["theta"], gp)
    res = 384
    cam = SY.orbit_camera(res, res)
    tf = SY.tf_density(P["value"])
    pix = SY.pixel_sample(res, res, 48, seed=57)
    R0 = oracle.render(P, lut, cam, tf, pix[:12], field_cap=1 << 16, grad=G)
    g = np.concatenate([R0["gfield"][r, :R0["stats"][r, 5], :, 0] for r in range(12)])
    g0 = 1e-3 * float(np.sqrt((g ** 2).sum(axis=1).mean()))
    shade = dict(shading=1, shade_ka=KA, shade_kd=KD, shade_g0=g0)
    yield dict(P=P, D=D, lut=lut, G=G, ctx=ctx, ds=ds, lt=lt, cam=cam, tf=tf, pix=pix, res=res, g0=g0, shade=shade)
    S.sphdvr_dataset_free(ds)
    S.sphdvr_lut_free(lt)
    S.sphdvr_destroy(ctx)


def test_shaded_field_gradient_and_pixels_match_the_oracle(S, setup):
    s = setup
    D, pix = s["D"], s["pix"]
    cap = 1 << 16
    R = oracle.render(s["P"], s["lut"], s["cam"], s["tf"], pix, field_cap=cap, grad=s["G"], shade=(KA, KD, s["g0"]))
    g = S.sphdvr_debug_rays_grad(s["ctx"], s["ds"], s["lt"], s["cam"], s["tf"], dict(ert_eps=0.0, **s["shade"]),
                                 pix, cap, D)
    assert not g["overflow"]
    fe, ge = [], []
    for r in range(len(pix)):
        if not R["stats"][r, 0]:
            continue
        n_o, n_g = R["stats"][r, 5], g["counts"][r, 2]
        fe.append(field_rel_l2(g["field"][r, :n_g], R["field"][r, :n_o], D))
        ge.append(grad_rel_l2(g["field"][r, :n_g], g["grad"][r, :n_g], R["field"][r, :n_o], R["gfield"][r, :n_o], D))
    print("g0 %.4g: field worst %.3g, gradient worst %.3g median %.3g" % (s["g0"], max(fe), max(ge), np.median(ge)))
    assert max(fe) <= FIELD_REL_L2
    assert max(ge) <= GRAD_REL_L2
    pe = np.abs(g["rgba"].astype(np.float64) - R["rgba"]).max()
    assert pe <= PIXEL_ABS, pe
    # the shading is visible: the shaded image differs from the unshaded one
    U = oracle.render(s["P"], s["lut"], s["cam"], s["tf"], pix)
    assert np.abs(U["rgba"] - R["rgba"]).max() > 10 * PIXEL_ABS


def test_unit_shading_gives_the_unshaded_image(S, setup):
    s = setup
    res = s["res"]
    import torch

    a = torch.zeros((res, res, 4), dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    S.sphdvr_render(s["ctx"], s["ds"], s["lt"], s["cam"], s["tf"], dict(ert_eps=0.0), a.data_ptr())
    S.sphdvr_render(s["ctx"], s["ds"], s["lt"], s["cam"], s["tf"],
                    dict(ert_eps=0.0, shading=1, shade_ka=1.0, shade_kd=0.0), b.data_ptr())
    torch.cuda.synchronize()
    assert (a - b).abs().max().item() <= 1e-5


def test_shaded_frame_matches_the_parity_hook_and_the_fallback_pass(S, setup):
    import torch

    s = setup
    res, pix = s["res"], s["pix"]
    o = dict(ert_eps=0.0, **s["shade"])
    img = torch.zeros((res, res, 4), dtype=torch.float32, device="cuda")
    S.sphdvr_render(s["ctx"], s["ds"], s["lt"], s["cam"], s["tf"], o, img.data_ptr())
    torch.cuda.synchronize()
    st = S.sphdvr_frame_stats(s["ctx"])
    assert st["overflow"] == 0
    g = S.sphdvr_debug_rays_grad(s["ctx"], s["ds"], s["lt"], s["cam"], s["tf"], o, pix, 1 << 16, s["D"])
    full = img.cpu().numpy().reshape(-1, 4)[pix]
    assert np.abs(full - g["rgba"]).max() <= 1e-5
    # a small per-ray capacity sends rays to the fallback pass: same image (a small frame, so that the
    # abandoned rays fit the fallback pass's list of 65,536 rays)
    cam = SY.orbit_camera(96, 72)
    a = torch.zeros((72, 96, 4), dtype=torch.float32, device="cuda")
    fb = torch.zeros_like(a)
    S.sphdvr_render(s["ctx"], s["ds"], s["lt"], cam, s["tf"], o, a.data_ptr())
    S.sphdvr_render(s["ctx"], s["ds"], s["lt"], cam, s["tf"], dict(o, ray_capacity=64), fb.data_ptr())
    torch.cuda.synchronize()
    assert S.sphdvr_frame_stats(s["ctx"])["overflow"] == 0
    assert (fb - a).abs().max().item() <= 1e-5


def test_shading_argument_errors(S, setup):
    import torch

    s = setup
    out = torch.zeros((s["res"], s["res"], 4), dtype=torch.float32, device="cuda")
    lt2 = S.sphdvr_lut_create(s["ctx"], "wendland_c2", 4, s["D"], 4096, s["lut"]["theta"], s["lut"]["pieces"])
    try:
        with pytest.raises(S.SphdvrError) as e:  # no gradient table
            S.sphdvr_render(s["ctx"], s["ds"], lt2, s["cam"], s["tf"], dict(shading=1, shade_ka=1.0), out.data_ptr())
        assert e.value.status == S.EINVAL
        with pytest.raises(S.SphdvrError) as e:  # knots that are not the table's
            th = s["lut"]["theta"].copy()
            th[5, 0] *= 1.01
            S.sphdvr_lut_set_gradient(lt2, th, np.zeros_like(s["lut"]["pieces"]))
        assert e.value.status == S.EINVAL
    finally:
        S.sphdvr_lut_free(lt2)
    for bad in (dict(shading=1, precision="fp64_naive"), dict(shading=2), dict(shading=1, shade_kd=-1.0),
                dict(shading=1, shade_g0=float("inf"))):
        with pytest.raises(S.SphdvrError) as e:
            S.sphdvr_render(s["ctx"], s["ds"], s["lt"], s["cam"], s["tf"], bad, out.data_ptr())
        assert e.value.status == S.EINVAL
    with pytest.raises(S.SphdvrError) as e:
        S.sphdvr_render_batch(s["ctx"], s["ds"], s["lt"], [s["cam"]], s["tf"], dict(shading=1, shade_ka=1.0),
                              [out.data_ptr()])
    assert e.value.status == S.EINVAL
