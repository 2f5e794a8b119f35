"""Parity at the full sizes of the larger workloads, on seeded pixel samples.

* 16,777,216-particle halo mixture (h over ~3 decades), Wendland C2, K=4 D=3,
  4096-entry table, perspective 2048x2048 -- the benchmark's frame;
* the same 16,777,216 positions prepared as an SPH code would: h = distance to the
  32nd nearest neighbour, value = the SPH density estimate (noisy h and values);
* 64,000,000-particle dam-break slab (dense graded layer + sparse splash),
  Wendland C4, K=4 D=4, perspective 4096x4096, a high-opacity transfer function.

Each frame is checked three ways on the same 48 seeded pixels:
1. the parity hook (sphdvr_debug_rays, no early termination): candidate sets,
   field pieces and pixels against the oracle, which computes the sampled rays
   one by one (FP64, all particles); the particles within 1e-6 h of tangency
   are counted on the GPU side and reported;
2. the production frame (sphdvr_render: the persistent 4-warp kernel, the
   dynamic work queue, early ray termination at the default 1e-5) -- the image
   the benchmark times -- against the oracle within 2e-4 + 1e-5;
3. the production frame without early termination equals the parity hook's
   pixels bit for bit (same per-ray arithmetic in both instantiations).
"""
import numpy as np
import pytest

import oracle
from paper_2401_02896_b300 import synthetic as SY

from test_gpu_parity import _check_rays, _mk, _orc_particles  # noqa: F401  (shared checking code)
from _helpers import PIXEL_ABS, oracle_lut

pytestmark = pytest.mark.gpu

ERT_EPS = 1e-5


@pytest.fixture(scope="module")
def S():
    from paper_2401_02896_b300 import sphdvr

    return sphdvr


@pytest.fixture(scope="module")
def ctx(S):
    c = S.sphdvr_create(0)
    yield c
    S.sphdvr_destroy(c)


def _production(S, ctx, ds, lt, cam, tf, ert):
    import torch

    out = torch.full((cam["height"], cam["width"], 4), -1.0, dtype=torch.float32, device="cuda")
    S.sphdvr_render(ctx, ds, lt, cam, tf, dict(ert_eps=ert), out.data_ptr())
    torch.cuda.synchronize()
    st = S.sphdvr_frame_stats(ctx)
    img = out.reshape(-1, 4).cpu().numpy()
    del out
    return img, st


def _three_way(S, ctx, ds, lt, P, lut, cam, tf, pix, name):
    wf, wp = _check_rays(S, ctx, ds, lt, P, lut, cam, tf, pix, cand_cap=1 << 16, field_cap=1 << 18)
    g = S.sphdvr_debug_rays(ctx, ds, lt, cam, tf, dict(ert_eps=0.0), pix)
    cands, tang = g["counts"][:, 0], g["counts"][:, 4]
    # tangency band: counted, reported, and a negligible share of the candidates
    assert tang.sum() <= max(4, 1e-3 * cands.sum()), (tang.sum(), cands.sum())
    R = oracle.render(_orc_particles(P), lut, cam, tf, pix)
    img, st = _production(S, ctx, ds, lt, cam, tf, ERT_EPS)
    assert st["overflow"] == 0, st
    err_prod = np.abs(img[pix].astype(np.float64) - R["rgba"]).max()
    assert err_prod <= PIXEL_ABS + ERT_EPS, err_prod
    img0, st0 = _production(S, ctx, ds, lt, cam, tf, 0.0)
    assert st0["overflow"] == 0, st0
    # without early termination every knot of every candidate is composited exactly once
    assert st0["knots"] == (lut["K"] + 1) * st0["segments"], st0
    assert np.array_equal(img0[pix], g["rgba"]), np.abs(img0[pix] - g["rgba"]).max()
    print("%s: field rel-L2 worst %.3g, hook pixel worst %.3g, production pixel worst %.3g (ERT %g, %d rays "
          "terminated), tangency-band tests %d of %d candidates on %d rays"
          % (name, wf, wp, err_prod, ERT_EPS, st["ert_rays"], int(tang.sum()), int(cands.sum()), len(pix)))
    return st


def test_halo_16m_2048_sampled_pixels(S, ctx):
    P = SY.halo_mixture(16_777_216, a_range=(5e-4, 0.05), seed=SY.BASE_SEED + 2, device="cuda")
    lut = oracle_lut("wendland_c2", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(2048, 2048, azimuth_deg=30.0, elevation_deg=20.0)  # the benchmark's camera
    tf = SY.tf_density(P["value"])
    pix = SY.pixel_sample(2048, 2048, 48, seed=21)
    try:
        _three_way(S, ctx, ds, lt, P, lut, cam, tf, pix, "halo16m")
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_halo_knn_16m_2048_sampled_pixels(S, ctx):
    P = SY.halo_mixture_knn(16_777_216, a_range=(5e-4, 0.05), seed=SY.BASE_SEED + 2)
    lut = oracle_lut("wendland_c2", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(2048, 2048, azimuth_deg=30.0, elevation_deg=20.0)
    tf = SY.tf_density(P["value"])
    pix = SY.pixel_sample(2048, 2048, 48, seed=23)
    try:
        _three_way(S, ctx, ds, lt, P, lut, cam, tf, pix, "halo16m kNN")
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_dam_break_64m_4096_sampled_pixels(S, ctx):
    P = SY.dam_break_slab(64_000_000)
    lut = oracle_lut("wendland_c4", 4, 4, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(4096, 4096, azimuth_deg=-60.0, elevation_deg=25.0, distance=1.6, center=(0.5, 0.25, 0.3))
    tf = SY.tf_density(P["value"], sigma_scale=500.0)
    pix = SY.pixel_sample(4096, 4096, 48, seed=22)
    try:
        st = _three_way(S, ctx, ds, lt, P, lut, cam, tf, pix, "dam-break 64M")
        assert st["ert_rays"] > 0  # the high-opacity frame exercises early termination
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)
