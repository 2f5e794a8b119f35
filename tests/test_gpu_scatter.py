"""The paper's pass order (scatter per particle, sort per ray, accumulate per ray) against the oracle and
against the ray-gathering path (anchored windows): same candidates and knots, pixels within the parity
tolerance, on uniform data and on a halo mixture whose h spans decades (where a plain recurrence over FP32
difference coefficients would drift)."""
import numpy as np
import pytest

import oracle
from paper_2401_02896_b300 import synthetic as SY

from _helpers import PIXEL_ABS, oracle_lut

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2401_02896_b300 import sphdvr

    return sphdvr


@pytest.fixture(scope="module")
def ctx(S):
    c = S.sphdvr_create(0)
    yield c
    S.sphdvr_destroy(c)


@pytest.mark.parametrize("case", ["cube_ortho", "cube_odd_K", "halo_perspective"])
def test_scatter_order_matches_oracle_and_gather(S, ctx, case):
    import torch

    if case == "cube_ortho":
        P, cam, lut, tf = SY.uniform_cube(), SY.ortho_camera_z(64, 64), oracle_lut("m4", 4, 3, 1025), SY.tf_bumps()
    elif case == "cube_odd_K":
        P, cam, lut, tf = SY.uniform_cube(), SY.orbit_camera(48, 40), oracle_lut("m4", 3, 2, 1025), SY.tf_bumps()
    else:
        P = SY.halo_mixture(60_000, seed=SY.BASE_SEED + 71)
        cam, lut, tf = SY.orbit_camera(96, 64, azimuth_deg=50.0), oracle_lut("wendland_c2", 4, 3, 1025), None
        tf = SY.tf_density(P["value"])
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    lt = S.sphdvr_lut_create(ctx, lut["kernel"], lut["K"], lut["D"], lut["n_lambda"], lut["theta"], lut["pieces"])
    H, W = cam["height"], cam["width"]
    try:
        opts = dict(ert_eps=0.0)
        a = torch.full((H, W, 4), -1.0, dtype=torch.float32, device="cuda")
        b = torch.zeros_like(a)
        S.sphdvr_render_scatter(ctx, ds, lt, cam, tf, opts, a.data_ptr())
        torch.cuda.synchronize()
        st_s = S.sphdvr_frame_stats(ctx)
        S.sphdvr_render(ctx, ds, lt, cam, tf, opts, b.data_ptr())  # FP32 anchored: drift-free
        torch.cuda.synchronize()
        st_g = S.sphdvr_frame_stats(ctx)
        assert st_s["rays"] == W * H
        assert abs(st_s["knots"] - st_g["knots"]) <= 1e-4 * st_g["knots"]
        assert float((a - b).abs().max()) <= PIXEL_ABS
        pix = SY.pixel_sample(W, H, 16, seed=72)
        parts = dict(pos=P["pos"], h=P["h"], mass=P["mass"], value=P["value"], density=P["density"])
        R = oracle.render(parts, lut, cam, tf, pix)
        assert np.abs(a.cpu().numpy().reshape(-1, 4)[pix] - R["rgba"]).max() <= PIXEL_ABS
        assert a[..., 3].max().item() > 0.05
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_scatter_argument_errors(S, ctx):
    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 1025)
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    lt = S.sphdvr_lut_create(ctx, lut["kernel"], lut["K"], lut["D"], lut["n_lambda"], lut["theta"], lut["pieces"])
    try:
        with pytest.raises(S.SphdvrError) as e:
            S.sphdvr_render_scatter(ctx, ds, lt, SY.ortho_camera_z(8, 8), SY.tf_bumps(), None, 0)
        assert e.value.status == S.EINVAL
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_scatter_degenerate_frames(S, ctx):
    """No particle in view: a transparent image; a 1x1 frame equals the gathering path's pixel."""
    import torch

    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 1025)
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    lt = S.sphdvr_lut_create(ctx, lut["kernel"], lut["K"], lut["D"], lut["n_lambda"], lut["theta"], lut["pieces"])
    try:
        away = SY.orbit_camera(16, 16)
        away = dict(away, target=[2 * away["eye"][i] - 0.5 for i in range(3)])
        o = torch.full((16, 16, 4), -1.0, dtype=torch.float32, device="cuda")
        S.sphdvr_render_scatter(ctx, ds, lt, away, SY.tf_bumps(), None, o.data_ptr())
        torch.cuda.synchronize()
        assert float(o.abs().max()) == 0.0
        one = SY.orbit_camera(1, 1)
        a = torch.zeros((1, 1, 4), dtype=torch.float32, device="cuda")
        b = torch.zeros_like(a)
        S.sphdvr_render_scatter(ctx, ds, lt, one, SY.tf_bumps(), dict(ert_eps=0.0), a.data_ptr())
        S.sphdvr_render(ctx, ds, lt, one, SY.tf_bumps(), dict(ert_eps=0.0), b.data_ptr())
        torch.cuda.synchronize()
        assert float((a - b).abs().max()) <= PIXEL_ABS
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)
