"""The allocation-free render entry point (sphdvr_render_static_scratch).

It runs the same binning and render kernels as sphdvr_render with all frame
scratch carved from the library's fixed device array, so two calls in a row
must give the image sphdvr_render gives, within the pixel tolerance.
"""
import numpy as np
import pytest

from paper_2401_02896_b300 import synthetic as SY

from _helpers import PIXEL_ABS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2401_02896_b300 import sphdvr as S

    ctx = S.sphdvr_create(0)
    P = SY.halo_mixture(200_000, seed=11)
    tf = SY.tf_density(P["value"])
    th, pc, _ = S.sphdvr_lut_build("wendland_c2", 4, 3, 1025)
    lut = S.sphdvr_lut_create(ctx, "wendland_c2", 4, 3, 1025, th, pc)
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    yield S, torch, ctx, ds, lut, tf
    S.sphdvr_dataset_free(ds)
    S.sphdvr_lut_free(lut)
    S.sphdvr_destroy(ctx)


def test_static_scratch_matches_render_twice(setup):
    S, torch, ctx, ds, lut, tf = setup
    cam = SY.orbit_camera(200, 136)  # ragged tiles in both directions
    ref = torch.zeros((136, 200, 4), dtype=torch.float32, device="cuda")
    S.sphdvr_render(ctx, ds, lut, cam, tf, None, ref.data_ptr())
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    assert r[..., 3].max() > 0.05  # the view is not empty
    for _ in range(2):
        out = torch.full((136, 200, 4), -1.0, dtype=torch.float32, device="cuda")
        S.sphdvr_render_static_scratch(ctx, ds, lut, cam, tf, None, out.data_ptr())
        torch.cuda.synchronize()
        err = np.abs(out.cpu().numpy() - r).max()
        assert err <= PIXEL_ABS, err


def test_static_scratch_persistent_queue_and_ortho(setup):
    S, torch, ctx, ds, lut, tf = setup
    cam = SY.orbit_camera(96, 96)
    cam = dict(cam, projection="ortho", half_w=0.6, half_h=0.6)
    opts = dict(persistent=1)
    ref = torch.zeros((96, 96, 4), dtype=torch.float32, device="cuda")
    S.sphdvr_render(ctx, ds, lut, cam, tf, opts, ref.data_ptr())
    out = torch.zeros_like(ref)
    S.sphdvr_render_static_scratch(ctx, ds, lut, cam, tf, opts, out.data_ptr())
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref.cpu().numpy()).max() <= PIXEL_ABS


def test_static_scratch_rejects_frames_beyond_its_limits(setup):
    S, torch, ctx, ds, lut, tf = setup
    out = torch.zeros(4, dtype=torch.float32, device="cuda")
    big = SY.orbit_camera(4112, 4096)  # 257 x 256 tiles > 65536
    with pytest.raises(S.SphdvrError) as e:
        S.sphdvr_render_static_scratch(ctx, ds, lut, big, tf, None, out.data_ptr())
    assert e.value.status == S.EINVAL
    with pytest.raises(S.SphdvrError) as e:
        S.sphdvr_render_static_scratch(ctx, ds, lut, SY.orbit_camera(8, 8), tf, None, 0)
    assert e.value.status == S.EINVAL
