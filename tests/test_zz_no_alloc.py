"""The allocation-free render entry point (sphdvr_render_static_scratch).

Some callers cannot allocate device memory while they render (a server whose
memory is all in its own pool, a process at its memory limit, a caller that
cannot take the synchronisation cudaMalloc/cudaFree bring).  This entry point
runs the same binning and render kernels as sphdvr_render with all frame
scratch carved from the library's fixed device array.  The tests check, on a
context that never rendered any other way, that the call leaves the context's
buffers as they were and the device's free memory unchanged after its first call,
that two calls in a row give the image sphdvr_render gives bit for bit, and
that its limits and frame flags are reported.  (Building a data set grows the
context's sort scratch, so "leaves the buffers alone" is checked as the held
bytes unchanged across the calls.)
"""
import numpy as np
import pytest

from paper_2401_02896_b300 import synthetic as SY

from _helpers import oracle_lut

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2401_02896_b300 import sphdvr as S

    P = SY.halo_mixture(200_000, seed=11)
    tf = SY.tf_density(P["value"])
    th, pc, _ = S.sphdvr_lut_build("wendland_c2", 4, 3, 1025)
    objs = []
    for _ in range(2):  # [0] renders only through the static entry point, [1] the reference images
        c = S.sphdvr_create(0)
        lut = S.sphdvr_lut_create(c, "wendland_c2", 4, 3, 1025, th, pc)
        ds = S.sphdvr_dataset_create(c, P["pos"], P["h"], P["mass"], P["density"], P["value"])
        objs.append((c, ds, lut))
    (ctx, ds, lut), ref = objs
    yield S, torch, ctx, ref, ds, lut, tf
    for c, d, l in objs:
        S.sphdvr_dataset_free(d)
        S.sphdvr_lut_free(l)
        S.sphdvr_destroy(c)


def _reference(S, torch, ref, cam, tf, opts):
    ref_ctx, ds, lut = ref
    img = torch.full((cam["height"], cam["width"], 4), -1.0, dtype=torch.float32, device="cuda")
    S.sphdvr_render(ref_ctx, ds, lut, cam, tf, opts, img.data_ptr())
    torch.cuda.synchronize()
    return img


def test_static_scratch_allocates_nothing_and_matches_render(setup):
    S, torch, ctx, ref_ctx, ds, lut, tf = setup
    cam = SY.orbit_camera(200, 136)  # ragged tiles in both directions
    outs = [torch.full((136, 200, 4), -1.0, dtype=torch.float32, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    held = S.sphdvr_ctx_info(ctx)["held_bytes"]
    S.sphdvr_render_static_scratch(ctx, ds, lut, cam, tf, None, outs[0].data_ptr())  # first call: set-up
    torch.cuda.synchronize()
    free_after_first = torch.cuda.mem_get_info()[0]
    S.sphdvr_render_static_scratch(ctx, ds, lut, cam, tf, None, outs[1].data_ptr())
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_after_first  # no device memory taken by the second call
    assert S.sphdvr_ctx_info(ctx)["held_bytes"] == held  # nor by the context's buffers
    st = S.sphdvr_frame_stats(ctx)  # the counters come from the static array
    assert st["rays"] == 200 * 136 and st["overflow"] == 0 and st["segments"] > 0
    img = _reference(S, torch, ref_ctx, cam, tf, None)
    assert img[..., 3].max().item() > 0.05  # the view is not empty
    for o in outs:
        assert torch.equal(o, img)
    assert S.sphdvr_frame_stats(ref_ctx[0])["segments"] == st["segments"]


def test_static_scratch_schedules_and_ortho(setup):
    """The work queue and the static ray stride (persistent=0) under the 64-CTA cap, orthographic rays."""
    S, torch, ctx, ref_ctx, ds, lut, tf = setup
    cam = dict(SY.orbit_camera(96, 80), projection="ortho", half_w=0.6, half_h=0.5)
    held = S.sphdvr_ctx_info(ctx)["held_bytes"]
    for opts in (dict(persistent=1), dict(persistent=0)):
        img = _reference(S, torch, ref_ctx, cam, tf, opts)
        out = torch.zeros_like(img)
        S.sphdvr_render_static_scratch(ctx, ds, lut, cam, tf, opts, out.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(out, img), opts
    assert S.sphdvr_ctx_info(ctx)["held_bytes"] == held


def test_static_scratch_reports_quantised_flags(setup):
    """A value quantum far below the field's bound sets flag bit 4; the static entry point reports it."""
    S, torch, ctx, ref_ctx, ds, lut, tf = setup
    P = SY.uniform_cube()
    L = oracle_lut("m4", 4, 3, 1025)
    dsq = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    ltq = S.sphdvr_lut_create(ctx, "m4", 4, 3, 1025, L["theta"], L["pieces"])
    cam = SY.ortho_camera_z(16, 16)
    o = torch.zeros((16, 16, 4), dtype=torch.float32, device="cuda")
    try:
        qp = S.sphdvr_dataset_quant_params(ctx, dsq, "m4", 3, 64)
        fine = dict(precision="int64_quant", quant_tau=qp["tau"], quant_sigma=qp["sigma"] * 1e-9)
        S.sphdvr_render_static_scratch(ctx, dsq, ltq, cam, SY.tf_bumps(), fine, o.data_ptr())
        torch.cuda.synchronize()
        assert S.sphdvr_frame_stats(ctx)["overflow"] & 16
        ok = dict(precision="int64_quant", quant_tau=qp["tau"], quant_sigma=qp["sigma"])
        S.sphdvr_render_static_scratch(ctx, dsq, ltq, cam, SY.tf_bumps(), ok, o.data_ptr())
        torch.cuda.synchronize()
        assert not S.sphdvr_frame_stats(ctx)["overflow"] & 16
    finally:
        S.sphdvr_dataset_free(dsq)
        S.sphdvr_lut_free(ltq)


def test_static_scratch_rejects_frames_beyond_its_limits(setup):
    S, torch, ctx, ref_ctx, ds, lut, tf = setup
    out = torch.zeros(4, dtype=torch.float32, device="cuda")
    held = S.sphdvr_ctx_info(ctx)["held_bytes"]
    big = SY.orbit_camera(4112, 4096)  # 257 x 256 tiles > 65536
    with pytest.raises(S.SphdvrError) as e:
        S.sphdvr_render_static_scratch(ctx, ds, lut, big, tf, None, out.data_ptr())
    assert e.value.status == S.EINVAL
    with pytest.raises(S.SphdvrError) as e:
        S.sphdvr_render_static_scratch(ctx, ds, lut, SY.orbit_camera(8, 8), tf, None, 0)
    assert e.value.status == S.EINVAL
    # large particles seen close up: every chunk covers many tiles, more than 2,097,152 chunk-tile pairs
    P = SY.uniform_cube(200_000, h=0.05, seed=SY.BASE_SEED + 31)
    dsb = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    held = S.sphdvr_ctx_info(ctx)["held_bytes"]  # the build may have grown the sort scratch
    img = torch.zeros((4096, 4096, 4), dtype=torch.float32, device="cuda")
    try:
        with pytest.raises(S.SphdvrError) as e:
            S.sphdvr_render_static_scratch(ctx, dsb, lut, SY.orbit_camera(4096, 4096, distance=1.2), tf, None,
                                           img.data_ptr())
        assert e.value.status == S.EOVERFLOW
    finally:
        S.sphdvr_dataset_free(dsb)
    assert S.sphdvr_ctx_info(ctx)["held_bytes"] == held
    assert float(img.abs().max()) == 0.0  # nothing was rendered
