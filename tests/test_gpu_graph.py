"""Frame plans: preallocated, capacity-bound frames that can be captured into a CUDA graph.

A plan's frame runs the same binning and render kernels as sphdvr_render; its
pairs are sorted inside a fixed-capacity buffer whose unused entries carry the
largest key, so the sorted pairs, the tile ranges and the image are identical
to sphdvr_render's.  Captured into a CUDA graph (stream capture), a replay
renders the same image again.
"""
import pytest

from paper_2401_02896_b300 import synthetic as SY

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2401_02896_b300 import sphdvr as S

    ctx = S.sphdvr_create(0)
    th, pc, _ = S.sphdvr_lut_build("wendland_c2", 4, 3, 1025)
    lt = S.sphdvr_lut_create(ctx, "wendland_c2", 4, 3, 1025, th, pc)
    P = SY.halo_mixture(80_000, seed=SY.BASE_SEED + 51)
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    yield S, torch, ctx, lt, ds, SY.tf_density(P["value"])
    S.sphdvr_dataset_free(ds)
    S.sphdvr_lut_free(lt)
    S.sphdvr_destroy(ctx)


def _ref(S, torch, ctx, lt, ds, tf, cam, opts=None):
    o = torch.zeros((cam["height"], cam["width"], 4), dtype=torch.float32, device="cuda")
    S.sphdvr_render(ctx, ds, lt, cam, tf, opts, o.data_ptr())
    torch.cuda.synchronize()
    return o, S.sphdvr_frame_stats(ctx)["pairs"]


@pytest.mark.parametrize("opts", [None, dict(precision="fp64_naive")], ids=["anchored", "fp64"])
def test_plan_frames_equal_render_and_replay_from_a_cuda_graph(env, opts):
    S, torch, ctx, lt, ds, tf = env
    cams = [SY.orbit_camera(160, 120, azimuth_deg=40.0), SY.orbit_camera(77, 200, azimuth_deg=130.0)]
    refs = [_ref(S, torch, ctx, lt, ds, tf, c, opts) for c in cams]
    plan = S.FramePlan(ctx, ds, lt, tf, opts, 256, 256, 2 * max(p for _, p in refs) + 64)
    try:
        for c, (ref, _) in zip(cams, refs):
            out = torch.full_like(ref, -1.0)
            plan.render(c, out.data_ptr())
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
        assert not plan.overflowed()
        # capture both frames into one graph on a side stream, then replay it
        imgs = [torch.full_like(ref, -1.0) for ref, _ in refs]
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            for c, img in zip(cams, imgs):
                plan.render(c, img.data_ptr(), stream=s.cuda_stream)
        torch.cuda.synchronize()
        assert all(float(img.min()) == -1.0 for img in imgs)  # capturing runs nothing
        for _ in range(2):
            for img in imgs:
                img.fill_(-1.0)
            g.replay()
            torch.cuda.synchronize()
            for img, (ref, _) in zip(imgs, refs):
                assert torch.equal(img, ref)
        assert not plan.overflowed()
    finally:
        plan.destroy()


def test_plan_overflow_and_argument_errors(env):
    S, torch, ctx, lt, ds, tf = env
    cam = SY.orbit_camera(96, 96)
    ref, pairs = _ref(S, torch, ctx, lt, ds, tf, cam)
    assert pairs > 64
    plan = S.FramePlan(ctx, ds, lt, tf, None, 96, 96, 64)
    try:
        out = torch.zeros_like(ref)
        plan.render(cam, out.data_ptr())
        torch.cuda.synchronize()
        assert plan.overflowed()
        assert not plan.overflowed()  # read and cleared
        with pytest.raises(S.SphdvrError) as e:
            plan.render(SY.orbit_camera(97, 96), out.data_ptr())
        assert e.value.status == S.EINVAL
    finally:
        plan.destroy()
    for bad in ((0, 96, 100), (96, 96, 1), (96, 40000, 100)):
        with pytest.raises(S.SphdvrError) as e:
            S.FramePlan(ctx, ds, lt, tf, None, *bad)
        assert e.value.status == S.EINVAL
