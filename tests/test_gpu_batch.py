"""Batched rendering: several frames in one launch of the render kernel.

The frames of a batch share data set, table, transfer function and options;
their rays are taken from one work queue.  Each ray's arithmetic does not
depend on which warp takes it, so a batch must reproduce the images of
separate sphdvr_render calls bit for bit, and its sampled pixels must match
the oracle like any frame.  The server groups compatible queued requests into
such launches.
"""
import numpy as np
import pytest

import oracle
from paper_2401_02896_b300 import synthetic as SY

from _helpers import PIXEL_ABS, oracle_lut

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2401_02896_b300 import sphdvr as S

    ctx = S.sphdvr_create(0)
    lut = oracle_lut("wendland_c2", 4, 3, 4096)
    lt = S.sphdvr_lut_create(ctx, lut["kernel"], lut["K"], lut["D"], lut["n_lambda"], lut["theta"], lut["pieces"])
    P = SY.halo_mixture(60_000, seed=SY.BASE_SEED + 23)
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    P2 = SY.halo_mixture(20_000, seed=SY.BASE_SEED + 24)
    ds2 = S.sphdvr_dataset_create(ctx, P2["pos"], P2["h"], P2["mass"], P2["density"], P2["value"])
    yield S, torch, ctx, lut, lt, P, ds, ds2, SY.tf_density(P["value"]), SY.tf_density(P2["value"])
    S.sphdvr_dataset_free(ds)
    S.sphdvr_dataset_free(ds2)
    S.sphdvr_lut_free(lt)
    S.sphdvr_destroy(ctx)


def _cams():
    # mixed sizes, ragged tiles, perspective and orthographic
    return [SY.orbit_camera(96, 64, azimuth_deg=10.0), SY.orbit_camera(128, 128, azimuth_deg=75.0, elevation_deg=-30.0),
            SY.orbit_camera(37, 53, azimuth_deg=200.0), SY.ortho_camera_z(80, 48),
            SY.orbit_camera(200, 120, azimuth_deg=300.0, elevation_deg=60.0)]


def _single(S, torch, ctx, ds, lt, cams, tf, opts):
    out = []
    for c in cams:
        o = torch.full((c["height"], c["width"], 4), -1.0, dtype=torch.float32, device="cuda")
        S.sphdvr_render(ctx, ds, lt, c, tf, opts, o.data_ptr())
        out.append(o)
    torch.cuda.synchronize()
    return out


def _batch(S, torch, ctx, ds, lt, cams, tf, opts):
    out = [torch.full((c["height"], c["width"], 4), -1.0, dtype=torch.float32, device="cuda") for c in cams]
    S.sphdvr_render_batch(ctx, ds, lt, cams, tf, opts, [o.data_ptr() for o in out])
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("opts", [None, dict(precision="fp64_naive"), dict(precision="fp32_reinit", reinit_dt=0.05),
                                  dict(precision="fp32_kahan"), dict(persistent=0)],
                         ids=["anchored", "fp64", "reinit", "kahan", "static"])
def test_batch_equals_separate_frames(env, opts):
    S, torch, ctx, lut, lt, P, ds, _, tf, _ = env
    cams = _cams()
    ref = _single(S, torch, ctx, ds, lt, cams, tf, opts)
    got = _batch(S, torch, ctx, ds, lt, cams, tf, opts)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    assert max(o[..., 3].max().item() for o in got) > 0.05
    st = S.sphdvr_frame_stats(ctx)
    assert st["rays"] == sum(c["width"] * c["height"] for c in cams)


@pytest.mark.parametrize("prec", ["fp32_anchored", "fp32_naive", "fp32_kahan"])
def test_every_knot_composited_once(env, prec):
    """Without early termination the window kernel composites each knot of each candidate exactly once: the
    frame's knot count is K + 1 times its candidate count, separately and batched (a particle dropped from
    the waiting list or the active set, or a knot taken twice, breaks the count)."""
    S, torch, ctx, lut, lt, P, ds, _, tf, _ = env
    cams = _cams()
    opts = dict(precision=prec, ert_eps=0.0)
    for c in cams:
        _single(S, torch, ctx, ds, lt, [c], tf, opts)
        st = S.sphdvr_frame_stats(ctx)
        assert st["knots"] == (lut["K"] + 1) * st["segments"] and st["segments"] > 0, st
    _batch(S, torch, ctx, ds, lt, cams, tf, opts)
    st = S.sphdvr_frame_stats(ctx)
    assert st["knots"] == (lut["K"] + 1) * st["segments"], st


def test_batch_of_one_and_of_eight(env):
    S, torch, ctx, lut, lt, P, ds, _, tf, _ = env
    cams = [SY.orbit_camera(40 + 8 * i, 56, azimuth_deg=45.0 * i) for i in range(S.MAX_BATCH)]
    ref = _single(S, torch, ctx, ds, lt, cams, tf, None)
    for a, b in zip(_batch(S, torch, ctx, ds, lt, cams, tf, None), ref):
        assert torch.equal(a, b)
    assert torch.equal(_batch(S, torch, ctx, ds, lt, cams[3:4], tf, None)[0], ref[3])


def test_batch_sampled_pixels_match_the_oracle(env):
    S, torch, ctx, lut, lt, P, ds, _, tf, _ = env
    cams = _cams()[:3]
    got = _batch(S, torch, ctx, ds, lt, cams, tf, dict(ert_eps=0.0))
    parts = dict(pos=P["pos"], h=P["h"], mass=P["mass"], value=P["value"], density=P["density"])
    for f, (c, img) in enumerate(zip(cams, got)):
        pix = SY.pixel_sample(c["width"], c["height"], 10, seed=40 + f)
        R = oracle.render(parts, lut, c, tf, pix)
        mine = img.reshape(-1, 4)[torch.as_tensor(pix, dtype=torch.long, device="cuda")].cpu().numpy()
        assert np.abs(mine - R["rgba"]).max() <= PIXEL_ABS


def test_batch_argument_errors(env):
    S, torch, ctx, lut, lt, P, ds, _, tf, _ = env
    o = torch.zeros((32, 32, 4), dtype=torch.float32, device="cuda")
    cam = SY.orbit_camera(32, 32)
    for cams, outs in (([], []), ([cam] * (S.MAX_BATCH + 1), [o.data_ptr()] * (S.MAX_BATCH + 1)),
                       ([cam, cam], [o.data_ptr(), 0]), ([cam, dict(cam, width=0)], [o.data_ptr()] * 2)):
        with pytest.raises(S.SphdvrError) as e:
            S.sphdvr_render_batch(ctx, ds, lt, cams, tf, None, outs)
        assert e.value.status == S.EINVAL


def test_server_groups_compatible_requests(env):
    """One worker, requests queued faster than it renders: compatible ones share launches, others do not."""
    S, torch, ctx, lut, lt, P, ds, ds2, tf, tf2 = env
    r = np.random.default_rng(7)
    reqs = []
    for i in range(14):
        k = int(r.integers(3)) == 0  # about a third on the second data set
        res = int(r.choice([48, 96, 160]))
        reqs.append((ds2 if k else ds, tf2 if k else tf, SY.orbit_camera(res, res, azimuth_deg=360 * r.random())))
    refs = []
    for d, t, c in reqs:
        refs.append(_single(S, torch, ctx, d, lt, [c], t, None)[0])
    srv = S.Server(ctx, 8 << 30, max_inflight=1)
    try:
        srv.set_batch(S.MAX_BATCH)
        outs = [torch.full((c["height"], c["width"], 4), -1.0, dtype=torch.float32, device="cuda") for _, _, c in reqs]
        tickets = [srv.submit(d, lt, c, t, None, o.data_ptr()) for (d, t, c), o in zip(reqs, outs)]
        for tk in tickets:
            assert srv.wait(tk, 120_000)
        bs = srv.batch_stats()
        st = srv.stats()
        for bad in ((0, 1000), (S.MAX_BATCH + 1, 1000), (2, -1)):
            with pytest.raises(S.SphdvrError):
                srv.set_batch(*bad)
    finally:
        srv.destroy()
    for o, ref in zip(outs, refs):
        assert torch.equal(o, ref)
    assert st["completed"] == len(reqs)
    assert bs["frames"] == len(reqs)
    assert bs["launches"] < len(reqs) and 2 <= bs["largest"] <= S.MAX_BATCH


@pytest.mark.parametrize("limits", [(1, 1 << 20), (8, 0)], ids=["one_frame", "no_rays_beyond_the_first"])
def test_server_without_batching(env, limits):
    """Batching off, by the frame limit or by the ray limit: one launch per request."""
    S, torch, ctx, lut, lt, P, ds, _, tf, _ = env
    cams = [SY.orbit_camera(64, 64, azimuth_deg=30.0 * i) for i in range(5)]
    refs = _single(S, torch, ctx, ds, lt, cams, tf, None)
    srv = S.Server(ctx, 8 << 30, max_inflight=1)
    try:
        srv.set_batch(*limits)
        outs = [torch.zeros((64, 64, 4), dtype=torch.float32, device="cuda") for _ in cams]
        tickets = [srv.submit(ds, lt, c, tf, None, o.data_ptr()) for c, o in zip(cams, outs)]
        for tk in tickets:
            assert srv.wait(tk, 60_000)
        bs = srv.batch_stats()
    finally:
        srv.destroy()
    for o, ref in zip(outs, refs):
        assert torch.equal(o, ref)
    assert bs["launches"] == len(cams) and bs["largest"] == 1


def test_batch_with_degenerate_frames(env):
    """A 1x1 frame and a frame that sees no particle, batched with an ordinary one."""
    S, torch, ctx, lut, lt, P, ds, _, tf, _ = env
    away = SY.orbit_camera(24, 16, distance=2.0)
    away = dict(away, target=[2 * away["eye"][i] - 0.5 for i in range(3)])  # looking away from the data
    cams = [SY.orbit_camera(1, 1), away, SY.orbit_camera(33, 17, azimuth_deg=123.0)]
    ref = _single(S, torch, ctx, ds, lt, cams, tf, None)
    for a, b in zip(_batch(S, torch, ctx, ds, lt, cams, tf, None), ref):
        assert torch.equal(a, b)
    assert float(ref[1].abs().max()) == 0.0
