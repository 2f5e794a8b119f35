"""The frame server: continuous batching over worker streams with a device-memory budget.

Requests mix two resident data sets, seeded orbit cameras and several image
sizes, and arrive with seeded exponential gaps (a Poisson process).  Every
served image must equal the image sphdvr_render gives for the same inputs
(the same kernels run; only the stream and the worker's buffers differ).
"""
import time

import numpy as np
import pytest

from paper_2401_02896_b300 import synthetic as SY

from _helpers import PIXEL_ABS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2401_02896_b300 import sphdvr as S

    ctx = S.sphdvr_create(0)
    th, pc, _ = S.sphdvr_lut_build("wendland_c2", 4, 3, 1025)
    lut = S.sphdvr_lut_create(ctx, "wendland_c2", 4, 3, 1025, th, pc)
    sets = []
    for n, seed in ((150_000, 31), (40_000, 32)):
        P = SY.halo_mixture(n, seed=seed)
        ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
        sets.append((ds, SY.tf_density(P["value"])))
    yield S, torch, ctx, lut, sets
    for ds, _ in sets:
        S.sphdvr_dataset_free(ds)
    S.sphdvr_lut_free(lut)
    S.sphdvr_destroy(ctx)


def _requests(count, seed):
    r = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        res = int(r.choice([48, 96, 128, 200]))
        cam = SY.orbit_camera(res, res, azimuth_deg=360 * r.random(), elevation_deg=-50 + 100 * r.random())
        out.append((int(r.integers(2)), cam, float(r.exponential(0.002))))
    return out


def _reference(S, torch, ctx, lut, sets, reqs):
    refs = []
    for k, cam, _ in reqs:
        ds, tf = sets[k]
        o = torch.zeros((cam["height"], cam["width"], 4), dtype=torch.float32, device="cuda")
        S.sphdvr_render(ctx, ds, lut, cam, tf, None, o.data_ptr())
        refs.append(o)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in refs]


def test_server_matches_render_under_poisson_arrivals(env):
    S, torch, ctx, lut, sets = env
    reqs = _requests(24, 5)
    refs = _reference(S, torch, ctx, lut, sets, reqs)
    srv = S.Server(ctx, 8 << 30, max_inflight=3)
    try:
        outs, tickets = [], []
        for k, cam, gap in reqs:
            ds, tf = sets[k]
            o = torch.full((cam["height"], cam["width"], 4), -1.0, dtype=torch.float32, device="cuda")
            outs.append(o)
            tickets.append(srv.submit(ds, lut, cam, tf, None, o.data_ptr()))
            time.sleep(gap)
        for t in tickets:
            assert srv.wait(t, 60_000)
        st = srv.stats()
    finally:
        srv.destroy()
    for o, ref in zip(outs, refs):
        assert np.abs(o.cpu().numpy() - ref).max() <= PIXEL_ABS
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["rays_per_s"] > 0
    assert st["held_bytes"] <= 8 << 30


def test_server_tight_budget_serialises_frames(env):
    """A budget that holds one frame's buffers but not two: workers take turns, results unchanged."""
    S, torch, ctx, lut, sets = env
    reqs = _requests(8, 9)
    refs = _reference(S, torch, ctx, lut, sets, reqs)
    # one 200x200 frame needs the render grid's per-ray scratch (~0.7 GB) plus small buffers
    srv = S.Server(ctx, 1200 << 20, max_inflight=3)
    try:
        outs, tickets = [], []
        for k, cam, _ in reqs:
            ds, tf = sets[k]
            o = torch.zeros((cam["height"], cam["width"], 4), dtype=torch.float32, device="cuda")
            outs.append(o)
            tickets.append(srv.submit(ds, lut, cam, tf, None, o.data_ptr()))
        for t in tickets:
            assert srv.wait(t, 120_000)
        st = srv.stats()
    finally:
        srv.destroy()
    for o, ref in zip(outs, refs):
        assert np.abs(o.cpu().numpy() - ref).max() <= PIXEL_ABS
    assert st["completed"] == len(reqs)
    assert st["held_bytes"] <= 1200 << 20


def test_server_refuses_frames_beyond_the_budget_and_unknown_tickets(env):
    S, torch, ctx, lut, sets = env
    srv = S.Server(ctx, 1 << 20, max_inflight=1)
    try:
        o = torch.zeros((64, 64, 4), dtype=torch.float32, device="cuda")
        ds, tf = sets[0]
        with pytest.raises(S.SphdvrError) as e:
            srv.submit(ds, lut, SY.orbit_camera(64, 64), tf, None, o.data_ptr())
        assert e.value.status == S.EBUSY
        with pytest.raises(S.SphdvrError) as e:
            srv.wait(12345, 0)
        assert e.value.status == S.ENOTFOUND
    finally:
        srv.destroy()
    with pytest.raises(S.SphdvrError) as e:
        S.Server(ctx, 1 << 30, max_inflight=9)
    assert e.value.status == S.EINVAL


def test_server_timeout_then_completion_and_destroy_with_pending(env):
    S, torch, ctx, lut, sets = env
    srv = S.Server(ctx, 8 << 30, max_inflight=1)
    ds, tf = sets[0]
    outs = [torch.zeros((256, 256, 4), dtype=torch.float32, device="cuda") for _ in range(4)]
    tickets = [srv.submit(ds, lut, SY.orbit_camera(256, 256, azimuth_deg=10 * i), tf, None, o.data_ptr())
               for i, o in enumerate(outs)]
    first = srv.wait(tickets[-1], 0)  # four frames queued on one worker: the last is not done yet
    assert first is False
    assert srv.wait(tickets[-1], -1)
    # the earlier tickets are not waited for: destroy retires them
    srv.destroy()
