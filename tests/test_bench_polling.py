"""The serving stream's completion polling on CPU, against a fake frame server: a frame in
flight answers wait(ticket, 0) with False, a completed one with True, a failed one raises;
every latency is measured from the frame's own submission to the poll that saw it done."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeServer:
    """Frames complete at given clock times; ticket 'bad' fails."""

    def __init__(self, clock, done_at):
        self.clock, self.done_at = clock, done_at

    def wait(self, ticket, timeout_ms):
        assert timeout_ms == 0
        if ticket == "bad":
            raise RuntimeError("frame failed")
        return self.clock() >= self.done_at[ticket]


def test_latencies_wait_for_completion():
    clk = FakeClock()
    srv = FakeServer(clk, {1: 0.5, 2: 0.05, 3: 2.0})
    tix = [(0.0, 256, 1), (0.01, 512, 2), (0.2, 2048, 3)]
    lat = bench.poll_completions(srv, tix, clock=clk, sleep=clk.sleep, period=0.01)
    got = {r: t for t, r in lat}
    assert [r for _, r in lat] == [512, 256, 2048]  # completion order
    assert got[512] == pytest.approx(0.05 - 0.01, abs=0.011)
    assert got[256] == pytest.approx(0.5, abs=0.011)
    assert got[2048] == pytest.approx(1.8, abs=0.011)
    assert all(t >= 0.0 for t, _ in lat)


def test_failed_frame_raises():
    clk = FakeClock()
    srv = FakeServer(clk, {1: 0.1})
    with pytest.raises(RuntimeError):
        bench.poll_completions(srv, [(0.0, 256, 1), (0.0, 256, "bad")], clock=clk, sleep=clk.sleep)
