"""Parity at the full sizes of the larger workloads, on seeded pixel samples.

* 16,777,216-particle halo mixture (h over ~3 decades), Wendland C2, K=4 D=3,
  4096-entry table, perspective 2048x2048 -- the benchmark's frame;
* 64,000,000-particle dam-break slab (dense graded layer + sparse splash),
  Wendland C4, K=4 D=4, perspective 4096x4096, a high-opacity transfer function.

The oracle computes the sampled rays one by one (FP64, all particles); the CUDA
path renders the same rays through the parity hook (same kernels, no early
termination, so that complete rays are compared).
"""
import pytest

from paper_2401_02896_b300 import synthetic as SY

from test_gpu_parity import _check_rays, _mk  # noqa: F401  (shared checking code of the parity tests)
from _helpers import oracle_lut

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


def test_halo_16m_2048_sampled_pixels(S, ctx):
    P = SY.halo_mixture(16_777_216, a_range=(5e-4, 0.05), seed=SY.BASE_SEED + 2, device="cuda")
    lut = oracle_lut("wendland_c2", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(2048, 2048)
    tf = SY.tf_density(P["value"])
    pix = SY.pixel_sample(2048, 2048, 24, seed=21)
    try:
        wf, wp = _check_rays(S, ctx, ds, lt, P, lut, cam, tf, pix, cand_cap=1 << 16, field_cap=1 << 18)
        print("halo16m: field rel-L2 worst %.3g, pixel worst %.3g" % (wf, wp))
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_dam_break_64m_4096_sampled_pixels(S, ctx):
    P = SY.dam_break_slab(64_000_000)
    lut = oracle_lut("wendland_c4", 4, 4, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(4096, 4096, azimuth_deg=-60.0, elevation_deg=25.0, distance=1.6, center=(0.5, 0.25, 0.3))
    tf = SY.tf_density(P["value"], sigma_scale=500.0)
    pix = SY.pixel_sample(4096, 4096, 16, seed=22)
    try:
        wf, wp = _check_rays(S, ctx, ds, lt, P, lut, cam, tf, pix, cand_cap=1 << 16, field_cap=1 << 18)
        print("dam-break 64M: field rel-L2 worst %.3g, pixel worst %.3g" % (wf, wp))
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)
