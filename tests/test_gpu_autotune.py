"""The autotuner (sphdvr_autotune): parameters chosen by timing real frames still render the image the
oracle computes, and the JSON-lines cache returns the same choice without timing again."""
import json

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


def test_tuned_options_render_like_the_oracle_and_are_cached(S, tmp_path):
    import torch

    ctx = S.sphdvr_create(0)
    P = SY.halo_mixture(150_000, seed=SY.BASE_SEED + 41)
    lut = oracle_lut("wendland_c2", 4, 3, 4096)
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    lt = S.sphdvr_lut_create(ctx, "wendland_c2", 4, 3, 4096, lut["theta"], lut["pieces"])
    cam = SY.orbit_camera(200, 150)
    tf = SY.tf_density(P["value"])
    cache = str(tmp_path / "autotune.jsonl")
    try:
        tuned, (ms0, ms1) = S.sphdvr_autotune(ctx, ds, lt, cam, tf, dict(ert_eps=0.0), cache_path=cache)
        assert 0 < ms1 <= ms0 * 1.05, (ms0, ms1)
        assert 0 <= tuned["ctas_per_sm"] <= 3 and 1.0 <= tuned["window_h"] <= 2.0, tuned
        lines = [json.loads(x) for x in open(cache)]
        assert len(lines) == 1 and lines[0]["ctas_per_sm"] == tuned["ctas_per_sm"]
        # a cache hit returns the same choice and appends nothing
        again, ms_again = S.sphdvr_autotune(ctx, ds, lt, cam, tf, dict(ert_eps=0.0), cache_path=cache)
        assert again["ctas_per_sm"] == tuned["ctas_per_sm"] and again["window_h"] == pytest.approx(tuned["window_h"])
        assert len(open(cache).readlines()) == 1 and ms_again[1] == pytest.approx(ms1, rel=1e-3)
        # the tuned frame matches the oracle and the default frame
        out = torch.zeros((150, 200, 4), dtype=torch.float32, device="cuda")
        ref = torch.zeros_like(out)
        S.sphdvr_render(ctx, ds, lt, cam, tf, tuned, out.data_ptr())
        S.sphdvr_render(ctx, ds, lt, cam, tf, dict(ert_eps=0.0), ref.data_ptr())
        torch.cuda.synchronize()
        assert (out - ref).abs().max().item() <= 1e-5
        pix = SY.pixel_sample(200, 150, 40, seed=81)
        R = oracle.render(P, lut, cam, tf, pix)
        assert np.abs(out.cpu().numpy().reshape(-1, 4)[pix] - R["rgba"]).max() <= PIXEL_ABS
        with pytest.raises(S.SphdvrError) as e:
            S.sphdvr_autotune(ctx, ds, lt, cam, tf, dict(precision="fp64_naive"))
        assert e.value.status == S.EINVAL
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)
        S.sphdvr_destroy(ctx)
