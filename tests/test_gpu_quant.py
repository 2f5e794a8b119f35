"""GPU parity of the quantised fixed-point path (precision INT64_QUANT, Sec. 4.2-4.4).

The CUDA path quantises every candidate's knots and difference coefficients
(Sec. 4.3) and runs the coefficient update in exact 64-bit integers inside its
windows; the oracle (``oracle.quant``) quantises the same candidates with
Python integers and sums each interval's coefficients explicitly.  The two
take their rounding decisions from different FP arithmetic (device: FP32
table, FP64 products; oracle: FP64 table), so a knot may land one quantum
apart and a free coefficient differ in its last bits: the field is compared in
relative L2 (1e-5), the pixels per channel (2e-4), like the other modes.
"""
import numpy as np
import pytest

from oracle import quant as Q
from paper_2401_02896_b300 import synthetic as SY

from _helpers import FIELD_REL_L2, PIXEL_ABS, field_rel_l2, oracle_lut

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


def _parts(P):
    return dict(pos=P["pos"], h=P["h"], mass=P["mass"], value=P["value"], density=P["density"])


def _quanta(S, P, kernel, D, lut, cam, pix, margin=2.0):
    """tau and sigma of Sec. 4.4 for 64-bit integers: sigma = A_max / 2^63 with A_max `margin` times
    the largest field value the oracle finds on the sampled rays, tau minimising Q_E for the median
    particle."""
    import oracle

    parts = _parts(P)
    R = oracle.render(parts, lut, cam, SY.tf_bumps(), np.asarray(pix, np.int32), field_cap=1 << 14)
    fmax = 0.0
    for r in range(len(pix)):
        F = R["field"][r][: int(R["stats"][r, 5])]
        if len(F):
            ts = np.linspace(F[0, 0], F[-1, 1], 4001)
            fmax = max(fmax, float(np.abs(oracle.field_eval(F, ts)).max()))
    h_rep = float(np.median(P["h"]))
    pc_rep = float(np.median(oracle.particle_amplitude(parts) / P["h"].astype(np.float64) ** 3))
    ratio = margin * fmax / (float(oracle.kernel_w(kernel, 0.0)) * pc_rep)
    tau_rel, sig_rel, qe = S.sphdvr_quant_params(kernel, D, 64, ratio)
    return tau_rel * h_rep, sig_rel * pc_rep, qe


def _mk(S, ctx, P, lut):
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    lt = S.sphdvr_lut_create(ctx, lut["kernel"], lut["K"], lut["D"], lut["n_lambda"], lut["theta"], lut["pieces"])
    return ds, lt


@pytest.mark.parametrize("kernel,K,D", [("m4", 4, 3), ("m4", 3, 3), ("wendland_c2", 4, 2)])
def test_quantised_rays_match_the_quantised_oracle(S, ctx, kernel, K, D):
    P = SY.uniform_cube()
    lut = oracle_lut(kernel, K, D, 1025)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(32, 32)
    tf = SY.tf_bumps()
    pix = np.concatenate([SY.pixel_sample(32, 32, 14, seed=61), [0, 31, 32 * 31, 32 * 32 - 1]]).astype(np.int32)
    tau, sigma, qe = _quanta(S, P, kernel, D, lut, cam, pix)
    opts = dict(precision="int64_quant", quant_tau=tau, quant_sigma=sigma, ert_eps=0.0)
    try:
        g = S.sphdvr_debug_rays(ctx, ds, lt, cam, tf, opts, pix, cand_cap=4096, field_cap=1 << 14, D=D)
        assert not g["overflow"]
        R = Q.quant_render(_parts(P), lut, cam, tf, pix, tau, sigma)
        worst_f, worst_p = 0.0, 0.0
        for r in range(len(pix)):
            mine = g["field"][r, : int(g["counts"][r, 2])]
            ref = R["field"][r]
            if len(ref) == 0:
                assert np.abs(mine[:, 2:]).max(initial=0.0) == 0.0
                continue
            worst_f = max(worst_f, field_rel_l2(mine, ref, D))
        worst_p = float(np.abs(g["rgba"] - R["rgba"]).max())
        print("quantised %s K=%d D=%d: tau %.3g sigma %.3g Q_E %.2g; field %.3g, pixel %.3g"
              % (kernel, K, D, tau, sigma, qe, worst_f, worst_p))
        assert worst_f <= FIELD_REL_L2
        assert worst_p <= PIXEL_ABS
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_quantised_frame_through_the_render_entry(S, ctx):
    """The full-frame kernel (work queue, 4 warps per CTA) gives the parity hook's pixels and agrees with the
    other drift-free mode, FP32 with re-anchored windows, within the quantisation error.  (The naive FP64
    recurrence is not a reference at scale: its coefficients keep the FP32 rounding residue of every finished
    particle and drift, Sec. 4.1.)  One length quantum serves all particles (Sec. 4.4), so the data set has
    one smoothing length; sigma bounds the field with a margin of 4 over the sampled rays' maximum."""
    import torch

    P = SY.uniform_cube(4000, h=0.05, seed=SY.BASE_SEED + 41)
    lut = oracle_lut("m4", 4, 3, 1025)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(64, 48)
    tf = SY.tf_bumps()
    pix = SY.pixel_sample(64, 48, 12, seed=62)
    tau, sigma, qe = _quanta(S, P, "m4", 3, lut, cam, pix, margin=4.0)
    opts = dict(precision="int64_quant", quant_tau=tau, quant_sigma=sigma, ert_eps=0.0)
    try:
        a = torch.zeros((48, 64, 4), dtype=torch.float32, device="cuda")
        b = torch.zeros_like(a)
        S.sphdvr_render(ctx, ds, lt, cam, tf, opts, a.data_ptr())
        S.sphdvr_render(ctx, ds, lt, cam, tf, dict(ert_eps=0.0), b.data_ptr())
        torch.cuda.synchronize()
        g = S.sphdvr_debug_rays(ctx, ds, lt, cam, tf, opts, pix)
        img = a.cpu().numpy().reshape(-1, 4)
        assert np.abs(img[pix] - g["rgba"]).max() <= 1e-6
        assert float((a - b).abs().max()) <= 1e-3
        assert a[..., 3].max().item() > 0.05
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_quantised_batch_equals_separate_frames(S, ctx):
    """The batched launch (one work queue over several frames) gives the separate frames' quantised images."""
    import torch

    P = SY.uniform_cube(2000, h=0.06, seed=SY.BASE_SEED + 42)
    lut = oracle_lut("m4", 4, 3, 1025)
    ds, lt = _mk(S, ctx, P, lut)
    cams = [SY.orbit_camera(40, 56, azimuth_deg=30.0 * i) for i in range(3)] + [SY.ortho_camera_z(48, 32)]
    tau, sigma, _ = _quanta(S, P, "m4", 3, lut, cams[0], SY.pixel_sample(40, 56, 8, seed=63), margin=4.0)
    opts = dict(precision="int64_quant", quant_tau=tau, quant_sigma=sigma)
    try:
        ref = []
        for c in cams:
            o = torch.zeros((c["height"], c["width"], 4), dtype=torch.float32, device="cuda")
            S.sphdvr_render(ctx, ds, lt, c, SY.tf_bumps(), opts, o.data_ptr())
            ref.append(o)
        got = [torch.full_like(o, -1.0) for o in ref]
        S.sphdvr_render_batch(ctx, ds, lt, cams, SY.tf_bumps(), opts, [o.data_ptr() for o in got])
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
        assert max(o[..., 3].max().item() for o in ref) > 0.05
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_quantised_option_errors(S, ctx):
    import torch

    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 1025)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(16, 16)
    o = torch.zeros((16, 16, 4), dtype=torch.float32, device="cuda")
    try:
        for bad in (dict(precision="int64_quant"), dict(precision="int64_quant", quant_tau=1e-4),
                    dict(precision="int64_quant", quant_tau=-1.0, quant_sigma=1e-12),
                    dict(precision="int64_quant", quant_tau=float("inf"), quant_sigma=1e-12)):
            with pytest.raises(S.SphdvrError) as e:
                S.sphdvr_render(ctx, ds, lt, cam, SY.tf_bumps(), bad, o.data_ptr())
            assert e.value.status == S.EINVAL
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def _field_max(P, lut, cam, pix):
    import oracle

    R = oracle.render(_parts(P), lut, cam, SY.tf_bumps(), np.asarray(pix, np.int32), field_cap=1 << 15)
    fmax = 0.0
    for r in range(len(pix)):
        F = R["field"][r][: int(R["stats"][r, 5])]
        if len(F):
            ts = np.linspace(F[0, 0], F[-1, 1], 8001)
            fmax = max(fmax, float(np.abs(oracle.field_eval(F, ts)).max()))
    return fmax


def test_dataset_quanta_bound_the_field_and_render_like_the_oracle(S, ctx):
    """sphdvr_dataset_quant_params: a_max bounds the field (on uniform and halo data), sigma = a_max / 2^63,
    tau is Q_E's minimiser for the median particle, and frames rendered with these quanta match the oracle's."""
    import oracle

    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 1025)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(32, 32)
    tf = SY.tf_bumps()
    pix = SY.pixel_sample(32, 32, 12, seed=64)
    try:
        qp = S.sphdvr_dataset_quant_params(ctx, ds, "m4", 3, 64)
        fmax = _field_max(P, lut, cam, pix)
        assert fmax <= qp["a_max"] <= 100 * fmax
        assert abs(qp["sigma"] * 2.0 ** 63 / qp["a_max"] - 1) < 1e-12
        # the representative particle: the upper medians (element n // 2 in order) of h and c
        n = len(P["h"])
        h_med = float(np.sort(P["h"].astype(np.float64))[n // 2])
        amp = P["mass"].astype(np.float32) * P["value"].astype(np.float32) / P["density"].astype(np.float32)
        c_med = float(np.sort(amp.astype(np.float64) / P["h"].astype(np.float64) ** 3)[n // 2])
        t_rel, s_rel, qe = S.sphdvr_quant_params("m4", 3, 64, qp["a_max"] / (oracle.kernel_w("m4", 0.0) * c_med))
        assert abs(qp["tau"] / (t_rel * h_med) - 1) < 1e-5 and abs(qp["qe"] / qe - 1) < 1e-5
        opts = dict(precision="int64_quant", quant_tau=qp["tau"], quant_sigma=qp["sigma"], ert_eps=0.0)
        g = S.sphdvr_debug_rays(ctx, ds, lt, cam, tf, opts, pix)
        R = Q.quant_render(_parts(P), lut, cam, tf, pix, qp["tau"], qp["sigma"])
        assert np.abs(g["rgba"] - R["rgba"]).max() <= PIXEL_ABS
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)
    P2 = SY.halo_mixture(60_000, seed=SY.BASE_SEED + 43)
    lut2 = oracle_lut("wendland_c2", 4, 3, 1025)
    ds2, lt2 = _mk(S, ctx, P2, lut2)
    try:
        qp2 = S.sphdvr_dataset_quant_params(ctx, ds2, "wendland_c2", 3, 64)
        cam2 = SY.orbit_camera(64, 64)
        assert _field_max(P2, lut2, cam2, SY.pixel_sample(64, 64, 16, seed=65)) <= qp2["a_max"]
    finally:
        S.sphdvr_dataset_free(ds2)
        S.sphdvr_lut_free(lt2)


def test_quanta_too_fine_are_flagged(S, ctx):
    """A value quantum far below the field's bound makes the particles' integers exceed 2^62: flag bit 4."""
    import torch

    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 1025)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(16, 16)
    o = torch.zeros((16, 16, 4), dtype=torch.float32, device="cuda")
    try:
        qp = S.sphdvr_dataset_quant_params(ctx, ds, "m4", 3, 64)
        S.sphdvr_render(ctx, ds, lt, cam, SY.tf_bumps(),
                        dict(precision="int64_quant", quant_tau=qp["tau"], quant_sigma=qp["sigma"]), o.data_ptr())
        torch.cuda.synchronize()
        assert not S.sphdvr_frame_stats(ctx)["overflow"] & 16
        S.sphdvr_render(ctx, ds, lt, cam, SY.tf_bumps(),
                        dict(precision="int64_quant", quant_tau=qp["tau"], quant_sigma=qp["sigma"] * 1e-9),
                        o.data_ptr(), allow_overflow=True)
        torch.cuda.synchronize()
        assert S.sphdvr_frame_stats(ctx)["overflow"] & 16
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)
