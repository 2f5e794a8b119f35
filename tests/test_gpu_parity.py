"""GPU parity of the CUDA path (through the C ABI) against the oracle.

Every input is seeded and synthetic.  Each test renders with the library and
with the oracle on the same particles, table, camera and transfer function and
checks: candidate sets identical apart from particles within 1e-6 h of
tangency; field per ray within relative L2 1e-5; composited pixels within
2e-4 per channel.
"""

import numpy as np
import pytest

import oracle
from paper_2401_02896_b300 import synthetic as SY

from _helpers import FIELD_REL_L2, PIXEL_ABS, field_rel_l2, oracle_lut, tangency_band

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


def _mk(S, ctx, P, lut):
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    lt = S.sphdvr_lut_create(ctx, lut["kernel"], lut["K"], lut["D"], lut["n_lambda"], lut["theta"], lut["pieces"])
    return ds, lt


def _orc_particles(P):
    return dict(pos=P["pos"], h=P["h"], mass=P["mass"], value=P["value"], density=P["density"])


def _check_rays(S, ctx, ds, lt, P, lut, cam, tf, pix, opts=None, cand_cap=4096, field_cap=1 << 15, q=2.0,
                field_tol=FIELD_REL_L2, pixel_tol=PIXEL_ABS, ert=1e-5):
    D = lut["D"]
    opts = dict(opts or {})
    opts.setdefault("ert_eps", 0.0)  # compare complete rays with the oracle (no early termination)
    g = S.sphdvr_debug_rays(ctx, ds, lt, cam, tf, opts, pix, cand_cap=cand_cap, field_cap=field_cap, D=D)
    assert not g["overflow"], g["counts"][:, 3].max()
    R = oracle.render(_orc_particles(P), lut, cam, tf, pix, cand_cap=cand_cap, field_cap=field_cap)
    assert not R["truncated"]
    worst_field = 0.0
    for r, p in enumerate(pix):
        o, v = oracle.camera_ray(cam, int(p))
        nc_g, nc_o = int(g["counts"][r, 0]), int(R["stats"][r, 0])
        gc = set(g["cand_ids"][r, :nc_g].tolist())
        oc = set(R["cand_ids"][r, :nc_o].tolist())
        band = tangency_band(P, o, v, q, np.array(sorted(gc ^ oc), dtype=np.int64)) if gc != oc else set()
        assert gc - band == oc - band, (p, len(gc ^ oc))
        if nc_o == 0:
            assert np.all(g["rgba"][r] == 0)
            continue
        nf_g, nf_o = int(g["counts"][r, 2]), int(R["stats"][r, 5])
        e = field_rel_l2(g["field"][r, :nf_g], R["field"][r, :nf_o], D)
        worst_field = max(worst_field, e)
        assert e <= field_tol, (p, e)
    err = np.abs(g["rgba"].astype(np.float64) - R["rgba"]).max()
    assert err <= pixel_tol, err
    return worst_field, err


def test_small_uniform_full_frame_debug(S, ctx):
    """1,000 uniform particles, h = 0.08, cubic B-spline, K=4 D=3, ortho 64x64 along +z, every pixel."""
    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(64, 64)
    tf = SY.tf_bumps()
    try:
        wf, wp = _check_rays(S, ctx, ds, lt, P, lut, cam, tf, np.arange(64 * 64))
        print("field rel-L2 worst %.3g, pixel worst %.3g" % (wf, wp))
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_small_uniform_full_frame_render(S, ctx):
    """The production render path (not the debug hook) on the same frame: every pixel within 2e-4."""
    import torch

    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(64, 64)
    tf = SY.tf_bumps()
    try:
        out = torch.zeros((64, 64, 4), dtype=torch.float32, device="cuda")
        S.sphdvr_render(ctx, ds, lt, cam, tf, dict(ert_eps=0.0), out.data_ptr())
        torch.cuda.synchronize()
        img = out.cpu().numpy().reshape(-1, 4).astype(np.float64)
        R = oracle.render(_orc_particles(P), lut, cam, tf, np.arange(64 * 64))
        assert np.abs(img - R["rgba"]).max() <= PIXEL_ABS
        st = S.sphdvr_frame_stats(ctx)
        assert st["rays"] == 64 * 64
        assert st["segments"] == int(R["stats"][:, 0].sum())
        assert st["knots"] == int(R["stats"][:, 1].sum())
        assert st["overflow"] == 0
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_clustered_1m_sampled_pixels(S, ctx):
    """1M-particle halo mixture, Wendland C2, K=4 D=3, perspective 1024x1024: 48 seeded pixels."""
    P = SY.halo_mixture(1_000_000)
    lut = oracle_lut("wendland_c2", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(1024, 1024)
    tf = SY.tf_density(P["value"])
    pix = SY.pixel_sample(1024, 1024, 48, seed=11)
    try:
        wf, wp = _check_rays(S, ctx, ds, lt, P, lut, cam, tf, pix, cand_cap=16384, field_cap=1 << 17)
        print("field rel-L2 worst %.3g, pixel worst %.3g" % (wf, wp))
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


@pytest.mark.parametrize("K,D", [(4, 1), (4, 2), (4, 4), (3, 3), (2, 3), (1, 4)])
def test_small_uniform_degree_and_pieces_sweep(S, ctx, K, D):
    """Other (K, D): odd K has no middle knot, K = 1 a single even piece."""
    P = SY.uniform_cube()
    lut = oracle_lut("m4", K, D, 1025)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(24, 24)
    tf = SY.tf_bumps()
    try:
        _check_rays(S, ctx, ds, lt, P, lut, cam, tf, np.arange(24 * 24))
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_perspective_inside_volume_with_t_near(S, ctx):
    """Eye inside the particle cloud, t_near = 0.25: clipping of the first pieces and knots behind the eye."""
    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(32, 24, azimuth_deg=15, elevation_deg=10, distance=0.35, fovy_deg=60, t_near=0.25)
    tf = SY.tf_bumps()
    try:
        _check_rays(S, ctx, ds, lt, P, lut, cam, tf, np.arange(32 * 24))
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_wendland_c4_degree4(S, ctx):
    P = SY.uniform_cube(2000, h=0.06, seed=SY.BASE_SEED + 9)
    lut = oracle_lut("wendland_c4", 4, 4, 2049)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(32, 32, azimuth_deg=50, elevation_deg=35, distance=1.6)
    tf = SY.tf_bumps(lo=0.0, hi=2.0)
    try:
        _check_rays(S, ctx, ds, lt, P, lut, cam, tf, np.arange(32 * 32))
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_precision_modes_order(S, ctx):
    """The plain recurrence (Sec. 4.1) drifts; re-anchored FP32 windows do not."""
    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(32, 32)
    tf = SY.tf_bumps()
    pix = np.arange(32 * 32)
    R = oracle.render(_orc_particles(P), lut, cam, tf, pix, field_cap=4096)
    worst = {}
    try:
        for prec in ("fp32_anchored", "fp32_naive", "fp64_naive"):
            g = S.sphdvr_debug_rays(ctx, ds, lt, cam, tf, dict(precision=prec, ert_eps=0.0), pix, field_cap=4096,
                                    D=3)
            e = [field_rel_l2(g["field"][r, :g["counts"][r, 2]], R["field"][r, :R["stats"][r, 5]], 3)
                 for r in range(len(pix)) if R["stats"][r, 0]]
            worst[prec] = max(e)
        assert worst["fp32_anchored"] <= FIELD_REL_L2
        # both plain recurrences drift (knot positions are FP32 offsets either way)
        assert worst["fp32_naive"] > 10 * worst["fp32_anchored"]
        assert worst["fp64_naive"] > 10 * worst["fp32_anchored"]
        print(worst)
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_early_ray_termination_bound(S, ctx):
    """Opaque transfer function: terminated rays differ from the complete oracle by at most ert_eps."""
    import torch

    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(32, 32)
    tf = SY.tf_bumps(sigma_scale=40.0)
    eps = 1e-4
    try:
        out = torch.zeros((32, 32, 4), dtype=torch.float32, device="cuda")
        S.sphdvr_render(ctx, ds, lt, cam, tf, dict(ert_eps=eps), out.data_ptr())
        torch.cuda.synchronize()
        st = S.sphdvr_frame_stats(ctx)
        assert st["ert_rays"] > 0
        R = oracle.render(_orc_particles(P), lut, cam, tf, np.arange(32 * 32))
        err = np.abs(out.cpu().numpy().reshape(-1, 4) - R["rgba"]).max()
        assert err <= eps + PIXEL_ABS, err
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_library_tables_end_to_end(S, ctx):
    """Each side with its own table (library builder vs oracle builder): pixels within 2e-4."""
    import torch

    P = SY.uniform_cube()
    th, pc, _ = S.sphdvr_lut_build("m4", 4, 3, 2049)
    lt = S.sphdvr_lut_create(ctx, "m4", 4, 3, 2049, th, pc)
    ds = S.sphdvr_dataset_create(ctx, P["pos"], P["h"], P["mass"], P["density"], P["value"])
    cam = SY.ortho_camera_z(32, 32)
    tf = SY.tf_bumps()
    try:
        out = torch.zeros((32, 32, 4), dtype=torch.float32, device="cuda")
        S.sphdvr_render(ctx, ds, lt, cam, tf, dict(ert_eps=0.0), out.data_ptr())
        torch.cuda.synchronize()
        R = oracle.render(_orc_particles(P), oracle_lut("m4", 4, 3, 2049), cam, tf, np.arange(32 * 32))
        assert np.abs(out.cpu().numpy().reshape(-1, 4) - R["rgba"]).max() <= PIXEL_ABS
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_no_particles_in_view_is_transparent(S, ctx):
    import torch

    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(16, 16, lo=(3.0, 3.0), hi=(4.0, 4.0))
    try:
        out = torch.full((16, 16, 4), 7.0, dtype=torch.float32, device="cuda")
        S.sphdvr_render(ctx, ds, lt, cam, SY.tf_bumps(), None, out.data_ptr())
        torch.cuda.synchronize()
        assert torch.all(out == 0)
        assert S.sphdvr_frame_stats(ctx)["segments"] == 0
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_invalid_inputs_are_rejected(S, ctx):
    P = SY.uniform_cube(64)
    bad = dict(P)
    bad["h"] = P["h"].copy()
    bad["h"][5] = 0.0
    with pytest.raises(S.SphdvrError) as e:
        S.sphdvr_dataset_create(ctx, bad["pos"], bad["h"], bad["mass"], bad["density"], bad["value"])
    assert e.value.status == S.EINVAL
    bad["h"][5] = np.nan
    with pytest.raises(S.SphdvrError):
        S.sphdvr_dataset_create(ctx, bad["pos"], bad["h"], bad["mass"], bad["density"], bad["value"])
    lut = oracle_lut("m4", 4, 3, 257)
    ds, lt = _mk(S, ctx, P, lut)
    try:
        cam = SY.ortho_camera_z(8, 8)
        tf = SY.tf_bumps()
        import torch

        out = torch.zeros((8, 8, 4), dtype=torch.float32, device="cuda")
        for c in [dict(cam, width=0), dict(cam, target=cam["eye"]), dict(cam, half_w=0.0)]:
            with pytest.raises(S.SphdvrError) as e:
                S.sphdvr_render(ctx, ds, lt, c, tf, None, out.data_ptr())
            assert e.value.status == S.EINVAL
        for t in [dict(tf, lo=2.0, hi=1.0), dict(tf, rgba=tf["rgba"][:1])]:
            with pytest.raises(S.SphdvrError) as e:
                S.sphdvr_render(ctx, ds, lt, cam, t, None, out.data_ptr())
            assert e.value.status == S.EINVAL
        with pytest.raises(S.SphdvrError):
            S.sphdvr_render(ctx, ds, lt, cam, tf, dict(precision=7), out.data_ptr())
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_static_and_dynamic_schedules_agree(S, ctx):
    """The static ray stride and the atomic work queue render the same image (same per-ray arithmetic)."""
    import torch

    P = SY.halo_mixture(100_000, seed=SY.BASE_SEED + 17)
    lut = oracle_lut("wendland_c2", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(120, 88)
    tf = SY.tf_density(P["value"])
    try:
        a = torch.zeros((88, 120, 4), dtype=torch.float32, device="cuda")
        b = torch.zeros_like(a)
        S.sphdvr_render(ctx, ds, lt, cam, tf, dict(persistent=0), a.data_ptr())
        S.sphdvr_render(ctx, ds, lt, cam, tf, dict(persistent=1), b.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        assert a[..., 3].max().item() > 0.05
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_reinitialisation_knots(S, ctx):
    """FP32 recurrence with reinitialisation knots every reinit_dt along t (Sec. 4.1): dense knots bound the
    drift like re-anchored windows, knots farther apart than the rays let it grow as in the plain recurrence."""
    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.ortho_camera_z(32, 32)
    tf = SY.tf_bumps()
    pix = np.arange(32 * 32)
    R = oracle.render(_orc_particles(P), lut, cam, tf, pix, field_cap=4096)

    def worst(opts):
        g = S.sphdvr_debug_rays(ctx, ds, lt, cam, tf, dict(opts, ert_eps=0.0), pix, field_cap=4096, D=3)
        return max(field_rel_l2(g["field"][r, :g["counts"][r, 2]], R["field"][r, :R["stats"][r, 5]], 3)
                   for r in range(len(pix)) if R["stats"][r, 0])

    try:
        dense = worst(dict(precision="fp32_reinit", reinit_dt=0.02))
        sparse = worst(dict(precision="fp32_reinit", reinit_dt=100.0))
        naive = worst(dict(precision="fp32_naive"))
        print(dense, sparse, naive)
        assert dense <= FIELD_REL_L2
        assert sparse > 10 * dense
        # without reinitialisation the drift is the plain recurrence's (its size depends on the order of
        # the FP32 operations, which differs between the kernels that run the two modes)
        assert naive / 3 <= sparse <= 3 * naive
        with pytest.raises(S.SphdvrError):
            S.sphdvr_debug_rays(ctx, ds, lt, cam, tf, dict(precision="fp32_reinit"), pix[:4], D=3)
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_table_file_load_renders_like_create(S, ctx, tmp_path):
    """A table saved to a file and loaded back (sphdvr_lut_load) renders the same image bit for bit."""
    import torch

    P = SY.uniform_cube()
    lut = oracle_lut("m4", 4, 3, 1025)
    path = str(tmp_path / "m4.lut")
    S.sphdvr_lut_save(path, "m4", 4, 3, 1025, lut["theta"], lut["pieces"], lut["err"])
    ds, lt = _mk(S, ctx, P, lut)
    lt2 = S.sphdvr_lut_load(ctx, path)
    cam = SY.orbit_camera(64, 48)
    tf = SY.tf_bumps()
    try:
        a = torch.zeros((48, 64, 4), dtype=torch.float32, device="cuda")
        b = torch.full_like(a, -1.0)
        S.sphdvr_render(ctx, ds, lt, cam, tf, None, a.data_ptr())
        S.sphdvr_render(ctx, ds, lt2, cam, tf, None, b.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(a, b) and a[..., 3].max().item() > 0.05
    finally:
        S.sphdvr_lut_free(lt2)
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)


def test_capacity_fallback_renders_the_same_image(S, ctx):
    """Rays that overflow the frame pass's per-ray capacity (forced small here) are abandoned, listed and
    rendered again by the fallback pass with larger capacities: the image matches the default frame and the
    oracle, and every ray is counted once.  (A smaller capacity also makes a ray flush its new particles
    earlier, which moves window ends: the two images agree to rounding, not bit for bit.)"""
    import torch

    P = SY.halo_mixture(100_000, seed=SY.BASE_SEED + 17)
    lut = oracle_lut("wendland_c2", 4, 3, 4096)
    ds, lt = _mk(S, ctx, P, lut)
    cam = SY.orbit_camera(72, 56)
    tf = SY.tf_density(P["value"])
    try:
        a = torch.zeros((56, 72, 4), dtype=torch.float32, device="cuda")
        b = torch.full_like(a, -1.0)
        S.sphdvr_render(ctx, ds, lt, cam, tf, dict(ert_eps=0.0), a.data_ptr())
        torch.cuda.synchronize()
        sa = S.sphdvr_frame_stats(ctx)
        S.sphdvr_render(ctx, ds, lt, cam, tf, dict(ert_eps=0.0, ray_capacity=64), b.data_ptr())
        torch.cuda.synchronize()
        sb = S.sphdvr_frame_stats(ctx)
        assert sa["max_table"] > 64  # the small capacity does not hold every ray
        assert sa["overflow"] == 0 and sb["overflow"] == 0, (sa["overflow"], sb["overflow"])
        assert (a - b).abs().max().item() <= 1e-5
        for k in ("rays", "segments", "knots"):
            assert sa[k] == sb[k], k
        pix = SY.pixel_sample(72, 56, 40, seed=71)
        R = oracle.render(_orc_particles(P), lut, cam, tf, pix)
        assert np.abs(b.cpu().numpy().reshape(-1, 4)[pix] - R["rgba"]).max() <= PIXEL_ABS
        with pytest.raises(S.SphdvrError):
            S.sphdvr_render(ctx, ds, lt, cam, tf, dict(ray_capacity=8), b.data_ptr())
    finally:
        S.sphdvr_dataset_free(ds)
        S.sphdvr_lut_free(lt)
