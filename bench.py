#!/usr/bin/env python
"""Benchmark of the per-ray higher-order SPH field reconstruction + DVR path.

Default workload (one B300): 16,777,216 particles from a Plummer-halo mixture
with a uniform background (h spans about three decades), Wendland C2 kernel,
K = 4 pieces of degree D = 3 per particle, a 4096-entry table, perspective
camera 2048 x 2048.  One step = one frame rendered through the library
(binning + render kernel); the particle set (384 MB, larger than L2) is
resident.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sphdvr|reference]

Under torchrun (N > 1) every rank renders its own frames (different cameras)
of the same resident data: weak scaling, no data-path collective; the value
is all ranks' rays over the slowest rank's time.  ``--impl reference`` times
the FP64 CPU oracle on a bounded sample of the same frame's pixels.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2401_02896_b300 import synthetic as SY  # noqa: E402

WORKLOADS = {
    "halo16m": dict(n=16_777_216, a_range=(5e-4, 0.05), seed=SY.BASE_SEED + 2, kernel="wendland_c2", K=4, D=3,
                    n_lambda=4096, res=2048,
                    desc="halo mixture 16,777,216 particles (64 Plummer halos + 20% uniform background, "
                         "h = expected 32-NN distance, ~3 decades), Wendland C2, K=4, D=3, 4096-entry table, "
                         "perspective 2048x2048, FP32 anchored"),
    # the same positions with h = the true 32nd-neighbour distance and the SPH density estimate as value
    "halo16m_knn": dict(n=16_777_216, a_range=(5e-4, 0.05), seed=SY.BASE_SEED + 2, knn=True, kernel="wendland_c2",
                        K=4, D=3, n_lambda=4096, res=2048,
                        desc="halo mixture 16,777,216 particles (64 Plummer halos + 20% uniform background), "
                             "h = distance to the 32nd nearest neighbour (k-d tree), value = SPH density estimate, "
                             "Wendland C2, K=4, D=3, 4096-entry table, perspective 2048x2048, FP32 anchored"),
    "halo1m": dict(n=1_000_000, a_range=(5e-3, 0.05), seed=SY.BASE_SEED + 1, kernel="wendland_c2", K=4, D=3,
                   n_lambda=4096, res=1024,
                   desc="halo mixture 1,000,000 particles, Wendland C2, K=4, D=3, perspective 1024x1024"),
    # the large single frame: dam-break slab, high-opacity transfer function (early ray termination)
    "slab64m": dict(n=64_000_000, slab=True, kernel="wendland_c4", K=4, D=4, n_lambda=4096, res=4096, sigma_scale=500.0,
                    desc="dam-break slab 64,000,000 particles (dense graded layer + 5% splash, h 1e-4..1e-2), "
                         "Wendland C4, K=4, D=4, 4096-entry table, perspective 4096x4096, transfer function "
                         "sigma x500 (early ray termination), FP32 anchored"),
}

# DRAM bytes (read + write) of one frame-pass launch of the render kernel, from the
# ncu capture named in profiles/ (launches_halo16m_2048.md) of the kernel as it is in
# this tree, keyed by (workload, image size, precision, window_h); None where no
# capture of the current kernel and options exists.
PROFILED_DRAM_BYTES = {
    ("halo16m", 2048, "fp32_anchored", 2.0): 8.46e9 + 256.28e9,
}


def replica_rate(total_ms, rays, dist=None, device="cpu"):
    """Whole-job rate of N replicas (one frame stream per rank, no data-path collective):
    (slowest rank's time in ms, all ranks' rays / that time in Mrays/s).  The only
    collectives are a MAX over the ranks' times and a SUM of their rays."""
    t_max, rays_all = float(total_ms), float(rays)
    if dist is not None:
        import torch

        t = torch.tensor([t_max], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        r = torch.tensor([rays_all], dtype=torch.float64, device=device)
        dist.all_reduce(r, op=dist.ReduceOp.SUM)
        t_max, rays_all = float(t.item()), float(r.item())
    return t_max, rays_all / (t_max / 1e3) / 1e6


def flops_per_segment(K, D):
    """Algorithmic FP32 operations per particle-ray segment (an FMA counts 2), counted from the
    arithmetic the render kernel performs on its common path:
      candidate test 20 (chi - o, t = p.v, w = p - t v, |w|^2 against (q h)^2), table entry and
      amplitude 10;
      per knot (K + 1 per segment): its position 2; its difference coefficients 2D + 1
      (a h^-3 s_kd / h^d); the coefficient update of Sec. 2, a Taylor shift D(D + 1) plus D adds;
      per piece (one per knot) the compositing of Sec. 1 on one transfer-function cell: the end value
      2D, the curvature bound 3D, two cell lookups 4, optical depth 3(D + 1) + 2, and two
      Gauss-Legendre nodes of 3(D + 1) + 2D + 22 each (field, optical depth, exp, emission in RGB)."""
    per_knot = 2 + (2 * D + 1) + D * (D + 1) + D
    per_piece = 2 * D + 3 * D + 4 + 3 * (D + 1) + 2 + 2 * (3 * (D + 1) + 2 * D + 22)
    return 30 + (K + 1) * (per_knot + per_piece)


def clocks_start(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def clocks_stop(proc, f, path, device):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        c = [x.strip() for x in line.split(",")]
        if len(c) < 9 or c[0] != str(device):
            continue
        try:
            sm.append(float(c[1]))
            mx = max(mx, float(c[2]))
        except ValueError:
            continue
        for n, v in zip(names, c[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return None
    return dict(sm_mhz=float(np.median(sm)), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(sm))


def make_inputs(w, device):
    if w.get("slab"):
        P = SY.dam_break_slab(w["n"])
    elif w.get("knn"):
        P = SY.halo_mixture_knn(w["n"], a_range=w["a_range"], seed=w["seed"])
    else:
        P = SY.halo_mixture(w["n"], a_range=w["a_range"], seed=w["seed"], device=device)
    tf = SY.tf_density(P["value"], sigma_scale=w.get("sigma_scale", 1.0)) if w.get("sigma_scale") else \
        SY.tf_density(P["value"])
    return P, tf


def camera_for(w, rank, step=0):
    if w.get("slab"):
        return SY.orbit_camera(w["res"], w["res"], azimuth_deg=-60.0 + 7.0 * rank, elevation_deg=25.0, distance=1.6,
                               center=(0.5, 0.25, 0.3))
    return SY.orbit_camera(w["res"], w["res"], azimuth_deg=30.0 + 7.0 * rank, elevation_deg=20.0)


def log_dir():
    """Directory for the run's side files (clock samples, autotune cache): $SPHDVR_BENCH_LOG_DIR or the temp dir."""
    return os.environ.get("SPHDVR_BENCH_LOG_DIR") or tempfile.gettempdir()


def plain_vs_served(S, torch, ctx, ds, lut, tf, opts, dev, stream, n=16, sizes=(128, 256, 512), seed=4321):
    """The same mixed request set rendered (a) in the plain form -- one render launch per frame with a static
    ray schedule (persistent=0), frames one after another -- and (b) through the frame server -- two worker
    streams, the persistent work queue, compatible requests batched into one launch -- all requests queued at
    once.  Wall time from the first request to the last image; rays/s of each form and their ratio."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n):
        r_ = int(rng.choice(sizes))
        cams.append(SY.orbit_camera(r_, r_, azimuth_deg=360 * rng.random(), elevation_deg=-40 + 80 * rng.random()))
    rays = sum(c["width"] * c["height"] for c in cams)
    a_out = [torch.empty((c["height"], c["width"], 4), dtype=torch.float32, device=dev) for c in cams]
    b_out = [torch.empty_like(o) for o in a_out]
    plain = dict(opts, persistent=0)
    S.sphdvr_render(ctx, ds, lut, cams[0], tf, plain, a_out[0].data_ptr(), stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, o in zip(cams, a_out):
        S.sphdvr_render(ctx, ds, lut, c, tf, plain, o.data_ptr(), stream=stream)
        torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    srv = S.Server(ctx, 16 << 30, max_inflight=2)
    t0 = time.perf_counter()
    tickets = [srv.submit(ds, lut, c, tf, dict(opts, persistent=1), o.data_ptr()) for c, o in zip(cams, b_out)]
    for t_ in tickets:
        srv.wait(t_, -1)
    t_served = time.perf_counter() - t0
    bs = srv.batch_stats()
    srv.destroy()
    diff = max(float((a - b).abs().max()) for a, b in zip(a_out, b_out))
    return dict(requests=n, sizes=list(sizes), rays=rays, plain_ms=t_plain * 1e3, served_ms=t_served * 1e3,
                plain_mrays_per_s=rays / t_plain / 1e6, served_mrays_per_s=rays / t_served / 1e6,
                ratio=t_plain / t_served, served_launches=bs["launches"], largest_batch=bs["largest"],
                max_pixel_diff=diff,
                note="plain: one sphdvr_render per frame, static ray schedule, synchronised frame by frame; served: "
                     "frame server, 2 workers, work queue, batched launches, all requests queued at once; wall time")


def cpu_oracle_rate(P, w, tf, n_pix, seed, threads=None):
    """Oracle (FP64, C + OpenMP) rays/s on a seeded sample of pixels of the frame."""
    import oracle

    if threads:
        oracle.set_threads(threads)
    lut = oracle.lut_build(w["kernel"], w["K"], w["D"], w["n_lambda"])
    cam = camera_for(w, 0)
    pix = SY.pixel_sample(cam["width"], cam["height"], n_pix, seed)
    part = dict(pos=P["pos"], h=P["h"], mass=P["mass"], value=P["value"], density=P["density"])
    t = time.perf_counter()
    R = oracle.render(part, lut, cam, tf, pix)
    dt = time.perf_counter() - t
    return dict(rays_per_s=n_pix / dt, seconds=dt, segments=int(R["stats"][:, 0].sum()), cores=oracle.num_threads(),
                lut=lut, part=part, cam=cam)


def run_reference(args, w, rank, world):
    """The oracle as it stands, on the host cores: each step a 16-pixel sample of the frame."""
    if rank != 0:
        return
    import oracle

    P, tf = make_inputs(w, None)
    lut = oracle.lut_build(w["kernel"], w["K"], w["D"], w["n_lambda"])
    part = dict(pos=P["pos"], h=P["h"], mass=P["mass"], value=P["value"], density=P["density"])
    cam = camera_for(w, 0)
    per_step = 16
    for i in range(args.warmup):
        oracle.render(part, lut, cam, tf, SY.pixel_sample(cam["width"], cam["height"], per_step, 1000 + i))
    t = time.perf_counter()
    segs = 0
    for i in range(args.steps):
        R = oracle.render(part, lut, cam, tf, SY.pixel_sample(cam["width"], cam["height"], per_step, 2000 + i))
        segs += int(R["stats"][:, 0].sum())
    dt = time.perf_counter() - t
    mrays = per_step * args.steps / dt / 1e6
    line = dict(metric="Mrays/s", value=mrays, unit="Mrays/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * dt / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=w["desc"], particles=w["n"], width=w["res"], height=w["res"],
                            sample="%d seeded pixels per step" % per_step),
                segments_per_s=segs / dt,
                cpu_baseline=dict(value=mrays, unit="Mrays/s", cores=oracle.num_threads(), kind="oracle",
                                  sample="%d seeded pixels per step, %d steps" % (per_step, args.steps)),
                e2e=dict(value=mrays, unit="Mrays/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def poll_completions(srv, tickets, clock=time.perf_counter, sleep=time.sleep, period=0.005):
    """Latencies of submitted frames, polled: `tickets` holds (submission time, size, ticket); the server's
    wait(ticket, 0) returns False while a frame is in flight and True once it has completed (it raises for a
    failed frame).  Returns [(completion - submission, size)] in completion order."""
    lat, pending = [], list(tickets)
    while pending:
        still = []
        for ts, r_, t_ in pending:
            if srv.wait(t_, 0):
                lat.append((clock() - ts, r_))
            else:
                still.append((ts, r_, t_))
        pending = still
        if pending:
            sleep(period)
    return lat


def serving_stream(S, torch, ctx, tf_all, dev, per_rate=20, seed=2024, workers=3):
    """Serving stream: four resident clustered data sets (1M, 4M, 16M, 32M particles of the halo generator, seeds +0..3),
    requests with random orbit cameras and sizes uniform over {256, 512, 1024, 2048} squared, Poisson arrivals.
    The service rate is measured first (a burst of requests queued at once); then three arrival rates
    (0.5, 0.8 and 1.2 times it) with `per_rate` requests each: p50/p99 submission-to-completion latency per
    rate and per size."""
    sets, luts = [], {}
    th, pc, _ = S.sphdvr_lut_build("wendland_c2", 4, 3, 4096)
    lut = S.sphdvr_lut_create(ctx, "wendland_c2", 4, 3, 4096, th, pc)
    for i, n in enumerate((1_000_000, 4_000_000, 16_000_000, 32_000_000)):
        P = SY.halo_mixture(n, seed=SY.BASE_SEED + 1 + i, device="cuda")
        t = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(dev) for k in ("pos", "h", "mass", "density", "value")}
        ds = S.sphdvr_dataset_create(ctx, t["pos"], t["h"], t["mass"], t["density"], t["value"])
        sets.append((n, ds, SY.tf_density(P["value"])))
        del t, P
    resident = sum(S.sphdvr_dataset_info(ds)["bytes"] for _, ds, _ in sets)
    rng = np.random.default_rng(seed)
    sizes = (256, 512, 1024, 2048)

    def request():
        k = int(rng.integers(len(sets)))
        r_ = int(rng.choice(sizes))
        return k, r_, SY.orbit_camera(r_, r_, azimuth_deg=360 * rng.random(), elevation_deg=-40 + 80 * rng.random())

    def run(reqs, gaps):
        srv = S.Server(ctx, 64 << 30, max_inflight=workers)
        outs, tix = [], []
        t0 = time.perf_counter()
        for (k, r_, c_), g in zip(reqs, gaps):
            time.sleep(g)
            o_ = torch.empty((r_, r_, 4), dtype=torch.float32, device=dev)
            outs.append(o_)
            tix.append((time.perf_counter(), r_, srv.submit(sets[k][1], lut, c_, sets[k][2], dict(ert_eps=1e-5),
                                                            o_.data_ptr())))
        lat = poll_completions(srv, tix)
        wall = time.perf_counter() - t0
        srv.destroy()
        rays = sum(r_ * r_ for _, r_, _ in reqs)
        return lat, wall, rays

    burst = [request() for _ in range(2 * workers + 2)]
    lat, wall, rays = run(burst, [0.0] * len(burst))
    capacity = len(burst) / wall  # requests per second at saturation
    out = dict(datasets="halo generator 1M/4M/16M/32M, seeds +0..3, resident together (%.2f GB)" % (resident / 1e9),
               sizes=list(sizes), workers=workers, burst=dict(requests=len(burst), requests_per_s=capacity,
                                                              mrays_per_s=rays / wall / 1e6), rates=[])
    for f in (0.5, 0.8, 1.2):
        lam = f * capacity
        reqs = [request() for _ in range(per_rate)]
        gaps = list(rng.exponential(1.0 / lam, size=per_rate))
        lat, wall, rays = run(reqs, gaps)
        ms = np.array([x[0] for x in lat]) * 1e3
        per_size = {}
        for r_ in sizes:
            v = np.array([x[0] for x in lat if x[1] == r_]) * 1e3
            if len(v):
                per_size[str(r_)] = dict(n=int(len(v)), p50_ms=float(np.percentile(v, 50)),
                                         p99_ms=float(np.percentile(v, 99)))
        out["rates"].append(dict(load=f, requests_per_s=lam, requests=per_rate, p50_ms=float(np.percentile(ms, 50)),
                                 p99_ms=float(np.percentile(ms, 99)), mrays_per_s=rays / wall / 1e6,
                                 per_size=per_size))
    for _, ds, _ in sets:
        S.sphdvr_dataset_free(ds)
    S.sphdvr_lut_free(lut)
    return out


def precision_sweep_times(S, torch, ctx, ds, w, tf, cam, dev, stream, degrees=(1, 2, 3, 4)):
    """Precision / degree sweep frame times: each precision mode x degree D on the workload's frame (kernel time, CUDA events),
    and each mode's largest pixel difference from the FP32 anchored frame of the same D.  (The errors against
    the FP64 oracle are measured by tests/test_gpu_precision_sweep.py.)"""
    W, H = cam["width"], cam["height"]
    rows = []
    for D in degrees:
        th, pc, _ = S.sphdvr_lut_build(w["kernel"], w["K"], D, w["n_lambda"])
        lt = S.sphdvr_lut_create(ctx, w["kernel"], w["K"], D, w["n_lambda"], th, pc)
        imgs = {}
        for mode in ("fp32_anchored", "fp32_naive", "fp32_kahan", "fp64_naive", "fp32_reinit", "int64_quant"):
            o = dict(precision=mode, ert_eps=1e-5)
            if mode == "fp32_reinit":
                o["reinit_dt"] = 0.02 if D <= 3 else 0.005  # the spacing the parity sweep validates
            if mode == "int64_quant":
                q = S.sphdvr_dataset_quant_params(ctx, ds, w["kernel"], D, 64)
                o.update(quant_tau=q["tau"], quant_sigma=q["sigma"])
            img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
            S.sphdvr_render(ctx, ds, lt, cam, tf, o, img.data_ptr(), stream=stream)
            torch.cuda.synchronize()
            st = S.sphdvr_frame_stats(ctx)
            imgs[mode] = img
            rows.append(dict(D=D, mode=mode, render_ms=st["render_ns"] / 1e6,
                             mrays_per_s=W * H / (st["render_ns"] / 1e9) / 1e6, segments=st["segments"],
                             flags=st["overflow"]))
        for r in rows:
            if r["D"] == D:
                r["max_pixel_diff_vs_anchored"] = float((imgs[r["mode"]] - imgs["fp32_anchored"]).abs().max())
        del imgs
        S.sphdvr_lut_free(lt)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sphdvr", choices=["sphdvr", "reference"])
    ap.add_argument("--workload", default="halo16m", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-pixels", type=int, default=48)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp32_anchored")
    ap.add_argument("--res", type=int, default=0, help="override the workload's image size (square)")
    ap.add_argument("--serve-requests", type=int, default=12,
                    help="frames pushed through the frame server after the timed region (0: skip)")
    ap.add_argument("--batch-frames", type=int, default=8,
                    help="small frames timed separately and as one batched launch after the timed region (<2: skip)")
    ap.add_argument("--batch-res", type=int, default=128)
    ap.add_argument("--scatter-frame", type=int, default=1,
                    help="time the paper's scatter-sort pass order against ray gathering on a 1M-particle frame (0: skip)")
    ap.add_argument("--quant-frame", type=int, default=1,
                    help="time the quantised integer path against FP32 anchored on a 1M-particle frame (0: skip)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="tune the render options on the workload's frame before timing (sphdvr_autotune; 0: defaults)")
    ap.add_argument("--plain-vs-served", type=int, default=16,
                    help="requests of the plain-vs-served comparison (0: skip)")
    ap.add_argument("--shading-frame", type=int, default=1,
                    help="time a shaded frame beside the unshaded one (1M-particle halo mixture, 512x512; 0: skip)")
    ap.add_argument("--precision-sweep", action="store_true",
                    help="also time every precision mode x D in {1,2,3,4} on the workload's frame")
    ap.add_argument("--serving-stream", type=int, default=0,
                    help="requests per arrival rate of the serving stream over four resident data sets (0: skip)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.res > 0:
        w["res"] = args.res
        r0 = WORKLOADS[args.workload]["res"]
        w["desc"] = w["desc"].replace("%dx%d" % (r0, r0), "%dx%d" % (args.res, args.res))
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, w, rank, world)

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2401_02896_b300 import sphdvr as S

    P, tf = make_inputs(w, "cuda")
    ctx = S.sphdvr_create(local)
    th, pc, _err = S.sphdvr_lut_build(w["kernel"], w["K"], w["D"], w["n_lambda"])
    lut = S.sphdvr_lut_create(ctx, w["kernel"], w["K"], w["D"], w["n_lambda"], th, pc)
    dev = torch.device("cuda", local)
    tens = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(dev) for k in ("pos", "h", "mass", "density", "value")}
    torch.cuda.synchronize()
    t_build = time.perf_counter()
    ds = S.sphdvr_dataset_create(ctx, tens["pos"], tens["h"], tens["mass"], tens["density"], tens["value"])
    t_build = time.perf_counter() - t_build  # the call returns after the build has completed
    del tens
    cam = camera_for(w, rank)
    opts = dict(precision=args.precision, ert_eps=1e-5)
    # roofline denominator: the device's FP32 FMA rate, measured (FFMA loop, CUDA events; no clock is set)
    fp32_peak = S.sphdvr_measure_fp32_peak(ctx, torch.cuda.current_stream(dev).cuda_stream)
    W, H = cam["width"], cam["height"]
    out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    # ---- autotuning: the timed frames use the options the autotuner picks for this frame
    autotune = None
    if args.autotune and args.precision in ("fp32_anchored", "fp32_naive"):
        default_opts = dict(opts)
        opts, (ms0, ms1) = S.sphdvr_autotune(ctx, ds, lut, cam, tf, default_opts,
                                             cache_path=os.path.join(log_dir(), "sphdvr_autotune_r%d.jsonl" % rank),
                                             stream=stream)
        # the default options once at the full size, for the speed-up the tuning brings there
        S.sphdvr_render(ctx, ds, lut, cam, tf, default_opts, out.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        full_default_ms = S.sphdvr_frame_stats(ctx)["render_ns"] / 1e6
        autotune = dict(chosen=dict(ctas_per_sm=opts["ctas_per_sm"], window_h=opts["window_h"],
                                    window_fill=opts["window_fill"]),
                        tuning_frame_ms=dict(default=ms0, tuned=ms1), full_frame_default_ms=full_default_ms,
                        note="coordinate descent over CTAs per SM, window_h, window_fill on the frame's view at "
                             "<= 512x512 (render-kernel time, CUDA events); the timed frames use the chosen options")

    def frame():
        S.sphdvr_render(ctx, ds, lut, cam, tf, opts, out.data_ptr(), stream=stream)

    for _ in range(max(3, args.warmup)):
        frame()
    torch.cuda.synchronize()
    st0 = S.sphdvr_frame_stats(ctx)
    # ---- timed region: device time, CUDA events on the render stream
    # the clock samples of the timed region (directory: $SPHDVR_BENCH_LOG_DIR, else the temp directory)
    clk_path = os.path.join(os.environ.get("SPHDVR_BENCH_LOG_DIR") or tempfile.gettempdir(),
                            "bench_clocks_r%d.csv" % rank)
    proc, fh = clocks_start(clk_path)
    time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    render_ns, launches, segs, knots = [], 0, 0, 0
    evs[0].record()
    for i in range(args.steps):
        frame()
        evs[i + 1].record()
        st = S.sphdvr_frame_stats(ctx)  # reads the render kernel's own CUDA events
        render_ns.append(st["render_ns"])
        launches += st["launches"]
        segs += st["segments"]
        knots += st["knots"]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    frame_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = sum(frame_ms)
    clocks = clocks_stop(proc, fh, clk_path, local)
    t_max, value = replica_rate(total_ms, W * H * args.steps, dist, dev)

    # ---- end to end: host output buffer, copies inside the call
    host = torch.empty((H, W, 4), dtype=torch.float32, pin_memory=True).numpy()
    S.sphdvr_render_host(ctx, ds, lut, cam, tf, opts, host, stream=stream)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.sphdvr_render_host(ctx, ds, lut, cam, tf, opts, host, stream=stream)
    e2e_s = time.perf_counter() - t0
    e2e_val = W * H * args.steps / e2e_s / 1e6
    if dist:
        dist.barrier()

    # ---- serving: seeded orbit cameras of mixed sizes, Poisson arrivals, two worker streams
    serving = None
    if args.serve_requests > 0:
        rng = np.random.default_rng(1234 + rank)
        sizes = [s_ for s_ in (256, 512, 1024) if s_ <= W] or [W]
        srv = S.Server(ctx, 16 << 30, max_inflight=2)
        outs, tickets = [], []
        for i in range(args.serve_requests):
            r_ = int(rng.choice(sizes))
            c_ = SY.orbit_camera(r_, r_, azimuth_deg=360 * rng.random(), elevation_deg=-40 + 80 * rng.random())
            o_ = torch.empty((r_, r_, 4), dtype=torch.float32, device=dev)
            outs.append(o_)
            tickets.append(srv.submit(ds, lut, c_, tf, opts, o_.data_ptr()))
            time.sleep(float(rng.exponential(1.5)))
        for t_ in tickets:
            srv.wait(t_, -1)
        sv = srv.stats()
        bs = srv.batch_stats()
        srv.destroy()
        serving = dict(requests=args.serve_requests, sizes=sizes, arrivals="Poisson, mean gap 1.5 s", workers=2,
                       p50_ms=sv["p50_ms"], p99_ms=sv["p99_ms"], mrays_per_s=sv["rays_per_s"] / 1e6,
                       failed=int(sv["failed"]), render_launches=bs["launches"], largest_batch=bs["largest"])
        del outs

    # ---- plain one-launch-per-frame form against the served form on one mixed request set
    pvs = None
    if args.plain_vs_served > 0:
        pvs = plain_vs_served(S, torch, ctx, ds, lut, tf, opts, dev, stream, n=args.plain_vs_served)

    # ---- batching: the same small frames rendered one launch each and as one batched launch
    batching = None
    if args.batch_frames > 1:
        nb, rb = args.batch_frames, args.batch_res
        cams_b = [SY.orbit_camera(rb, rb, azimuth_deg=360.0 * i / nb, elevation_deg=-30 + 60.0 * i / nb)
                  for i in range(nb)]
        outs_b = [torch.empty((rb, rb, 4), dtype=torch.float32, device=dev) for _ in cams_b]

        def separate():
            for c_, o_ in zip(cams_b, outs_b):
                S.sphdvr_render(ctx, ds, lut, c_, tf, opts, o_.data_ptr(), stream=stream)

        def batched():
            S.sphdvr_render_batch(ctx, ds, lut, cams_b, tf, opts, [o_.data_ptr() for o_ in outs_b], stream=stream)

        # the same frames from a frame plan captured into one CUDA graph
        pairs_max = 0
        for c_, o_ in zip(cams_b, outs_b):
            S.sphdvr_render(ctx, ds, lut, c_, tf, opts, o_.data_ptr(), stream=stream)
            pairs_max = max(pairs_max, S.sphdvr_frame_stats(ctx)["pairs"])
        plan = S.FramePlan(ctx, ds, lut, tf, opts, rb, rb, int(1.5 * pairs_max) + 64)
        gs = torch.cuda.Stream(dev)
        graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=gs, capture_error_mode="thread_local"):
            for c_, o_ in zip(cams_b, outs_b):
                plan.render(c_, o_.data_ptr(), stream=gs.cuda_stream)
        tb = {}
        for name, fn in (("separate", separate), ("batched", batched), ("graph", graph.replay)):
            fn()
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(3):
                t0 = time.perf_counter()
                fn()
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            tb[name] = best
        plan_overflow = plan.overflowed()
        del graph
        plan.destroy()
        batching = dict(frames=nb, size=rb, separate_ms=tb["separate"] * 1e3, batched_ms=tb["batched"] * 1e3,
                        speedup=tb["separate"] / tb["batched"], graph_ms=tb["graph"] * 1e3,
                        graph_pair_overflow=plan_overflow,
                        note="wall time incl. binning, best of 3; batched = one render launch for all frames; "
                             "graph = one replay of the frames captured from a frame plan")
        del outs_b

    # ---- quantised fixed-point path (Sec. 4.2-4.4) beside FP32 anchored: uniform 1M particles, one
    # smoothing length (one length quantum serves every particle), 512x512
    quant = None
    if args.quant_frame:
        nq, hq, rq = 1_000_000, 0.012, 512
        PQ = SY.uniform_cube(nq, h=hq, seed=SY.BASE_SEED + 90)
        dsq = S.sphdvr_dataset_create(ctx, PQ["pos"], PQ["h"], PQ["mass"], PQ["density"], PQ["value"])
        # representative particle amplitude m v / (rho h^3): the median over the particles
        pc_rep = float(np.median(PQ["mass"].astype(np.float64) * PQ["value"] / PQ["density"]
                                 / PQ["h"].astype(np.float64) ** 3))
        # A_max: 8 times the particles overlapping a point at the mean density, each at its peak value
        ratio = 8 * nq * 4.0 / 3.0 * math.pi * (2 * hq) ** 3
        tau_rel, sig_rel, qe = S.sphdvr_quant_params(w["kernel"], w["D"], 64, ratio)
        camq = SY.orbit_camera(rq, rq)
        tfq = SY.tf_bumps()  # three opacity bumps across the field's range: every piece is classified
        oq = torch.empty((rq, rq, 4), dtype=torch.float32, device=dev)
        ref_q = torch.empty_like(oq)
        qopts = dict(precision="int64_quant", quant_tau=tau_rel * hq, quant_sigma=sig_rel * pc_rep, ert_eps=1e-5)
        tq = {}
        for name, op_, img in (("fp32_anchored", None, ref_q), ("int64_quant", qopts, oq)):
            S.sphdvr_render(ctx, dsq, lut, camq, tfq, op_, img.data_ptr(), stream=stream)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(2):
                t0 = time.perf_counter()
                S.sphdvr_render(ctx, dsq, lut, camq, tfq, op_, img.data_ptr(), stream=stream)
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            tq[name] = (best, S.sphdvr_frame_stats(ctx)["segments"])
        quant = dict(workload="uniform cube 1,000,000 particles, h 0.012, perspective 512x512, transfer function with "
                              "three opacity bumps", int_bits=64,
                     tau=tau_rel * hq, sigma=sig_rel * pc_rep, quant_error_estimate=qe,
                     anchored_ms=tq["fp32_anchored"][0] * 1e3, quant_ms=tq["int64_quant"][0] * 1e3,
                     quant_segments_per_s=tq["int64_quant"][1] / tq["int64_quant"][0],
                     max_pixel_diff_vs_anchored=float((oq - ref_q).abs().max()),
                     note="wall time incl. binning, best of 2")
        S.sphdvr_dataset_free(dsq)
        del oq, ref_q

    # ---- the paper's pass order (scatter knots per particle, one sort, accumulate per ray) against ray
    # gathering on the 1M-particle halo mixture, 256x256
    scatter = None
    if args.scatter_frame:
        w1 = WORKLOADS["halo1m"]
        P1, tf1 = make_inputs(w1, "cuda")
        t1 = {k: torch.from_numpy(np.ascontiguousarray(P1[k])).to(dev) for k in ("pos", "h", "mass", "density", "value")}
        ds1 = S.sphdvr_dataset_create(ctx, t1["pos"], t1["h"], t1["mass"], t1["density"], t1["value"])
        del t1
        cam1 = SY.orbit_camera(256, 256)
        ga = torch.empty((256, 256, 4), dtype=torch.float32, device=dev)
        sc = torch.empty_like(ga)
        ts_ = {}
        for name, fn in (("gather", lambda: S.sphdvr_render(ctx, ds1, lut, cam1, tf1, None, ga.data_ptr(),
                                                             stream=stream)),
                         ("scatter", lambda: S.sphdvr_render_scatter(ctx, ds1, lut, cam1, tf1, None, sc.data_ptr(),
                                                                     stream=stream))):
            fn()
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(2):
                t0 = time.perf_counter()
                fn()
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            ts_[name] = (best, S.sphdvr_frame_stats(ctx)["knots"])
        scatter = dict(workload="halo mixture 1,000,000 particles, perspective 256x256", gather_ms=ts_["gather"][0] * 1e3,
                       scatter_ms=ts_["scatter"][0] * 1e3, knots=ts_["scatter"][1],
                       slowdown=ts_["scatter"][0] / ts_["gather"][0],
                       max_pixel_diff=float((ga - sc).abs().max()),
                       note="wall time incl. binning / scatter and sort, best of 2")
        S.sphdvr_dataset_free(ds1)
        del ga, sc

    # ---- shaded rendering (the across-ray gradient reconstructed beside the field) against the unshaded frame
    shading = None
    if args.shading_frame:
        w1 = WORKLOADS["halo1m"]
        P1, tf1 = make_inputs(w1, "cuda")
        ds1 = S.sphdvr_dataset_create(ctx, P1["pos"], P1["h"], P1["mass"], P1["density"], P1["value"])
        th1, pc1, _ = S.sphdvr_lut_build(w1["kernel"], w1["K"], w1["D"], w1["n_lambda"])
        lt1 = S.sphdvr_lut_create(ctx, w1["kernel"], w1["K"], w1["D"], w1["n_lambda"], th1, pc1)
        gp1, _ = S.sphdvr_lut_build_grad(w1["kernel"], w1["K"], w1["D"], w1["n_lambda"], th1)
        S.sphdvr_lut_set_gradient(lt1, th1, gp1)
        # softening gradient: 1e-3 of the data's typical gradient scale (median value / median h)
        g0 = 1e-3 * float(np.median(P1["value"])) / float(np.median(P1["h"]))
        cam1 = SY.orbit_camera(512, 512)
        imgs_ = {k: torch.empty((512, 512, 4), dtype=torch.float32, device=dev) for k in ("plain", "shaded", "unit")}
        modes_ = (("plain", dict(ert_eps=1e-5)),
                  ("shaded", dict(ert_eps=1e-5, shading=1, shade_ka=0.3, shade_kd=0.7, shade_g0=g0)),
                  ("unit", dict(ert_eps=1e-5, shading=1, shade_ka=1.0, shade_kd=0.0, shade_g0=g0)))
        tsh = {}
        for name, o_ in modes_:
            S.sphdvr_render(ctx, ds1, lt1, cam1, tf1, o_, imgs_[name].data_ptr(), stream=stream)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(2):
                S.sphdvr_render(ctx, ds1, lt1, cam1, tf1, o_, imgs_[name].data_ptr(), stream=stream)
                torch.cuda.synchronize()
                best = min(best, S.sphdvr_frame_stats(ctx)["render_ns"] / 1e6)
            tsh[name] = best
        shading = dict(workload="halo mixture 1,000,000 particles, Wendland C2, K=4, D=3, perspective 512x512",
                       ka=0.3, kd=0.7, g0=g0, unshaded_ms=tsh["plain"], shaded_ms=tsh["shaded"],
                       ratio=tsh["shaded"] / tsh["plain"],
                       unit_shading_max_pixel_diff=float((imgs_["unit"] - imgs_["plain"]).abs().max()),
                       note="render-kernel time (CUDA events), best of 2; unit shading = ka 1, kd 0")
        S.sphdvr_dataset_free(ds1)
        S.sphdvr_lut_free(lt1)
        del imgs_

    sweep = precision_sweep_times(S, torch, ctx, ds, w, tf, cam, dev, stream) if args.precision_sweep else None
    stream_c4 = serving_stream(S, torch, ctx, tf, dev, per_rate=args.serving_stream) if args.serving_stream > 0 else None

    if rank == 0:
        seg_per_frame = segs / args.steps
        fps = flops_per_segment(w["K"], w["D"])
        kern_s = np.mean(render_ns) / 1e9
        achieved = seg_per_frame * fps / kern_s / 1e12
        lat = np.array(frame_ms)
        line = dict(
            metric="Mrays/s", value=value, unit="Mrays/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
            data="synthetic",
            config=dict(workload=w["desc"], particles=w["n"], width=W, height=H, kernel=w["kernel"], K=w["K"],
                        D=w["D"], n_lambda=w["n_lambda"], precision=args.precision, ert_eps=1e-5,
                        l2="inputs larger than L2 (resident particles %.0f MB)" % (S.sphdvr_dataset_info(ds)["bytes"] / 1e6),
                        parallelism="replicas: one frame stream per GPU" if world > 1 else "1 GPU"),
            segments_per_s=seg_per_frame * args.steps * world / (t_max / 1e3),
            p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
            frame_stats=dict(segments=int(seg_per_frame), knots=int(knots / args.steps), pairs=st0["pairs"],
                             max_table=st0["max_table"], overflow=st0["overflow"], ert_rays=st0["ert_rays"],
                             render_kernel_ms=kern_s * 1e3),
            roofline=dict(bound="alu", achieved=achieved, peak=fp32_peak, unit="TFLOP/s",
                          frac=achieved / fp32_peak,
                          traffic=PROFILED_DRAM_BYTES.get((args.workload, w["res"], args.precision,
                                                           round(float(opts.get("window_h") or 1.0), 3))),
                          note="peak: FP32 FMA rate measured in this run (sphdvr_measure_fp32_peak, an FFMA "
                               "loop on every resident thread; MEASURED_PEAKS.json has no FP32 figure); "
                               "achieved: %d algorithmic FLOP per segment x segments per frame / render "
                               "kernel time (CUDA events)" % fps),
            e2e=dict(value=e2e_val, unit="Mrays/s", h2d_bytes_per_step=int(tf["rgba"].nbytes),
                     d2h_bytes_per_step=int(W * H * 16)),
            gpu_launches=int(launches),
            clocks=clocks,
        )
        if autotune:
            autotune["full_frame_tuned_ms"] = kern_s * 1e3
            autotune["full_frame_speedup"] = autotune["full_frame_default_ms"] / (kern_s * 1e3)
            line["autotune"] = autotune
        if pvs:
            line["plain_vs_served"] = pvs
        if sweep:
            line["precision_sweep"] = sweep
        if stream_c4:
            line["serving_stream"] = stream_c4
        if serving:
            line["serving"] = serving
        if batching:
            line["batching"] = batching
        if quant:
            line["quantised"] = quant
        if scatter:
            line["scatter_order"] = scatter
        if shading:
            line["shading"] = shading
        info = S.sphdvr_dataset_info(ds)
        line["dataset_build"] = dict(ms=t_build * 1e3, particles_per_s=w["n"] / t_build,
                                     input_bytes=int(w["n"] * 28), resident_bytes=int(info["bytes"]),
                                     note="inputs already on the device; levels, Morton keys, radix sort, chunks")
        if not args.no_cpu_baseline:
            cb = cpu_oracle_rate(P, w, tf, args.cpu_pixels, seed=77)
            line["cpu_baseline"] = dict(value=cb["rays_per_s"] / 1e6, unit="Mrays/s", cores=cb["cores"], kind="oracle",
                                        sample="%d seeded pixels of the same frame (%.1f s, %d segments)" % (
                                            args.cpu_pixels, cb["seconds"], cb["segments"]))
        print(json.dumps(line), flush=True)
    S.sphdvr_dataset_free(ds)
    S.sphdvr_lut_free(lut)
    S.sphdvr_destroy(ctx)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
