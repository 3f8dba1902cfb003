#!/usr/bin/env python
"""Benchmark of the chunked Gaussian-splatting mapper hot path on one B300.

Workload (default): one keyframe window of 8 views of mixed size
(4 x 1200x680, 2 x 640x480, 2 x 320x240 = 4,032,000 pixels) over 2M Gaussians
(SH degree 3, FP32) in 64 chunks of 4 m.  One step = the optimisation pass of
Sec. III-E for the window: cull chunks, gather the visible Gaussians, render
RGB + depth (forward), L1 loss of Eq. 2-4, backward to every parameter and
the pose, scatter the active set back to its chunks.

  batched : all 8 views in one render call (one preprocess over the Gaussians,
            one sort, one persistent blend launch per direction)
  plain   : the per-keyframe method, 8 sequential passes with one view each
            (cull, gather, forward, loss, backward, scatter per keyframe)

Prints one JSON line (metric, value = batched Mpix/s, ...).  `--impl
reference` times the CPU FP64 oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd render Mpix/s per keyframe window (batched vs plain); % HBM roofline"
UNIT = "Mpix/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--gaussians", type=int, default=2_000_000)
    ap.add_argument("--tile", default="auto", help="WxH, or auto (autotuned)")
    ap.add_argument("--stage", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="batched timing only (no plain/e2e/CPU legs), for profilers")
    ap.add_argument("--workload", default="window", choices=["window", "corridor", "sampling", "loopclosure", "loss"])
    ap.add_argument("--bwd", default="warp", choices=["warp", "slots", "pixel"],
                    help="backward blend: default, lane slots, or (half-warp launch) pixels on the lanes")
    ap.add_argument("--length", type=float, default=5000.0, help="corridor: metres of road (1 m per frame)")
    ap.add_argument("--per-m", type=int, default=8000, help="corridor: Gaussians per metre (40M per 5 km)")
    ap.add_argument("--propose-every", type=int, default=4, help="corridor: frames between prefetch proposals")
    ap.add_argument("--cpu-pixels", type=int, default=48, help="oracle sample: pixels per sampled view")
    ap.add_argument("--no-side-workloads", action="store_true",
                    help="window only: skip the indoor-room and 1 km corridor legs of the default run")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2032.0)), "measured"
    except Exception:
        return 6400.0, 2032.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"dcg_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (every rank gets it); identity on one rank."""
    if world <= 1:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- our implementation
def run_ours(args, rank, world):
    import torch

    from paper_2511_23030_b300 import build, dcg, synth

    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    sc = synth.window_scene(0, n=args.gaussians)
    P = sc["params"]
    cams = sc["cams"]
    deg = sc["deg"]
    n_all = P.shape[0]
    F = P.shape[1]
    npix = sum(c.W * c.H for c in cams)
    # capacities sized to the scene (the window makes about 10 instances per Gaussian)
    cfg = dcg.config(sh_degree=deg, max_active=n_all + 1024, max_views=8, max_pixels=npix,
                     max_instances=max(32 << 20, 24 * n_all), chunk_size=sc["chunk_size"],
                     device_budget=n_all + 1024, host_capacity=n_all + 1024, dfar=60.0,
                     flags={"warp": 0, "slots": 1, "pixel": 2}[args.bwd])
    ctx = dcg.dcg_create(cfg)
    stream = torch.cuda.current_stream()
    g_t = torch.from_numpy(np.ascontiguousarray(P.T)).cuda()
    dcg.dcg_chunk_table_update(ctx, g_t, n_all)
    del g_t
    # targets (pinned host copies for the end-to-end run)
    trgb_h = torch.from_numpy(np.concatenate([t.reshape(-1) for t in sc["target_rgb"]])).pin_memory()
    tdep_h = torch.from_numpy(np.concatenate([t.reshape(-1) for t in sc["target_depth"]])).pin_memory()
    trgb, tdep = trgb_h.cuda(), tdep_h.cuda()
    rgb = torch.zeros(3 * npix, device="cuda")
    depth = torch.zeros(npix, device="cuda")
    dr = torch.zeros_like(rgb)
    dd = torch.zeros_like(depth)
    loss = torch.zeros(1, device="cuda")
    loss_h = torch.zeros(1).pin_memory()
    grads_t = torch.zeros((F, n_all + 1024), device="cuda")
    grads = dcg.gaussians(grads_t, deg)
    dpose = torch.zeros(8 * 6, device="cuda")
    lam = sc["lambda_depth"]
    offs = np.cumsum([0] + [c.W * c.H for c in cams])

    # launch shape: autotuned over tile x staging depth on this window (forward + backward)
    tune = None
    if args.tile == "auto":
        lst = dcg.dcg_cull_chunks(ctx, cams)
        g, n = dcg.dcg_gather_active(ctx, lst)
        dcg.dcg_render_fwd(ctx, g, n, cams, rgb, depth)
        dcg.dcg_loss_l1(ctx, rgb, depth, trgb, tdep, cams, lam, dr, dd, loss)
        tune = dcg.dcg_autotune(ctx, g, n, cams, rgb, depth, dr, dd, grads, reps=2)
        tile = tuple(tune["tile"])
        stage = tune["stage"]
    else:
        tile = tuple(int(x) for x in args.tile.split("x"))
        stage = args.stage or 128
        dcg.dcg_set_launch(ctx, tile[0], tile[1], stage)

    graph = {"n": -1}

    def step_batched():
        # cull -> gather -> [render fwd, loss, render bwd: one CUDA graph] -> scatter
        lst = dcg.dcg_cull_chunks(ctx, cams)
        g, n = dcg.dcg_gather_active(ctx, lst)
        if graph["n"] != n:
            dcg.dcg_window_capture(ctx, g, n, cams, rgb, depth, trgb, tdep, lam, dr, dd, loss, grads, dpose)
            graph["n"] = n
        dcg.dcg_window_run(ctx, cams)
        dcg.dcg_scatter_back(ctx, g, n)
        return n

    def step_batched_direct():
        lst = dcg.dcg_cull_chunks(ctx, cams)
        g, n = dcg.dcg_gather_active(ctx, lst)
        dcg.dcg_render_fwd(ctx, g, n, cams, rgb, depth)
        loss.zero_()
        dcg.dcg_loss_l1(ctx, rgb, depth, trgb, tdep, cams, lam, dr, dd, loss)
        dcg.dcg_render_bwd(ctx, dr, dd, grads, dpose)
        dcg.dcg_scatter_back(ctx, g, n)
        return n

    def step_plain():
        n = 0
        for v, c in enumerate(cams):
            lst = dcg.dcg_cull_chunks(ctx, [c])
            g, n = dcg.dcg_gather_active(ctx, lst)
            o = int(offs[v])
            Pv = c.W * c.H
            r = rgb[3 * o: 3 * (o + Pv)]
            d = depth[o: o + Pv]
            dcg.dcg_render_fwd(ctx, g, n, [c], r, d)
            dcg.dcg_loss_l1(ctx, r, d, trgb[3 * o: 3 * (o + Pv)], tdep[o: o + Pv], [c], lam, dr[3 * o: 3 * (o + Pv)],
                            dd[o: o + Pv], loss)
            dcg.dcg_render_bwd(ctx, dr[3 * o: 3 * (o + Pv)], dd[o: o + Pv], grads, dpose[6 * v: 6 * v + 6])
            dcg.dcg_scatter_back(ctx, g, n)
        return n

    # End to end through the public API: every step copies its targets from
    # pinned host memory and reads its loss back.  The copy for step t+1 runs on
    # a copy stream as soon as step t's loss has read the target buffer, i.e.
    # under step t's backward and step t+1's forward; the loss of each step is
    # copied to its own pinned slot and read after the run.
    copy_stream = torch.cuda.Stream()
    ev_free, ev_ready = torch.cuda.Event(), torch.cuda.Event()
    loss_slots = {}

    def issue_targets():
        copy_stream.wait_event(ev_free)
        with torch.cuda.stream(copy_stream):
            trgb.copy_(trgb_h, non_blocking=True)
            tdep.copy_(tdep_h, non_blocking=True)
            ev_ready.record(copy_stream)

    def step_e2e(t, last):
        lst = dcg.dcg_cull_chunks(ctx, cams)
        g, n = dcg.dcg_gather_active(ctx, lst)
        dcg.dcg_render_fwd(ctx, g, n, cams, rgb, depth)
        stream.wait_event(ev_ready)
        loss.zero_()
        dcg.dcg_loss_l1(ctx, rgb, depth, trgb, tdep, cams, lam, dr, dd, loss)
        ev_free.record(stream)
        if not last:
            issue_targets()
        dcg.dcg_render_bwd(ctx, dr, dd, grads, dpose)
        dcg.dcg_scatter_back(ctx, g, n)
        loss_slots["buf"][t: t + 1].copy_(loss, non_blocking=True)
        return n

    def timed_e2e(k, w):
        loss_slots["buf"] = torch.zeros(max(k, w) + 1).pin_memory()
        for rep, steps in ((0, w), (1, k)):
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            ev_free.record(stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            issue_targets()
            for t in range(steps):
                step_e2e(t, t == steps - 1)
            e1.record(stream)
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
        losses = loss_slots["buf"][:k].numpy()
        assert np.isfinite(losses).all() and (losses > 0).all()
        return max_over_ranks(e0.elapsed_time(e1), world, "cuda")

    def timed(fn, k, w, profile=False):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        if profile:
            dcg.dcg_profile(ctx, True)
            dcg.dcg_profile_read(ctx)
        l0 = dcg.dcg_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # the phase timers hold 4096 intervals between reads (a plain step of 8
        # views records about 80): a long profiled run reads and sums them
        # every 25 steps
        prof = {} if profile else None

        def read_timers():
            for key, (v, c) in dcg.dcg_profile_read(ctx).items():
                a = prof.setdefault(key, [0.0, 0])
                a[0] += v
                a[1] += c

        e0.record(stream)
        for j in range(k):
            fn()
            if profile and j % 25 == 24 and j + 1 < k:
                read_timers()
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = e0.elapsed_time(e1)
        launches = dcg.dcg_launch_count() - l0
        if profile:
            read_timers()
            dcg.dcg_profile(ctx, False)
            prof = {key: (v[0], v[1]) for key, v in prof.items()}
        return max_over_ranks(ms, world, "cuda"), launches, prof

    K, W = args.steps, args.warmup
    # per-phase device times of the direct (uncaptured) calls; the graph replays the same kernels
    _, _, prof = timed(step_batched_direct, K, W, profile=True)
    K_p = max(2, K // 2)
    # clocks are sampled over the three timed legs (batched, plain, end to end)
    with Clocks(torch.cuda.current_device()) as clk:
        ms_b, launches_b, _ = timed(step_batched, K, W)
        n_vis, n_inst, n_tiles = dcg.dcg_state_stats(ctx)
        n_eval, n_blend = dcg.dcg_state_evals(ctx)
        if args.quick:
            ms_p = ms_e = None  # not measured: profiler runs time the batched window only
        else:
            ms_p, launches_p, _ = timed(step_plain, K_p, max(1, W // 2))
            ms_e = timed_e2e(K, 2)
    clocks = clk.summary()
    dcg.dcg_sync(ctx)
    # per-phase device times of the plain path (outside the timed legs): the plain
    # path gathers and writes back per view, so the render phases alone say how
    # much of the batched/plain ratio comes from batching the render itself
    prof_p = None
    if not args.quick:
        _, _, prof_p = timed(step_plain, K_p, 1, profile=True)

    mpix_b = npix * K * world / (ms_b / 1e3) / 1e6
    mpix_p = npix * K_p * world / (ms_p / 1e3) / 1e6 if ms_p else None
    mpix_e = npix * K * world / (ms_e / 1e3) / 1e6 if ms_e else None
    phases = {k: round(v[0] / K, 4) for k, v in prof.items() if k not in ("log_sample", "loop_closure")}
    render_phases = ("preprocess_fwd", "binning", "blend_fwd", "blend_bwd", "preprocess_bwd")
    plain_phases = ({k: round(v[0] / K_p, 4) for k, v in prof_p.items() if k not in ("log_sample", "loop_closure")}
                    if prof_p else None)
    render_b = sum(phases[k] for k in render_phases)
    render_p = sum(plain_phases[k] for k in render_phases) if plain_phases else None
    n_act = n_all
    roof = roofline(phases, n_act, n_vis, n_inst, n_blend, npix, deg, F, clocks, f"{tile[0]}x{tile[1]}/{stage}",
                    n_views=len(cams), n_eval=n_eval)
    out = {
        "metric": METRIC, "value": round(mpix_b, 2), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(ms_b / K, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded; stands in for KITTI/Replica-shaped keyframe windows)",
        "config": {"workload": "keyframe window: 8 views (4x1200x680, 2x640x480, 2x320x240) = 4,032,000 px over "
                               f"{n_all} Gaussians (SH3, FP32) in 64 chunks of 4 m",
                   "gaussians": n_all, "views": 8, "pixels": npix, "tile": f"{tile[0]}x{tile[1]}", "stage": stage,
                   "autotune": tune, "bwd_accumulation": args.bwd,
                   "l2": "inputs larger than L2 (parameters 472 MB per step)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "batched_direct_calls_ms_per_step": round(sum(v[0] for v in prof.values()) / K, 4),
        "plain": {"value": round(mpix_p, 2), "unit": UNIT, "ms_per_step": round(ms_p / K_p, 4),
                  "speedup_batched_over_plain": round(mpix_b / mpix_p, 3),
                  "phases_ms_per_step": plain_phases,
                  "render_only": {"phases": list(render_phases), "batched_ms": round(render_b, 4),
                                  "plain_ms": round(render_p, 4),
                                  "speedup_batched_over_plain": round(render_p / render_b, 3)}} if ms_p else None,
        "phases_ms_per_step": phases,
        "counts": {"visible_pairs": n_vis, "instances": n_inst, "tiles": n_tiles, "blend_evaluations": n_eval,
                   "blended_pairs": n_blend},
        "roofline": roof,
        "e2e": {"value": round(mpix_e, 2), "unit": UNIT, "h2d_bytes_per_step": int(4 * 4 * npix),
                "d2h_bytes_per_step": 4} if ms_e else None,
        "gpu_launches": int(launches_b),
        "clocks": clocks,
    }
    dcg.dcg_destroy(ctx)
    if not args.quick:
        out["train_step"] = train_leg(args, sc, cfg, tile, stage, trgb, tdep, rgb, depth, dr, dd, loss, grads, grads_t,
                                      dpose, npix, K, W)
        out["log_sample"] = sampling_leg(sc, npix, trgb, rgb, depth, K, W)
        out["loop_closure"] = loop_closure_leg(sc, max(4, K // 4))
        if not args.no_side_workloads:
            out["indoor"] = indoor_leg(K, W)
            out["mlp"] = mlp_leg()
            out["corridor"] = corridor_bench(1000.0, 8000, args.propose_every, train_length=1000.0)
    return out


def indoor_leg(K, W, cpu_pixels=24):
    """The indoor-room workload: 640x480 views and 500k Gaussians on the walls,
    floor and ceiling of a 10x8x3 m room (5 cm jitter, 4 m chunks, SH degree 3),
    one keyframe per step along a smooth random-walk trajectory: cull, gather,
    render fwd, L1 RGB + 0.1 L1 depth against the step's target, bwd, scatter.
    Mpix/s of the step, its phases and the dominant kernel's roofline; the FP64
    oracle times fwd + bwd on a pixel sample of one keyframe (all 500k
    Gaussians projected) on the host cores."""
    import torch

    import oracle
    from paper_2511_23030_b300 import dcg, synth

    steps = K + W
    sc = synth.room_indoor(0, n=500_000, n_steps=steps)
    P, cams, deg = sc["params"], sc["cams"], sc["deg"]
    n, F = P.shape
    Wd, Hd = cams[0].W, cams[0].H
    npx = Wd * Hd
    cfg = dcg.config(sh_degree=deg, max_active=n, max_views=1, max_pixels=npx, max_instances=48 << 20,
                     chunk_size=sc["chunk_size"], device_budget=n, host_capacity=n, dfar=20.0)
    ctx = dcg.dcg_create(cfg)
    try:
        g_t = torch.from_numpy(np.ascontiguousarray(P.T)).cuda()
        dcg.dcg_chunk_table_update(ctx, g_t, n)
        del g_t
        trgb = torch.from_numpy(np.stack([t.reshape(-1) for t in sc["target_rgb"]])).cuda()
        tdep = torch.from_numpy(np.stack([t.reshape(-1) for t in sc["target_depth"]])).cuda()
        rgb, depth = torch.zeros(3 * npx, device="cuda"), torch.zeros(npx, device="cuda")
        dr, dd = torch.zeros_like(rgb), torch.zeros_like(depth)
        loss = torch.zeros(1, device="cuda")
        grads_t = torch.zeros((F, n), device="cuda")
        grads = dcg.gaussians(grads_t, deg)
        dpose = torch.zeros(6, device="cuda")
        lam = sc["lambda_depth"]
        act = []

        def step(t):
            c = cams[t]
            g, na = dcg.dcg_gather_active(ctx, dcg.dcg_cull_chunks(ctx, [c]))
            dcg.dcg_render_fwd(ctx, g, na, [c], rgb, depth)
            loss.zero_()
            dcg.dcg_loss_l1(ctx, rgb, depth, trgb[t], tdep[t], [c], lam, dr, dd, loss)
            dcg.dcg_render_bwd(ctx, dr, dd, grads, dpose)
            dcg.dcg_scatter_back(ctx, g, na)
            act.append(na)

        stream = torch.cuda.current_stream()
        for t in range(W):
            step(t)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        act.clear()
        e0.record(stream)
        for t in range(W, steps):
            step(t)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        n_act = int(np.mean(act))
        # phases of the same steps (the library's event timers)
        dcg.dcg_profile(ctx, True)
        dcg.dcg_profile_read(ctx)
        vis = inst = blend = 0
        prof = {}
        for t in range(W, steps):
            step(t)
            nv, ni, _ = dcg.dcg_state_stats(ctx)
            _, nb = dcg.dcg_state_evals(ctx)
            vis, inst, blend = vis + nv, inst + ni, blend + nb
            if (t - W) % 100 == 99 or t + 1 == steps:  # the timers hold 4096 intervals between reads
                for key, (v, c) in dcg.dcg_profile_read(ctx).items():
                    a = prof.setdefault(key, [0.0, 0])
                    a[0] += v
                    a[1] += c
        dcg.dcg_profile(ctx, False)
        phases = {k: round(v[0] / K, 4) for k, v in prof.items() if k not in ("log_sample", "loop_closure")}
        roof = roofline(phases, n_act, vis // K, inst // K, blend // K, npx, deg, F, None, "", n_views=1)
    finally:
        dcg.dcg_destroy(ctx)
    # the oracle on a bounded sample of one keyframe
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    c = cams[W]
    pix = synth.pixel_sample(np.random.default_rng(3), Wd, Hd, cpu_pixels)
    t0 = time.perf_counter()
    o = oracle.render(P, deg, c, pix=pix, n_threads=cores)
    oracle.render_bwd(P, deg, c, np.sign(o["rgb"] - 0.5) / (3.0 * npx), lam * np.sign(o["depth"] - 3.0) / npx,
                      pix=pix, n_threads=cores)
    dt = time.perf_counter() - t0
    return {"what": "indoor room: one 640x480 keyframe per step (cull, gather, fwd, L1 + 0.1 L1 depth, bwd, "
                    "scatter) over 500k Gaussians (SH3) in 4 m chunks",
            "value": round(npx / (ms / 1e3) / 1e6, 2), "unit": UNIT, "ms_per_step": round(ms, 4), "steps": K,
            "warmup": W, "active_gaussians_mean": n_act, "phases_ms_per_step": phases, "roofline": roof,
            "cpu_baseline": {"value": round(len(pix) / dt / 1e6, 9), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(pix)} pixels of one keyframe, fwd+bwd, 500000 Gaussians projected",
                             "seconds": round(dt, 2)}}


def mlp_leg(reps=50):
    """The prefetch MLP's GEMMs on the two tensor-core paths (tcgen05 with TMA-staged operands, and
    mma.sync): forward of a 4096-candidate batch and one training step of a 2048-sample batch,
    timed with CUDA events over `reps` calls each.  FLOPs per forward: 2 x (128 x 256 + 2 x 256 x
    256) per row (the three hidden layers); a training step adds the two backward products per
    layer (about 3 x the forward)."""
    import torch

    from paper_2511_23030_b300 import dcg, synth

    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.normal(0, 1, (4096, 128)).astype(np.float32)).cuda().to(torch.bfloat16).view(torch.int16)
    y = torch.from_numpy((rng.uniform(size=4096) < 0.4).astype(np.float32)).cuda()
    prob = torch.zeros(4096, device="cuda")
    loss = torch.zeros(1, device="cuda")
    flop_row = 2 * (128 * 256 + 2 * 256 * 256)
    _, _, _ = peaks()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak = float(json.load(f)["bf16_tflops"])
            src = "measured"
    except Exception:
        bf16_peak, src = 1800.0, "fallback"
    out = {"what": "prefetch MLP 128-256-256-256-1, BF16 products, FP32 accumulation", "peak_bf16_tflops": bf16_peak,
           "peak_source": src}
    stream = torch.cuda.current_stream()
    for gemm in ("tcgen05", "mma_sync"):
        m = dcg.dcg_mlp_create(4096)
        try:
            dcg.dcg_mlp_set_gemm(m, gemm)
            dcg.dcg_mlp_set_params(m, synth.mlp_init_params(0))
            res = {}
            for name, fn, rows, mult in (("forward_4096", lambda: dcg.dcg_mlp_forward(m, x, 4096, prob), 4096, 1),
                                         ("train_step_2048",
                                          lambda: dcg.dcg_mlp_train_step(m, x[:2048], y[:2048], 2048, 1e-4, loss),
                                          2048, 3)):
                for _ in range(5):
                    fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    fn()
                e1.record(stream)
                torch.cuda.synchronize()
                us = e0.elapsed_time(e1) * 1e3 / reps
                tf = mult * flop_row * rows / (us * 1e-6) / 1e12
                res[name] = {"us": round(us, 2), "tflops": round(tf, 2), "frac": round(tf / bf16_peak, 4)}
            dcg.dcg_mlp_get_params(m)  # raises if a bounded wait of the tensor-core path gave up
            out[gemm] = res
        finally:
            dcg.dcg_mlp_destroy(m)
    return out


LAMBDA_S = 0.2  # weight of the SSIM term of Eq. 3 in the training leg (the 3DGS value)


def lr_per_component(F: int):
    """3DGS-style learning rates per parameter component (means, log-scales, quaternion,
    opacity logit, SH DC, SH rest)."""
    lr = np.zeros(F, np.float32)
    lr[0:3], lr[3:6], lr[6:10], lr[10] = 1.6e-4, 5e-3, 1e-3, 5e-2
    lr[11:14] = 2.5e-3
    lr[14:] = 2.5e-3 / 20
    return lr


def train_leg(args, sc, cfg, tile, stage, trgb, tdep, rgb, depth, dr, dd, loss, grads, grads_t, dpose, npix, K, W):
    """The whole training step of the window with Adam moments stored per Gaussian (they are
    gathered and scattered with the parameters): cull, gather, [fwd, loss of Eq. 2-4 with the SSIM
    term, bwd: graph], Adam, scatter.  Also times the Adam kernel and the loss alone."""
    import torch

    from paper_2511_23030_b300 import dcg

    cfg.with_moments = 1
    ctx = dcg.dcg_create(cfg)
    try:
        P, cams, deg = sc["params"], sc["cams"], sc["deg"]
        n_all, F = P.shape
        g_t = torch.from_numpy(np.ascontiguousarray(P.T)).cuda()
        dcg.dcg_chunk_table_update(ctx, g_t, n_all)
        del g_t
        dcg.dcg_set_launch(ctx, tile[0], tile[1], stage)
        lam = sc["lambda_depth"]
        lr = lr_per_component(F)
        stream = torch.cuda.current_stream()
        st = {"n": -1, "t": 0}

        def step():
            lst = dcg.dcg_cull_chunks(ctx, cams)
            g, n = dcg.dcg_gather_active(ctx, lst)
            if st["n"] != n:
                dcg.dcg_window_capture(ctx, g, n, cams, rgb, depth, trgb, tdep, lam, dr, dd, loss, grads, dpose,
                                       lambda_s=LAMBDA_S)
                st["n"] = n
            dcg.dcg_window_run(ctx, cams)
            st["t"] += 1
            dcg.dcg_adam_step(ctx, g, grads, n, lr, 0.9, 0.999, 1e-15, st["t"])
            dcg.dcg_scatter_back(ctx, g, n)
            return g, n

        for _ in range(W):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            g, n = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        # the Adam kernel alone (parameters, gradients and both moments exceed L2)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(3, K)
        a0.record(stream)
        for _ in range(reps):
            st["t"] += 1
            dcg.dcg_adam_step(ctx, g, grads, n, lr, 0.9, 0.999, 1e-15, st["t"])
        a1.record(stream)
        torch.cuda.synchronize()
        ms_adam = a0.elapsed_time(a1) / reps
        # the loss of Eq. 2-4 with and without its SSIM term
        ms_loss = {}
        for ls in (0.0, LAMBDA_S):
            a0.record(stream)
            for _ in range(reps):
                dcg.dcg_loss(ctx, rgb, depth, trgb, tdep, cams, ls, lam, dr, dd, loss)
            a1.record(stream)
            torch.cuda.synchronize()
            ms_loss[ls] = a0.elapsed_time(a1) / reps
        hbm, _, src = peaks()
        gbs = 28.0 * F * n / (ms_adam / 1e3) / 1e9  # read p, g, m, v; write p, m, v (FP32)
        return {"value": round(npix / (ms / 1e3) / 1e6, 2), "unit": UNIT, "ms_per_step": round(ms, 4),
                "optimizer": "Adam, moments stored per Gaussian in the chunks (3 F floats per Gaussian)",
                "loss": f"Eq. 2-4: lambda_s {LAMBDA_S} (SSIM, 11x11 Gaussian window), lambda_depth {lam}",
                "loss_ms": round(ms_loss[LAMBDA_S], 4), "loss_l1_only_ms": round(ms_loss[0.0], 4),
                "adam_ms": round(ms_adam, 4), "adam_roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm,
                                                                 "unit": "GB/s", "frac": round(gbs / hbm, 4),
                                                                 "bytes_per_launch": int(28 * F * n),
                                                                 "peak_source": src}}
    finally:
        dcg.dcg_destroy(ctx)


SAMPLE_FRACTION = 0.05  # sampling leg: kappa of Eq. 1 is set so that about this share of pixels is sampled


def sampling_leg(sc, npix, trgb, rgb, depth, K, W):
    """LoG penalty sampling of Eq. 1 over the window's 8 views in one call (the targets against the
    images the window rendered) and back-projection of the sampled pixels at the rendered depth in
    another.  The paper gives no kappa; it is set to SAMPLE_FRACTION / mean(P_s) over the window
    (from one pass that writes P_s and samples nothing), so about that share of pixels is sampled.
    Device time from the library's phase timers; algorithmic bytes per pixel: both images (24 B),
    the uniform (4 B), the flag written and read twice by the ordered compaction (12 B); per sample
    the index written and read (8 B), its depth and colour (16 B) and the new Gaussian (4 F B)."""
    import torch

    from paper_2511_23030_b300 import dcg

    cams, deg = sc["cams"], sc["deg"]
    F = sc["params"].shape[1]
    cap = npix // 4
    cfg = dcg.config(sh_degree=deg, max_active=1024, max_views=1, max_pixels=npix, max_instances=1 << 20,
                     chunk_size=sc["chunk_size"], device_budget=1024, host_capacity=1024, dfar=60.0)
    ctx = dcg.dcg_create(cfg)
    try:
        u = torch.rand(npix, generator=torch.Generator(device="cuda").manual_seed(7), device="cuda")
        idx = torch.zeros(cap, dtype=torch.int32, device="cuda")
        out = torch.zeros((F, cap), device="cuda")
        hbm, _, src = peaks()
        ps = torch.zeros(npix, device="cuda")
        dcg.dcg_log_sample_views(ctx, cams, trgb, rgb, 0.0, u, idx, ps_out=ps)
        mean_ps = float(ps.mean())
        kappa = SAMPLE_FRACTION / mean_ps if mean_ps > 0 else 0.0
        del ps

        def window():
            n, _ = dcg.dcg_log_sample_views(ctx, cams, trgb, rgb, kappa, u, idx)
            dcg.dcg_backproject_views(ctx, idx, n, depth, trgb, cams, -2.0, out)
            return n

        for _ in range(W):
            window()
        torch.cuda.synchronize()
        dcg.dcg_profile(ctx, True)
        dcg.dcg_profile_read(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ns = 0
        for _ in range(K):
            ns = window()
        e1.record()
        torch.cuda.synchronize()
        prof = dcg.dcg_profile_read(ctx)
        dcg.dcg_profile(ctx, False)
        dev_ms = prof["log_sample"][0] / K
        api_ms = e0.elapsed_time(e1) / K
        algo = 40 * npix + ns * (8 + 16 + 4 * F)
        gbs = algo / (dev_ms / 1e3) / 1e9
        return {"what": "Eq. 1 LoG penalty sampling of the 8 window views in one call (targets vs rendered) "
                        "+ back-projection",
                "pixels": npix, "kappa": round(kappa, 4), "mean_penalty": round(mean_ps, 5),
                "samples_per_window": int(ns), "sampled_fraction": round(ns / npix, 4),
                "device_ms_per_window": round(dev_ms, 4), "api_ms_per_window": round(api_ms, 4),
                "value": round(npix / (dev_ms / 1e3) / 1e6, 1), "unit": "Mpix/s",
                "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(gbs / hbm, 4), "bytes_per_window": int(algo), "peak_source": src},
                "launches_per_window": 6}
    finally:
        dcg.dcg_destroy(ctx)


def _rigid(deg_z, t):
    a = np.deg2rad(deg_z)
    C = np.eye(4, dtype=np.float32)
    C[:2, :2] = [[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]]
    C[:3, 3] = t
    return C


def loop_closure_leg(sc, K):
    """Loop-closure correction (Sec. III-F) of the window map: two keyframes' Gaussians move with
    their pose corrections and are redistributed over the chunks; corrections alternate with their
    inverses so the map stays near its start.  Wall time per call (host planning of the moved rows
    included) and the device phases; algorithmic device bytes per gathered Gaussian: the transform
    (10 floats read, 7 written), the keys (12 B read, 8 B written), the moved flags (flag and key read,
    flag written), their ordered compaction (flag read twice), the destinations (flag read, index
    written), the row permutation and the page writes (each 4 F B read and written)."""
    import time

    import torch

    from paper_2511_23030_b300 import dcg

    P, cams, deg = sc["params"], sc["cams"], sc["deg"]
    n_all, F = P.shape
    cfg = dcg.config(sh_degree=deg, max_active=n_all + 1024, max_views=8, max_pixels=max(c.W * c.H for c in cams),
                     max_instances=1 << 20, chunk_size=sc["chunk_size"], device_budget=n_all + (n_all >> 1),
                     host_capacity=2 * n_all, dfar=60.0)
    ctx = dcg.dcg_create(cfg)
    try:
        g_t = torch.from_numpy(np.ascontiguousarray(P.T)).cuda()
        dcg.dcg_chunk_table_update(ctx, g_t, n_all)
        del g_t
        kfs = [cams[0], cams[3]]
        fwd = [_rigid(0.5, (0.2, -0.1, 0.05)), _rigid(-0.4, (-0.15, 0.1, 0.02))]
        inv = [np.linalg.inv(C).astype(np.float32) for C in fwd]
        hbm, _, src = peaks()
        dcg.dcg_loop_closure(ctx, kfs, fwd)  # warm-up (allocations, host tier pages)
        dcg.dcg_loop_closure(ctx, kfs, inv)
        dcg.dcg_sync(ctx)
        dcg.dcg_profile(ctx, True)
        dcg.dcg_profile_read(ctx)
        wall, nts, nms, ngs = [], [], [], []
        for r in range(K):
            counts = dcg.dcg_chunk_info(ctx)["counts"]
            ngs.append(int(counts[dcg.dcg_cull_chunks(ctx, kfs)].sum()))  # the union the call gathers
            dcg.dcg_sync(ctx)
            t0 = time.perf_counter()
            nt, nm = dcg.dcg_loop_closure(ctx, kfs, fwd if r % 2 == 0 else inv)
            wall.append((time.perf_counter() - t0) * 1e3)
            nts.append(nt)
            nms.append(nm)
        prof = dcg.dcg_profile_read(ctx)
        dcg.dcg_profile(ctx, False)
        dev_ms = prof["loop_closure"][0] / K
        gather_ms = (prof["gather"][0] + prof["stall"][0]) / K
        n_g = float(np.mean(ngs))
        algo = int(n_g * (40 + 28 + 20 + 36 + 16 * F))
        gbs = algo / (dev_ms / 1e3) / 1e9
        return {"what": "loop-closure correction + chunk redistribution of the 2-keyframe union (synchronous call)",
                "gaussians": n_all, "gathered": int(n_g), "transformed": int(np.mean(nts)), "moved": int(np.mean(nms)),
                "wall_ms": round(float(np.median(wall)), 3), "device_ms": round(dev_ms, 4),
                "gather_ms": round(gather_ms, 4),
                "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(gbs / hbm, 4), "bytes_per_call": int(algo), "peak_source": src}}
    finally:
        dcg.dcg_destroy(ctx)


TRAFFIC_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "dram_traffic.json")
RASTER_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2511_23030_b300", "csrc", "raster.cu")


def measured_traffic(phase: str, launch: str, units: int, field: str = "dram_bytes_per_launch",
                     unit_key: str = "instances"):
    """A per-launch figure of the phase's kernel from the committed ncu capture (DRAM bytes, or warp
    instructions), scaled from the captured workload to this one by the units the kernel processes
    (instances for DRAM bytes: the blends read one record per instance; pixel-Gaussian evaluations
    for warp instructions: the per-pixel loops dominate them); None unless the capture is of this
    launch shape and of the rasteriser source as it is now."""
    import hashlib

    try:
        rec = json.load(open(TRAFFIC_FILE))
        sha = hashlib.sha256(open(RASTER_SRC, "rb").read()).hexdigest()
    except (OSError, ValueError):
        return None
    k = rec.get("kernels", {}).get(phase)
    if not k or field not in k or rec.get("raster_cu_sha256") != sha or rec.get("launch") != launch:
        return None
    if not rec.get(unit_key) or not units:
        return None
    return int(k[field] * units / rec[unit_key])


def roofline(phases, n_act, n_vis, n_inst, n_blend, npix, deg, F, clocks, launch="", n_views=8, n_eval=0):
    """Dominant phase with its algorithmic bytes (or FLOPs) per launch over its live duration."""
    hbm, sm_max, src = peaks()
    rec = 48
    algo_bytes = {
        # parameters once per call; per visible pair the record; per pair depth, tiles touched, rectangle
        "preprocess_fwd": 4 * F * n_act + n_vis * rec + 16 * n_views * n_act,
        # key write/read per visible pair and per instance (4 + 2 radix passes, 3 touches each), emission,
        # ranges and masks (instance read and write)
        "binning": 8 * 3 * n_vis * 4 + 8 * 3 * n_inst * 2 + 8 * n_inst + 12 * n_vis + 16 * n_inst,
        "blend_fwd": n_inst * (8 + rec) + npix * (4 * 4 + 8),
        "blend_bwd": n_inst * (8 + rec + 40) + npix * (4 * 4 + 8),
        # parameters read and gradients written once; per visible pair the 2D gradient slot read and
        # zeroed; per pair the tiles-touched flag
        "preprocess_bwd": 4 * F * n_act + n_vis * 2 * 48 + 4 * F * n_act + 4 * n_views * n_act,
        "gather": 2 * 4 * F * n_act,
        "scatter": 2 * 4 * F * n_act,
    }
    dom = max((k for k in algo_bytes), key=lambda k: phases.get(k, 0.0))
    t = phases[dom] / 1e3
    # every phase against the HBM peak (algorithmic bytes over its live time)
    by_phase = {k: {"gbs": round(b / (phases[k] / 1e3) / 1e9, 1), "frac": round(b / (phases[k] / 1e3) / 1e9 / hbm, 4)}
                for k, b in algo_bytes.items() if phases.get(k, 0.0) > 0.01}
    if dom in ("blend_fwd", "blend_bwd"):
        # FP32 issue bound: 148 SMs x 128 lanes x 2 FLOP per clock.  The algorithmic work is the
        # composited (pixel, Gaussian) pairs, independent of how the kernel culls: 22 FLOP per pair
        # forward, 55 backward (MUFU ex2 and the division counted as one FLOP each)
        flop_per_pair = 22 if dom == "blend_fwd" else 55
        peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12
        ach = n_blend * flop_per_pair / t / 1e12
        out = {"kernel": dom, "bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
               "frac": round(ach / peak, 4), "traffic": measured_traffic(dom, launch, n_inst),
               "hbm_gbs": round(algo_bytes[dom] / t / 1e9, 1),
               "hbm_frac": round(algo_bytes[dom] / t / 1e9 / hbm, 4), "peak_source": f"derived (sm_max {sm_max} MHz)",
               "hbm_by_phase": by_phase}
        # what bounds it: the warp-instruction issue rate (148 SMs x 4 schedulers x 1 per clock) against
        # the instructions ncu counted per launch (scaled by pixel-Gaussian evaluations)
        inst = measured_traffic(dom, launch, n_eval, "warp_instructions_per_launch", "evaluations")
        if inst is not None:
            ipeak = 148 * 4 * sm_max * 1e6
            out["issue"] = {"warp_instructions": inst, "achieved_ginst_s": round(inst / t / 1e9, 1),
                            "peak_ginst_s": round(ipeak / 1e9, 1), "frac": round(inst / t / ipeak, 4)}
        return out
    ach = algo_bytes[dom] / t / 1e9
    return {"kernel": dom, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(ach / hbm, 4), "traffic": measured_traffic(dom, launch, n_inst), "peak_source": src,
            "hbm_by_phase": by_phase}


# ----------------------------------------------------------------------------- CPU baseline (oracle)
def cpu_baseline(pix_per_view: int, views=None, n_gaussians=2_000_000, seed=0, scene=None, single_thread_pixels=0):
    """FP64 oracle fwd+bwd on a bounded pixel sample of the window (the whole
    scene is projected for every sampled view)."""
    import oracle

    from paper_2511_23030_b300 import synth

    oracle.build()
    sc = synth.window_scene(0, n=n_gaussians) if scene is None else scene
    P, cams = sc["params"], sc["cams"]
    views = range(len(cams)) if views is None else views
    rng = np.random.default_rng(seed)
    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    m = 0
    for v in views:
        c = cams[v]
        pix = synth.pixel_sample(rng, c.W, c.H, pix_per_view)
        o = oracle.render(P, sc["deg"], c, pix=pix, n_threads=cores)
        gr = np.sign(o["rgb"] - 0.5) / (3.0 * c.W * c.H)
        gd = 0.1 * np.sign(o["depth"] - 10.0) / (c.W * c.H)
        oracle.render_bwd(P, sc["deg"], c, gr, gd, pix=pix, n_threads=cores)
        m += len(pix)
    dt = time.perf_counter() - t0
    out = {"value": round(m / dt / 1e6, 8), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{m} pixels ({pix_per_view} per view, views {list(views)}) of the window, fwd+bwd, "
                     f"{n_gaussians} Gaussians projected per view", "seconds": round(dt, 2)}
    if single_thread_pixels:
        # the same on one host thread, on a smaller sample of the last view
        c = cams[list(views)[-1]]
        pix = synth.pixel_sample(rng, c.W, c.H, single_thread_pixels)
        t0 = time.perf_counter()
        o = oracle.render(P, sc["deg"], c, pix=pix, n_threads=1)
        gr = np.sign(o["rgb"] - 0.5) / (3.0 * c.W * c.H)
        gd = 0.1 * np.sign(o["depth"] - 10.0) / (c.W * c.H)
        oracle.render_bwd(P, sc["deg"], c, gr, gd, pix=pix, n_threads=1)
        dt1 = time.perf_counter() - t0
        out["single_thread"] = {"value": round(len(pix) / dt1 / 1e6, 9), "unit": UNIT, "cores": 1,
                                "sample": f"{len(pix)} pixels of view {list(views)[-1]}, fwd+bwd",
                                "seconds": round(dt1, 2)}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2511_23030_b300 import synth

    K, W = args.steps, args.warmup
    sc = synth.window_scene(0, n=args.gaussians)
    views = [5]  # one 640x480 view per step keeps the whole run within minutes
    for _ in range(min(W, 1)):
        cpu_baseline(4, views=views, n_gaussians=args.gaussians, scene=sc)
    t0 = time.perf_counter()
    m = 0
    cb = None
    for k in range(K):
        cb = cpu_baseline(16, views=views, n_gaussians=args.gaussians, seed=k, scene=sc)
        m += 16
    dt = time.perf_counter() - t0
    val = m / dt / 1e6
    cb["value"] = round(val, 8)
    cb["sample"] = f"per step 16 pixels of view 5 (640x480) of the window, fwd+bwd, {args.gaussians} Gaussians"
    return {"metric": METRIC, "value": round(val, 8), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": round(dt / K * 1e3, 2), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "keyframe window: 8 views (4x1200x680, 2x640x480, 2x320x240) = 4,032,000 px over "
                                   f"{args.gaussians} Gaussians (SH3) in 64 chunks of 4 m",
                       "parallelism": "host cores"},
            "cpu_baseline": cb, "e2e": {"value": round(val, 8), "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def run_corridor(args):
    return corridor_bench(args.length, args.per_m, args.propose_every, train_length=3000.0)


def corridor_bench(length, per_m, propose_every, train_length=3000.0):
    """Out-of-core mapping along a driving corridor (1241x376 views, 8 m chunks,
    5 km and 40 M Gaussians by default, device budget 15 % of the map capped
    at 6 M Gaussians, pinned host tier), one keyframe per metre:
    cull, gather, render fwd, L1 loss, bwd, scatter, then a prefetch proposal:
    none, constant-velocity extrapolation, or the learned MLP (trained here on
    a different drive, `train_length` metres, with samples the mapper
    generates from its exact cull).  Both predictors propose on a side stream
    every `propose_every` frames."""
    import torch

    from paper_2511_23030_b300 import build, dcg, prefetch, synth

    build.build()
    zfar, s = 60.0, 8.0
    W, H = 1241, 376
    t0 = time.perf_counter()
    # training drive (seed 1): chunk layout only, sparse Gaussians
    xy, head = synth.corridor_path(1, train_length)
    Ptr = synth.corridor_gaussians(np.random.default_rng(6), xy, head, 40, deg=0)
    cams_tr = synth.corridor_cameras(xy, head, W=W, H=H)
    for c in cams_tr:
        c.zfar = zfar
    ctx = dcg.dcg_create(dcg.config(sh_degree=0, max_active=Ptr.shape[0], max_views=1, max_pixels=W * H,
                                    chunk_size=s, device_budget=Ptr.shape[0], host_capacity=Ptr.shape[0], dfar=zfar,
                                    max_chunks=16384, page_gaussians=256))
    dcg.dcg_chunk_table_update(ctx, torch.from_numpy(np.ascontiguousarray(Ptr.T)).cuda(), Ptr.shape[0])
    X, y, n, pos = prefetch.make_dataset(ctx, cams_tr, s, 1.5 * zfar, max_samples=200_000)
    pm = prefetch.PrefetchMLP(max_batch=4096)
    dcg.dcg_mlp_set_params(pm.m, synth.mlp_init_params(0))
    t1 = time.perf_counter()
    losses = prefetch.train(pm, X, y, n, epochs=6, batch=2048, lr=1e-3)
    t_train = time.perf_counter() - t1
    dcg.dcg_destroy(ctx)
    del X, y
    # evaluation drive (seed 0)
    xy, head = synth.corridor_path(0, length)
    P = synth.corridor_gaussians(np.random.default_rng(5), xy, head, per_m, deg=3)
    cams = synth.corridor_cameras(xy, head, W=W, H=H)
    for c in cams:
        c.zfar = zfar
    N, F = P.shape
    # device active set: 6 M Gaussians on the 5 km drive; at least 1.2 M, which holds the chunks one
    # frame sees (about 0.5-0.7 M Gaussians at 8000 per metre), so that short drives run too
    budget = min(6_000_000, max(int(0.15 * N), 1_200_000))
    Pt = torch.from_numpy(np.ascontiguousarray(P.T))
    del P
    t_gen = time.perf_counter() - t0
    out = {"workload": "corridor", "metric": "out-of-core mapping Mpix/s, stall and hidden chunk-load share",
           "unit": UNIT, "config": {"length_m": length, "gaussians": N, "view": f"{W}x{H}", "chunk_m": s,
                                    "budget_gaussians": budget, "frames": len(cams),
                                    "propose_every": propose_every, "train_drive_m": train_length},
           "train": {"samples": n, "positive_frac": round(pos, 4), "loss_per_epoch": [round(v, 4) for v in losses],
                     "seconds": round(t_train, 2)}, "setup_seconds": round(t_gen, 1), "modes": {}}
    for mode in ("none", "cv", "mlp"):
        ctx = dcg.dcg_create(dcg.config(sh_degree=3, max_active=budget, max_views=1, max_pixels=W * H, chunk_size=s,
                                        device_budget=budget, host_capacity=N, dfar=zfar, max_chunks=16384,
                                        page_gaussians=512, max_instances=64 << 20))
        g_t = Pt.cuda()
        dcg.dcg_chunk_table_update(ctx, g_t, N)
        del g_t
        torch.cuda.empty_cache()
        pm.bind(ctx)
        rgb = torch.zeros(3 * W * H, device="cuda")
        depth = torch.zeros(W * H, device="cuda")
        dr, dd = torch.zeros_like(rgb), torch.zeros_like(depth)
        trgb = torch.rand(3 * W * H, device="cuda")
        tdep = torch.rand(W * H, device="cuda") * 30
        loss = torch.zeros(1, device="cuda")
        grads_t = torch.zeros((synth.n_fields(3), budget), device="cuda")
        grads = dcg.gaussians(grads_t, 3)

        def render(g, na, cam):
            dcg.dcg_render_fwd(ctx, g, na, [cam], rgb, depth)
            dcg.dcg_loss_l1(ctx, rgb, depth, trgb, tdep, [cam], 0.1, dr, dd, loss)
            dcg.dcg_render_bwd(ctx, dr, dd, grads, None)

        out["config"]["chunks"] = dcg.dcg_chunk_count(ctx)
        r = prefetch.run_corridor(ctx, cams, mode, s, 1.5 * zfar, pm=pm, render=render, every=propose_every)
        dcg.dcg_sync(ctx)
        r["ms_per_step"] = round(r["ms"] / r["steps"], 4)
        r["value"] = round(W * H * r["steps"] / (r["ms"] / 1e3) / 1e6, 2)
        r["io_frac"] = round(r["stall_ms"] / r["ms"], 4)
        r["hidden_load_frac"] = round(r["hidden_load_frac"], 4)
        out["modes"][mode] = r
        dcg.dcg_destroy(ctx)
    none_stall = out["modes"]["none"]["stall_ms"]
    for mode in ("cv", "mlp"):
        out["modes"][mode]["stall_hidden_vs_none"] = round(1 - out["modes"][mode]["stall_ms"] / max(none_stall, 1e-9), 4)
    pm.close()
    return out


def run_sampling(args):
    """The LoG sampling leg alone: the window is rendered once (forward) to give the rendered
    images and depth, then Eq. 1 sampling and back-projection of all 8 views are timed."""
    import torch

    from paper_2511_23030_b300 import build, dcg, synth

    build.build()
    sc = synth.window_scene(0, n=args.gaussians)
    P, cams = sc["params"], sc["cams"]
    n_all = P.shape[0]
    npix = sum(c.W * c.H for c in cams)
    cfg = dcg.config(sh_degree=sc["deg"], max_active=n_all + 1024, max_views=8, max_pixels=npix,
                     max_instances=160 << 20, chunk_size=sc["chunk_size"], device_budget=6_000_000,
                     host_capacity=n_all + 1024, dfar=60.0)
    ctx = dcg.dcg_create(cfg)
    try:
        g_t = torch.from_numpy(np.ascontiguousarray(P.T)).cuda()
        dcg.dcg_chunk_table_update(ctx, g_t, n_all)
        del g_t
        g, n = dcg.dcg_gather_active(ctx, dcg.dcg_cull_chunks(ctx, cams))
        rgb, depth = torch.zeros(3 * npix, device="cuda"), torch.zeros(npix, device="cuda")
        dcg.dcg_render_fwd(ctx, g, n, cams, rgb, depth)
        dcg.dcg_sync(ctx)
    finally:
        dcg.dcg_destroy(ctx)
    trgb = torch.from_numpy(np.concatenate([t.reshape(-1) for t in sc["target_rgb"]])).cuda()
    out = sampling_leg(sc, npix, trgb, rgb, depth, args.steps, args.warmup)
    out.update({"workload": "sampling", "metric": "LoG penalty sampling (Eq. 1) Mpix/s per keyframe window",
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
                "data": "synthetic window scene (8 views, 4,032,000 px)"})
    return out


def run_loss(args):
    """The image loss of Eq. 2-4 alone (L1 colour and depth plus the SSIM term, lambda_s = 0.2) and
    its gradient over the window's 8 views: the window is rendered once, then dcg_loss is timed with
    the library's phase timers.  SSIM bound: FP32 issue; its work is ~290 FMA per pixel and channel
    (the window passes of the 32 x 32-tile kernel), its bytes 24 per pixel and channel plus the L1
    parts (40 per pixel)."""
    import torch

    from paper_2511_23030_b300 import build, dcg, synth

    build.build()
    sc = synth.window_scene(0, n=args.gaussians)
    P, cams = sc["params"], sc["cams"]
    n_all = P.shape[0]
    npix = sum(c.W * c.H for c in cams)
    cfg = dcg.config(sh_degree=sc["deg"], max_active=n_all + 1024, max_views=8, max_pixels=npix,
                     max_instances=160 << 20, chunk_size=sc["chunk_size"], device_budget=6_000_000,
                     host_capacity=n_all + 1024, dfar=60.0)
    ctx = dcg.dcg_create(cfg)
    try:
        g_t = torch.from_numpy(np.ascontiguousarray(P.T)).cuda()
        dcg.dcg_chunk_table_update(ctx, g_t, n_all)
        del g_t
        g, n = dcg.dcg_gather_active(ctx, dcg.dcg_cull_chunks(ctx, cams))
        rgb, depth = torch.zeros(3 * npix, device="cuda"), torch.zeros(npix, device="cuda")
        dcg.dcg_render_fwd(ctx, g, n, cams, rgb, depth)
        trgb = torch.from_numpy(np.concatenate([t.reshape(-1) for t in sc["target_rgb"]])).cuda()
        tdep = torch.from_numpy(np.concatenate([t.reshape(-1) for t in sc["target_depth"]])).cuda()
        dr, dd, loss = torch.zeros_like(rgb), torch.zeros_like(depth), torch.zeros(1, device="cuda")

        def step():
            loss.zero_()
            dcg.dcg_loss(ctx, rgb, depth, trgb, tdep, cams, LAMBDA_S, sc["lambda_depth"], dr, dd, loss)

        for _ in range(args.warmup):
            step()
        dcg.dcg_sync(ctx)
        dcg.dcg_profile(ctx, True)
        dcg.dcg_profile_read(ctx)
        for _ in range(args.steps):
            step()
        prof = dcg.dcg_profile_read(ctx)
        dcg.dcg_profile(ctx, False)
        ms = prof["loss"][0] / args.steps
        hbm, sm_max, src = peaks()
        flops = 2 * 290 * 3 * npix
        peak = 148 * 128 * 2 * sm_max * 1e6 / 1e12
        return {"workload": "loss", "metric": "image loss (L1 + SSIM, Eq. 2-4) and gradient, Mpix/s per keyframe window",
                "value": round(npix / (ms / 1e3) / 1e6, 1), "unit": "Mpix/s", "ms_per_window": round(ms, 4),
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
                "lambda_s": LAMBDA_S, "loss": float(loss),
                "roofline": {"bound": "alu", "achieved": round(flops / (ms / 1e3) / 1e12, 2), "peak": round(peak, 1),
                             "unit": "TFLOP/s", "frac": round(flops / (ms / 1e3) / 1e12 / peak, 4),
                             "hbm_gbs": round((24 * 3 + 40) * npix / (ms / 1e3) / 1e9, 1), "hbm_peak": hbm,
                             "peak_source": f"derived (sm_max {sm_max} MHz); HBM {src}"},
                "data": "synthetic window scene (8 views, 4,032,000 px)"}
    finally:
        dcg.dcg_destroy(ctx)


def main():
    args = parse()
    if args.workload == "loss":
        print(json.dumps(run_loss(args)))
        return
    if args.workload == "corridor":
        print(json.dumps(run_corridor(args)))
        return
    if args.workload == "sampling":
        print(json.dumps(run_sampling(args)))
        return
    if args.workload == "loopclosure":
        from paper_2511_23030_b300 import build, synth

        build.build()
        out = loop_closure_leg(synth.window_scene(0, n=args.gaussians), args.steps)
        out.update({"workload": "loopclosure", "metric": "loop-closure correction ms per call (2M-Gaussian map)",
                    "steps": args.steps, "higher_is_better": False, "dtype": "f32",
                    "data": "synthetic window scene (2 keyframes corrected)"})
        print(json.dumps(out))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch

        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group(backend)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world)
        if rank == 0 and not args.no_cpu_baseline and not args.quick:
            out["cpu_baseline"] = cpu_baseline(args.cpu_pixels, views=[0, 5], n_gaussians=args.gaussians,
                                               single_thread_pixels=4)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
