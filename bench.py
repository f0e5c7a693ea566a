#!/usr/bin/env python
"""Post-densification refinement throughput with the SkipGS gate vs the
always-backward loop, on the 3M-Gaussian synthetic workload (SH degree 3,
200 ring views at 1297x840, views drawn uniformly, targets rendered from a
ground-truth scene; the gate with W=500, beta=0.95, eps=1e-8, rho_lo=0.5).

A step is one refinement iteration: view selection, projection, binning and
sort, compositing, loss, gate decision, and - when the gate opens - the loss
gradient, raster and projection adjoint and Adam, then the EMA update.  Each
loop runs as one captured CUDA graph per iteration (the backward branch is an
IF node set on the device).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gsr|reference]

Under torchrun every rank runs its own replica on its own GPU (the loop
does not shard); value = all ranks' iterations / max wall time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "post-densif. iters/s fwd+gated bwd vs full bwd; bwd ms/view at 3M Gaussians"
WORKLOAD = ("3M Gaussians SH3, 200 jittered-ring views 1297x840, post-densification refinement loop "
            "started after 5000 always-backward iterations, SkipGS gate W=500 beta=0.95 eps=1e-8 rho_lo=0.5, "
            "views uniform (seed 0), FP32 params + Adam")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gsr", choices=["gsr", "reference"])
    ap.add_argument("--n", type=int, default=3_000_000)
    ap.add_argument("--views", type=int, default=200)
    ap.add_argument("--width", type=int, default=1297)
    ap.add_argument("--height", type=int, default=840)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="budget of the oracle CPU baseline")
    ap.add_argument("--ref-seconds", type=float, default=150.0, help="budget of the reference arm")
    ap.add_argument("--pre", type=int, default=5000, help="always-backward iterations before the measured loop")
    ap.add_argument("--c4", action="store_true",
                    help="batched workload instead of the default line: 8 ring views per iteration at mixed "
                         "resolutions (640x360 .. 1600x1063), launch shape autotuned; prints its own JSON line")
    ap.add_argument("--rho-sweep", action="store_true",
                    help="NEXT-1: gated loop for rho_lo in (no budget, 0.3, 0.5, 0.7, 0.9) against the "
                         "always-backward loop; prints its own JSON line")
    ap.add_argument("--stages-once", action="store_true",
                    help="run two eager iterations of every stage on one view of the workload and exit "
                         "(a small, fixed launch sequence for hardware-counter captures)")
    return ap.parse_args()


def run_c4(args) -> None:
    """Batched refinement: B = 8 views per iteration, each of the 200 ring
    cameras at a resolution drawn from the four C4 sizes; launch shape chosen
    by the autotuner; gated vs always-backward loops from the same
    post-pre-phase snapshot (graph replays, CUDA events)."""
    import numpy as np
    import torch

    import synth
    from paper_2603_08997_gb300 import autotune, build, raster
    from paper_2603_08997_gb300.refine import RefinementLoop

    build.build()
    B = 8
    K = args.steps if args.steps != 5000 else 300
    pre_iters = args.pre if args.pre != 5000 else 300
    gt, start, cams, seq = synth.case_c4_ring(n=args.n, n_views=args.views, n_iters=max(K, pre_iters) + 64,
                                              views_per_step=B)
    dev = torch.device("cuda", 0)
    cap = 512 * 1024 * 1024
    # targets: renders of the ground-truth scene at each camera's own size
    mgt = raster.GaussianModel.from_scene(gt, dev)
    targets = []
    for cam in cams:
        r = raster.Renderer(args.n, 3, raster.Views([cam], 16, dev), raster.RasterSettings(), 40 * args.n, dev)
        r.forward(mgt.c_params())
        targets.append(r.image.view(3, cam.height, cam.width).clone())
        del r
    torch.cuda.synchronize()
    del mgt
    torch.cuda.empty_cache()
    model = raster.GaussianModel.from_scene(start, dev)
    cands = tuple((t, b, 1, 2) for t in (8, 16, 32) for b in (128, 256))
    st, tune_ms = autotune.autotune(model, cams, targets, candidates=cands, views_per_step=B, reps=2,
                                    pair_capacity=cap)
    pre = RefinementLoop(model, cams, targets, synth.pre_sequence(pre_iters * B, args.views), st, gated=False,
                         pair_capacity=cap, views_per_step=B)
    pre.capture()
    for _ in range(pre_iters):
        pre.step_graph()
    init = pre.snapshot()
    pre.close()
    del pre

    def timed(gated: bool):
        loop = RefinementLoop(model, cams, targets, seq, st, gated=gated, pair_capacity=cap, views_per_step=B)
        loop.restore(init)
        loop.capture()
        for _ in range(args.warmup):
            loop.step_graph()
        loop.restore(init)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(loop.stream)
        for _ in range(K):
            loop.step_graph()
        e1.record(loop.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        final = float(np.mean(loop.evaluate()))
        gs = loop.gate.read(loop.stream)
        status = int(loop.renderer.status.item())
        loop.close()
        return ms, final, gs, status

    ms_full, loss_full, _, s_full = timed(False)
    ms_gated, loss_gated, gs, s_gated = timed(True)
    print(json.dumps({
        "metric": "batched refinement: iters/s with 8 views per iteration (gated vs always-backward)",
        "value": K / (ms_gated * 1e-3), "unit": "iters/s", "views_per_s": B * K / (ms_gated * 1e-3),
        "full_bwd_iters_per_s": K / (ms_full * 1e-3), "gated_speedup": ms_full / ms_gated,
        "steps": K, "views_per_step": B, "pre_iterations": pre_iters,
        "gate": {"decisions": gs["t"], "backward_views": gs["b"], "rho_cum": gs["b"] / max(gs["t"], 1)},
        "final_loss_gated": loss_gated, "final_loss_full": loss_full,
        "final_loss_rel_diff": (loss_gated - loss_full) / loss_full,
        "autotuned": {"tile": st.tile, "batch": st.batch, "pixels_per_thread_fwd": st.pixels_per_thread_fwd,
                      "pixels_per_thread_bwd": st.pixels_per_thread,
                      "candidates_ms": {f"{t}/{b}/{pf}/{pb}": v for (t, b, pf, pb), v in tune_ms.items()}},
        "device_status": [s_full, s_gated], "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.n // 1000000}M Gaussians SH3, {args.views} ring views at resolutions drawn "
                               "from 640x360/980x545/1297x840/1600x1063, 8 views per iteration",
                   "n_gaussians": args.n}}))


def setup_c3(args, dev):
    """The C3 workload: ground-truth targets rendered on the GPU, the start
    scene, and the untimed always-backward pre-phase (stand-in for
    densification) whose end state both timed loops start from.  Returns
    (model, cameras, targets, view sequence, snapshot, settings, capacity,
    start scene)."""
    import torch

    import synth
    from paper_2603_08997_gb300 import raster
    from paper_2603_08997_gb300.refine import RefinementLoop

    seq_len = max(args.steps, 5000)
    gt, start, cams, seq = synth.case_c3(n=args.n, n_views=args.views, n_iters=seq_len,
                                         width=args.width, height=args.height)
    st = raster.RasterSettings()
    cap = 24 * args.n
    # targets: renders of the ground-truth scene (device-resident)
    mgt = raster.GaussianModel.from_scene(gt, dev)
    slot = raster.Views([cams[0]], st.tile, dev)
    rgt = raster.Renderer(args.n, 3, slot, st, cap, dev)
    targets = torch.empty((args.views, 3, args.height, args.width), dtype=torch.float32, device=dev)
    for v, cam in enumerate(cams):
        rgt.views = raster.Views([cam], st.tile, dev)
        rgt.forward(mgt.c_params())
        targets[v].copy_(rgt.image.view(3, args.height, args.width))
    torch.cuda.synchronize()
    del mgt, rgt
    model = raster.GaussianModel.from_scene(start, dev)
    # the measured loops start from the pre-phase's end state, parameters and
    # Adam moments carried over
    pre = RefinementLoop(model, cams, targets, synth.pre_sequence(max(args.pre, 1), args.views), st,
                         gated=False, pair_capacity=cap)
    pre.capture()
    for _ in range(args.pre):
        pre.step_graph()
    init = pre.snapshot()
    pre.close()
    del pre
    return model, cams, targets, seq, init, st, cap, start


def run_rho_sweep(args) -> None:
    """NEXT-1: the gated loop from the same snapshot for several budget floors
    rho_lo (rho_lo < 0: no budget, Table 4's ablation): realised rho_cum,
    iterations/s and final loss, plus the always-backward reference; the
    gated runs log the per-iteration gradient and update norms."""
    import numpy as np
    import torch

    from paper_2603_08997_gb300 import build
    from paper_2603_08997_gb300.refine import RefinementLoop

    build.build()
    dev = torch.device("cuda", 0)
    model, cams, targets, seq, init, st, cap, _ = setup_c3(args, dev)
    K = args.steps

    def run(gated: bool, rho_lo: float):
        loop = RefinementLoop(model, cams, targets, seq, st, gated=gated, rho_lo=rho_lo, pair_capacity=cap,
                              log_capacity=K)
        loop.restore(init)
        loop.capture()
        torch.cuda.synchronize()
        # timed in segments ending at the final-loss checkpoints K-3s .. K (as
        # the headline loops); the evaluations between segments are not timed
        seg = max(1, min(250, K // 4))
        marks = sorted({m for m in (K - 3 * seg, K - 2 * seg, K - seg, K) if m > 0})
        ms, done, evals = 0.0, 0, []
        for mark in marks:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(loop.stream)
            for _ in range(mark - done):
                loop.step_graph()
            e1.record(loop.stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            done = mark
            if mark == K:
                log = loop.read_log(K)
            evals.append(float(np.mean(loop.evaluate())))
        final = float(np.mean(evals))
        gs = loop.gate.read(loop.stream)
        loop.close()
        tenth = max(1, K // 10)
        stepped = log["g"][:, 0] > 0
        gn = np.sqrt(log["grad_sq"][stepped]) if stepped.any() else np.zeros(1)
        un = np.sqrt(log["update_sq"][stepped]) if stepped.any() else np.zeros(1)
        return {"rho_lo": rho_lo if gated else None, "gated": gated, "iters_per_s": K / (ms * 1e-3),
                "rho_cum": gs["b"] / max(gs["t"], 1), "rho_min": gs["rho_min"], "final_loss": final,
                "grad_norm_first_tenth": float(np.mean(gn[:tenth])), "grad_norm_last_tenth": float(np.mean(gn[-tenth:])),
                "update_norm_first_tenth": float(np.mean(un[:tenth])),
                "update_norm_last_tenth": float(np.mean(un[-tenth:]))}

    rows = [run(False, 0.5)] + [run(True, r) for r in (-1.0, 0.3, 0.5, 0.7, 0.9)]
    full = rows[0]
    for r in rows[1:]:
        r["speedup"] = r["iters_per_s"] / full["iters_per_s"]
        r["final_loss_rel_diff"] = (r["final_loss"] - full["final_loss"]) / full["final_loss"]
    print(json.dumps({"metric": "rho_lo sweep of the gated refinement loop (NEXT-1)", "steps": K,
                      "workload": WORKLOAD, "rows": rows}))


def stages_once(args) -> None:
    """Two eager forward + backward iterations of every stage (and of the
    unfused projection adjoint + Adam) on view 0 of the workload's scene
    (perturbed start, ground-truth target), for counters."""
    import torch

    import synth
    from paper_2603_08997_gb300 import build, raster

    build.build()
    gt, start, cams, _ = synth.case_c3(n=args.n, n_views=4, n_iters=10, width=args.width, height=args.height)
    views = raster.Views([cams[0]], 16)
    r = raster.Renderer(args.n, 3, views, raster.RasterSettings(), pair_capacity=24 * args.n)
    r.forward(raster.GaussianModel.from_scene(gt).c_params())
    torch.cuda.synchronize()
    target = r.image.clone()
    m = raster.GaussianModel.from_scene(start)
    adam = raster.AdamState(m)
    p, gr = m.c_params(), m.c_grads(adam.grad)
    for _ in range(2):
        r.forward(p)
        r.compute_loss(target)
        r.loss_backward(target)
        r.raster_bwd()
        r.project_bwd_adam(m, adam)  # the loop's backward branch
        r.project_bwd(p, gr)         # its unfused alternative
        adam.step()
    torch.cuda.synchronize()
    print(json.dumps({"stages_once": True, "status": int(r.status.item()), "pairs": int(r.pair_count.item())}))


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.f = open(self.path, "w")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self) -> dict:
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------- CPU oracle arm

def oracle_sample_step(scene, cam, frac: float, seed: int = 0):
    """One oracle refinement iteration on a bounded sample of the workload: the
    crop of the view covering `frac` of its pixels (centred) with the Gaussians
    whose projected centres fall in it (plus a 16-pixel border), against a
    seeded target.  Returns (seconds, pixels of the crop)."""
    import numpy as np

    import oracle
    import synth

    rc = oracle.RasterConfig()
    W, H = cam.width, cam.height
    cw = max(16, int(round(W * math.sqrt(frac))))
    ch = max(16, int(round(H * math.sqrt(frac))))
    x0, y0 = (W - cw) // 2, (H - ch) // 2
    crop = synth.Camera(cam.R, cam.t, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, cw, ch, cam.znear)
    key = ("proj_full", id(cam))
    if key not in scene.extra:
        scene.extra[key] = oracle.project(scene, cam, rc)  # sample selection only, untimed
    skey = ("sample", id(cam), cw, ch)  # the crop's Gaussians, untimed, reused by later steps of one size
    if skey not in scene.extra:
        pr = scene.extra[key]
        m = pr["mean2d"]
        sel = np.nonzero((pr["touched"] > 0) & (m[:, 0] > x0 - 16) & (m[:, 0] < x0 + cw + 16) &
                         (m[:, 1] > y0 - 16) & (m[:, 1] < y0 + ch + 16))[0]
        scene.extra[skey] = synth.Scene(scene.means[sel], scene.log_scales[sel], scene.quats[sel],
                                        scene.opacity_logit[sel], scene.sh[sel])
    sub = scene.extra[skey]
    target = np.random.default_rng(seed).uniform(0, 1, (3, ch, cw))
    from oracle.adam import AdamConfig, adam_step, lr_vector
    cfg = AdamConfig()
    p = sub.flat().astype(np.float64)
    lr = lr_vector(sub.n, sub.sh.shape[1], cfg)
    t0 = time.perf_counter()
    f = oracle.forward(sub, crop, rc)
    L, dL = oracle.loss_and_grad(f["image"], target)
    g = oracle.backward(sub, crop, rc, f, dL)
    gflat = np.concatenate([g["means"].ravel(), g["log_scales"].ravel(), g["quats"].ravel(),
                            g["opacity_logit"].ravel(), g["sh"].ravel()])
    adam_step(p, gflat, np.zeros_like(p), np.zeros_like(p), 0, lr, cfg)
    return time.perf_counter() - t0, cw * ch


def cpu_baseline(args, scene, cam, budget_s: float) -> dict:
    """The FP64 oracle timed on this host's cores on bounded crops of one view,
    scaled to iterations/s of the full view (the oracle's cost grows with the
    crop's pixels and the Gaussians over them)."""
    import oracle
    oracle.core.build()
    cores = oracle.num_threads()
    dt, px = oracle_sample_step(scene, cam, 0.01)
    full_px = cam.width * cam.height
    frac = min(1.0, 0.01 * (budget_s / 3.0) / max(dt, 1e-3))
    total, pix, runs = 0.0, 0, 0
    while total < budget_s * 0.5 and runs < 3:
        dt, px = oracle_sample_step(scene, cam, frac, seed=runs)
        total += dt
        pix += px
        runs += 1
    its = (pix / full_px) / total
    return {"value": its, "unit": "iters/s", "cores": cores, "kind": "oracle",
            "sample": f"{runs} oracle iteration(s) on a centred crop of {pix // runs} px of view 0 "
                      f"({100.0 * pix / runs / full_px:.1f}% of 1297x840) with the Gaussians over it; "
                      f"{total:.1f} s CPU wall time, scaled to the full view by the pixel fraction"}


def run_reference(args) -> None:
    import synth
    K, W = args.steps, args.warmup
    gt, start, cams, seq = synth.case_c3(n=args.n, n_views=args.views, n_iters=max(K, 1),
                                         width=args.width, height=args.height)
    cam = cams[int(seq[0])]
    import oracle
    oracle.core.build()
    cores = oracle.num_threads()
    dt, _ = oracle_sample_step(start, cam, 0.002)
    per_step = args.ref_seconds / (K + W)
    frac = max(1e-4, min(1.0, 0.002 * per_step / max(dt, 1e-4)))
    for w in range(W):
        oracle_sample_step(start, cam, frac, seed=w)
    total, pix = 0.0, 0
    for k in range(K):
        dt, px = oracle_sample_step(start, cam, frac, seed=100 + k)
        total += dt
        pix += px
    value = (pix / (args.width * args.height)) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_gaussians": args.n, "views": args.views,
                       "width": args.width, "height": args.height},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: one FP64 oracle iteration on a centred crop covering "
                                       f"{100 * frac:.3f}% of the view's pixels with the Gaussians over it, "
                                       f"scaled to the full view by the pixel fraction"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU arm

PEAK_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # FP32 lanes x FMA x max SM clock
BACKWARD_STAGES = ("loss_bwd", "raster_bwd", "project_bwd_adam")
UNFUSED_STAGES = ("project_bwd", "adam")  # the loop's fused=False alternative to project_bwd_adam


def stage_times(loop, targets, b_frac: float, reps: int = 10) -> dict:
    """Time every entry point of one refinement iteration on the loop's stream
    (CUDA events, `reps` launches each, state of the loop's last view)."""
    import torch
    r, s, adam = loop.renderer, loop.stream, loop.adam
    params, grads = loop.params, loop.grads
    snap = loop.snapshot()
    fns = {
        "project": lambda: r.project(params, s),
        "bin_sort": lambda: r.bin_sort(s),
        "render_fwd": lambda: r.render_fwd(s),
        "loss": lambda: r.compute_loss(loop.targets, loop.target_offsets, loop.view_ids, stream=s),
        "loss_bwd": lambda: r.loss_backward(loop.targets, loop.target_offsets, loop.view_ids, stream=s),
        "raster_bwd": lambda: r.raster_bwd(stream=s),
        "project_bwd": lambda: r.project_bwd(params, grads, stream=s),
        "adam": lambda: adam.step(stream=s),
        "project_bwd_adam": lambda: r.project_bwd_adam(loop.model, adam, stream=s),
    }
    out = {}
    with torch.cuda.stream(s):
        for name, fn in fns.items():
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
            torch.cuda.synchronize()
            out[name] = {"ms": e0.elapsed_time(e1) / reps}
    loop.restore(snap)
    return weigh_stages(out, b_frac)


def weigh_stages(out: dict, b_frac: float) -> dict:
    """Each stage's weight in a gated iteration (1 every step, b_frac for the
    backward branch, 0 for the unfused alternative the loop does not run) and
    its share of the weighted sum; `out` maps stage -> {"ms": ...}."""
    tot = 0.0
    for name, v in out.items():
        v["weight"] = 0.0 if name in UNFUSED_STAGES else (b_frac if name in BACKWARD_STAGES else 1.0)
        tot += v["weight"] * v["ms"]
    for v in out.values():
        v["share"] = v["weight"] * v["ms"] / tot
    return out


def roofline_of(stages: dict, loop, args) -> dict:
    """Roofline of the stage with the largest share of the gated iteration.
    Algorithmic work per launch: HBM stages count bytes
    a launch must move; compositing stages count FLOPs per evaluated
    (pixel, Gaussian) pair, with the evaluated pairs counted as sum(n_last)."""
    import json as _json
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_note = "of measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "of fallback 6.8 TB/s"
    r = loop.renderer
    N = r.n
    E = N * r.views.n
    P = int(r.pair_count.item())
    px = r.views.total_pixels
    evals = float(r.n_last.double().sum().item())
    T = r.views.total_tiles
    chunk = max(1024, -(-(-(-N // 304)) // 256) * 256)  # entries per chunk of the tile counting sort
    n_c = -(-N // chunk) * r.views.n
    params = loop.model.flat.numel()
    work = {
        "project": ("hbm", N * (236 + 68), "bytes: 236 B parameters read + 68 B record, rectangle, count written per Gaussian"),
        "bin_sort": ("hbm", 148 * E + 4 * P + 16 * n_c * T + 8 * T,
                     "bytes: 148 B per (view, Gaussian) entry (depth keys 16, four radix passes 80, clipped "
                     "rectangles 32, counting 8, placement 12) + 4 B per (Gaussian, tile) pair + 16 B per "
                     "(chunk, tile) count-matrix cell + 8 B per tile range"),
        "render_fwd": ("alu", 12.0 * evals, "FLOP: 12 per evaluated pair"),
        "loss": ("hbm", 60 * px, "bytes: 60 B per pixel"),
        "loss_bwd": ("hbm", 72 * px, "bytes: 72 B per pixel"),
        "raster_bwd": ("alu", 40.0 * evals, "FLOP: 40 per evaluated pair"),
        "project_bwd": ("hbm", N * (236 + 48 + 236), "bytes: 520 B per Gaussian"),
        "adam": ("hbm", 28 * params, "bytes: 28 B per parameter (read p, g, m, v; write p, m, v)"),
        "project_bwd_adam": ("hbm", N * 48 * r.views.n + 24 * params,
                             "bytes: 48 B of 2D gradients per (view, Gaussian) + 24 B per parameter "
                             "(read p, m, v; write p, m, v)"),
    }
    name = max(stages, key=lambda k: stages[k]["share"])
    bound, units, note = work[name]
    traffic, traffic_note = stage_traffic(name)
    t = stages[name]["ms"] * 1e-3
    if bound == "hbm":
        achieved, peak, unit, pk_note = units / t / 1e9, hbm, "GB/s", hbm_note
    else:
        achieved, peak, unit = units / t / 1e12, PEAK_ALU_TFLOPS, "TFLOP/s"
        pk_note = "derived FP32 peak: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz"
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": traffic, "traffic_note": traffic_note, "work_per_launch": units, "work_def": note, "launch_ms": t * 1e3,
            "share_of_gated_iteration": stages[name]["share"], "peak_note": pk_note,
            "all_stages": {k: {"bound": w[0], "achieved": (w[1] / (stages[k]["ms"] * 1e-3)) / (1e9 if w[0] == "hbm" else 1e12),
                               "frac": (w[1] / (stages[k]["ms"] * 1e-3)) / (1e9 if w[0] == "hbm" else 1e12) /
                               (hbm if w[0] == "hbm" else PEAK_ALU_TFLOPS)} for k, w in work.items()}}


def sources_sha256() -> str:
    """Digest of the CUDA sources (any kernel change invalidates stored counters)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2603_08997_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def stage_traffic(stage: str):
    """DRAM bytes per launch of a stage from the committed ncu summary, or
    None when the kernels changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "stage_traffic_3M.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None, "no stored capture"
    if rec.get("sources_sha256") != sources_sha256():
        return None, "kernels changed since the stored capture"
    b = rec.get("per_launch_bytes", {}).get(stage)
    return (float(b) if b is not None else None), "profiles/stage_traffic_3M.json (ncu dram__bytes_read.sum + dram__bytes_write.sum)"


def aggregate_time(t_local: float, dist, device) -> float:
    """Job time = the slowest rank's timed region (replicas, no data exchange)."""
    if dist is None:
        return t_local
    import torch
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps: int, world: int, t_max: float) -> float:
    """Iterations of all ranks per second of the slowest rank."""
    return steps * world / t_max


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if args.stages_once:
        stages_once(args)
        return
    if args.c4:
        run_c4(args)
        return
    if args.rho_sweep:
        run_rho_sweep(args)
        return

    import numpy as np
    import torch

    import synth
    from paper_2603_08997_gb300 import build, gsr, raster
    from paper_2603_08997_gb300.refine import HostTargets, RefinementLoop

    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    K, W = args.steps, args.warmup
    dev = torch.device("cuda", local)
    model, cams, targets, seq, init, st, cap, start = setup_c3(args, dev)

    def timed_loop(gated: bool):
        loop = RefinementLoop(model, cams, targets, seq, st, gated=gated, pair_capacity=cap)
        loop.restore(init)
        loop.capture()
        for _ in range(W):
            loop.step_graph()
        loop.restore(init)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clock = ClockSampler(local) if (gated and rank == 0) else None
        # timed in segments that end at the final-loss checkpoints K-3s, K-2s,
        # K-s and K; the all-view evaluations between segments are not timed
        seg = max(1, min(250, K // 4))
        marks = sorted({m for m in (K - 3 * seg, K - 2 * seg, K - seg, K) if m > 0})
        ms, done, evals = 0.0, 0, []
        t0 = time.perf_counter()
        for mark in marks:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("timed_gated" if gated else "timed_full")
            e0.record(loop.stream)
            for _ in range(mark - done):
                loop.step_graph()
            e1.record(loop.stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            ms += e0.elapsed_time(e1)
            done = mark
            if mark >= K - 3 * seg:
                evals.append(float(np.mean(loop.evaluate())))
        wall = time.perf_counter() - t0
        clocks = clock.stop() if clock else None
        gs = loop.gate.read(loop.stream)
        status = int(loop.renderer.status.item())
        final = float(np.mean(evals))
        return loop, ms, wall, gs, status, final, clocks

    full, ms_full, wall_full, gs_full, st_full, loss_full, _ = timed_loop(False)
    kc_full = full.kernels_per_step
    full.close()
    gated, ms_gated, wall_gated, gs_gated, st_gated, loss_gated, clocks = timed_loop(True)
    kc_gated = gated.kernels_per_step

    # per-stage timing on the loop's stream (CUDA events, after the timed loops),
    # weighted by how often each stage runs in the gated loop
    stages = stage_times(gated, targets, b_frac=gs_gated["b"] / K)
    roofline = roofline_of(stages, gated, args)
    # end-to-end through the C ABI with host-resident targets
    e2e = None
    if not args.no_e2e:
        host_targets = targets.cpu().pin_memory()
        del targets
        torch.cuda.empty_cache()
        slot_target = torch.empty((1, 3, args.height, args.width), dtype=torch.float32, device=dev)
        gated.close()
        del gated
        loop = RefinementLoop(model, cams, slot_target, seq, st, gated=True, pair_capacity=cap)
        # every view's target is the slot the host fills each step
        loop.target_offsets = torch.zeros(len(cams), dtype=torch.int64, device=dev)
        loop.restore(init)
        loop.capture()
        loss_host = torch.empty(K, dtype=torch.float32).pin_memory()
        g_host = torch.empty(K, dtype=torch.uint8).pin_memory()
        seq_np = np.asarray(seq)

        feeder = HostTargets(loop, host_targets, seq_np)

        def e2e_step(k):
            feeder.step()  # target from pinned host memory, copied while the previous iteration runs
            with torch.cuda.stream(loop.stream):
                loss_host[k:k + 1].copy_(loop.renderer.loss, non_blocking=True)
                g_host[k:k + 1].copy_(loop.g, non_blocking=True)

        for k in range(W):
            e2e_step(k)
        loop.restore(init)
        feeder.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(K):
            e2e_step(k)
        torch.cuda.synchronize()
        wall_e2e = time.perf_counter() - t0
        e2e = {"value": K / wall_e2e, "unit": "iters/s",
               "h2d_bytes_per_step": 3 * args.height * args.width * 4, "d2h_bytes_per_step": 4 + 1}
        loop.close()

    # aggregate over ranks: max time
    t_gated = aggregate_time(ms_gated * 1e-3, dist, dev)
    if dist:
        dist.barrier()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    b = gs_gated["b"]
    it_full = K / (ms_full * 1e-3)
    it_gated = job_value(K, 1, t_gated)
    t_bwd = (ms_full - ms_gated) / max(K - b, 1)          # ms per backward (per view)
    t_fwd_ms = ms_full / K - t_bwd
    launches = kc_gated[0] * K + kc_gated[1] * b
    line = {
        "metric": METRIC, "value": job_value(K, world, t_gated), "unit": "iters/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_gated / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_gaussians": args.n, "views": args.views, "width": args.width,
                   "height": args.height, "iterations_timed": K, "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (2.8 GB of parameters and Adam state, 2.6 GB of targets)"},
        "full_bwd_iters_per_s": it_full * world, "gated_speedup": it_gated / it_full,
        "bwd_ms_per_view": t_bwd, "fwd_ms_per_view": t_fwd_ms,
        "backward_passes": b, "rho_cum": b / K, "rho_min": gs_gated["rho_min"],
        "final_loss_gated": loss_gated, "final_loss_full": loss_full,
        "final_loss_def": "mean over all 200 views, averaged over the checkpoints at K-750, K-500, K-250, K",
        "final_loss_rel_diff": (loss_gated - loss_full) / loss_full,
        "device_status": [st_full, st_gated],
        "wall_s": {"full": wall_full, "gated": wall_gated},
        "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
        "kernels_per_step": {"always": kc_gated[0], "backward_branch": kc_gated[1],
                             "full_loop": kc_full[0] + kc_full[1]},
        "roofline": roofline,
        "stage_ms": {k: round(v["ms"], 4) for k, v in stages.items()},
        "stage_share_gated": {k: round(v["share"], 4) for k, v in stages.items()},
    }
    try:
        line["cpu_baseline"] = cpu_baseline(args, start, cams[int(seq[0])], args.cpu_seconds)
    except Exception as e:  # the baseline is a report, not the product
        line["cpu_baseline"] = {"error": repr(e)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
