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
    ap.add_argument("--steps", type=int, default=1000,
                    help="timed iterations: the last K of the --iters-iteration post-densification loop")
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
    ap.add_argument("--iters", type=int, default=5000,
                    help="length of each measured post-densification loop (both arms run all of it; the last "
                         "--steps iterations are timed)")
    ap.add_argument("--c4", action="store_true",
                    help="batched workload instead of the default line: 8 ring views per iteration at mixed "
                         "resolutions (640x360 .. 1600x1063), launch shape autotuned; prints its own JSON line")
    ap.add_argument("--c4-slots", action="store_true",
                    help="with --c4: every slot a grid of the largest view's size, a block per tile (the "
                         "non-persistent form, for comparison)")
    ap.add_argument("--rho-sweep", action="store_true",
                    help="NEXT-1: gated loop for rho_lo in (no budget, 0.3, 0.5, 0.7, 0.9) against the "
                         "always-backward loop; prints its own JSON line")
    ap.add_argument("--densify", action="store_true",
                    help="NEXT-3: densification phase from a sparse start, then gated vs always-backward post phase")
    ap.add_argument("--densify-iters", type=int, default=5000, help="length of the densification phase")
    ap.add_argument("--densify-grad", type=float, default=1e-8,
                    help="gradient threshold of the density control, pixels (0: the vanilla 2e-4 NDC value in "
                         "pixels, 3.1e-7 at 1297 px, which lies above the 99th percentile of this synthetic "
                         "scene's statistic; 1e-8 lies between its 90th and 99th at the first density step)")
    ap.add_argument("--prune", action="store_true",
                    help="NEXT-4: opacity prune + compaction at eps_alpha in (0.005, 0.05, 0.2), then SkipGS")
    ap.add_argument("--c2", action="store_true", help="C2: 200k-Gaussian fwd+bwd+Adam iteration timing")
    ap.add_argument("--c5", action="store_true", help="C5: 6M Gaussians, 4x1080p fwd+bwd batch timing and memory")
    ap.add_argument("--lists", default="coarse", choices=["coarse", "tile", "auto"],
                    help="coarse: the binning writes super-tile lists and the compositing kernels filter each "
                         "tile's entries from them; tile: per-tile lists (gs_bin_sort); auto (the --c2 and --c4 "
                         "modes): the faster of the two on the mode's workload (autotune.choose_list_form)")
    ap.add_argument("--oracle-timing", action="store_true",
                    help="the FP64 oracle's stages timed on C2 on one host core and on all of them")
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
    # the batch as one persistent launch per compositing stage: resident
    # blocks take (view, tile) items longest-first from a device queue, each
    # view with its own tile grid
    import dataclasses
    st = dataclasses.replace(st, persistent=not args.c4_slots, coarse_lists=args.lists == "coarse")
    form_ms = None
    if args.lists == "auto":  # the faster list form for this batch shape
        st, form_ms = autotune.choose_list_form(model, cams[:B], targets[:B], st, pair_capacity=cap)
    pre = RefinementLoop(model, cams, targets, synth.pre_sequence(pre_iters * B, args.views), st, gated=False,
                         pair_capacity=cap, views_per_step=B)
    pre.capture()
    for _ in range(pre_iters):
        pre.step_graph()
    init = pre.snapshot()
    pre.close()
    del pre

    def timed(gated: bool, lr_scale: bool = False, per_view: bool = False):
        loop = RefinementLoop(model, cams, targets, seq, st, gated=gated, pair_capacity=cap, views_per_step=B,
                              batch_lr_scale=lr_scale, compact_tiles=not args.c4_slots, per_view_steps=per_view)
        loop.restore(init)
        loop.capture()
        for _ in range(args.warmup):
            loop.step_graph()
        loop.restore(init)
        # the whole loop timed; final loss averaged over four checkpoints
        res = run_measured_loop(loop, plan_loop(K, K))
        loop.close()
        return res["ms_loop"], float(np.mean(res["evals"])), res["gate_end"], res["status"]

    # one Adam step per batch on the summed gradient of the opened views,
    # its rates scaled by the opened share (the line's reading)
    ms_full, loss_full, _, s_full = timed(False)
    ms_gated, loss_gated, gs, s_gated = timed(True, lr_scale=True)
    ms_g1, loss_g1, gs1, s_g1 = timed(True)  # full rate whenever any view opened
    # each opened view its own Adam step (the always-backward loop: every view)
    ms_fp, loss_fp, _, s_fp = timed(False, per_view=True)
    ms_gp, loss_gp, gsp, s_gp = timed(True, per_view=True)
    print(json.dumps({
        "metric": "batched refinement: iters/s with 8 views per iteration (gated vs always-backward)",
        "value": K / (ms_gated * 1e-3), "unit": "iters/s", "views_per_s": B * K / (ms_gated * 1e-3),
        "full_bwd_iters_per_s": K / (ms_full * 1e-3), "gated_speedup": ms_full / ms_gated,
        "steps": K, "views_per_step": B, "pre_iterations": pre_iters,
        "gate": {"decisions": gs["t"], "backward_views": gs["b"], "rho_cum": gs["b"] / max(gs["t"], 1)},
        "final_loss_gated": loss_gated, "final_loss_full": loss_full,
        "final_loss_rel_diff": (loss_gated - loss_full) / loss_full,
        "step_reading": "one Adam step per batch when any view opened, on the summed gradient of the opened "
                        "views, its learning rates scaled by the opened share (gs_adam_config.lr_scale_den)",
        "unscaled_step": {"iters_per_s": K / (ms_g1 * 1e-3), "speedup": ms_full / ms_g1,
                          "rho_cum": gs1["b"] / max(gs1["t"], 1), "final_loss": loss_g1,
                          "final_loss_rel_diff": (loss_g1 - loss_full) / loss_full},
        "per_view_steps": {"reading": "each opened view its own Adam step in slot order (gs_view_steps); the "
                                      "always-backward loop steps for every view",
                           "full_bwd_iters_per_s": K / (ms_fp * 1e-3), "final_loss_full": loss_fp,
                           "iters_per_s": K / (ms_gp * 1e-3), "speedup": ms_fp / ms_gp,
                           "rho_cum": gsp["b"] / max(gsp["t"], 1), "final_loss": loss_gp,
                           "final_loss_rel_diff": (loss_gp - loss_fp) / loss_fp},
        "launch": "block per tile, largest-view slots" if args.c4_slots else
                  "persistent: resident blocks take (view, tile) items longest-first from a queue; per-view tile grids",
        "autotuned": {"tile": st.tile, "batch": st.batch, "pixels_per_thread_fwd": st.pixels_per_thread_fwd,
                      "pixels_per_thread_bwd": st.pixels_per_thread,
                      "candidates_ms": {f"{t}/{b}/{pf}/{pb}": v for (t, b, pf, pb), v in tune_ms.items()},
                      "lists": "super-tile" if st.coarse_lists else "tile", "list_form_ms": form_ms},
        "device_status": [s_full, s_gated, s_g1, s_fp, s_gp], "dtype": "f32", "data": "synthetic",
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

    seq_len = max(args.steps, getattr(args, "iters", 5000), 5000)
    gt, start, cams, seq = synth.case_c3(n=args.n, n_views=args.views, n_iters=seq_len,
                                         width=args.width, height=args.height)
    st = raster.RasterSettings(coarse_lists=args.lists == "coarse")
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
    K = max(args.iters, args.steps)  # the whole loop is timed here

    def run(gated: bool, rho_lo: float):
        loop = RefinementLoop(model, cams, targets, seq, st, gated=gated, rho_lo=rho_lo, pair_capacity=cap,
                              log_capacity=K)
        loop.restore(init)
        loop.capture()
        res = run_measured_loop(loop, plan_loop(K, K))
        log = loop.read_log(K)
        final = float(np.mean(res["evals"]))
        gs = res["gate_end"]
        loop.close()
        tenth = max(1, K // 10)
        stepped = log["g"][:, 0] > 0 if gated else np.ones(K, bool)
        gn = np.sqrt(log["grad_sq"][stepped]) if stepped.any() else np.zeros(1)
        un = np.sqrt(log["update_sq"][stepped]) if stepped.any() else np.zeros(1)
        # the always-backward loop runs every backward pass; its gate still
        # decides (and would have skipped where g = 0), reported separately
        return {"rho_lo": rho_lo if gated else None, "gated": gated, "iters_per_s": K / (res["ms_loop"] * 1e-3),
                "backward_passes": gs["b"] if gated else K, "rho_cum": gs["b"] / max(gs["t"], 1) if gated else 1.0,
                "gate_open_rate": gs["b"] / max(gs["t"], 1), "rho_min": gs["rho_min"], "final_loss": final,
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


def gated_vs_full(model, cams, targets, seq, st, cap, plan, adam=None, W=3):
    """The post-densification loop from the model's current state (and
    optional Adam state), always-backward then gated, both from the same
    snapshot, each run through plan_loop's marks (whole loop timed).
    Returns {"full": result, "gated": result} as run_measured_loop gives."""
    import torch
    from paper_2603_08997_gb300.refine import RefinementLoop
    base = RefinementLoop(model, cams, targets, seq, st, gated=False, pair_capacity=cap, adam=adam)
    init = base.snapshot()
    base.close()
    del base
    out = {}
    for gated in (False, True):
        loop = RefinementLoop(model, cams, targets, seq, st, gated=gated, pair_capacity=cap, adam=adam)
        loop.restore(init)
        loop.capture()
        for _ in range(W):
            loop.step_graph()
        loop.restore(init)
        res = run_measured_loop(loop, plan)
        res["kernels_per_step"] = loop.kernels_per_step
        loop.close()
        out["gated" if gated else "full"] = res
        torch.cuda.synchronize()
    return out


def loop_summary(r: dict, iters: int) -> dict:
    f, g = r["full"], r["gated"]
    lf, lg = float(sum(f["evals"]) / len(f["evals"])), float(sum(g["evals"]) / len(g["evals"]))
    return {"full_iters_per_s": iters / (f["ms_loop"] * 1e-3), "gated_iters_per_s": iters / (g["ms_loop"] * 1e-3),
            "speedup": f["ms_loop"] / g["ms_loop"], "rho_cum": g["gate_end"]["b"] / iters,
            "final_loss_full": lf, "final_loss_gated": lg, "final_loss_rel_diff": (lg - lf) / lf,
            "device_status": [f["status"], g["status"]]}


def run_densify(args) -> None:
    """NEXT-3: a densification phase before T_d, then the post phase.  The
    start is a sparse perturbed subset (a third) of the 3M ground truth;
    always-backward refinement with adaptive density control every 100
    iterations from iteration 500 (clone / split / prune, Sec. 3) up to
    --densify-iters, the set capped at --n; then the gated and the
    always-backward post-densification loops of --iters iterations from the
    densified state (parameters and Adam moments carried over)."""
    import math
    import torch

    import synth
    from paper_2603_08997_gb300 import build, raster
    from paper_2603_08997_gb300.refine import densification_phase

    build.build()
    dev = torch.device("cuda", 0)
    gt, _, cams, seq = synth.case_c3(n=args.n, n_views=args.views, n_iters=max(args.iters, args.densify_iters),
                                     width=args.width, height=args.height)
    st = raster.RasterSettings(coarse_lists=args.lists == "coarse")
    mgt = raster.GaussianModel.from_scene(gt, dev)
    rgt = raster.Renderer(args.n, 3, raster.Views([cams[0]], st.tile, dev), st, 24 * args.n, dev)
    targets = torch.empty((args.views, 3, args.height, args.width), dtype=torch.float32, device=dev)
    for v, cam in enumerate(cams):
        rgt.views = raster.Views([cam], st.tile, dev)
        rgt.forward(mgt.c_params())
        targets[v].copy_(rgt.image.view(3, args.height, args.width))
    torch.cuda.synchronize()
    del mgt, rgt
    n0 = args.n // 3
    start = synth.sparse_start(gt, n0, seed=11)
    del gt
    model = raster.GaussianModel.from_scene(start, dev)
    # thresholds: the gradient threshold from --densify-grad (pixels; the
    # vanilla 2e-4 on the NDC-space gradient is 2e-4 * 2 / W = 3.1e-7 here);
    # 1% of the scene extent (1.1 x the camera radius 3); opacity 0.005
    grad_thr = args.densify_grad if args.densify_grad > 0 else 2e-4 * 2.0 / args.width
    cfg = raster.densify_config(grad_thr=grad_thr, max_scale=0.01 * 1.1 * 3.0, eps_alpha=0.005)
    pre_seq = synth.pre_sequence(args.densify_iters, args.views)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    model, adam, hist = densification_phase(model, cams, targets, pre_seq, args.densify_iters, cfg, st,
                                            interval=100, start=500, max_gaussians=args.n,
                                            capacity_per_gaussian=48)
    torch.cuda.synchronize()
    t_d = time.perf_counter() - t0
    iters = max(args.iters, 1)
    r = gated_vs_full(model, cams, targets, seq, st, 48 * model.n, plan_loop(iters, iters), adam=adam)
    print(json.dumps({
        "metric": "densification phase then post phase (NEXT-3): gated vs always-backward iters/s",
        "densify": {"start_gaussians": n0, "iterations": args.densify_iters, "interval": 100, "from": 500,
                    "grad_thr_px": grad_thr, "max_scale": 0.033, "eps_alpha": 0.005, "cap": args.n,
                    "wall_s": t_d, "iters_per_s_wall": args.densify_iters / t_d,
                    "history": [dict(zip(("iteration", "n_before", "clone", "split", "prune", "n_after",
                                          "grad_p50_p90_p99"), h)) for h in hist]},
        "post": dict(loop_summary(r, iters), iterations=iters, n_gaussians=model.n),
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "sparse perturbed third of the 3M-Gaussian SH3 scene, 200 ring views 1297x840, "
                               "density control then SkipGS W=500 beta=0.95 eps=1e-8 rho_lo=0.5"}}))


def run_prune(args) -> None:
    """NEXT-4: an opacity-threshold prune (alpha < eps_alpha, Sec. 3) with
    compaction of the parameters and Adam moments before the post phase,
    then SkipGS on top: for each threshold, the gated and always-backward
    loops on the pruned set against the unpruned ones (same snapshot, same
    view sequence)."""
    import torch

    from paper_2603_08997_gb300 import build, raster

    build.build()
    dev = torch.device("cuda", 0)
    model, cams, targets, seq, init, st, cap, _ = setup_c3(args, dev)
    iters = max(args.iters, 1)
    plan = plan_loop(iters, iters)
    adam = raster.AdamState(model)

    def load(snap):
        model.flat.copy_(snap["flat"])
        adam.m.copy_(snap["m"])
        adam.v.copy_(snap["v"])
        adam.step_count.copy_(snap["step"])

    rows = []
    load(init)
    rows.append(dict(loop_summary(gated_vs_full(model, cams, targets, seq, st, cap, plan, adam=adam), iters),
                     eps_alpha=None, n_gaussians=model.n))
    for eps in (0.005, 0.05, 0.2):
        load(init)
        stats = raster.DensityStats(model.n, dev)
        cfg = raster.densify_config(grad_thr=float("inf"), max_scale=1.0, eps_alpha=eps)
        noise = torch.zeros((model.n, 2, 3), dtype=torch.float32, device=dev)
        pm, pa, action = raster.densify(model, adam, stats, cfg, noise)
        del stats, noise
        torch.cuda.synchronize()
        rows.append(dict(loop_summary(gated_vs_full(pm, cams, targets, seq, st, cap, plan, adam=pa), iters),
                         eps_alpha=eps, n_gaussians=pm.n))
        del pm, pa
        torch.cuda.empty_cache()
    base_full = rows[0]["full_iters_per_s"]
    base_loss = rows[0]["final_loss_full"]
    for r in rows:
        r["gated_speedup_vs_unpruned_full"] = r["gated_iters_per_s"] / base_full
        r["full_speedup_vs_unpruned_full"] = r["full_iters_per_s"] / base_full
        r["final_loss_gated_vs_unpruned_full"] = (r["final_loss_gated"] - base_loss) / base_loss
    print(json.dumps({"metric": "opacity prune + compaction, then SkipGS (NEXT-4)", "iterations": iters,
                      "workload": WORKLOAD, "rows": rows, "dtype": "f32", "data": "synthetic"}))


def run_c2(args) -> None:
    """C2: one view of the 200,000-Gaussian SH3 unit-ball scene at 980x545, a
    forward + loss + backward + Adam iteration (the always-backward loop as a
    captured graph, 1 view per iteration), target = render of a perturbed copy
    plus N(0, 0.01) noise; per-stage times and the peak device memory."""
    import numpy as np
    import torch

    import synth
    from paper_2603_08997_gb300 import build, raster
    from paper_2603_08997_gb300.refine import RefinementLoop

    build.build()
    dev = torch.device("cuda", 0)
    scene, tscene, cam, noise = synth.case_c2()
    st = raster.RasterSettings(coarse_lists=args.lists == "coarse")
    mt = raster.GaussianModel.from_scene(tscene, dev)
    rt = raster.Renderer(scene.n, 3, raster.Views([cam], st.tile, dev), st, 48 * scene.n, dev)
    rt.forward(mt.c_params())
    target = (rt.image.view(1, 3, cam.height, cam.width) + torch.from_numpy(noise).to(dev)).contiguous()
    del mt, rt
    torch.cuda.synchronize()
    model = raster.GaussianModel.from_scene(scene, dev)
    form_ms = None
    if args.lists == "auto":  # the faster list form on this workload
        from paper_2603_08997_gb300 import autotune
        st, form_ms = autotune.choose_list_form(model, [cam], [target[0]], st, pair_capacity=48 * scene.n)
    torch.cuda.reset_peak_memory_stats(dev)
    K = max(args.steps, 1)
    loop = RefinementLoop(model, [cam], target, np.zeros(K + args.warmup, np.int32), st, gated=False,
                          pair_capacity=48 * scene.n)
    loop.capture()
    for _ in range(max(args.warmup, 3)):
        loop.step_graph()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(loop.stream)
    for _ in range(K):
        loop.step_graph()
    e1.record(loop.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    stages = stage_times(loop, target, b_frac=1.0)
    print(json.dumps({"metric": "C2 fwd+bwd+Adam iteration (200k Gaussians SH3, 980x545)", "value": 1000.0 / ms,
                      "unit": "iters/s", "ms_per_iteration": ms, "steps": K,
                      "stage_ms": {k: round(v["ms"], 4) for k, v in stages.items()},
                      "pairs": int(loop.renderer.pair_count.item()), "status": int(loop.renderer.status.item()),
                      "peak_device_bytes": int(torch.cuda.max_memory_allocated(dev)),
                      "lists": "super-tile" if st.coarse_lists else "tile", "list_form_ms": form_ms,
                      "dtype": "f32", "data": "synthetic"}))


def run_oracle_timing(args) -> None:
    """The FP64 oracle's stages (the baseline the kernels are compared with,
    not a target) timed on the C2 scene (200k Gaussians SH3, 980x545) on one
    host core and on all of them: projection, binning, compositing, loss and
    its gradient, raster adjoint, projection adjoint, the Adam step over
    every parameter, and the gate's decision and EMA update over 5000 losses.
    Wall time of each call on this host (CPU work; no GPU is used)."""
    import time

    import numpy as np

    import oracle
    import synth
    from oracle.adam import AdamConfig, adam_step, lr_vector
    from oracle.gate import Gate, GateConfig

    oracle.core.build()
    scene, tscene, cam, noise = synth.case_c2()
    rc = oracle.RasterConfig()
    target = (oracle.forward(tscene, cam, rc)["image"] + noise).astype(np.float32)
    all_cores = oracle.num_threads()
    rows = {}
    # The first pass only warms the host's allocator (first-touch page faults
    # are not the oracle's arithmetic); the two after it are reported.
    for threads in (all_cores, 1, all_cores):
        oracle.set_num_threads(threads)
        t = {}

        def timed(name, fn):
            t0 = time.perf_counter()
            out = fn()
            t[name] = (time.perf_counter() - t0) * 1e3
            return out

        proj = timed("project", lambda: oracle.project(scene, cam, rc))
        _, vals, ranges, _ = timed("bin_sort", lambda: oracle.bin_sort([proj], [cam], rc.tile))
        f = timed("render_fwd", lambda: oracle.render(proj, cam, vals, ranges, rc, 0))
        L, dL = timed("loss", lambda: oracle.loss_and_grad(f["image"], target))
        g2d = timed("raster_bwd", lambda: oracle.raster_bwd(proj, cam, vals, ranges, rc, dL, 0))
        grads = timed("project_bwd", lambda: oracle.project_bwd(scene, cam, rc, g2d))
        cfg = AdamConfig()
        lr = lr_vector(scene.means.shape[0], scene.sh.shape[1], cfg)
        flat_p = np.concatenate([np.asarray(getattr(scene, k), np.float64).ravel()
                                 for k in ("means", "log_scales", "quats", "opacity_logit", "sh")])
        flat_g = np.concatenate([np.asarray(grads[k], np.float64).ravel()
                                 for k in ("means", "log_scales", "quats", "opacity_logit", "sh")])
        zeros = np.zeros_like(flat_p)
        timed("adam", lambda: adam_step(flat_p, flat_g, zeros, zeros, 0, lr, cfg))
        rng = np.random.default_rng(0)
        views, losses = rng.integers(0, 200, 5000), rng.uniform(0.004, 0.006, 5000)

        def gate_run():
            gt = Gate(GateConfig(W=500, beta=0.95, eps=1e-8, rho_lo=0.5, n_views=200))
            for v_, l_ in zip(views, losses):
                gt.decide(int(v_), float(l_))
                gt.update(int(v_), float(l_))
        timed("gate_5000_iterations", gate_run)
        t["iteration_fwd_loss_bwd_adam"] = sum(t[k] for k in ("project", "bin_sort", "render_fwd", "loss",
                                                               "raster_bwd", "project_bwd", "adam"))
        rows[f"{threads}_thread{'s' if threads > 1 else ''}"] = {k: round(v, 2) for k, v in t.items()}
    print(json.dumps({"metric": "FP64 oracle stage times on C2 (200k Gaussians SH3, 980x545), ms",
                      "host_cores": os.cpu_count(), "threads_all": all_cores, "pairs": int(len(vals)),
                      "rows": rows, "kind": "oracle", "data": "synthetic"}))


def run_c5(args) -> None:
    """C5: 6M Gaussians SH3, 4 views of 1920x1080 per batch through the
    torch.autograd.Function path (render -> per-view loss -> backward with
    per-tile transmittance checkpoints), targets = renders of a perturbed copy;
    ms per batch for forward and backward, pairs, and the peak device memory
    (parameters, gradients, pairs, checkpoints, images)."""
    import torch

    import synth
    from paper_2603_08997_gb300 import autograd, build, raster

    build.build()
    dev = torch.device("cuda", 0)
    scene, cams = synth.case_c5()
    views = raster.Views(cams, 16, dev)
    cap = 200_000_000 * len(cams)
    r = raster.Renderer(scene.n, 3, views, raster.RasterSettings(), pair_capacity=cap, device=dev)
    mt = raster.GaussianModel.from_scene(synth.perturb_scene(scene, 5, 0.2), dev)
    r.forward(mt.c_params())
    target = r.image.clone()
    del mt
    model = raster.GaussianModel.from_scene(scene, dev)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    flat = model.flat.clone().requires_grad_(True)
    ms_f, ms_b = [], []
    for k in range(max(args.warmup, 2) + max(args.steps, 1)):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        img = autograd.render(flat, model, r)
        losses = autograd.photometric_loss(img, target, r)
        e[1].record()
        flat.grad = None
        losses.sum().backward()
        e[2].record()
        torch.cuda.synchronize()
        if k >= max(args.warmup, 2):
            ms_f.append(e[0].elapsed_time(e[1]))
            ms_b.append(e[1].elapsed_time(e[2]))
    print(json.dumps({"metric": "C5 fwd+bwd per 4x1920x1080 batch (6M Gaussians SH3, autograd path)",
                      "value": 1000.0 / (sum(ms_f) / len(ms_f) + sum(ms_b) / len(ms_b)), "unit": "batches/s",
                      "fwd_ms": sum(ms_f) / len(ms_f), "bwd_ms": sum(ms_b) / len(ms_b), "batches": len(ms_f),
                      "pairs": int(r.pair_count.item()), "status": int(r.status.item()),
                      "peak_device_bytes": int(torch.cuda.max_memory_allocated(dev)),
                      "param_bytes": int(model.flat.numel() * 4), "dtype": "f32", "data": "synthetic"}))


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
    r = raster.Renderer(args.n, 3, views, raster.RasterSettings(coarse_lists=args.lists == "coarse"),
                        pair_capacity=24 * args.n)
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
    crop of the view covering `frac` of its pixels (centred) with every
    Gaussian whose support box reaches it, against a seeded target.  Returns
    (seconds, pixels of the crop)."""
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
        m, r = pr["mean2d"], pr["radius"]
        # every Gaussian whose support box (mean2D +- half-extents) reaches the
        # crop, wherever its centre lies
        sel = np.nonzero((pr["touched"] > 0) & (m[:, 0] + r[:, 0] >= x0) & (m[:, 0] - r[:, 0] <= x0 + cw) &
                         (m[:, 1] + r[:, 1] >= y0) & (m[:, 1] - r[:, 1] <= y0 + ch))[0]
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
                      f"({100.0 * pix / runs / full_px:.1f}% of 1297x840) with every Gaussian whose support "
                      f"box reaches it; "
                      f"{total:.1f} s CPU wall time, scaled to the full view by the pixel fraction"}


def workload_config(args, plan: dict, world: int) -> dict:
    """The `config` object of the bench line (both arms print the same one)."""
    return {"workload": WORKLOAD, "n_gaussians": args.n, "views": args.views, "width": args.width,
            "height": args.height, "loop_iterations": plan["iters"],
            "timed": f"the last {plan['K']} of {plan['iters']} post-densification iterations "
                     f"(t = {plan['start'] + 1}..{plan['iters']})",
            "parallelism": "replicas" if world > 1 else "1 GPU",
            "lists": ("super-tile lists, each tile's entries filtered by the compositing kernels"
                      if getattr(args, "lists", "tile") == "coarse" else "per-tile lists"),
            "l2": "inputs larger than L2 (2.8 GB of parameters and Adam state, 2.6 GB of targets)"}


def run_reference(args) -> None:
    """The oracle arm: each step one FP64 oracle refinement iteration on a
    bounded crop of the workload's view (the same crop size every step, sized
    so the whole run takes about --ref-seconds), scaled to full-view
    iterations/s by the pixel fraction."""
    import synth
    K, W = args.steps, args.warmup
    plan = plan_loop(max(args.iters, args.steps), args.steps)
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
            "steps": K, "warmup": W, "ms_per_step": 1000.0 * total / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "value_def": "full-view iterations/s: the crop's pixel fraction per timed second; ms_per_step is the "
                         "wall time of one timed sample step",
            "config": workload_config(args, plan, 1),
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: one FP64 oracle iteration on a centred crop covering "
                                       f"{100 * frac:.3f}% of the view's pixels with every Gaussian whose support "
                                       f"box reaches it, scaled to the full view by the pixel fraction"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU arm

# FP32 work per (pixel, Gaussian) pair of the compositing kernels, counted from
# the operations Eq. (alpha) and Eq. (blend) and their adjoint need (a fused
# multiply-add counts two):
#   evaluating alpha' at a pixel inside the support box: offset (2), |U dp|^2
#   (7), exponent scale and opacity (2), clamp and cut-off tests (2) = 13, plus
#   one exponential on the special-function unit;
#   forward, per contributing pair: 1 - alpha', T (1 - alpha') and its test,
#   alpha' T, three colour FMAs = 10;
#   adjoint, per contributing pair: T rebuilt (2 + a reciprocal), weight (1),
#   colour gradients (6), dL/dalpha' (14), colour-behind suffix sums (6),
#   opacity, mean2D and conic gradients (23), and the nine sums over pixels
#   per Gaussian (9) = 61.
FLOP_EVAL, FLOP_FWD_CONTRIB, FLOP_BWD_CONTRIB = 13, 10, 61


def peak_alu_tflops(sm_count: int, sm_mhz: float) -> float:
    """FP32 peak from unit counts and the clock: SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


def device_alu_peak(peaks: dict):
    """(TFLOP/s, note) for the current device: its SM count and the maximum SM
    clock the driver measured (else 2070 MHz, the part's maximum)."""
    sms = 152
    try:
        import torch
        if torch.cuda.is_available():
            sms = int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    except Exception:
        pass
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return peak_alu_tflops(sms, mhz), f"derived FP32 peak: {sms} SMs x 128 FP32 lanes x 2 FLOP x {mhz:.0f} MHz"


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


def coarse_pairs(r, fallback: int) -> int:
    """(entry, super-tile of 4 x 4 tiles) pairs of the last binning, from the
    packed tile rectangles the projection wrote (x0, y0, width, height in
    tiles); `fallback` (the pair count, an upper bound) when unavailable."""
    try:
        import torch
        if not getattr(r, "aux_valid", False):
            return int(fallback)
        q = r.rect16.view(-1, 4).to(torch.int64)
        w, h = q[:, 2], q[:, 3]
        live = (w > 0) & (h > 0)
        cx = (q[:, 0] + w - 1) // 4 - q[:, 0] // 4 + 1
        cy = (q[:, 1] + h - 1) // 4 - q[:, 1] // 4 + 1
        return int(torch.where(live, cx * cy, torch.zeros_like(cx)).sum().item())
    except Exception:
        return int(fallback)


def atomic_probe_rate(n_records: int, n_updates: int, reps: int = 3) -> float:
    """Peak rate (updates/s) of the raster adjoint's global atomic pattern -
    two float4 and one float reduction per update into scattered 48-byte
    records (gs_atomic_probe) - over a buffer of n_records records; best of
    `reps` launches timed with CUDA events."""
    import torch
    from paper_2603_08997_gb300 import gsr
    buf = torch.zeros(n_records * 12, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    best = float("inf")
    gsr.call("gs_atomic_probe", gsr.ptr(buf), n_records, n_updates, gsr.stream_handle(s))
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        gsr.call("gs_atomic_probe", gsr.ptr(buf), n_records, n_updates, gsr.stream_handle(s))
        e1.record(s)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    del buf
    return n_updates / best


def roofline_of(stages: dict, loop, args, census: dict | None = None, atomic_peak: float | None = None) -> dict:
    """Roofline of the stage with the largest share of the gated iteration, and
    of every stage.  Algorithmic work per launch: HBM stages count the bytes a
    launch must move; the compositing kernels count FP32 operations per
    (pixel, Gaussian) pair the method needs (FLOP_* above) over the pairs the
    work census found: evaluations inside support boxes and contributing
    pairs.  The raster adjoint also reports its global atomic rate against the
    probe's peak, and the bytes its pairs move through L2."""
    import json as _json
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_note = "of measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "of fallback 6.8 TB/s"
    alu_peak, alu_note = device_alu_peak(peaks)
    r = loop.renderer
    N = r.n
    E = N * r.views.n
    P = int(r.pair_count.item())
    px = r.views.total_pixels
    T = r.views.total_tiles
    if census is None:  # no census: every list position up to n_last, all contributing (an upper bound)
        ev = float(r.n_last.double().sum().item())
        census = dict(sum_n_last=ev, evaluated=ev, contributing=ev, tile_pairs=P, staged=P)
    ev, con = float(census["evaluated"]), float(census["contributing"])
    Pc = coarse_pairs(r, P)
    params = loop.model.flat.numel()
    work = {
        "project": ("hbm", N * (236 + 68), "bytes: 236 B parameters read + 68 B record, rectangle, count written per Gaussian"),
        "bin_sort": (("hbm", 124 * E + 6 * Pc + 20 * T,
                      f"bytes: 124 B per (view, Gaussian) entry (four radix passes 76, rectangle gather 20, tile "
                      f"and super-tile counts 16, super-tile scatter reads 12) + 6 B per (entry, super-tile) pair "
                      f"({Pc:.4g}: Gaussian index and covered-tile mask written; the compositing kernels filter the "
                      f"tiles' entries from these lists, no (Gaussian, tile) pair is placed) + 20 B per tile "
                      f"(totals, starts, range)") if getattr(r, "coarse", False) else
                     ("hbm", 124 * E + 14 * Pc + 4 * P + 20 * T,
                      f"bytes: 124 B per (view, Gaussian) entry (four radix passes 76, rectangle gather 20, tile "
                      f"and super-tile counts 16, super-tile scatter reads 12) + 14 B per (entry, super-tile) pair "
                      f"({Pc:.4g}: 6 B record written, the mask read by the count pass, both read by the place "
                      f"pass) + 4 B per (Gaussian, tile) pair ({P:.4g}) + 20 B per tile (totals, starts, range)")),
        "render_fwd": ("alu", FLOP_EVAL * ev + FLOP_FWD_CONTRIB * con,
                       f"FLOP: {FLOP_EVAL} per evaluated (pixel, Gaussian) pair inside its support box "
                       f"({ev:.4g}) + {FLOP_FWD_CONTRIB} per contributing pair ({con:.4g}), from the work census"),
        "loss": ("hbm", 60 * px, "bytes: 60 B per pixel"),
        "loss_bwd": ("hbm", 72 * px, "bytes: 72 B per pixel"),
        "raster_bwd": ("alu", FLOP_EVAL * ev + FLOP_BWD_CONTRIB * con,
                       f"FLOP: {FLOP_EVAL} per evaluated pair ({ev:.4g}) + {FLOP_BWD_CONTRIB} per contributing "
                       f"pair ({con:.4g}), from the work census"),
        "project_bwd": ("hbm", N * (236 + 48 + 236), "bytes: 520 B per Gaussian"),
        "adam": ("hbm", 28 * params, "bytes: 28 B per parameter (read p, g, m, v; write p, m, v)"),
        "project_bwd_adam": ("hbm", N * 48 * r.views.n + 24 * params,
                             "bytes: 48 B of 2D gradients per (view, Gaussian) + 24 B per parameter "
                             "(read p, m, v; write p, m, v)"),
    }

    def frac_of(k):
        w = work[k]
        a = (w[1] / (stages[k]["ms"] * 1e-3)) / (1e9 if w[0] == "hbm" else 1e12)
        return a, a / (hbm if w[0] == "hbm" else alu_peak)

    all_stages = {}
    for k, w in work.items():
        if k not in stages:
            continue
        a, f = frac_of(k)
        all_stages[k] = {"bound": w[0], "achieved": a, "frac": f, "ms": stages[k]["ms"]}
    # the raster adjoint: global atomics (three instructions per (tile,
    # Gaussian) pair with a contributor) against the probe's peak, and the
    # bytes its pairs move (40 B record re-read per staged entry, 36 B of
    # atomic read-modify-write per contributing (tile, Gaussian) pair), which
    # L2 serves
    if "raster_bwd" in stages:
        t_b = stages["raster_bwd"]["ms"] * 1e-3
        tp = float(census["tile_pairs"])
        at = {"updates_per_s": tp / t_b, "atomic_instructions_per_launch": 3 * tp}
        if atomic_peak:
            at.update(peak_updates_per_s=atomic_peak, frac=tp / t_b / atomic_peak,
                      peak_note="gs_atomic_probe: the same three-atomic update at hashed records of a "
                                "[N][12]-float buffer, best of 3 launches")
        l2_bytes = 40.0 * float(census["staged"]) + 36.0 * tp
        all_stages["raster_bwd"].update(atomic=at, pair_bytes_per_launch=l2_bytes,
                                        pair_bytes_gbs=l2_bytes / t_b / 1e9)
    name = max(stages, key=lambda k: stages[k]["share"])
    bound, units, note = work[name]
    traffic, traffic_note = stage_traffic(name)
    t = stages[name]["ms"] * 1e-3
    if bound == "hbm":
        achieved, peak, unit, pk_note = units / t / 1e9, hbm, "GB/s", hbm_note
    else:
        achieved, peak, unit, pk_note = units / t / 1e12, alu_peak, "TFLOP/s", alu_note
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": traffic, "traffic_note": traffic_note, "work_per_launch": units, "work_def": note,
            "launch_ms": t * 1e3, "share_of_gated_iteration": stages[name]["share"], "peak_note": pk_note,
            "census": census, "all_stages": all_stages}


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


def plan_loop(iters: int, K: int) -> dict:
    """Where one measured loop stops.  The loop runs `iters` iterations from
    the post-pre-phase snapshot; its last K form the timed window.  The
    final-loss checkpoints sit at iters - 3s, iters - 2s, iters - s and iters
    (s = min(250, iters // 4)); the all-view evaluations there are not timed,
    so the window is split where a checkpoint falls inside it.
    Returns {"iters", "K", "start", "marks", "evals"}: run to each mark in
    turn; the window is [start, iters)."""
    iters = max(1, int(iters))
    K = max(1, min(int(K), iters))
    start = iters - K
    seg = max(1, min(250, iters // 4))
    evals = sorted({m for m in (iters - 3 * seg, iters - 2 * seg, iters - seg, iters) if m > 0})
    marks = sorted(({start} if start > 0 else set()) | set(evals))
    return {"iters": iters, "K": K, "start": start, "marks": marks, "evals": evals}


def backward_split(ms_full: float, ms_gated: float, iters: int, n_bwd: int, min_skip_frac: float = 0.1):
    """Forward and backward ms per view from two loops over the same `iters`
    iterations, one always-backward (t_full = iters (f + b)) and one gated with
    n_bwd backward passes (t_gated = iters f + n_bwd b).  The system is only
    determined when the gated loop skipped enough of them: with fewer than
    min_skip_frac * iters skips the difference is timing noise and (None, None)
    comes back."""
    skipped = iters - n_bwd
    if iters <= 0 or skipped < max(1.0, min_skip_frac * iters):
        return None, None
    b = (ms_full - ms_gated) / skipped
    f = ms_full / iters - b
    return f, b


def run_measured_loop(loop, plan: dict, dist=None, on_window=None, nvtx: str | None = None) -> dict:
    """Runs a restored, captured RefinementLoop through plan_loop's marks
    (graph replays; CUDA events on the loop's stream around every segment).
    Returns the window's and the whole loop's device ms, the gate counters at
    the window's start and end, and the final-loss evaluations.  nvtx: name
    of an NVTX range around each segment of the timed window only."""
    import numpy as np
    import torch
    done, ms_all, ms_win, evals = 0, 0.0, 0.0, []
    g0 = {"t": 0, "b": 0}
    wall0 = None
    for mark in plan["marks"]:
        in_window = done >= plan["start"]
        torch.cuda.synchronize()
        if in_window and done == plan["start"]:
            if dist:
                dist.barrier()
            if on_window:
                on_window()
            wall0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if nvtx and in_window:
            torch.cuda.nvtx.range_push(nvtx)
        e0.record(loop.stream)
        for _ in range(mark - done):
            loop.step_graph()
        e1.record(loop.stream)
        torch.cuda.synchronize()
        if nvtx and in_window:
            torch.cuda.nvtx.range_pop()
        ms = e0.elapsed_time(e1)
        ms_all += ms
        if in_window:
            ms_win += ms
        done = mark
        if mark == plan["start"]:
            g0 = loop.gate.read(loop.stream)
        if mark in plan["evals"]:
            evals.append(float(np.mean(loop.evaluate())))
    if dist:
        dist.barrier()
    g1 = loop.gate.read(loop.stream)
    return {"ms_window": ms_win, "ms_loop": ms_all, "gate_start": g0, "gate_end": g1, "evals": evals,
            "wall_window": time.perf_counter() - wall0 if wall0 is not None else None,
            "status": int(loop.renderer.status.item())}


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
    if args.oracle_timing:
        if rank == 0:
            run_oracle_timing(args)
        return
    if args.c4:
        run_c4(args)
        return
    if args.rho_sweep:
        run_rho_sweep(args)
        return
    if args.densify:
        run_densify(args)
        return
    if args.c2:
        run_c2(args)
        return
    if args.c5:
        run_c5(args)
        return
    if args.prune:
        run_prune(args)
        return

    import numpy as np
    import torch

    from paper_2603_08997_gb300 import build
    from paper_2603_08997_gb300.refine import HostTargets, RefinementLoop

    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    W = args.warmup
    plan = plan_loop(max(args.iters, args.steps), args.steps)
    K, iters = plan["K"], plan["iters"]
    dev = torch.device("cuda", local)
    model, cams, targets, seq, init, st, cap, start = setup_c3(args, dev)

    def measured(gated: bool):
        loop = RefinementLoop(model, cams, targets, seq, st, gated=gated, pair_capacity=cap)
        loop.restore(init)
        loop.capture()
        for _ in range(W):  # untimed warm-up replays (graph upload), then back to the snapshot
            loop.step_graph()
        loop.restore(init)
        clock = ClockSampler(local) if (gated and rank == 0) else None
        res = run_measured_loop(loop, plan, dist, nvtx="timed_gated" if gated else "timed_full")
        res["clocks"] = clock.stop() if clock else None
        return loop, res

    full, r_full = measured(False)
    kc_full = full.kernels_per_step
    full.close()
    del full
    gated, r_gated = measured(True)
    kc_gated = gated.kernels_per_step
    b_loop = r_gated["gate_end"]["b"]
    b_win = b_loop - r_gated["gate_start"]["b"]

    # per-stage timing on the loop's stream (CUDA events, after the timed loops),
    # weighted by how often each stage runs in the gated loop
    stages = stage_times(gated, targets, b_frac=b_loop / iters)
    census = gated.renderer.census(gated.stream)
    atomic_peak = atomic_probe_rate(args.n, max(census["tile_pairs"], 1 << 20))
    roofline = roofline_of(stages, gated, args, census, atomic_peak)
    # end to end through the C ABI with host-resident targets: the same loop,
    # each step's target copied from pinned host memory, loss and decision
    # copied back; wall clock over the same window
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
        loss_host = torch.empty(iters + W, dtype=torch.float32).pin_memory()
        g_host = torch.empty(iters + W, dtype=torch.uint8).pin_memory()
        feeder = HostTargets(loop, host_targets, np.asarray(seq))

        def e2e_step(k):
            feeder.step()  # target from pinned host memory, copied while the previous iteration runs
            with torch.cuda.stream(loop.stream):
                loss_host[k:k + 1].copy_(loop.renderer.loss, non_blocking=True)
                g_host[k:k + 1].copy_(loop.g, non_blocking=True)

        for k in range(W):
            e2e_step(k)
        loop.restore(init)
        feeder.reset()
        for k in range(plan["start"]):
            e2e_step(k)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(plan["start"], iters):
            e2e_step(k)
        torch.cuda.synchronize()
        wall_e2e = time.perf_counter() - t0
        e2e = {"value": K * world / aggregate_time(wall_e2e, dist, dev), "unit": "iters/s",
               "h2d_bytes_per_step": 3 * args.height * args.width * 4, "d2h_bytes_per_step": 4 + 1,
               "timed": f"wall clock over the last {K} of {iters} iterations, targets from pinned host memory"}
        loop.close()

    # aggregate over ranks: max time
    t_gated = aggregate_time(r_gated["ms_window"] * 1e-3, dist, dev)
    t_full = aggregate_time(r_full["ms_window"] * 1e-3, dist, dev)
    if dist:
        dist.barrier()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    it_full = job_value(K, world, t_full)
    it_gated = job_value(K, world, t_gated)
    f_reg, b_reg = backward_split(r_full["ms_loop"], r_gated["ms_loop"], iters, b_loop)
    bwd_stage = sum(stages[k]["ms"] for k in BACKWARD_STAGES)
    fwd_stage = sum(stages[k]["ms"] for k in ("project", "bin_sort", "render_fwd", "loss"))
    launches = kc_gated[0] * K + kc_gated[1] * b_win
    loss_gated, loss_full = float(np.mean(r_gated["evals"])), float(np.mean(r_full["evals"]))
    line = {
        "metric": METRIC, "value": it_gated, "unit": "iters/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_gated * 1e3 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, plan, world),
        "full_bwd_iters_per_s": it_full, "gated_speedup": it_gated / it_full,
        "gate_in_warmup": plan["start"] < 500 + 1,
        "backward_passes": b_win, "rho_cum_window": b_win / K, "rho_cum": b_loop / iters,
        "rho_min": r_gated["gate_end"]["rho_min"],
        "bwd_ms_per_view": bwd_stage, "fwd_ms_per_view": fwd_stage,
        "bwd_fwd_def": "stage times (CUDA events): backward = loss_bwd + raster_bwd + project_bwd_adam, "
                       "forward = project + bin_sort + render_fwd + loss",
        "bwd_ms_per_view_loop": b_reg, "fwd_ms_per_view_loop": f_reg,
        "loop": {"iterations": iters, "gated_iters_per_s": iters / (r_gated["ms_loop"] * 1e-3),
                 "full_bwd_iters_per_s": iters / (r_full["ms_loop"] * 1e-3),
                 "speedup": r_full["ms_loop"] / r_gated["ms_loop"], "backward_passes": b_loop,
                 "rho_cum": b_loop / iters, "ms": {"gated": r_gated["ms_loop"], "full": r_full["ms_loop"]}},
        "final_loss_gated": loss_gated, "final_loss_full": loss_full,
        "final_loss_def": "mean over all %d views, averaged over the checkpoints after iterations %s" % (
            args.views, ", ".join(str(m) for m in plan["evals"])),
        "final_loss_rel_diff": (loss_gated - loss_full) / loss_full,
        "device_status": [r_full["status"], r_gated["status"]],
        "clocks": r_gated["clocks"], "e2e": e2e, "gpu_launches": launches,
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
