"""Post-densification refinement loop with the SkipGS gate (Algorithm 1).

One iteration: select the view(s) of this iteration (device-side, from the
pre-drawn view sequence) -> project -> bin/sort -> render -> loss (value) ->
gate decision -> [loss gradient -> raster and projection adjoint -> Adam]
only when g = 1 -> per-view EMA update.

Batched form (views_per_step = B > 1): B views per iteration in B camera
slots sized for the largest training view; each slot takes its view's pose,
intrinsics and size on the device, the gate decides the B losses in order
(reading (vii)), the adjoint runs for the views with g = 1 only, and Adam
steps once if any did.  The backward branch issues gs_render_bwd_adam (the
raster adjoint, then the projection adjoint and Adam in one kernel, so the
parameter gradients never reach DRAM); fused=False issues gs_render_bwd then
gs_adam_step instead.

`step_graph` replays the iteration as one CUDA graph: the bracketed branch is
an IF conditional node that the gate kernel sets on the device, so no value
crosses to the host inside the loop.  `step_eager` issues the same calls
directly, with the branch predicated on the device flag.  With gated=False
the branch always runs (the vanilla always-backward loop).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import gsr
from .raster import AdamState, DensityStats, Gate, GaussianModel, RasterSettings, Renderer, Views, densify


class RefinementLoop:
    def __init__(self, model: GaussianModel, train_cams: list, targets, view_seq,
                 settings: RasterSettings | None = None, gated: bool = True, W: int = 500, beta: float = 0.95,
                 eps: float = 1e-8, rho_lo: float = 0.5, lr=None, pair_capacity: int | None = None,
                 fused: bool = True, views_per_step: int = 1, log_capacity: int = 0,
                 adam: AdamState | None = None, stats: DensityStats | None = None, batch_lr_scale: bool = False,
                 compact_tiles: bool = False, per_view_steps: bool = False):
        """targets: [n_train, 3, H, W] tensor (equal sizes) or a list of
        [3, H_v, W_v] tensors, one per training view.  adam: an existing
        optimizer state of `model` to continue (else a fresh one).  stats: the
        densification statistic, accumulated after every backward pass.
        batch_lr_scale (views_per_step > 1): each step's learning rates are
        scaled by the fraction of the iteration's views the gate opened.
        compact_tiles: the selected views' own tile grids are packed one after
        another (gs_select_views with the tile size) instead of each slot
        holding a grid of the largest view's size.
        per_view_steps (views_per_step > 1, fused backward): each opened view
        of the batch takes its own Adam step in slot order (the always-backward
        loop: every view), on its own gradient from the batch's forward pass."""
        import copy
        self.model = model
        self.fused = bool(fused)
        self.s = settings or RasterSettings()
        self.gated = bool(gated)
        self.B = int(views_per_step)
        dev = model.flat.device
        self.n_train = len(train_cams)
        # B slots with the capacity of the largest training view
        wmax = max(int(c.width) for c in train_cams)
        hmax = max(int(c.height) for c in train_cams)
        slot_cam = copy.copy(train_cams[0])
        slot_cam.width, slot_cam.height = wmax, hmax
        self.slot = Views([slot_cam] * self.B, self.s.tile, dev)
        self.poses = Views(train_cams, self.s.tile, dev)
        self.renderer = Renderer(model.n, model.sh_degree, self.slot, self.s, pair_capacity, dev)
        self.renderer.sizes_on_device = True
        if isinstance(targets, torch.Tensor):  # one stacked tensor: used in place (no copy)
            t = targets.contiguous()
            self.targets = t.view(-1)
            self.target_offsets = torch.arange(t.shape[0], dtype=torch.int64, device=dev) * t[0].numel()
        else:
            sizes = [int(x.numel()) for x in targets]
            self.targets = torch.cat([x.contiguous().view(-1) for x in targets]).to(dev)
            self.target_offsets = torch.as_tensor(np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64),
                                                  device=dev)
        self.seq = torch.as_tensor(np.asarray(view_seq, np.int32), device=dev)
        self.iter = torch.zeros(1, dtype=torch.int64, device=dev)
        self.view_ids = torch.zeros(self.B, dtype=torch.int32, device=dev)
        self.g = torch.zeros(self.B, dtype=torch.uint8, device=dev)
        self.any = torch.zeros(1, dtype=torch.int32, device=dev)
        self.gate = Gate(self.n_train, W, beta, eps, rho_lo, dev)
        if adam is not None:
            self.adam = adam
        else:
            self.adam = AdamState(model, lr) if lr is not None else AdamState(model)
        self.stats = stats
        self.select_tile = int(self.s.tile) if compact_tiles else 0
        self.per_view = bool(per_view_steps) and self.B > 1 and self.fused
        if self.per_view:
            self.view_gates = torch.zeros(self.B * self.B, dtype=torch.uint8, device=dev)
            self.view_do = torch.zeros(self.B, dtype=torch.int32, device=dev)
        self.lr_scale = bool(batch_lr_scale) and self.B > 1 and self.gated
        self.adam.cfg.lr_scale_den = self.B if self.lr_scale else 0
        self.params = model.c_params()
        self.grads = model.c_grads(self.adam.grad)
        self.stream = torch.cuda.Stream(device=dev)
        self.body_stream = torch.cuda.Stream(device=dev)
        self.graph = None
        # per-iteration log (losses, decisions, gradient and update norms), filled
        # on the device inside the step; log_capacity iterations, then it wraps
        self.log_cap = int(log_capacity)
        if self.log_cap > 0:
            self.loss_log = torch.zeros(self.log_cap * self.B, dtype=torch.float32, device=dev)
            self.g_log = torch.zeros(self.log_cap * self.B, dtype=torch.uint8, device=dev)
            self.norm_log = torch.zeros(2 * self.log_cap, dtype=torch.float64, device=dev)
            self.norms2 = torch.zeros(2, dtype=torch.float64, device=dev)
        else:
            self.loss_log = self.g_log = self.norm_log = self.norms2 = None

    # ---- pieces of one iteration
    def _front(self, s):
        gsr.call("gs_select_views", gsr.ptr(self.seq), int(self.seq.numel()), gsr.ptr(self.iter), self.B,
                 gsr.ptr(self.view_ids), gsr.ptr(self.poses.dev), gsr.ptr(self.slot.dev), self.select_tile,
                 gsr.stream_handle(s))
        self.renderer.forward(self.params, s)
        self.renderer.compute_loss(self.targets, self.target_offsets, self.view_ids, with_grad=False, stream=s)

    def _back(self, s, predicated: bool):
        """predicated: the branch is issued unconditionally and each part checks
        the device flags; otherwise it runs inside the gate's IF node (any g =
        1), where only a batch still needs the per-view gate."""
        r = self.renderer
        gate = self.g if (predicated or self.B > 1) and self.gated else None
        r.loss_backward(self.targets, self.target_offsets, self.view_ids, stream=s)
        # the step-gate word (number of opened views) is passed when the step
        # is predicated on it, or when it scales the step
        do_step = self.any if (predicated or self.lr_scale) else None
        if self.per_view:
            # the raster adjoint of the opened views, then one projection
            # adjoint + Adam step per opened view, in slot order
            gsr.call("gs_view_steps", gsr.ptr(self.g), self.B, int(not self.gated), gsr.ptr(self.view_gates),
                     gsr.ptr(self.view_do), gsr.stream_handle(s))
            r.raster_bwd(view_gate=gate, stream=s)
            for k in range(self.B):
                r.project_bwd_adam(self.model, self.adam, view_gate=self.view_gates[k * self.B:(k + 1) * self.B],
                                   do_step=self.view_do[k:k + 1], norms2=self.norms2, stream=s)
        elif self.fused:
            r.backward_adam(self.model, self.adam, view_gate=gate, do_step=do_step, norms2=self.norms2, stream=s)
        else:
            r.backward(self.params, self.grads, view_gate=gate, accumulate=False, stream=s)
            self.adam.step(do_step=do_step, norms2=self.norms2, stream=s)
        if self.stats is not None:  # the 2D gradients are still in the workspace
            self.stats.accumulate(r, view_gate=self.g if (predicated or self.B > 1) and self.gated else None,
                                  stream=s)

    def _update(self, s):
        self.gate.update(self.view_ids, self.renderer.loss, stream=s)
        if self.log_cap > 0:
            gsr.call("gs_log_step", gsr.ptr(self.iter), self.B, gsr.ptr(self.renderer.loss), gsr.ptr(self.g),
                     gsr.ptr(self.norms2), gsr.ptr(self.loss_log), gsr.ptr(self.g_log), gsr.ptr(self.norm_log),
                     self.log_cap, gsr.stream_handle(s))

    def read_log(self, iters: int) -> dict:
        """The last `iters` (<= log_capacity) logged iterations, oldest first:
        losses [iters, B], decisions [iters, B], sum g^2 and sum dp^2 [iters]."""
        assert 0 < iters <= self.log_cap
        torch.cuda.synchronize()
        it = int(self.iter.item())
        idx = [(k % self.log_cap) for k in range(it - iters, it)]
        L = self.loss_log.view(self.log_cap, self.B).cpu().numpy()[idx]
        G = self.g_log.view(self.log_cap, self.B).cpu().numpy()[idx]
        Nm = self.norm_log.view(self.log_cap, 2).cpu().numpy()[idx]
        return dict(loss=L, g=G, grad_sq=Nm[:, 0], update_sq=Nm[:, 1])

    # ---- eager
    def step_eager(self) -> None:
        s = self.stream
        self._front(s)
        self.gate.decide(self.view_ids, self.renderer.loss, self.g, self.any, stream=s)
        self._back(s, predicated=self.gated)
        self._update(s)

    # ---- graph
    def capture(self) -> None:
        s, b = self.stream, self.body_stream
        hs, hb = gsr.stream_handle(s), gsr.stream_handle(b)
        torch.cuda.synchronize()
        gsr.call("gs_graph_begin", hs)
        try:
            self._front(s)
            if self.gated:
                cond = C.c_uint64()
                gsr.call("gs_graph_cond_create", hs, C.byref(cond))
                self.gate.decide(self.view_ids, self.renderer.loss, self.g, self.any, cond=cond.value, stream=s)
                gsr.call("gs_graph_if_begin", hs, cond, hb)
                self._back(b, predicated=False)
                gsr.call("gs_graph_if_end", hs, hb)
            else:
                self.gate.decide(self.view_ids, self.renderer.loss, self.g, self.any, stream=s)
                self._back(s, predicated=False)
            self._update(s)
        finally:
            g = C.c_void_p()
            code = gsr.lib().gs_graph_end(hs, C.byref(g))
        gsr.check("gs_graph_end", code)
        self.graph = g
        kc = (C.c_int64 * 2)()
        gsr.call("gs_graph_kernel_counts", self.graph, kc)
        self.kernels_per_step = (int(kc[0]), int(kc[1]))

    def step_graph(self) -> None:
        if self.graph is None:
            self.capture()
        gsr.call("gs_graph_launch", self.graph, gsr.stream_handle(self.stream))

    def close(self) -> None:
        if self.graph is not None:
            gsr.lib().gs_graph_destroy(self.graph)
            self.graph = None

    # ---- state
    def reset(self, flat_params: torch.Tensor) -> None:
        """Back to iteration 0 from the given parameters (device-side copies)."""
        with torch.cuda.stream(self.stream):
            self.model.flat.copy_(flat_params)
            self.adam.m.zero_()
            self.adam.v.zero_()
            self.adam.grad.zero_()
            self.adam.step_count.zero_()
            self.iter.zero_()
        self.gate.reset(self.stream)

    def snapshot(self) -> dict:
        """Parameters and optimizer state (device copies)."""
        torch.cuda.synchronize()
        return dict(flat=self.model.flat.clone(), m=self.adam.m.clone(), v=self.adam.v.clone(),
                    step=self.adam.step_count.clone())

    def restore(self, snap: dict) -> None:
        """Continue from a snapshot: parameters and Adam state as saved, the gate
        empty and the iteration counter at 0 (the start of a post-densification
        phase)."""
        with torch.cuda.stream(self.stream):
            self.model.flat.copy_(snap["flat"])
            self.adam.m.copy_(snap["m"])
            self.adam.v.copy_(snap["v"])
            self.adam.step_count.copy_(snap["step"])
            self.adam.grad.zero_()
            self.iter.zero_()
        self.gate.reset(self.stream)

    def evaluate(self, view_ids=None) -> np.ndarray:
        """Loss of every training view (or the given ones) with the current
        parameters, B views per forward pass."""
        ids = list(range(self.n_train) if view_ids is None else view_ids)
        n = len(ids)
        seq = torch.as_tensor(np.asarray(ids, np.int32), device=self.model.flat.device)
        it = torch.zeros(1, dtype=torch.int64, device=seq.device)
        vid = torch.zeros(self.B, dtype=torch.int32, device=seq.device)
        out = torch.zeros(n + self.B, dtype=torch.float32, device=seq.device)
        s = self.stream
        with torch.cuda.stream(s):
            for k in range(0, n, self.B):
                gsr.call("gs_select_views", gsr.ptr(seq), n, gsr.ptr(it), self.B, gsr.ptr(vid),
                         gsr.ptr(self.poses.dev), gsr.ptr(self.slot.dev), self.select_tile, gsr.stream_handle(s))
                self.renderer.forward(self.params, s)
                self.renderer.compute_loss(self.targets, self.target_offsets, vid, stream=s)
                out[k:k + self.B].copy_(self.renderer.loss)
        s.synchronize()
        return out[:n].cpu().numpy()


class HostTargets:
    """Feeds a one-view-per-iteration RefinementLoop from per-view targets in
    pinned host memory.  The loop must have been built with a single device
    target slot that every view maps to (target_offsets all 0).  The target
    of iteration k + 1 is copied host -> device into a staging buffer on a
    copy stream while iteration k runs; at the start of iteration k + 1 it is
    moved into the slot with a device copy on the loop's stream, so the host
    transfer overlaps the previous iteration instead of preceding this one."""

    def __init__(self, loop: RefinementLoop, host_targets, view_seq):
        assert loop.B == 1, "one view per iteration"
        self.loop = loop
        self.host = host_targets
        self.seq = np.asarray(view_seq)
        self.slot = loop.targets
        self.stage = [torch.empty_like(self.slot) for _ in range(2)]
        self.copy_stream = torch.cuda.Stream(device=self.slot.device)
        self.ready = [torch.cuda.Event(), torch.cuda.Event()]
        self.free = [torch.cuda.Event(), torch.cuda.Event()]
        self.k = 0

    def reset(self) -> None:
        """Back to iteration 0 (with the loop's restore/reset)."""
        torch.cuda.synchronize()
        self.k = 0

    def _prefetch(self, k: int) -> None:
        b = k % 2
        v = int(self.seq[k % len(self.seq)])
        with torch.cuda.stream(self.copy_stream):
            self.copy_stream.wait_event(self.free[b])  # the slot copy out of this buffer is done
            self.stage[b].copy_(self.host[v].reshape(-1), non_blocking=True)
            self.ready[b].record(self.copy_stream)

    def step(self) -> None:
        """One iteration (graph replay) with its target fed from the host."""
        k = self.k
        if k == 0:
            self._prefetch(0)
        self._prefetch(k + 1)
        ls = self.loop.stream
        b = k % 2
        ls.wait_event(self.ready[b])
        with torch.cuda.stream(ls):
            self.slot.copy_(self.stage[b], non_blocking=True)
        self.free[b].record(ls)
        self.loop.step_graph()
        self.k += 1


def densification_phase(model: GaussianModel, train_cams: list, targets, view_seq, iters: int, cfg,
                        settings: RasterSettings | None = None, interval: int = 100, start: int = 500,
                        until: int | None = None, noise_seed: int = 0, capacity_per_gaussian: int = 24,
                        max_gaussians: int | None = None, adam: AdamState | None = None, on_step=None):
    """Iterations 0..iters of always-backward refinement with adaptive density
    control (Sec. 3, the phase before T_d): the statistic accumulates after
    every backward pass, and at every multiple of `interval` in [start,
    until) (until = iters) the set is cloned, split and pruned by
    gs_densify_decide / gs_densify_apply and the statistic restarts.  Between
    two density steps N is fixed and the iterations replay one captured
    graph.  When a step would grow the set beyond max_gaussians it only
    prunes.  Split noise: standard normal draws from a seeded CUDA generator.
    Returns (model, adam, history); history rows are (iteration, n_before,
    clones, splits, prunes, n_after, [median, 90th, 99th percentile of the
    mean gradient norm over the Gaussians seen])."""
    from . import gsr
    st = settings or RasterSettings()
    until = iters if until is None else until
    dev = model.flat.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(noise_seed))
    adam = adam if adam is not None else AdamState(model)
    stats = DensityStats(model.n, dev)
    steps = [k for k in range(max(start, interval), min(until, iters) + 1, interval) if k > 0]
    history, it = [], 0
    for end in steps + ([iters] if not steps or steps[-1] < iters else []):
        if end > it:
            loop = RefinementLoop(model, train_cams, targets, view_seq, st, gated=False,
                                  pair_capacity=capacity_per_gaussian * model.n, adam=adam, stats=stats)
            loop.iter.fill_(it)
            loop.capture()
            for _ in range(end - it):
                loop.step_graph()
            loop.close()
            torch.cuda.synchronize()
            status = int(loop.renderer.status.item())
            if status != 0:
                raise gsr.GsError("densification_phase", status)
            del loop
            it = end
        if end in steps:
            noise = torch.randn((model.n, 2, 3), generator=gen, device=dev, dtype=torch.float32)
            # the statistic's distribution over the Gaussians seen so far (for the log)
            seen = stats.denom > 0
            avg = stats.accum[seen] / stats.denom[seen].float()
            q = torch.quantile(avg[:1 << 24], torch.tensor([0.5, 0.9, 0.99], device=dev)).tolist() \
                if avg.numel() else [0.0, 0.0, 0.0]
            c = cfg
            if max_gaussians is not None:
                action, offsets = densify_decide_count(model, stats, cfg)
                if offsets > max_gaussians:  # prune only
                    c = gsr.gs_densify_config(float("inf"), cfg.log_size_thr, cfg.logit_prune_thr,
                                              cfg.log_split_shrink)
            n0 = model.n
            model, adam, action = densify(model, adam, stats, c, noise)
            counts = torch.bincount(action.long(), minlength=4).cpu().tolist()
            history.append((it, n0, counts[1], counts[2], counts[3], model.n, q))
            if on_step is not None:
                on_step(history[-1])
            stats = DensityStats(model.n, dev)
            del noise
    return model, adam, history


def densify_decide_count(model: GaussianModel, stats: DensityStats, cfg):
    """(actions, new count) of a density step without applying it (synchronises)."""
    from .raster import densify_decide
    action, offsets = densify_decide(model, stats, cfg)
    return action, int(offsets[model.n].item())
