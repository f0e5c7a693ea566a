"""Buffers and call sequence of the rasterizer, on top of the C ABI.

Everything here is memory management and argument marshalling; every
arithmetic step runs in libgsr's kernels:

  GaussianModel   the flat parameter buffer (gs_param_layout) with per-group views
  Views           gs_camera slots in device memory (+ host copy), tile/pixel layout
  Renderer        per-view buffers for project -> bin/sort -> render -> loss -> backward
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import gsr


@dataclass
class RasterSettings:
    tile: int = 16
    batch: int = 256
    lowpass: float = 0.3
    alpha_max: float = 0.99
    alpha_min: float = 1.0 / 255.0
    t_min: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)
    lambda_ssim: float = 0.2
    pixels_per_thread: int = 2      # raster adjoint
    pixels_per_thread_fwd: int = 1  # forward compositing
    longest_tiles_first: bool = True  # launch tiles by descending list length (gs_tile_order)
    persistent: bool = False  # compositing kernels as a persistent grid taking tiles from a device queue
    # the binning writes super-tile lists (gs_bin_sort_coarse) and the compositing
    # kernels filter each tile's entries from them (the *_coarse calls)
    coarse_lists: bool = False

    def struct(self, sh_degree: int) -> gsr.gs_raster_config:
        c = gsr.gs_raster_config()
        c.lowpass, c.alpha_max, c.alpha_min, c.t_min = self.lowpass, self.alpha_max, self.alpha_min, self.t_min
        for i in range(3):
            c.bg[i] = float(self.bg[i])
        c.tile, c.batch, c.sh_degree = int(self.tile), int(self.batch), int(sh_degree)
        c.pixels_per_thread = int(self.pixels_per_thread)
        return c


def param_layout(n: int, sh_degree: int):
    out = (C.c_int64 * 6)()
    gsr.call("gs_param_layout", n, sh_degree, out)
    return [int(x) for x in out]


class GaussianModel:
    """N Gaussians in one flat float32 buffer laid out by gs_param_layout."""

    def __init__(self, n: int, sh_degree: int, device="cuda"):
        self.n, self.sh_degree = int(n), int(sh_degree)
        self.K = (sh_degree + 1) ** 2
        self.offsets = param_layout(self.n, self.sh_degree)
        self.flat = torch.zeros(self.offsets[5], dtype=torch.float32, device=device)
        self.views = self.group_views(self.flat)

    def group_views(self, flat: torch.Tensor) -> dict:
        o, n = self.offsets, self.n
        return dict(means=flat[o[0]:o[0] + 3 * n].view(n, 3), log_scales=flat[o[1]:o[1] + 3 * n].view(n, 3),
                    quats=flat[o[2]:o[2] + 4 * n].view(n, 4), opacity_logit=flat[o[3]:o[3] + n],
                    sh=flat[o[4]:o[4] + 3 * self.K * n].view(n, self.K, 3))

    @classmethod
    def from_scene(cls, scene, device="cuda") -> "GaussianModel":
        m = cls(scene.n, scene.sh_degree, device)
        m.load_scene(scene)
        return m

    def load_scene(self, scene) -> None:
        for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
            self.views[k].copy_(torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)))

    def c_params(self, flat: torch.Tensor | None = None) -> gsr.gs_params:
        v = self.views if flat is None else self.group_views(flat)
        p = gsr.gs_params()
        p.means, p.log_scales, p.quats = v["means"].data_ptr(), v["log_scales"].data_ptr(), v["quats"].data_ptr()
        p.opacity_logit, p.sh = v["opacity_logit"].data_ptr(), v["sh"].data_ptr()
        p.n, p.sh_degree = self.n, self.sh_degree
        p._owner = (self, v)  # the struct holds raw pointers: keep their storage alive with it
        return p

    def c_grads(self, flat: torch.Tensor) -> gsr.gs_grads:
        v = self.group_views(flat)
        g = gsr.gs_grads()
        g.means, g.log_scales, g.quats = v["means"].data_ptr(), v["log_scales"].data_ptr(), v["quats"].data_ptr()
        g.opacity_logit, g.sh = v["opacity_logit"].data_ptr(), v["sh"].data_ptr()
        g._owner = v
        return g


def camera_struct(cam) -> gsr.gs_camera:
    c = gsr.gs_camera()
    R = np.asarray(cam.R, np.float32).ravel()
    t = np.asarray(cam.t, np.float32).ravel()
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.znear = int(cam.width), int(cam.height), float(cam.znear)
    return c


class Views:
    """Camera slots: host array (with tile/pixel offsets filled by
    gs_camera_layout) and its copy in device memory."""

    def __init__(self, cams: list, tile: int, device="cuda"):
        self.n = len(cams)
        self.host = (gsr.gs_camera * self.n)(*[camera_struct(c) for c in cams])
        tt, tp = C.c_int64(), C.c_int64()
        gsr.call("gs_camera_layout", self.host, self.n, int(tile), C.byref(tt), C.byref(tp))
        self.total_tiles, self.total_pixels = int(tt.value), int(tp.value)
        raw = bytes(C.string_at(C.addressof(self.host), C.sizeof(self.host)))
        self.dev = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)
        self.sizes = [(int(c.width), int(c.height)) for c in cams]
        self.max_view_tiles = max(-(-w // tile) * -(-h // tile) for w, h in self.sizes)
        # super-tiles of 4 x 4 tiles per view (the super-tile lists' tables)
        self.max_view_super_tiles = max(-(-(-(-w // tile)) // 4) * -(-(-(-h // tile)) // 4) for w, h in self.sizes)
        self.pix_offsets = [int(self.host[v].pix_offset) for v in range(self.n)]

    def image_view(self, flat: torch.Tensor, v: int) -> torch.Tensor:
        w, h = self.sizes[v]
        o = 3 * self.pix_offsets[v]
        return flat[o:o + 3 * w * h].view(3, h, w)


class Renderer:
    """All per-view buffers of one rasterization pipeline over `views`."""

    def __init__(self, n: int, sh_degree: int, views: Views, settings: RasterSettings | None = None,
                 pair_capacity: int | None = None, device="cuda", keep_keys: bool = False,
                 coarse_capacity: int | None = None):
        self.s = settings or RasterSettings()
        self.n, self.sh_degree, self.views = int(n), int(sh_degree), views
        # True when the device cameras are chosen on the device (slots filled by
        # gs_select_views): the loss then reads each view's size from them
        self.sizes_on_device = False
        self.cfg = self.s.struct(sh_degree)
        self.cfg_fwd = self.s.struct(sh_degree)
        self.cfg_fwd.pixels_per_thread = int(self.s.pixels_per_thread_fwd)
        V, T, P = views.n, views.total_tiles, views.total_pixels
        if pair_capacity is None:
            pair_capacity = max(1 << 16, 16 * n * V)
        self.cap = int(pair_capacity)
        dev = device
        self.rec = torch.empty(V * n * 12, dtype=torch.float32, device=dev)
        self.rect = torch.empty(V * n * 4, dtype=torch.int32, device=dev)
        self.touched = torch.empty(V * n, dtype=torch.int32, device=dev)
        # depth keys and packed rectangles written by gs_project for gs_bin_sort;
        # valid only after project() (records set by other means clear the flag)
        self.depth_key = torch.empty(V * n, dtype=torch.int32, device=dev)
        self.rect16 = torch.empty(V * n * 4, dtype=torch.int16, device=dev)
        self.aux_valid = False
        self.coarse = bool(self.s.coarse_lists)
        if self.coarse:  # super-tile lists (at most one entry per pair)
            self.ccap = int(coarse_capacity) if coarse_capacity is not None else self.cap
            n_st = T // 4 + V
            self.c_gid = torch.empty(max(self.ccap, 1), dtype=torch.int32, device=dev)
            self.c_mask = torch.empty(max(self.ccap, 1), dtype=torch.int16, device=dev)
            self.c_start = torch.empty(n_st, dtype=torch.int32, device=dev)
            self.c_count = torch.zeros(n_st, dtype=torch.int32, device=dev)
            self.c_view_first = torch.empty(V + 1, dtype=torch.int64, device=dev)
            self.c_total = torch.zeros(1, dtype=torch.int64, device=dev)
            self.lists = gsr.gs_coarse_lists(self.c_gid.data_ptr(), self.c_mask.data_ptr(), self.c_start.data_ptr(),
                                             self.c_count.data_ptr(), self.c_view_first.data_ptr(),
                                             self.c_total.data_ptr(), self.ccap)
            self.vals = None
        else:
            self.vals = torch.empty(max(self.cap, 1), dtype=torch.int32, device=dev)
        self.keys = torch.empty(max(self.cap, 1), dtype=torch.int64, device=dev) if keep_keys else None
        self.ranges = torch.empty(2 * T, dtype=torch.int32, device=dev)
        self.tile_order = torch.empty(T, dtype=torch.int32, device=dev) if self.s.longest_tiles_first else None
        self.queue = torch.zeros(1, dtype=torch.int32, device=dev) if self.s.persistent else None
        self.pair_count = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.image = torch.empty(3 * P, dtype=torch.float32, device=dev)
        self.T_final = torch.empty(P, dtype=torch.float32, device=dev)
        self.n_last = torch.empty(P, dtype=torch.int32, device=dev)
        self.ckpt_slots = int(gsr.lib().gs_ckpt_slots(self.cap, T, self.s.batch))
        self.ckpt = torch.empty(self.ckpt_slots * self.s.tile * self.s.tile, dtype=torch.float32, device=dev)
        self.batch_pos = torch.empty(self.ckpt_slots, dtype=torch.int32, device=dev) if self.coarse else None
        L = gsr.lib()
        if self.coarse:
            self.bin_ws_bytes = int(L.gs_bin_sort_coarse_workspace_size(n, V, T))
        else:
            self.bin_ws_bytes = int(L.gs_bin_sort_workspace_size(n, V, self.cap, T))
        self.bin_ws = torch.empty(self.bin_ws_bytes, dtype=torch.uint8, device=dev)
        self.loss_ws_bytes = int(L.gs_loss_workspace_size(views.host, V))
        self.loss_ws = torch.empty(self.loss_ws_bytes, dtype=torch.uint8, device=dev)
        self.bwd_ws_bytes = int(L.gs_render_bwd_workspace_size(n, V))
        self.bwd_ws = torch.empty(self.bwd_ws_bytes, dtype=torch.uint8, device=dev)
        self.dL_dimage = torch.empty(3 * P, dtype=torch.float32, device=dev)
        self.loss = torch.zeros(V, dtype=torch.float32, device=dev)

    # --- structs
    def c_proj(self, with_aux: bool | None = None) -> gsr.gs_projected:
        p = gsr.gs_projected()
        p.rec, p.rect, p.tiles_touched = self.rec.data_ptr(), self.rect.data_ptr(), self.touched.data_ptr()
        if self.aux_valid if with_aux is None else with_aux:
            p.depth_key, p.rect16 = self.depth_key.data_ptr(), self.rect16.data_ptr()
        return p

    def c_saved(self) -> gsr.gs_fwd_saved:
        s = gsr.gs_fwd_saved()
        s.T_final, s.n_last, s.ckpt, s.ckpt_slots = (self.T_final.data_ptr(), self.n_last.data_ptr(),
                                                     self.ckpt.data_ptr(), self.ckpt_slots)
        s.tile_order = self.tile_order.data_ptr() if self.tile_order is not None else None
        s.queue = self.queue.data_ptr() if self.queue is not None else None
        s.batch_pos = self.batch_pos.data_ptr() if self.batch_pos is not None else None
        return s

    # --- pipeline steps (each one C-ABI call)
    def project(self, params: gsr.gs_params, stream=None) -> None:
        gsr.call("gs_project", C.byref(params), gsr.ptr(self.views.dev), self.views.n, C.byref(self.cfg),
                 self.c_proj(with_aux=True), gsr.ptr(self.status), gsr.stream_handle(stream))
        self.aux_valid = True

    def bin_sort(self, stream=None) -> None:
        proj = self.c_proj()
        if self.coarse:
            gsr.call("gs_bin_sort_coarse", C.byref(proj), gsr.ptr(self.views.dev), self.views.n, self.n,
                     self.views.total_tiles, self.views.max_view_tiles, self.views.max_view_super_tiles,
                     C.byref(self.cfg), gsr.ptr(self.bin_ws),
                     self.bin_ws_bytes, C.byref(self.lists), self.cap, gsr.ptr(self.ranges),
                     gsr.ptr(self.pair_count), gsr.ptr(self.status), gsr.stream_handle(stream))
        else:
            gsr.call("gs_bin_sort", C.byref(proj), gsr.ptr(self.views.dev), self.views.n, self.n,
                     self.views.total_tiles, self.views.max_view_tiles, C.byref(self.cfg), gsr.ptr(self.bin_ws),
                     self.bin_ws_bytes, gsr.ptr(self.keys), gsr.ptr(self.vals), self.cap, gsr.ptr(self.ranges),
                     gsr.ptr(self.pair_count), gsr.ptr(self.status), gsr.stream_handle(stream))
        if self.tile_order is not None:
            gsr.call("gs_tile_order", gsr.ptr(self.ranges), self.views.total_tiles, gsr.ptr(self.tile_order),
                     gsr.stream_handle(stream))

    def render_fwd(self, stream=None) -> None:
        proj = self.c_proj()
        name, lists = self._lists("gs_render_fwd")
        gsr.call(name, C.byref(proj), self.n, lists, gsr.ptr(self.ranges),
                 gsr.ptr(self.views.dev), self.views.n, self.views.total_tiles, C.byref(self.cfg_fwd),
                 gsr.ptr(self.image), self.c_saved(), gsr.ptr(self.status), gsr.stream_handle(stream))

    def _lists(self, name: str):
        """The call for this renderer's list form and its list argument."""
        if self.coarse:
            return name + "_coarse", C.byref(self.lists)
        return name, gsr.ptr(self.vals)

    def forward(self, params: gsr.gs_params, stream=None) -> torch.Tensor:
        self.project(params, stream)
        self.bin_sort(stream)
        self.render_fwd(stream)
        return self.image

    def _cams_dev(self):
        return gsr.ptr(self.views.dev) if self.sizes_on_device else None

    def compute_loss(self, target: torch.Tensor, target_offsets=None, view_ids=None, with_grad=False,
                     stream=None) -> torch.Tensor:
        gsr.call("gs_loss", gsr.ptr(self.image), gsr.ptr(target), gsr.ptr(target_offsets), self.views.host,
                 self._cams_dev(), gsr.ptr(view_ids), self.views.n, float(self.s.lambda_ssim), gsr.ptr(self.loss_ws),
                 self.loss_ws_bytes, gsr.ptr(self.loss), gsr.ptr(self.dL_dimage) if with_grad else None,
                 gsr.stream_handle(stream))
        return self.loss

    def loss_backward(self, target: torch.Tensor, target_offsets=None, view_ids=None, stream=None) -> torch.Tensor:
        gsr.call("gs_loss_backward", gsr.ptr(self.image), gsr.ptr(target), gsr.ptr(target_offsets),
                 self.views.host, self._cams_dev(), gsr.ptr(view_ids), self.views.n, float(self.s.lambda_ssim),
                 gsr.ptr(self.loss_ws), self.loss_ws_bytes, gsr.ptr(self.dL_dimage), gsr.stream_handle(stream))
        return self.dL_dimage

    def backward(self, params: gsr.gs_params, grads: gsr.gs_grads, dL_dimage: torch.Tensor | None = None,
                 view_gate: torch.Tensor | None = None, accumulate: bool = False, stream=None) -> None:
        proj = self.c_proj()
        dl = self.dL_dimage if dL_dimage is None else dL_dimage
        name, lists = self._lists("gs_render_bwd")
        gsr.call(name, C.byref(params), C.byref(proj), lists, gsr.ptr(self.ranges),
                 gsr.ptr(self.views.dev), self.views.n, self.views.total_tiles, C.byref(self.cfg),
                 self.c_saved(), gsr.ptr(dl), gsr.ptr(view_gate), grads, int(bool(accumulate)),
                 gsr.ptr(self.bwd_ws), self.bwd_ws_bytes, gsr.ptr(self.status), gsr.stream_handle(stream))

    def raster_bwd(self, dL_dimage: torch.Tensor | None = None, view_gate: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
        """Raster adjoint only: per-view 2D gradients into self.bwd_ws ([V][N][12] floats)."""
        proj = self.c_proj()
        dl = self.dL_dimage if dL_dimage is None else dL_dimage
        name, lists = self._lists("gs_raster_bwd")
        gsr.call(name, C.byref(proj), self.n, lists, gsr.ptr(self.ranges),
                 gsr.ptr(self.views.dev), self.views.n, self.views.total_tiles, C.byref(self.cfg), self.c_saved(),
                 gsr.ptr(dl), gsr.ptr(view_gate), gsr.ptr(self.bwd_ws), self.bwd_ws_bytes, gsr.ptr(self.status),
                 gsr.stream_handle(stream))
        return self.bwd_ws.view(torch.float32).view(self.views.n, self.n, 12)

    def project_bwd(self, params: gsr.gs_params, grads: gsr.gs_grads, view_gate: torch.Tensor | None = None,
                    accumulate: bool = False, stream=None) -> None:
        """Projection adjoint from the 2D gradients that raster_bwd left in self.bwd_ws."""
        gsr.call("gs_project_bwd", C.byref(params), gsr.ptr(self.views.dev), self.views.n, C.byref(self.cfg),
                 gsr.ptr(self.bwd_ws), gsr.ptr(view_gate), grads, int(bool(accumulate)), gsr.ptr(self.status),
                 gsr.stream_handle(stream))

    def backward_adam(self, model: "GaussianModel", adam: "AdamState", dL_dimage: torch.Tensor | None = None,
                      view_gate: torch.Tensor | None = None, do_step: torch.Tensor | None = None,
                      norms2: torch.Tensor | None = None, stream=None) -> None:
        """Backward pass and Adam step in one call (gs_render_bwd_adam); norms2
        (2 float64, optional) receives the sums of g^2 and of the squared update."""
        proj = self.c_proj()
        dl = self.dL_dimage if dL_dimage is None else dL_dimage
        name, lists = self._lists("gs_render_bwd_adam")
        gsr.call(name, gsr.ptr(model.flat), gsr.ptr(adam.m), gsr.ptr(adam.v), model.n,
                 model.sh_degree, C.byref(proj), lists, gsr.ptr(self.ranges), gsr.ptr(self.views.dev),
                 self.views.n, self.views.total_tiles, C.byref(self.cfg), self.c_saved(), gsr.ptr(dl),
                 gsr.ptr(view_gate), C.byref(adam.cfg), gsr.ptr(do_step), gsr.ptr(adam.step_count), gsr.ptr(norms2),
                 gsr.ptr(self.bwd_ws), self.bwd_ws_bytes, gsr.ptr(self.status), gsr.stream_handle(stream))

    def project_bwd_adam(self, model: "GaussianModel", adam: "AdamState", view_gate: torch.Tensor | None = None,
                         do_step: torch.Tensor | None = None, norms2: torch.Tensor | None = None,
                         stream=None) -> None:
        """Projection adjoint of the 2D gradients in self.bwd_ws fused with the
        Adam step (gs_project_bwd_adam): raster_bwd then this = backward_adam."""
        gsr.call("gs_project_bwd_adam", gsr.ptr(model.flat), gsr.ptr(adam.m), gsr.ptr(adam.v), model.n,
                 model.sh_degree, gsr.ptr(self.views.dev), self.views.n, C.byref(self.cfg), gsr.ptr(self.bwd_ws),
                 gsr.ptr(view_gate), C.byref(adam.cfg), gsr.ptr(do_step), gsr.ptr(adam.step_count), gsr.ptr(norms2),
                 gsr.ptr(self.status), gsr.stream_handle(stream))

    def census(self, stream=None) -> dict:
        """Work of the last forward pass (gs_raster_census; synchronises):
        sum of n_last, support-box evaluations, contributing pairs, (tile,
        Gaussian) pairs with a contributor, staged list entries."""
        counts = torch.zeros(5, dtype=torch.int64, device=self.image.device)
        proj = self.c_proj()
        vals = self.vals
        if self.coarse:  # the census walks tile lists: bin the same projection into them once
            dev = self.image.device
            vals = torch.empty(max(self.cap, 1), dtype=torch.int32, device=dev)
            ranges = torch.empty_like(self.ranges)
            ws_bytes = int(gsr.lib().gs_bin_sort_workspace_size(self.n, self.views.n, self.cap, self.views.total_tiles))
            ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
            gsr.call("gs_bin_sort", C.byref(proj), gsr.ptr(self.views.dev), self.views.n, self.n,
                     self.views.total_tiles, self.views.max_view_tiles, C.byref(self.cfg), gsr.ptr(ws), ws_bytes, None,
                     gsr.ptr(vals), self.cap, gsr.ptr(ranges), gsr.ptr(self.pair_count), gsr.ptr(self.status),
                     gsr.stream_handle(stream))
        gsr.call("gs_raster_census", C.byref(proj), self.n, gsr.ptr(vals), gsr.ptr(self.ranges),
                 gsr.ptr(self.views.dev), self.views.n, self.views.total_tiles, C.byref(self.cfg),
                 gsr.ptr(self.n_last), gsr.ptr(counts), gsr.stream_handle(stream))
        torch.cuda.synchronize()  # the census ran on `stream`, not necessarily the current one
        c = [int(x) for x in counts.cpu().tolist()]
        return dict(sum_n_last=c[0], evaluated=c[1], contributing=c[2], tile_pairs=c[3], staged=c[4])

    # --- helpers for inspection (synchronise)
    def image_of(self, v: int = 0) -> torch.Tensor:
        return self.views.image_view(self.image, v)

    def records(self) -> torch.Tensor:
        return self.rec.view(self.views.n, self.n, 12)


class AdamState:
    """Adam moments and step counter for a GaussianModel (device memory)."""

    def __init__(self, model: GaussianModel, lr=(1.6e-5, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4), beta1=0.9,
                 beta2=0.999, eps=1e-15):
        self.model = model
        dev = model.flat.device
        self.m = torch.zeros_like(model.flat)
        self.v = torch.zeros_like(model.flat)
        self.grad = torch.zeros_like(model.flat)
        self.step_count = torch.zeros(1, dtype=torch.int64, device=dev)
        self.cfg = gsr.gs_adam_config()
        for i in range(6):
            self.cfg.lr[i] = float(lr[i])
        self.cfg.beta1, self.cfg.beta2, self.cfg.eps = float(beta1), float(beta2), float(eps)

    def step(self, do_step: torch.Tensor | None = None, zero_grad: bool = False, norms2: torch.Tensor | None = None,
             stream=None) -> None:
        """norms2: optional float64[2] device tensor that receives sum g^2 and
        sum (p_new - p_old)^2 of this step (added to it)."""
        m = self.model
        gsr.call("gs_adam_step", gsr.ptr(m.flat), gsr.ptr(self.grad), gsr.ptr(self.m), gsr.ptr(self.v), m.n,
                 m.sh_degree, C.byref(self.cfg), gsr.ptr(do_step), gsr.ptr(self.step_count), int(bool(zero_grad)),
                 gsr.ptr(norms2), gsr.stream_handle(stream))


class Gate:
    """SkipGS gate state in device memory (skipgs_gate_*)."""

    def __init__(self, n_views: int, W: int = 500, beta: float = 0.95, eps: float = 1e-8, rho_lo: float = 0.5,
                 device="cuda", stream=None):
        self.cfg = gsr.gs_gate_config()
        self.cfg.W, self.cfg.beta, self.cfg.eps, self.cfg.rho_lo, self.cfg.n_views = int(W), float(beta), float(eps), \
            float(rho_lo), int(n_views)
        nbytes = int(gsr.lib().skipgs_gate_state_size(int(n_views)))
        self.state = torch.zeros(nbytes, dtype=torch.uint8, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.reset(stream)

    def reset(self, stream=None) -> None:
        gsr.call("skipgs_gate_init", C.byref(self.cfg), gsr.ptr(self.state), gsr.stream_handle(stream))

    def decide(self, view_ids: torch.Tensor, losses: torch.Tensor, g: torch.Tensor, any_out=None, cond=None,
               stream=None) -> None:
        h = None
        if cond is not None:
            h = C.c_uint64(int(cond))
        gsr.call("skipgs_gate_decide", gsr.ptr(self.state), gsr.ptr(view_ids), gsr.ptr(losses), int(view_ids.numel()),
                 gsr.ptr(g), gsr.ptr(any_out), C.byref(h) if h is not None else None, gsr.ptr(self.status),
                 gsr.stream_handle(stream))

    def update(self, view_ids: torch.Tensor, losses: torch.Tensor, stream=None) -> None:
        gsr.call("skipgs_gate_update", gsr.ptr(self.state), gsr.ptr(view_ids), gsr.ptr(losses), int(view_ids.numel()),
                 gsr.stream_handle(stream))

    def read(self, stream=None) -> dict:
        out = (C.c_int64 * 7)()
        rho = C.c_double()
        gsr.call("skipgs_gate_read", gsr.ptr(self.state), out, C.byref(rho), gsr.stream_handle(stream))
        return dict(t=out[0], b=out[1], n_w=out[2], n_w1=out[3], calibrated=out[4], errors=out[5], n_views=out[6],
                    rho_min=rho.value)


def densify_config(grad_thr: float, max_scale: float, eps_alpha: float = 0.005,
                   split_factor: float = 1.6) -> gsr.gs_densify_config:
    """Thresholds of adaptive density control in the units gs_densify_decide
    compares: the mean view-space gradient norm (pixels), the largest scale
    (as a log-scale) and the opacity (as a logit); split children's scales
    are divided by split_factor (as a log)."""
    c = gsr.gs_densify_config()
    c.grad_thr = float(grad_thr)
    c.log_size_thr = float(math.log(max_scale))
    c.logit_prune_thr = float(math.log(eps_alpha / (1.0 - eps_alpha))) if eps_alpha > 0 else -float("inf")
    c.log_split_shrink = float(math.log(split_factor))
    return c


class DensityStats:
    """The densification statistic of N Gaussians (device): the summed norm of
    dL/dmean2D over the views each was visible in, and that view count."""

    def __init__(self, n: int, device="cuda"):
        self.n = int(n)
        self.accum = torch.zeros(self.n, dtype=torch.float32, device=device)
        self.denom = torch.zeros(self.n, dtype=torch.int32, device=device)

    def accumulate(self, renderer: "Renderer", view_gate: torch.Tensor | None = None, stream=None) -> None:
        """After a backward pass of `renderer` (its 2D gradients in the workspace)."""
        gsr.call("gs_densify_accumulate", gsr.ptr(renderer.bwd_ws), gsr.ptr(renderer.touched), self.n,
                 renderer.views.n, gsr.ptr(view_gate), gsr.ptr(self.accum), gsr.ptr(self.denom),
                 gsr.stream_handle(stream))

    def reset(self) -> None:
        self.accum.zero_()
        self.denom.zero_()


def densify_decide(model: GaussianModel, stats: DensityStats, cfg: gsr.gs_densify_config, stream=None):
    """Actions (u8[N]) and output offsets (int64[N+1]) on the device."""
    n = model.n
    dev = model.flat.device
    action = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
    offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
    ws_bytes = int(gsr.lib().gs_densify_workspace_size(n))
    ws = torch.empty(max(ws_bytes, 16), dtype=torch.uint8, device=dev)
    gsr.call("gs_densify_decide", gsr.ptr(model.flat), n, model.sh_degree, gsr.ptr(stats.accum),
             gsr.ptr(stats.denom), C.byref(cfg), gsr.ptr(action), gsr.ptr(offsets), gsr.ptr(ws), ws_bytes,
             gsr.stream_handle(stream))
    return action[:n], offsets


def densify(model: GaussianModel, adam: "AdamState", stats: DensityStats, cfg: gsr.gs_densify_config,
            noise: torch.Tensor, status: torch.Tensor | None = None, stream=None):
    """One density-control step: decide, read the new count (synchronises),
    allocate the resized parameter and Adam buffers, write the output set.
    noise: device float [N, 2, 3] standard normal draws for split children.
    Returns (model, adam, action) of the new set (statistics: new zeros)."""
    action, offsets = densify_decide(model, stats, cfg, stream)
    n_out = int(offsets[model.n].item())
    new = GaussianModel(n_out, model.sh_degree, model.flat.device)
    new_adam = AdamState(new)
    new_adam.cfg = adam.cfg
    new_adam.step_count.copy_(adam.step_count)
    gsr.call("gs_densify_apply", gsr.ptr(model.flat), gsr.ptr(adam.m), gsr.ptr(adam.v), model.n, model.sh_degree,
             gsr.ptr(action), gsr.ptr(offsets), gsr.ptr(noise), C.byref(cfg), gsr.ptr(new.flat), gsr.ptr(new_adam.m),
             gsr.ptr(new_adam.v), n_out, gsr.ptr(status), gsr.stream_handle(stream))
    return new, new_adam, action
