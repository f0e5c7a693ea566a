"""Thin ctypes binding of libgsr (include/gsr.h): same names, argument
marshalling only.  Every step of the rasterizer, loss, optimizer and gate runs
in the library's sm_103a kernels; this module only turns torch tensors into
device pointers and streams into handles.  There is no fallback: if the
library is missing, importing the bindings raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsr.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA, GS_ERR_CAPACITY, GS_ERR_NONFINITE, GS_ERR_UNSUPPORTED = range(7)


class GsError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {status_string(code)} ({code})")
        self.code = code


class gs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_float), ("tile_offset", C.c_int32), ("pix_offset", C.c_int64)]


class gs_raster_config(C.Structure):
    _fields_ = [("lowpass", C.c_float), ("alpha_max", C.c_float), ("alpha_min", C.c_float), ("t_min", C.c_float),
                ("bg", C.c_float * 3), ("tile", C.c_int32), ("batch", C.c_int32), ("sh_degree", C.c_int32),
                ("pixels_per_thread", C.c_int32)]


class gs_params(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64), ("sh_degree", C.c_int32)]


class gs_grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p)]


class gs_projected(C.Structure):
    _fields_ = [("rec", C.c_void_p), ("rect", C.c_void_p), ("tiles_touched", C.c_void_p), ("depth_key", C.c_void_p),
                ("rect16", C.c_void_p)]


class gs_fwd_saved(C.Structure):
    _fields_ = [("T_final", C.c_void_p), ("n_last", C.c_void_p), ("ckpt", C.c_void_p), ("ckpt_slots", C.c_int64),
                ("tile_order", C.c_void_p), ("queue", C.c_void_p), ("batch_pos", C.c_void_p)]


class gs_coarse_lists(C.Structure):
    _fields_ = [("gid", C.c_void_p), ("mask", C.c_void_p), ("start", C.c_void_p), ("count", C.c_void_p),
                ("view_first", C.c_void_p), ("total", C.c_void_p), ("capacity", C.c_int64)]


class gs_adam_config(C.Structure):
    _fields_ = [("lr", C.c_float * 6), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("lr_scale_den", C.c_int32)]


class gs_launch_shape(C.Structure):
    _fields_ = [("tile", C.c_int32), ("batch", C.c_int32), ("pixels_per_thread_fwd", C.c_int32),
                ("pixels_per_thread_bwd", C.c_int32)]


class gs_densify_config(C.Structure):
    _fields_ = [("grad_thr", C.c_float), ("log_size_thr", C.c_float), ("logit_prune_thr", C.c_float),
                ("log_split_shrink", C.c_float)]


GS_DENSIFY_KEEP, GS_DENSIFY_CLONE, GS_DENSIFY_SPLIT, GS_DENSIFY_PRUNE = range(4)


class gs_gate_config(C.Structure):
    _fields_ = [("W", C.c_int32), ("beta", C.c_double), ("eps", C.c_double), ("rho_lo", C.c_double),
                ("n_views", C.c_int32)]


_P = C.c_void_p
_S = C.c_void_p  # cudaStream_t
_I32, _I64, _F32, _SZ = C.c_int32, C.c_int64, C.c_float, C.c_size_t

# name -> (restype, argtypes)
_PROTOS = {
    "gs_status_string": (C.c_char_p, [C.c_int]),
    "gs_version": (C.c_int, []),
    "gs_param_layout": (C.c_int, [_I64, _I32, C.POINTER(C.c_int64)]),
    "gs_camera_layout": (C.c_int, [C.POINTER(gs_camera), _I32, _I32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "gs_ckpt_slots": (C.c_int64, [_I64, _I64, _I32]),
    "gs_project": (C.c_int, [C.POINTER(gs_params), _P, _I32, C.POINTER(gs_raster_config), gs_projected, _P, _S]),
    "gs_bin_sort_workspace_size": (C.c_size_t, [_I64, _I32, _I64, _I64]),
    "gs_bin_sort": (C.c_int, [C.POINTER(gs_projected), _P, _I32, _I64, _I64, _I32, C.POINTER(gs_raster_config), _P, _SZ,
                              _P, _P, _I64, _P, _P, _P, _S]),
    "gs_bin_sort_noalloc": (C.c_int, [C.POINTER(gs_projected), _P, _I32, _I64, _I64, _I32, C.POINTER(gs_raster_config),
                                      _P, _P, _I64, _P, _P, _P, _S]),
    "gs_bin_sort_coarse_workspace_size": (C.c_size_t, [_I64, _I32, _I64]),
    "gs_bin_sort_coarse": (C.c_int, [C.POINTER(gs_projected), _P, _I32, _I64, _I64, _I32, _I32,
                                     C.POINTER(gs_raster_config),
                                     _P, _SZ, C.POINTER(gs_coarse_lists), _I64, _P, _P, _P, _S]),
    "gs_tile_order": (C.c_int, [_P, _I64, _P, _S]),
    "gs_render_fwd_coarse": (C.c_int, [C.POINTER(gs_projected), _I64, C.POINTER(gs_coarse_lists), _P, _P, _I32, _I64,
                                       C.POINTER(gs_raster_config), _P, gs_fwd_saved, _P, _S]),
    "gs_render_bwd_coarse": (C.c_int, [C.POINTER(gs_params), C.POINTER(gs_projected), C.POINTER(gs_coarse_lists), _P,
                                       _P, _I32, _I64, C.POINTER(gs_raster_config), gs_fwd_saved, _P, _P, gs_grads,
                                       _I32, _P, _SZ, _P, _S]),
    "gs_raster_bwd_coarse": (C.c_int, [C.POINTER(gs_projected), _I64, C.POINTER(gs_coarse_lists), _P, _P, _I32, _I64,
                                       C.POINTER(gs_raster_config), gs_fwd_saved, _P, _P, _P, _SZ, _P, _S]),
    "gs_render_bwd_adam_coarse": (C.c_int, [_P, _P, _P, _I64, _I32, C.POINTER(gs_projected),
                                            C.POINTER(gs_coarse_lists), _P, _P, _I32, _I64,
                                            C.POINTER(gs_raster_config), gs_fwd_saved, _P, _P,
                                            C.POINTER(gs_adam_config), _P, _P, _P, _P, _SZ, _P, _S]),
    "gs_render_fwd": (C.c_int, [C.POINTER(gs_projected), _I64, _P, _P, _P, _I32, _I64, C.POINTER(gs_raster_config),
                                _P, gs_fwd_saved, _P, _S]),
    "gs_loss_workspace_size": (C.c_size_t, [C.POINTER(gs_camera), _I32]),
    "gs_loss": (C.c_int, [_P, _P, _P, C.POINTER(gs_camera), _P, _P, _I32, _F32, _P, _SZ, _P, _P, _S]),
    "gs_loss_backward": (C.c_int, [_P, _P, _P, C.POINTER(gs_camera), _P, _P, _I32, _F32, _P, _SZ, _P, _S]),
    "gs_render_bwd_workspace_size": (C.c_size_t, [_I64, _I32]),
    "gs_render_bwd": (C.c_int, [C.POINTER(gs_params), C.POINTER(gs_projected), _P, _P, _P, _I32, _I64,
                                C.POINTER(gs_raster_config), gs_fwd_saved, _P, _P, gs_grads, _I32, _P, _SZ, _P, _S]),
    "gs_raster_bwd": (C.c_int, [C.POINTER(gs_projected), _I64, _P, _P, _P, _I32, _I64, C.POINTER(gs_raster_config),
                                gs_fwd_saved, _P, _P, _P, _SZ, _P, _S]),
    "gs_project_bwd": (C.c_int, [C.POINTER(gs_params), _P, _I32, C.POINTER(gs_raster_config), _P, _P, gs_grads, _I32,
                                 _P, _S]),
    "gs_render_bwd_adam": (C.c_int, [_P, _P, _P, _I64, _I32, C.POINTER(gs_projected), _P, _P, _P, _I32, _I64,
                                     C.POINTER(gs_raster_config), gs_fwd_saved, _P, _P, C.POINTER(gs_adam_config), _P,
                                     _P, _P, _P, _SZ, _P, _S]),
    "gs_project_bwd_adam": (C.c_int, [_P, _P, _P, _I64, _I32, _P, _I32, C.POINTER(gs_raster_config), _P, _P,
                                      C.POINTER(gs_adam_config), _P, _P, _P, _P, _S]),
    "gs_adam_step": (C.c_int, [_P, _P, _P, _P, _I64, _I32, C.POINTER(gs_adam_config), _P, _P, _I32, _P, _S]),
    "gs_log_step": (C.c_int, [_P, _I32, _P, _P, _P, _P, _P, _P, _I64, _S]),
    "skipgs_gate_state_size": (C.c_size_t, [_I32]),
    "skipgs_gate_init": (C.c_int, [C.POINTER(gs_gate_config), _P, _S]),
    "skipgs_gate_decide": (C.c_int, [_P, _P, _P, _I32, _P, _P, C.POINTER(C.c_uint64), _P, _S]),
    "skipgs_gate_update": (C.c_int, [_P, _P, _P, _I32, _S]),
    "skipgs_gate_read": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_double), _S]),
    "gs_graph_begin": (C.c_int, [_S]),
    "gs_graph_cond_create": (C.c_int, [_S, C.POINTER(C.c_uint64)]),
    "gs_graph_if_begin": (C.c_int, [_S, C.c_uint64, _S]),
    "gs_graph_if_end": (C.c_int, [_S, _S]),
    "gs_graph_end": (C.c_int, [_S, C.POINTER(C.c_void_p)]),
    "gs_graph_launch": (C.c_int, [C.c_void_p, _S]),
    "gs_graph_kernel_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "gs_graph_destroy": (C.c_int, [C.c_void_p]),
    "gs_select_views": (C.c_int, [_P, _I64, _P, _I32, _P, _P, _P, _I32, _S]),
    "gs_view_steps": (C.c_int, [_P, _I32, _I32, _P, _P, _S]),
    "gs_raster_census": (C.c_int, [C.POINTER(gs_projected), _I64, _P, _P, _P, _I32, _I64, C.POINTER(gs_raster_config),
                                   _P, _P, _S]),
    "gs_atomic_probe": (C.c_int, [_P, _I64, _I64, _S]),
    "gs_densify_accumulate": (C.c_int, [_P, _P, _I64, _I32, _P, _P, _P, _S]),
    "gs_autotune_workspace_size": (C.c_size_t, [_I64, _I32, C.POINTER(gs_camera), _I32, _I64,
                                                C.POINTER(gs_launch_shape), _I32]),
    "gs_autotune": (C.c_int, [C.POINTER(gs_params), C.POINTER(gs_camera), _I32, _P, C.POINTER(gs_raster_config), _F32,
                              C.POINTER(gs_launch_shape), _I32, _I32, _I64, _P, _SZ, C.POINTER(C.c_float),
                              C.POINTER(C.c_int32), _S]),
    "gs_densify_workspace_size": (C.c_size_t, [_I64]),
    "gs_densify_decide": (C.c_int, [_P, _I64, _I32, _P, _P, C.POINTER(gs_densify_config), _P, _P, _P, _SZ, _S]),
    "gs_densify_apply": (C.c_int, [_P, _P, _P, _I64, _I32, _P, _P, _P, C.POINTER(gs_densify_config), _P, _P, _P,
                                   _I64, _P, _S]),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded libgsr.  Raises if it was not built (no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgsr.so not found at {LIB_PATH}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_PROTOS)


def status_string(code: int) -> str:
    return lib().gs_status_string(int(code)).decode()


def check(fn: str, code: int) -> None:
    if code != GS_OK:
        raise GsError(fn, code)


def ptr(t) -> C.c_void_p | None:
    """Device (or host) address of a tensor, or None."""
    if t is None:
        return None
    if isinstance(t, int):
        return C.c_void_p(t)
    return C.c_void_p(t.data_ptr())


def stream_handle(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def call(name: str, *args) -> int:
    """Calls a status-returning entry point and raises on failure."""
    code = getattr(lib(), name)(*args)
    check(name, code)
    return code
