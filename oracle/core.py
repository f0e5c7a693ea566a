"""ctypes wrapper of the FP64 C oracle (``gs_oracle.c``).

Test infrastructure only (see the package docstring).  Every function takes
and returns numpy arrays; inputs are widened exactly from float32 to float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Camera(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_double)]


class _Raster(C.Structure):
    _fields_ = [("lowpass", C.c_double), ("alpha_max", C.c_double), ("alpha_min", C.c_double),
                ("t_min", C.c_double), ("bg", C.c_double * 3), ("tile", C.c_int32)]


@dataclass
class RasterConfig:
    """Rasterizer constants.  The thresholds are the float32 values the CUDA
    path compares against, widened exactly, so both sides use the same numbers."""
    lowpass: float = float(np.float32(0.3))
    alpha_max: float = float(np.float32(0.99))
    alpha_min: float = float(np.float32(1.0) / np.float32(255.0))
    t_min: float = float(np.float32(1e-4))
    bg: tuple = (0.0, 0.0, 0.0)
    tile: int = 16

    def struct(self) -> _Raster:
        r = _Raster()
        r.lowpass, r.alpha_max, r.alpha_min, r.t_min = self.lowpass, self.alpha_max, self.alpha_min, self.t_min
        for i in range(3):
            r.bg[i] = float(self.bg[i])
        r.tile = int(self.tile)
        return r


_lib = None
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_sh_basis.argtypes = [C.c_int, _D, _D, _D]
        L.orc_project.argtypes = [C.c_int64, C.c_int, _D, _D, _D, _D, _D, C.POINTER(_Camera),
                                  C.POINTER(_Raster), _D, _D, _D, _D, _D, _D, _D, _I32, _I32, _I32]
        L.orc_bin_sort.argtypes = [C.c_int64, C.c_int, _I32, _U32, _I32, _I32, _I32, C.c_int64,
                                   _U64, _U32, _U32]
        L.orc_bin_sort.restype = C.c_int64
        L.orc_render.argtypes = [C.c_int, C.c_int, C.c_int32, _D, _D, _D, _D, _U32, _U32,
                                 C.POINTER(_Raster), C.c_double, _D, _D, _I32, _I32, _U8]
        L.orc_render.restype = C.c_uint64
        L.orc_render_brute.argtypes = [C.c_int, C.c_int, C.c_int64, _D, _D, _D, _D, _U32, _I32,
                                       C.POINTER(_Raster), _D, _D]
        L.orc_raster_bwd.argtypes = [C.c_int, C.c_int, C.c_int32, _D, _D, _D, _D, _U32, _U32,
                                     C.POINTER(_Raster), _D, _D]
        L.orc_project_bwd.argtypes = [C.c_int64, C.c_int, _D, _D, _D, _D, _D, C.POINTER(_Camera),
                                      C.POINTER(_Raster), _D, _D, _D, _D, _D, _D]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def camera_struct(cam) -> _Camera:
    c = _Camera()
    R = np.asarray(cam.R, np.float32).astype(np.float64).ravel()
    t = np.asarray(cam.t, np.float32).astype(np.float64).ravel()
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = t[i]
    c.fx, c.fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    c.cx, c.cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear = float(np.float32(cam.znear))
    return c


def tile_grid(cam, tile: int):
    return (int(cam.width) + tile - 1) // tile, (int(cam.height) + tile - 1) // tile


def _d(a):
    """float32 inputs widen exactly; float64 inputs (finite-difference probes) pass through."""
    return np.ascontiguousarray(a, dtype=np.float64)


def sh_basis(deg: int, d) -> tuple:
    """Real SH values Y[16] and their gradients dY[16,3] at direction d (x,y,z)."""
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    lib().orc_sh_basis(int(deg), np.ascontiguousarray(d, np.float64), Y, dY.ravel())
    return Y, dY


def project(scene, cam, rc: RasterConfig) -> dict:
    n, K = scene.n, scene.sh.shape[1]
    out = dict(mean2d=np.zeros((n, 2)), cov2d=np.zeros((n, 3)), conic=np.zeros((n, 3)),
               depth=np.zeros(n), rgb=np.zeros((n, 3)), opacity=np.zeros(n), radius=np.zeros((n, 2)),
               rect=np.zeros((n, 4), np.int32), touched=np.zeros(n, np.int32),
               flags=np.zeros(n, np.int32))
    cs, rs = camera_struct(cam), rc.struct()
    lib().orc_project(n, K, _d(scene.means), _d(scene.log_scales), _d(scene.quats),
                      _d(scene.opacity_logit), _d(scene.sh), C.byref(cs), C.byref(rs),
                      out["mean2d"], out["cov2d"], out["conic"], out["depth"], out["rgb"],
                      out["opacity"], out["radius"], out["rect"], out["touched"], out["flags"])
    # reading R3: the sort key uses the depth rounded to float32
    out["depth_bits"] = out["depth"].astype(np.float32).view(np.uint32).copy()
    return out


def bin_sort(projs: list, cams: list, tile: int):
    """Keys, values and per-tile ranges for one or more views (concatenated
    tile id space: view v's tiles start at the sum of the earlier views' tiles)."""
    n = int(projs[0]["touched"].shape[0])
    V = len(projs)
    grids = [tile_grid(c, tile) for c in cams]
    tiles_x = np.array([g[0] for g in grids], np.int32)
    counts = np.array([g[0] * g[1] for g in grids], np.int64)
    tile_offset = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int32)
    total = int(counts.sum())
    rect = np.ascontiguousarray(np.stack([p["rect"] for p in projs]), np.int32)
    dbits = np.ascontiguousarray(np.stack([p["depth_bits"] for p in projs]), np.uint32)
    touched = np.ascontiguousarray(np.stack([p["touched"] for p in projs]), np.int32)
    P = int(touched.astype(np.int64).sum())
    keys = np.zeros(max(P, 1), np.uint64)
    vals = np.zeros(max(P, 1), np.uint32)
    ranges = np.zeros(2 * total, np.uint32)
    got = lib().orc_bin_sort(n, V, rect.ravel(), dbits.ravel(), touched.ravel(), tile_offset, tiles_x,
                             total, keys, vals, ranges)
    assert got == P
    return keys[:P], vals[:P], ranges.reshape(total, 2), tile_offset


def render(proj: dict, cam, vals, ranges, rc: RasterConfig, tile_offset: int = 0,
           margin_rel: float = 1e-5) -> dict:
    W, H = int(cam.width), int(cam.height)
    out = dict(image=np.zeros((3, H, W)), T_final=np.zeros((H, W)), n_last=np.zeros((H, W), np.int32),
               n_contrib=np.zeros((H, W), np.int32), margin=np.zeros((H, W), np.uint8))
    rs = rc.struct()
    h = lib().orc_render(W, H, int(tile_offset), proj["mean2d"], proj["conic"], proj["rgb"], proj["opacity"],
                         np.ascontiguousarray(vals, np.uint32), np.ascontiguousarray(ranges, np.uint32).ravel(),
                         C.byref(rs), float(margin_rel), out["image"], out["T_final"], out["n_last"],
                         out["n_contrib"], out["margin"])
    out["hash"] = int(h)
    return out


def render_brute(proj: dict, cam, rc: RasterConfig) -> dict:
    W, H = int(cam.width), int(cam.height)
    n = int(proj["touched"].shape[0])
    out = dict(image=np.zeros((3, H, W)), T_final=np.zeros((H, W)))
    rs = rc.struct()
    lib().orc_render_brute(W, H, n, proj["mean2d"], proj["conic"], proj["rgb"], proj["opacity"],
                           proj["depth_bits"], proj["touched"], C.byref(rs), out["image"], out["T_final"])
    return out


def raster_bwd(proj: dict, cam, vals, ranges, rc: RasterConfig, dL_dimage, tile_offset: int = 0):
    """Per-Gaussian g2d[N,9]: dL/dmean2d(2), dL/dconic(a,b,c), dL/dopacity, dL/drgb(3)."""
    W, H = int(cam.width), int(cam.height)
    n = int(proj["touched"].shape[0])
    g2d = np.zeros((n, 9))
    rs = rc.struct()
    lib().orc_raster_bwd(W, H, int(tile_offset), proj["mean2d"], proj["conic"], proj["rgb"], proj["opacity"],
                         np.ascontiguousarray(vals, np.uint32), np.ascontiguousarray(ranges, np.uint32).ravel(),
                         C.byref(rs), np.ascontiguousarray(dL_dimage, np.float64), g2d)
    return g2d


def project_bwd(scene, cam, rc: RasterConfig, g2d, grads: dict | None = None) -> dict:
    n, K = scene.n, scene.sh.shape[1]
    if grads is None:
        grads = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                     opacity_logit=np.zeros(n), sh=np.zeros((n, K, 3)))
    cs, rs = camera_struct(cam), rc.struct()
    lib().orc_project_bwd(n, K, _d(scene.means), _d(scene.log_scales), _d(scene.quats),
                          _d(scene.opacity_logit), _d(scene.sh), C.byref(cs), C.byref(rs),
                          np.ascontiguousarray(g2d, np.float64), grads["means"], grads["log_scales"],
                          grads["quats"], grads["opacity_logit"], grads["sh"])
    return grads


def forward(scene, cam, rc: RasterConfig, margin_rel: float = 1e-5) -> dict:
    """project -> bin/sort -> tiled render for one view."""
    proj = project(scene, cam, rc)
    keys, vals, ranges, _ = bin_sort([proj], [cam], rc.tile)
    out = render(proj, cam, vals, ranges, rc, 0, margin_rel)
    out.update(proj=proj, keys=keys, vals=vals, ranges=ranges)
    return out


def backward(scene, cam, rc: RasterConfig, fwd: dict, dL_dimage, grads: dict | None = None) -> dict:
    g2d = raster_bwd(fwd["proj"], cam, fwd["vals"], fwd["ranges"], rc, dL_dimage)
    grads = project_bwd(scene, cam, rc, g2d, grads)
    grads["g2d"] = g2d
    return grads
