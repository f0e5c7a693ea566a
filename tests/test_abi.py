"""The C-ABI library builds for sm_103a, loads on the host and exports every
entry point include/gsr.h declares; host-side argument checks reject bad
input without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b((?:gs|skipgs)_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_08997_gb300 import build, gsr
    build.build()
    return gsr.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gs_project", "gs_bin_sort", "gs_render_fwd", "gs_render_bwd", "gs_loss", "gs_adam_step",
                     "skipgs_gate_decide", "skipgs_gate_update"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2603_08997_gb300 import gsr
    assert set(declared_functions()) <= set(gsr.exported_symbols())


def test_host_side_checks(lib):
    from paper_2603_08997_gb300 import gsr
    assert lib.gs_version() >= 100
    assert gsr.status_string(gsr.GS_ERR_CAPACITY) == "GS_ERR_CAPACITY"
    out = (C.c_int64 * 6)()
    assert lib.gs_param_layout(10, 3, out) == 0
    assert [out[i] % 64 for i in range(6)] == [0] * 6 and out[5] >= 59 * 10
    assert lib.gs_param_layout(10, 4, out) == gsr.GS_ERR_INVALID_ARG
    cams = (gsr.gs_camera * 2)()
    cams[0].width, cams[0].height, cams[1].width, cams[1].height = 33, 17, 16, 16
    tt, tp = C.c_int64(), C.c_int64()
    assert lib.gs_camera_layout(cams, 2, 16, C.byref(tt), C.byref(tp)) == 0
    assert (tt.value, tp.value) == (3 * 2 + 1, 33 * 17 + 256)
    assert cams[1].tile_offset == 6 and cams[1].pix_offset == 33 * 17
    assert lib.gs_camera_layout(cams, 2, 12, C.byref(tt), C.byref(tp)) == gsr.GS_ERR_INVALID_ARG
    # invalid arguments are refused before any launch
    assert lib.gs_project(None, None, 1, None, gsr.gs_projected(), None, None) == gsr.GS_ERR_INVALID_ARG
    assert lib.skipgs_gate_decide(None, None, None, 1, None, None, None, None, None) == gsr.GS_ERR_INVALID_ARG
    assert lib.gs_ckpt_slots(1000, 10, 256) == 1000 // 256 + 10 + 1
    assert lib.skipgs_gate_state_size(200) >= 200 * 9
    cfg = gsr.gs_gate_config()
    cfg.W, cfg.beta, cfg.eps, cfg.rho_lo, cfg.n_views = 10, 1.5, 1e-8, 0.5, 4
    assert lib.skipgs_gate_init(C.byref(cfg), C.c_void_p(16), None) == gsr.GS_ERR_INVALID_ARG


def test_fused_adjoint_adam_argument_checks(lib):
    """gs_project_bwd_adam refuses bad arguments before any launch: missing
    buffers, unaligned moments, degree mismatch, beta outside [0, 1)."""
    from paper_2603_08997_gb300 import gsr
    rc = gsr.gs_raster_config()
    rc.sh_degree = 3
    ac = gsr.gs_adam_config()
    ac.beta1, ac.beta2, ac.eps = 0.9, 0.999, 1e-15
    P = C.c_void_p
    fn = lib.gs_project_bwd_adam

    def call(flat=256, m=512, v=768, deg=3, cfg=rc, adam=ac, step=1024, g2d=2048):
        return fn(P(flat) if flat else None, P(m) if m else None, P(v), 100, deg, P(4096), 1, C.byref(cfg), P(g2d),
                  None, C.byref(adam), None, P(step) if step else None, None, None, None)

    assert call(flat=0) == gsr.GS_ERR_INVALID_ARG
    assert call(m=0) == gsr.GS_ERR_INVALID_ARG
    assert call(step=0) == gsr.GS_ERR_INVALID_ARG
    assert call(m=520) == gsr.GS_ERR_INVALID_ARG      # moments not 16-byte aligned
    assert call(g2d=2052) == gsr.GS_ERR_INVALID_ARG   # 2D gradients not 16-byte aligned
    assert call(deg=2) == gsr.GS_ERR_INVALID_ARG      # degree differs from the raster config
    bad = gsr.gs_adam_config()
    bad.beta1, bad.beta2, bad.eps = 0.9, 1.0, 1e-15
    assert call(adam=bad) == gsr.GS_ERR_INVALID_ARG


def test_workspace_too_small_is_refused(lib):
    from paper_2603_08997_gb300 import gsr
    proj = gsr.gs_projected(16, 16, 16)
    rc = gsr.gs_raster_config()
    rc.tile, rc.batch = 16, 256
    need = lib.gs_bin_sort_workspace_size(100, 1, 1000, 4)
    code = lib.gs_bin_sort(C.byref(proj), C.c_void_p(256), 1, 100, 4, 4, C.byref(rc), C.c_void_p(256), need - 1,
                           None, C.c_void_p(256), 1000, C.c_void_p(256), C.c_void_p(256), None, None)
    assert code == gsr.GS_ERR_WORKSPACE


def test_autotune_host_checks(lib):
    """gs_autotune sizes its workspace for the largest valid candidate and
    refuses a missing or short workspace, and mismatched arguments, before
    any launch."""
    from paper_2603_08997_gb300 import gsr
    cams = (gsr.gs_camera * 2)()
    cams[0].width, cams[0].height, cams[1].width, cams[1].height = 130, 70, 64, 64
    shapes = (gsr.gs_launch_shape * 3)(gsr.gs_launch_shape(8, 64, 1, 2), gsr.gs_launch_shape(32, 256, 2, 2),
                                      gsr.gs_launch_shape(12, 64, 1, 1))  # the last is not a valid shape
    big = lib.gs_autotune_workspace_size(1000, 3, cams, 2, 50000, shapes, 3)
    small = lib.gs_autotune_workspace_size(1000, 3, cams, 2, 50000, shapes, 1)
    only_invalid = lib.gs_autotune_workspace_size(1000, 3, cams, 2, 50000, C.byref(shapes[2]), 1)
    assert big >= small > 0 and only_invalid == 0
    assert lib.gs_autotune_workspace_size(1000, 4, cams, 2, 50000, shapes, 3) == 0
    assert cams[1].tile_offset == 0  # the caller's cameras are not modified
    p = gsr.gs_params()
    p.n, p.sh_degree = 1000, 3
    rc = gsr.gs_raster_config()
    rc.sh_degree = 3
    ms = (C.c_float * 3)()
    best = C.c_int32()
    args = (C.byref(p), cams, 2, C.c_void_p(256), C.byref(rc), 0.2, shapes, 3, 2, 50000)
    assert lib.gs_autotune(*args, None, big, ms, C.byref(best), None) == gsr.GS_ERR_WORKSPACE
    assert lib.gs_autotune(*args, C.c_void_p(1 << 20), big - 1, ms, C.byref(best), None) == gsr.GS_ERR_WORKSPACE
    rc.sh_degree = 2
    assert lib.gs_autotune(*args, C.c_void_p(1 << 20), big, ms, C.byref(best), None) == gsr.GS_ERR_INVALID_ARG


def test_super_tile_form_host_checks(lib):
    """The super-tile calls reject missing or misaligned list buffers, an
    oversized list capacity, a negative super-tile bound and a missing
    batch_pos before any launch; their workspace is smaller than the
    tile-list form's."""
    from paper_2603_08997_gb300 import gsr
    n, V, T = 100000, 2, 4000
    small = lib.gs_bin_sort_coarse_workspace_size(n, V, T)
    assert 0 < small < lib.gs_bin_sort_workspace_size(n, V, 24 * n, T)
    assert lib.gs_bin_sort_coarse_workspace_size(-1, V, T) == 0
    dev = C.c_void_p(1 << 20)  # a stand-in device address: every call below returns before using it
    proj = gsr.gs_projected(dev.value, dev.value, dev.value, None, None)
    cfg = gsr.gs_raster_config()
    cfg.tile, cfg.batch, cfg.pixels_per_thread = 16, 256, 2

    def lists(mask=1 << 20, cap=1000):
        return gsr.gs_coarse_lists(dev.value, mask, dev.value, dev.value, dev.value, dev.value, cap)

    def bin_call(lst, bound=0):
        return lib.gs_bin_sort_coarse(C.byref(proj), dev, V, n, T, 0, bound, C.byref(cfg), dev, 1 << 30,
                                      C.byref(lst) if lst is not None else None, 24 * n, dev, dev, dev, None)
    assert bin_call(None) == gsr.GS_ERR_INVALID_ARG
    assert bin_call(lists(mask=(1 << 20) + 2)) == gsr.GS_ERR_INVALID_ARG       # masks not 16-byte aligned
    assert bin_call(lists(cap=(1 << 32) - 1)) == gsr.GS_ERR_INVALID_ARG        # capacity above 2^32 - 65536
    assert bin_call(lists(), bound=-1) == gsr.GS_ERR_INVALID_ARG
    saved = gsr.gs_fwd_saved(dev.value, dev.value, dev.value, 100, None, None, None)  # no batch_pos
    assert lib.gs_render_fwd_coarse(C.byref(proj), n, C.byref(lists()), dev, dev, V, T, C.byref(cfg), dev, saved,
                                    None, None) == gsr.GS_ERR_INVALID_ARG
    saved.batch_pos = dev.value
    assert lib.gs_render_fwd_coarse(C.byref(proj), n, None, dev, dev, V, T, C.byref(cfg), dev, saved, None,
                                    None) == gsr.GS_ERR_INVALID_ARG
    assert lib.gs_raster_bwd_coarse(C.byref(proj), n, None, dev, dev, V, T, C.byref(cfg), saved, dev, None, dev,
                                    1 << 30, None, None) == gsr.GS_ERR_INVALID_ARG


def test_param_structs_keep_their_tensors_alive():
    """gs_params / gs_grads hold raw device pointers: the structs returned by
    c_params and c_grads keep the model and the gradient buffer alive, so a
    temporary model's storage cannot be reused while its struct is passed
    on (CPU tensors; no kernel runs)."""
    import gc
    import weakref

    import torch

    import synth
    from paper_2603_08997_gb300 import raster
    scene, _ = synth.scene_tiny(8, seed=1)
    m = raster.GaussianModel.from_scene(scene, torch.device("cpu"))
    ref = weakref.ref(m)
    p = m.c_params()
    del m
    gc.collect()
    assert ref() is not None and p.means == ref().views["means"].data_ptr()
    del p
    gc.collect()
    assert ref() is None
    flat = torch.zeros(raster.GaussianModel.from_scene(scene, torch.device("cpu")).flat.numel())
    fref = weakref.ref(flat)
    g = raster.GaussianModel.from_scene(scene, torch.device("cpu")).c_grads(flat)
    del flat
    gc.collect()
    assert fref() is not None
    del g
    gc.collect()
    assert fref() is None
