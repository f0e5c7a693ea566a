"""The super-tile list form (gs_bin_sort_coarse and the *_coarse compositing
calls) against the FP64 oracle and against the tile-list form.

* Lists, bit-exact: every super-tile's list filtered by a tile's mask bit (on
  the host) equals the oracle's depth-ordered list of that tile; each mask is
  the exact set of the super-tile's tiles that the entry's rectangle covers
  (never empty); ranges and the pair count equal the oracle's; the views'
  first super-tiles, the counts and the total follow the stated layout.
* Forward: image, final transmittance, last-contributor counts and
  checkpoints bit-identical to the tile-list form on the same records, and
  the pixels against the oracle at the bar of test_gpu_raster.
* Adjoint: 2D gradients equal to the tile-list form's up to the order of
  float atomics (1e-6 normwise) and to the oracle's at the gradient bar
  (1e-4 normwise, cosine >= 0.9999); the fused backward + Adam likewise.
* Edge cases: tiles of 8, 16 and 32, batches of 64 to 256, several views of
  ragged sizes, partial super-tiles at the grid's edges, a persistent grid,
  list capacity one short (GS_ERR_CAPACITY, ranges empty), all culled.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2603_08997_gb300 import gsr, raster
from tests import gpu_util

pytestmark = pytest.mark.gpu

SIZES = [(150, 97), (64, 40), (41, 70)]


def _renderer(cams, n, coarse, tile=16, batch=256, ppt=2, persistent=False, ccap=None, cap=None):
    gpu_util.lib()
    st = raster.RasterSettings(tile=tile, batch=batch, pixels_per_thread=ppt, pixels_per_thread_fwd=ppt,
                               persistent=persistent, coarse_lists=coarse)
    return raster.Renderer(n, 0, raster.Views(cams, tile), st, pair_capacity=cap, coarse_capacity=ccap)


def _case(nviews, n, seed, tile):
    sizes = SIZES[:nviews]
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    recs = [synth.projected_records(n, w, h, seed=seed + v) for v, (w, h) in enumerate(sizes)]
    dev, orc = gpu_util.records(recs, cams, tile)
    return sizes, cams, dev, orc


def _host_lists(r, cams, tile):
    """tile id -> the tile's Gaussian indices, filtered on the host from the
    super-tile lists (checking the layout and every mask on the way)."""
    total = int(r.c_total.item())
    gid = r.c_gid[:total].cpu().numpy().view(np.uint32)
    mask = r.c_mask[:total].cpu().numpy().view(np.uint16).astype(np.int64)
    start = r.c_start.cpu().numpy().view(np.uint32).astype(np.int64)
    count = r.c_count.cpu().numpy().view(np.uint32).astype(np.int64)
    vf = r.c_view_first.cpu().numpy()
    assert vf[0] == 0 and count.sum() == total
    lists, toff = {}, 0
    for v, cam in enumerate(cams):
        tx, ty = -(-cam.width // tile), -(-cam.height // tile)
        stx, sty = -(-tx // 4), -(-ty // 4)
        assert vf[v + 1] - vf[v] == stx * sty
        for sy in range(sty):
            for sx in range(stx):
                ct = vf[v] + sy * stx + sx
                seg = slice(start[ct], start[ct] + count[ct])
                g, m = gid[seg], mask[seg]
                assert np.all(m != 0)
                for k in range(16):
                    x, y = sx * 4 + k % 4, sy * 4 + k // 4
                    if x < tx and y < ty:
                        lists[toff + y * tx + x] = g[(m >> k) & 1 == 1]
                    else:
                        assert not np.any((m >> k) & 1)
                _check_masks(v, sx, sy, g, m, r._orc[v]["rect"])
        toff += tx * ty
    assert np.all(count[vf[len(cams)]:] == 0)
    return lists


def _check_masks(v, sx, sy, g, m, rect):
    """Each entry's mask = the tiles of super-tile (sx, sy) inside its rectangle."""
    x0, y0, x1, y1 = (rect[g, i].astype(np.int64) for i in range(4))
    want = np.zeros(len(g), np.int64)
    for k in range(16):
        x, y = sx * 4 + k % 4, sy * 4 + k // 4
        want |= ((x >= x0) & (x <= x1) & (y >= y0) & (y <= y1)).astype(np.int64) << k
    assert np.array_equal(m, want), (v, sx, sy)


@pytest.mark.parametrize("tile,nviews", [(8, 3), (16, 1), (16, 3), (32, 2)])
def test_super_tile_lists_bit_exact(tile, nviews):
    sizes, cams, dev, orc = _case(nviews, 3000, 101, tile)
    r = _renderer(cams, 3000, True, tile=tile)
    r._orc = orc
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    _, ovals, oranges, _ = oracle.bin_sort(orc, cams, tile)
    assert int(r.pair_count.item()) == len(ovals)
    assert np.array_equal(r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2), oranges)
    lists = _host_lists(r, cams, tile)
    assert len(lists) == r.views.total_tiles
    for t, g in lists.items():
        assert np.array_equal(g, ovals[oranges[t, 0]:oranges[t, 1]]), t


def test_super_tile_lists_dense_large():
    """A dense 700 x 560 view at tile 8 (4,900 tiles; long lists, several
    gather rounds per batch)."""
    cams = [synth.camera_pinhole(50, 50, 350, 280, 700, 560)]
    recs = [synth.projected_records(20000, 700, 560, seed=5)]
    dev, orc = gpu_util.records(recs, cams, 8)
    r = _renderer(cams, 20000, True, tile=8, cap=64 * 20000)
    r._orc = orc
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    _, ovals, oranges, _ = oracle.bin_sort(orc, cams, 8)
    for t, g in _host_lists(r, cams, 8).items():
        assert np.array_equal(g, ovals[oranges[t, 0]:oranges[t, 1]]), t


def _render_both(cams, dev, tile, batch, ppt, persistent=False, dl=None):
    out = []
    for coarse in (False, True):
        r = _renderer(cams, dev["touched"].numel() // len(cams), coarse, tile=tile, batch=batch, ppt=ppt,
                      persistent=persistent)
        gpu_util.set_projected(r, dev)
        r.ckpt.fill_(-1.0)
        r.bin_sort()
        r.render_fwd()
        g2d = r.raster_bwd(dL_dimage=dl).clone() if dl is not None else None
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        out.append(([t.clone().cpu() for t in (r.image, r.T_final, r.n_last, r.ckpt)], g2d, r))
    return out


@pytest.mark.parametrize("tile,batch,ppt,persistent", [(16, 256, 1, False), (16, 256, 2, True), (8, 64, 2, False),
                                                       (32, 128, 1, False), (8, 256, 1, True), (32, 64, 4, False)])
def test_forward_and_adjoint_equal_tile_lists(tile, batch, ppt, persistent):
    sizes, cams, dev, _ = _case(3, 4000, 211, tile)
    dl = torch.from_numpy(np.concatenate([synth.dl_dimage(w, h, seed=9 + v).ravel()
                                          for v, (w, h) in enumerate(sizes)])).cuda()
    (fa, ga, _), (fb, gb, _) = _render_both(cams, dev, tile, batch, ppt, persistent, dl)
    for a, b in zip(fa, fb):
        assert torch.equal(a, b)
    assert gpu_util.rel_err(gb.double().cpu().numpy(), ga.double().cpu().numpy()) < 1e-6


@pytest.mark.parametrize("tile,ppt", [(16, 2), (8, 1), (32, 2)])
def test_against_oracle(tile, ppt):
    """Pixels, last-contributor counts and 2D gradients of the super-tile form
    against the oracle on shared records."""
    sizes, cams, dev, orc = _case(2, 3000, 301, tile)
    dls = [synth.dl_dimage(w, h, seed=15 + v) for v, (w, h) in enumerate(sizes)]
    dl = torch.from_numpy(np.concatenate([d.ravel() for d in dls])).cuda()
    r = _renderer(cams, 3000, True, tile=tile, ppt=ppt)
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    r.render_fwd()
    g2d = r.raster_bwd(dL_dimage=dl).double().cpu().numpy()
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    rc = oracle.RasterConfig(tile=tile)
    _, ovals, oranges, toff = oracle.bin_sort(orc, cams, tile)
    from tests.test_gpu_raster import _compare_images
    for v, (cam, (w, h)) in enumerate(zip(cams, sizes)):
        o = oracle.render(orc[v], cam, ovals, oranges, rc, int(toff[v]))
        _compare_images(r.image_of(v).cpu().numpy(), o["image"], o["margin"])
        off = r.views.pix_offsets[v]
        nl = r.n_last[off:off + w * h].view(h, w).cpu().numpy()
        assert ((nl == o["n_last"]) | o["margin"].astype(bool)).all()
        og = oracle.raster_bwd(orc[v], cam, ovals, oranges, rc, dls[v].astype(np.float64), int(toff[v]))
        for sl in (slice(0, 2), slice(2, 5), slice(5, 6), slice(6, 9)):
            assert gpu_util.rel_err(g2d[v][:, sl], og[:, sl]) < 1e-4
            assert gpu_util.cosine(g2d[v][:, sl], og[:, sl]) > 0.9999


def test_fused_backward_adam_equals_tile_lists():
    """gs_render_bwd_adam_coarse against gs_render_bwd_adam: parameters and
    moments after one step equal up to the order of float atomics."""
    scene, cam = synth.scene_tiny(400, seed=12, sh_degree=3)
    dl = torch.from_numpy(synth.dl_dimage(cam.width, cam.height, 4).ravel()).cuda()
    res = []
    for coarse in (False, True):
        gpu_util.lib()
        st = raster.RasterSettings(coarse_lists=coarse)
        r = raster.Renderer(scene.n, 3, raster.Views([cam], 16), st)
        model = raster.GaussianModel.from_scene(scene)
        adam = raster.AdamState(model)
        r.forward(model.c_params())
        r.backward_adam(model, adam, dL_dimage=dl)
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        res.append([t.clone().cpu().double().numpy() for t in (model.flat, adam.m, adam.v)])
    for a, b in zip(*res):
        assert gpu_util.rel_err(b, a) < 1e-6


def test_capacity_one_short_and_all_culled():
    sizes, cams, dev, orc = _case(1, 800, 401, 16)
    r0 = _renderer(cams, 800, True)
    gpu_util.set_projected(r0, dev)
    r0.bin_sort()
    torch.cuda.synchronize()
    need = int(r0.c_total.item())
    assert need > 0 and int(r0.status.item()) == 0
    r = _renderer(cams, 800, True, ccap=need - 1)
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    torch.cuda.synchronize()
    assert int(r.status.item()) == gsr.GS_ERR_CAPACITY
    assert int(r.c_total.item()) == need
    assert int(r.ranges.abs().sum().item()) == 0
    # all culled: no entries, empty ranges, a black image, clean status
    r2 = _renderer(cams, 800, True)
    dev["touched"].zero_()
    gpu_util.set_projected(r2, dev)
    r2.bin_sort()
    r2.render_fwd()
    torch.cuda.synchronize()
    assert int(r2.status.item()) == 0 and int(r2.c_total.item()) == 0 and int(r2.pair_count.item()) == 0
    assert float(r2.image.abs().max().item()) == 0.0


def test_loop_equals_tile_lists():
    """The refinement loop (graph replay, gated) with the super-tile form:
    per-iteration losses equal the tile-list loop's up to the float-atomic
    order of the gradients (1e-5 relative), and so do the gate's decisions
    here (no loss of this run lies that close to the EMA)."""
    from paper_2603_08997_gb300.refine import RefinementLoop
    gpu_util.lib()
    scene, _, _ = synth.case_c1(n=1500)
    cams = [synth.camera_pinhole(64.0, 64.0, 32.0, 32.0, 64, 64) for _ in range(3)]
    for k, c in enumerate(cams):  # three poses: small rotations about y
        a = 0.05 * k
        c.R = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]], np.float32)
    rng = np.random.default_rng(9)
    tg = torch.from_numpy(rng.uniform(0, 1, (3, 3, 64, 64)).astype(np.float32)).cuda()
    seq = rng.integers(0, 3, size=40).astype(np.int32)
    logs = []
    for coarse in (False, True):
        model = raster.GaussianModel.from_scene(scene)
        st = raster.RasterSettings(coarse_lists=coarse)
        loop = RefinementLoop(model, cams, tg, seq, st, gated=True, W=6, log_capacity=40)
        loop.capture()
        for _ in range(40):
            loop.step_graph()
        torch.cuda.synchronize()
        assert int(loop.renderer.status.item()) == 0
        logs.append(loop.read_log(40))
        loop.close()
    np.testing.assert_allclose(logs[1]["loss"], logs[0]["loss"], rtol=1e-5)
    assert np.array_equal(logs[0]["g"], logs[1]["g"])


def test_super_tile_bound_too_small_is_an_error():
    """A view with more super-tiles than max_view_super_tiles: GS_ERR_INVALID_ARG
    in the status word and no entries or ranges for it; the exact bound works."""
    import ctypes as C
    sizes, cams, dev, _ = _case(1, 2000, 501, 16)
    r = _renderer(cams, 2000, True)
    gpu_util.set_projected(r, dev)
    exact = r.views.max_view_super_tiles
    for bound, want in ((exact, 0), (exact - 1, gsr.GS_ERR_INVALID_ARG)):
        r.status.zero_()
        r.ranges.fill_(7)
        proj = r.c_proj()
        gsr.call("gs_bin_sort_coarse", C.byref(proj), gsr.ptr(r.views.dev), r.views.n, r.n, r.views.total_tiles,
                 r.views.max_view_tiles, bound, C.byref(r.cfg), gsr.ptr(r.bin_ws), r.bin_ws_bytes,
                 C.byref(r.lists), r.cap, gsr.ptr(r.ranges), gsr.ptr(r.pair_count), gsr.ptr(r.status),
                 gsr.stream_handle())
        torch.cuda.synchronize()
        assert int(r.status.item()) == want
        if want:
            assert int(r.ranges.abs().sum().item()) == 0 and int(r.c_total.item()) == 0
        else:
            assert int(r.c_total.item()) > 0 and int(r.ranges.abs().sum().item()) > 0


@pytest.mark.parametrize("depths", ["equal", "wide", "one_visible"])
def test_depth_order_across_key_ranges(depths):
    """The depth sort works on keys relative to the visible keys' range and
    copies the passes above its bit length: all depths equal (every pass a
    copy: ties in index order), depths spanning 0.2..1e5 (no pass copied),
    and a single visible Gaussian.  Tile lists (both forms) bit-exact
    against the oracle's binning."""
    sizes = [(150, 97), (64, 40)]
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    recs = [synth.projected_records(3000, w, h, seed=601 + v) for v, (w, h) in enumerate(sizes)]
    rng = np.random.default_rng(7)
    for r in recs:
        if depths == "equal":
            r["depth"][:] = np.float32(3.5)
        elif depths == "wide":
            r["depth"][:] = np.exp(rng.uniform(np.log(0.2), np.log(1e5), r["depth"].shape)).astype(np.float32)
        else:
            r["culled"][:] = True
            r["culled"][17] = False
    dev, orc = gpu_util.records(recs, cams, 16)
    _, ovals, oranges, _ = oracle.bin_sort(orc, cams, 16)
    for coarse in (False, True):
        r = _renderer(cams, 3000, coarse)
        r._orc = orc
        gpu_util.set_projected(r, dev)
        r.bin_sort()
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        assert int(r.pair_count.item()) == len(ovals)
        assert np.array_equal(r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2), oranges)
        if coarse:
            for t, g in _host_lists(r, cams, 16).items():
                assert np.array_equal(g, ovals[oranges[t, 0]:oranges[t, 1]]), t
        else:
            P = int(r.pair_count.item())
            assert np.array_equal(r.vals[:P].cpu().numpy().view(np.uint32), ovals)


@pytest.mark.parametrize("depths", ["equal", "typical", "wide", "one_visible"])
def test_projected_single_view_depth_order(depths):
    """One view through gs_project's depth keys and packed rectangles, where
    the depth sort's last pass writes the depth order and the rectangles
    itself: the super-tile lists hold, tile for tile, the tile lists of the
    same projection (whose binning is bit-exact against the oracle's), and
    the images are equal, for key ranges of 0 bits (all depths equal), about
    23 bits (last pass the third), 28 bits (all four passes) and a single
    visible Gaussian."""
    depth = {"equal": (3.5, 3.5), "typical": (2.0, 4.0), "wide": (0.3, 1e5), "one_visible": (2.0, 4.0)}[depths]
    scene, cam = synth.scene_tiny(3000, seed=31, width=160, height=96, sh_degree=0, depth=depth)
    if depths == "one_visible":
        scene.means[1:, 2] = -1.0  # behind the camera: culled
    out = []
    for coarse in (False, True):
        gpu_util.lib()
        r = raster.Renderer(scene.n, 0, raster.Views([cam], 16), raster.RasterSettings(coarse_lists=coarse))
        r.forward(raster.GaussianModel.from_scene(scene).c_params())
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        out.append(r)
    rt, rc = out
    P = int(rt.pair_count.item())
    assert int(rc.pair_count.item()) == P
    if depths == "one_visible":
        assert 0 < P <= 4
    rg = rt.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert np.array_equal(rc.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2), rg)
    tv = rt.vals[:P].cpu().numpy().view(np.uint32)
    rc._orc = [{"rect": rc.rect.cpu().numpy().reshape(-1, 4)}]  # masks checked against the projection's rectangles
    lists = _host_lists(rc, [cam], 16)
    assert len(lists) == rt.views.total_tiles
    for t, g in lists.items():
        assert np.array_equal(g, tv[rg[t, 0]:rg[t, 1]]), t
    assert torch.equal(rc.image, rt.image)



@pytest.mark.parametrize("coarse,ppt", [(True, 2), (False, 2), (True, 1), (False, 4)])
def test_needles_against_oracle(coarse, ppt):
    """Long thin rotated footprints (aspect 15 to 40, long-axis sigma 4 to 14
    px): their support boxes cover many warp pixel blocks that their support
    ellipses miss, which the compositing kernels do not visit.  Pixels,
    last-contributor counts and 2D gradients against the oracle, both list
    forms."""
    w, h = 160, 120
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h)]
    rec = synth.projected_records(700, w, h, seed=77, sigma_range=(4.0, 14.0), aniso=(15.0, 40.0))
    # the case does what it is for: most (record, 8 x 8 block) pairs that a
    # box reaches lie outside the record's ellipse at 3 sigma
    c, s = np.cos(rec["theta"]), np.sin(rec["theta"])
    ex = 3 * np.sqrt((rec["sigma1"] * c) ** 2 + (rec["sigma2"] * s) ** 2)
    ey = 3 * np.sqrt((rec["sigma1"] * s) ** 2 + (rec["sigma2"] * c) ** 2)
    assert np.median(4 * ex * ey / (9 * np.pi * rec["sigma1"] * rec["sigma2"])) > 3.0  # box area / ellipse area
    dev, orc = gpu_util.records([rec], cams, 16)
    dl = synth.dl_dimage(w, h, seed=5)
    r = _renderer(cams, 700, coarse, tile=16, ppt=ppt)
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    r.render_fwd()
    g2d = r.raster_bwd(dL_dimage=torch.from_numpy(dl.ravel()).cuda()).double().cpu().numpy()[0]
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    rc = oracle.RasterConfig(tile=16)
    _, ovals, oranges, toff = oracle.bin_sort(orc, cams, 16)
    from tests.test_gpu_raster import _compare_images
    o = oracle.render(orc[0], cams[0], ovals, oranges, rc, 0)
    _compare_images(r.image_of(0).cpu().numpy(), o["image"], o["margin"])
    nl = r.n_last[:w * h].view(h, w).cpu().numpy()
    assert ((nl == o["n_last"]) | o["margin"].astype(bool)).all()
    og = oracle.raster_bwd(orc[0], cams[0], ovals, oranges, rc, dl.astype(np.float64), 0)
    for sl in (slice(0, 2), slice(2, 5), slice(5, 6), slice(6, 9)):
        assert gpu_util.rel_err(g2d[:, sl], og[:, sl]) < 1e-4
        assert gpu_util.cosine(g2d[:, sl], og[:, sl]) > 0.9999
