"""GPU projection, binning/sort and compositing against the FP64 oracle.

Tolerances: sort keys, values and tile ranges bit-exact given the same
stage inputs; pixels within 1e-5 relative (normwise over the image, and per
pixel against 1e-5 of the image's peak outside pixels the oracle flags as
within 1e-5 of a threshold); projected quantities within 1e-5 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2603_08997_gb300 import gsr, raster
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _renderer(cams, n, sh_degree=0, tile=16, batch=256, cap=None, keys=True, ppt=2, coarse=False):
    gpu_util.lib()
    views = raster.Views(cams, tile)
    st = raster.RasterSettings(tile=tile, batch=batch, pixels_per_thread=ppt, pixels_per_thread_fwd=ppt,
                               coarse_lists=coarse)
    return raster.Renderer(n, sh_degree, views, st, pair_capacity=cap, keep_keys=keys and not coarse)


def _sorted_pairs(r):
    P = int(r.pair_count.item())
    keys = r.keys[:P].cpu().numpy().view(np.uint64)
    vals = r.vals[:P].cpu().numpy().view(np.uint32)
    ranges = r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
    return P, keys, vals, ranges


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("nviews", [1, 3])
def test_bin_sort_bit_exact(tile, nviews):
    sizes = [(97, 61), (64, 64), (130, 33)][:nviews]
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    recs = [synth.projected_records(3000, w, h, seed=11 + v) for v, (w, h) in enumerate(sizes)]
    r = _renderer(cams, 3000, tile=tile)
    dev, orc = gpu_util.records(recs, cams, tile)
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    P, keys, vals, ranges = _sorted_pairs(r)
    okeys, ovals, oranges, _ = oracle.bin_sort(orc, cams, tile)
    assert P == len(okeys)
    assert np.array_equal(keys, okeys)
    assert np.array_equal(vals, ovals)
    assert np.array_equal(ranges, oranges)


@pytest.mark.parametrize("sizes,tile,n", [([(700, 560)], 8, 20000), ([(300, 200), (90, 300)], 16, 30000)])
def test_bin_sort_bit_exact_large(sizes, tile, n):
    """Larger tile grids (the 32-entry window path past about 4900 tiles per
    view) and dense scenes (many entries of one window on one tile, more than
    one window word)."""
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    recs = [synth.projected_records(n, w, h, seed=5 + v) for v, (w, h) in enumerate(sizes)]
    r = _renderer(cams, n, tile=tile, cap=64 * n)
    dev, orc = gpu_util.records(recs, cams, tile)
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    P, keys, vals, ranges = _sorted_pairs(r)
    okeys, ovals, oranges, _ = oracle.bin_sort(orc, cams, tile)
    assert P == len(okeys)
    assert np.array_equal(keys, okeys)
    assert np.array_equal(vals, ovals)
    assert np.array_equal(ranges, oranges)


def test_bin_sort_capacity_overflow_and_empty():
    cams = [synth.camera_pinhole(50, 50, 32, 32, 64, 64)]
    recs = [synth.projected_records(500, 64, 64, seed=2)]
    dev, orc = gpu_util.records(recs, cams, 16)
    need = int(sum(o["touched"].sum() for o in orc))
    r = _renderer(cams, 500, cap=need - 1)
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    torch.cuda.synchronize()
    assert int(r.status.item()) == gsr.GS_ERR_CAPACITY
    assert int(r.pair_count.item()) == need
    assert int(r.ranges.abs().sum().item()) == 0
    # all culled: no pairs, empty ranges, clean status
    r2 = _renderer(cams, 500)
    dev["touched"].zero_()
    gpu_util.set_projected(r2, dev)
    r2.bin_sort()
    r2.render_fwd()
    torch.cuda.synchronize()
    assert int(r2.pair_count.item()) == 0 and int(r2.status.item()) == 0
    assert float(r2.image.abs().max().item()) == 0.0


def _compare_images(img, ref, margin, tol=1e-5, cap=0.002, outliers=0.0):
    """Pixels against the oracle's:
    - normwise within tol relative, over all pixels and over the pixels the
      oracle does not flag as within its margin of a cut-off (alpha' near
      alpha_min or alpha_max, T (1 - alpha') near t_min);
    - per unflagged pixel within tol of the image's peak, except at most
      `outliers` of the pixels, which stay within 10 tol (end to end, the
      projection's float32 rounding of ill-conditioned footprints moves
      alphas by up to ~1e-4 relative; stage-wise, records are shared exactly
      and outliers = 0);
    - flagged pixels fewer than `cap` of the image.
    Returns (flagged, outlier) pixel counts."""
    img = np.asarray(img, np.float64)
    ref = np.asarray(ref, np.float64)
    flagged = margin.astype(bool)
    assert flagged.mean() < cap, (int(flagged.sum()), flagged.size)
    mask = flagged[None].repeat(3, 0)
    d = np.abs(img - ref)
    d[mask] = 0.0
    peak = np.abs(ref).max()
    over = d.max(0) > tol * peak
    assert over.mean() <= outliers, (int(over.sum()), d.max() / peak)
    assert d.max() <= 10 * tol * peak, (d.max(), peak)
    nd = np.linalg.norm(np.where(mask, 0.0, img - ref))
    assert nd <= tol * np.linalg.norm(ref), nd / np.linalg.norm(ref)
    assert np.linalg.norm(img - ref) <= tol * np.linalg.norm(ref), np.linalg.norm(img - ref) / np.linalg.norm(ref)
    return int(flagged.sum()), int(over.sum())


@pytest.mark.parametrize("tile,batch,ppt", [(16, 256, 2), (8, 64, 2), (32, 128, 2), (16, 128, 1), (8, 256, 1),
                                            (32, 64, 1)])
def test_render_synthetic_records(tile, batch, ppt):
    sizes = [(150, 97), (64, 40)]
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    recs = [synth.projected_records(4000, w, h, seed=21 + v) for v, (w, h) in enumerate(sizes)]
    r = _renderer(cams, 4000, tile=tile, batch=batch, ppt=ppt)
    dev, orc = gpu_util.records(recs, cams, tile)
    gpu_util.set_projected(r, dev)
    r.bin_sort()
    r.render_fwd()
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    rc = oracle.RasterConfig(tile=tile)
    _, ovals, oranges, toff = oracle.bin_sort(orc, cams, tile)
    for v, cam in enumerate(cams):
        o = oracle.render(orc[v], cam, ovals, oranges, rc, int(toff[v]))
        img = r.image_of(v).cpu().numpy()
        _compare_images(img, o["image"], o["margin"])
        off = r.views.pix_offsets[v]
        w, h = sizes[v]
        nl = r.n_last[off:off + w * h].view(h, w).cpu().numpy()
        agree = (nl == o["n_last"]) | o["margin"].astype(bool)
        assert agree.all()


@pytest.mark.parametrize("tile,ppt", [(8, 2), (16, 2), (32, 2), (16, 1)])
def test_render_end_to_end_c1(tile, ppt):
    scene, cam, _ = synth.case_c1()
    r = _renderer([cam], scene.n, tile=tile, ppt=ppt)
    model = raster.GaussianModel.from_scene(scene)
    r.forward(model.c_params())
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    # end to end, the projection's float32 rounding moves alphas by up to ~1e-4
    # relative for ill-conditioned footprints (test_projection_c2: conic error
    # below 1e-6 (1 + cond)): flag pixels within that of a cut-off
    o = oracle.forward(scene, cam, oracle.RasterConfig(tile=tile), margin_rel=1e-4)
    _compare_images(r.image_of(0).cpu().numpy(), o["image"], o["margin"], cap=0.01, outliers=1e-4)


def test_projection_c2():
    """Projection of the full C2 scene (200,000 Gaussians SH3, 980x545).
    The conic's float32 error grows with the condition number of Sigma2D (it
    is the inverse of a matrix rounded to float32): relative error at most
    1e-6 (1 + cond) for every footprint, and 1e-5 where cond <= 10.  Culling
    disagrees only where the oracle's wider rectangle inflation (x1.001 +
    0.01 px against x1.0001 + 0.001 px) keeps a Gaussian whose exact support
    reaches no pixel centre."""
    scene, _, cam, _ = synth.case_c2()
    r = _renderer([cam], scene.n, sh_degree=3)
    model = raster.GaussianModel.from_scene(scene)
    r.project(model.c_params())
    torch.cuda.synchronize()
    rec = r.records()[0].double().cpu().numpy()
    rect = r.rect.view(-1, 4).cpu().numpy()
    touched = r.touched.cpu().numpy()
    o = oracle.project(scene, cam, oracle.RasterConfig())
    vis = (o["touched"] > 0) & (touched > 0)
    r_ex = (o["radius"] - 0.01) / 1.001  # the oracle's exact support extents
    m = o["mean2d"]
    ex = np.stack([np.maximum(np.ceil(m[:, 0] - r_ex[:, 0] - 0.5), 0), np.maximum(np.ceil(m[:, 1] - r_ex[:, 1] - 0.5), 0),
                   np.minimum(np.floor(m[:, 0] + r_ex[:, 0] - 0.5), cam.width - 1),
                   np.minimum(np.floor(m[:, 1] + r_ex[:, 1] - 0.5), cam.height - 1)], 1)
    exact_empty = (ex[:, 0] > ex[:, 2]) | (ex[:, 1] > ex[:, 3])
    differ = (o["touched"] > 0) != (touched > 0)
    assert np.all(differ <= ((o["touched"] > 0) & exact_empty)), np.nonzero(differ & ~exact_empty)[0][:10]
    np.testing.assert_allclose(rec[vis, 0:2], o["mean2d"][vis], rtol=1e-6, atol=1e-4)
    np.testing.assert_allclose(rec[vis, 9], o["depth"][vis], rtol=1e-6)
    np.testing.assert_allclose(rec[vis, 5], o["opacity"][vis], rtol=1e-5)
    np.testing.assert_allclose(rec[vis, 6:9], o["rgb"][vis], rtol=1e-5, atol=1e-6)
    U = rec[vis, 2:5]
    Q = np.stack([U[:, 0] ** 2, U[:, 0] * U[:, 1], U[:, 1] ** 2 + U[:, 2] ** 2], 1)
    Qo = o["conic"][vis]
    err = np.linalg.norm(Q - Qo, axis=1) / np.linalg.norm(Qo, axis=1)
    cov = o["cov2d"][vis]
    tr, det = cov[:, 0] + cov[:, 2], cov[:, 0] * cov[:, 2] - cov[:, 1] ** 2
    disc = np.sqrt(np.maximum(tr * tr / 4 - det, 0.0))
    cond = (tr / 2 + disc) / (tr / 2 - disc)
    assert np.all(err <= 1e-6 * (1.0 + cond)), (err.max(), cond[np.argmax(err / (1 + cond))])
    well = cond <= 10.0
    assert well.mean() > 0.5 and err[well].max() <= 1e-5, err[well].max()
    # the GPU rectangle contains the exact support box
    gr = rect[vis]
    exv = ex[vis] // 16
    assert ((gr[:, 0] <= exv[:, 0]) & (gr[:, 1] <= exv[:, 1]) & (gr[:, 2] >= exv[:, 2]) & (gr[:, 3] >= exv[:, 3])).all()


@pytest.mark.parametrize("coarse", [False, True])
def test_render_end_to_end_c2(coarse):
    """The full C2 scene rendered end to end (tile lists and super-tile lists);
    flagged pixels (within 1e-4 of a cut-off, the projection's float32 reach)
    below 1% of the image, pixels beyond 1e-5 of the peak at most 0.01% (each
    within 1e-4)."""
    scene, _, cam, _ = synth.case_c2()
    r = _renderer([cam], scene.n, sh_degree=3, cap=24 * scene.n, coarse=coarse)
    model = raster.GaussianModel.from_scene(scene)
    r.forward(model.c_params())
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    o = oracle.forward(scene, cam, oracle.RasterConfig(), margin_rel=1e-4)
    _compare_images(r.image_of(0).cpu().numpy(), o["image"], o["margin"], cap=0.01, outliers=1e-4)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_pixels_per_thread_is_bit_invariant(tile):
    """The per-pixel arithmetic does not depend on how pixels map to threads:
    images, final transmittance, last-contributor counts and checkpoints are
    bit-identical for 1, 2 and (tiles of 16 or more) 4 pixels per thread."""
    sizes = [(150, 97), (41, 70)]
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    recs = [synth.projected_records(4000, w, h, seed=41 + v) for v, (w, h) in enumerate(sizes)]
    dev, _ = gpu_util.records(recs, cams, tile)
    out = []
    for ppt in ((1, 2) if tile < 16 else (1, 2, 4)):
        r = _renderer(cams, 4000, tile=tile, batch=64, ppt=ppt)
        gpu_util.set_projected(r, dev)
        r.ckpt.fill_(-1.0)
        r.bin_sort()
        r.render_fwd()
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        out.append([t.clone().cpu() for t in (r.image, r.T_final, r.n_last, r.ckpt)])
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert torch.equal(a, b)


def test_tile_order_is_a_permutation_by_work_and_changes_nothing():
    """gs_tile_order: a permutation of the tiles, list lengths non-increasing
    across the logarithmic groups; rendering in that order gives the same
    image, final transmittance, last-contributor counts and checkpoints."""
    sizes = [(150, 97), (64, 40)]
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    recs = [synth.projected_records(4000, w, h, seed=61 + v) for v, (w, h) in enumerate(sizes)]
    dev, _ = gpu_util.records(recs, cams, 8)
    out = []
    for ordered in (False, True):
        gpu_util.lib()
        views = raster.Views(cams, 8)
        st = raster.RasterSettings(tile=8, batch=64, longest_tiles_first=ordered)
        r = raster.Renderer(4000, 0, views, st)
        gpu_util.set_projected(r, dev)
        r.ckpt.fill_(-1.0)
        r.bin_sort()
        r.render_fwd()
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        out.append([t.clone().cpu() for t in (r.image, r.T_final, r.n_last, r.ckpt)])
        if ordered:
            order = r.tile_order.cpu().numpy().astype(np.int64)
            T = r.views.total_tiles
            assert np.array_equal(np.sort(order), np.arange(T))
            rg = r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
            length = (rg[:, 1] - rg[:, 0])[order]
            # group: 8 x (bit length of len + 1, minus one) + the three bits after its leading one
            x = length + 1
            e = np.floor(np.log2(x)).astype(np.int64)
            frac = np.where(e >= 3, (x >> np.maximum(e - 3, 0)) & 7, (x << np.maximum(3 - e, 0)) & 7)
            group = 8 * e + frac
            assert np.all(np.diff(group) <= 0)
    for a, b in zip(*out):
        assert torch.equal(a, b)


@pytest.mark.parametrize("tile,batch,ppt", [(16, 256, 1), (8, 64, 2), (32, 128, 2)])
def test_persistent_compositing_is_bit_invariant(tile, batch, ppt):
    """A persistent grid taking tiles from the queue gives the same image,
    final transmittance, last-contributor counts and checkpoints as a block
    per tile, and the same 2D gradients up to the order of float atomics."""
    sizes = [(150, 97), (41, 70)]
    cams = [synth.camera_pinhole(50, 50, w / 2, h / 2, w, h) for w, h in sizes]
    recs = [synth.projected_records(4000, w, h, seed=71 + v) for v, (w, h) in enumerate(sizes)]
    dev, _ = gpu_util.records(recs, cams, tile)
    dls = torch.from_numpy(np.concatenate([synth.dl_dimage(w, h, seed=3 + v).ravel()
                                           for v, (w, h) in enumerate(sizes)])).cuda()
    out = []
    for persistent in (False, True):
        gpu_util.lib()
        st = raster.RasterSettings(tile=tile, batch=batch, pixels_per_thread=ppt, pixels_per_thread_fwd=ppt,
                                   persistent=persistent)
        r = raster.Renderer(4000, 0, raster.Views(cams, tile), st)
        gpu_util.set_projected(r, dev)
        r.ckpt.fill_(-1.0)
        r.bin_sort()
        r.render_fwd()
        g2d = r.raster_bwd(dL_dimage=dls).clone()
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        out.append([t.clone().cpu() for t in (r.image, r.T_final, r.n_last, r.ckpt)] + [g2d.cpu()])
    for a, b in zip(out[0][:4], out[1][:4]):
        assert torch.equal(a, b)
    assert gpu_util.rel_err(out[1][4].double().numpy(), out[0][4].double().numpy()) < 1e-6


def test_bin_sort_from_projection_keys_equals_from_records():
    """gs_bin_sort reading the depth keys and packed rectangles gs_project
    wrote gives the same pairs and ranges as deriving them from the records."""
    scene, _, cam, _ = synth.case_c2(n=50_000)
    r = _renderer([cam], scene.n, sh_degree=3)
    model = raster.GaussianModel.from_scene(scene)
    r.project(model.c_params())
    out = []
    for aux in (True, False):
        r.aux_valid = aux
        r.bin_sort()
        torch.cuda.synchronize()
        assert int(r.status.item()) == 0
        out.append(_sorted_pairs(r))
    assert out[0][0] == out[1][0] > 0
    for a, b in zip(out[0][1:], out[1][1:]):
        assert np.array_equal(a, b)
