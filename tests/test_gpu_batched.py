"""Batched views (several views per iteration, uneven sizes, each chosen on
the device into a slot sized for the largest): every view of a batch renders
and scores as it does alone, and the batch's adjoint is the sum of the
views' adjoints over the views the gate opened."""
import numpy as np
import pytest
import torch

import synth
from paper_2603_08997_gb300 import gsr, raster
from paper_2603_08997_gb300.refine import RefinementLoop
from tests import gpu_util

pytestmark = pytest.mark.gpu

SIZES = [(64, 64), (48, 40), (80, 56)]


def _cams():
    return [synth.camera_pinhole(64.0 * w / 64, 64.0 * w / 64, w / 2, h / 2, w, h) for w, h in SIZES]


def _single(scene, cam, target, dl=None):
    """Image, loss and gradient of one view rendered alone."""
    r = raster.Renderer(scene.n, scene.sh_degree, raster.Views([cam], 16))
    model = raster.GaussianModel.from_scene(scene)
    grad = torch.zeros_like(model.flat)
    r.forward(model.c_params())
    r.compute_loss(torch.from_numpy(target.ravel()).cuda(), with_grad=True)
    r.backward(model.c_params(), model.c_grads(grad))
    torch.cuda.synchronize()
    return r.image_of(0).cpu().numpy(), float(r.loss[0].item()), grad.cpu().numpy()


def _slots(scene, cams, order, compact=False, persistent=False):
    """A renderer over len(order) slots of the largest size, filled on the
    device with the cameras of `order` (compact: the views' own tile grids
    packed one after another; persistent: compositing through a tile queue)."""
    import copy
    wmax, hmax = max(c.width for c in cams), max(c.height for c in cams)
    slot = copy.copy(cams[0])
    slot.width, slot.height = wmax, hmax
    slots = raster.Views([slot] * len(order), 16)
    poses = raster.Views(cams, 16)
    r = raster.Renderer(scene.n, scene.sh_degree, slots, raster.RasterSettings(persistent=persistent))
    r.sizes_on_device = True
    seq = torch.tensor(order, dtype=torch.int32, device="cuda")
    it = torch.zeros(1, dtype=torch.int64, device="cuda")
    vid = torch.zeros(len(order), dtype=torch.int32, device="cuda")
    gsr.call("gs_select_views", gsr.ptr(seq), len(order), gsr.ptr(it), len(order), gsr.ptr(vid),
             gsr.ptr(poses.dev), gsr.ptr(slots.dev), 16 if compact else 0, None)
    return r, vid


@pytest.mark.parametrize("compact,persistent", [(False, False), (True, True), (True, False), (False, True)])
def test_batch_matches_views_alone(compact, persistent):
    """Every view of a batch renders bit-identically to the view alone, with
    the slots' tile grids sized for the largest view or packed per view, and
    with one block per tile or a persistent grid taking tiles from a queue."""
    gpu_util.lib()
    scene, _, _ = synth.case_c1(n=1500)
    cams = _cams()
    rng = np.random.default_rng(4)
    targets = [rng.uniform(0, 1, (3, h, w)).astype(np.float32) for w, h in SIZES]
    alone = [_single(scene, c, t) for c, t in zip(cams, targets)]
    order = [2, 0, 1]
    r, vid = _slots(scene, cams, order, compact, persistent)
    flat_t = torch.from_numpy(np.concatenate([t.ravel() for t in targets])).cuda()
    offs = torch.tensor(np.concatenate([[0], np.cumsum([t.size for t in targets])[:-1]]), dtype=torch.int64,
                        device="cuda")
    model = raster.GaussianModel.from_scene(scene)
    grad = torch.zeros_like(model.flat)
    gate = torch.tensor([1, 0, 1], dtype=torch.uint8, device="cuda")  # slot 1 (view 0) closed
    r.forward(model.c_params())
    r.compute_loss(flat_t, offs, vid, with_grad=True)
    r.backward(model.c_params(), model.c_grads(grad), view_gate=gate)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    for k, v in enumerate(order):
        w, h = SIZES[v]
        off = r.views.pix_offsets[k]
        img = r.image[3 * off:3 * off + 3 * w * h].view(3, h, w).cpu().numpy()
        assert np.array_equal(img, alone[v][0])  # pixels are independent of the batch
        assert abs(float(r.loss[k].item()) - alone[v][1]) <= 1e-6 * alone[v][1]
    want = alone[2][2] + alone[1][2]  # the views in open slots 0 and 2
    assert gpu_util.rel_err(grad.cpu().numpy(), want) < 1e-5


def test_batch_slot_against_oracle():
    """One slot of a batch (a view chosen on the device into a slot larger than
    itself, between two other views; compact tile grids, persistent
    compositing) against the FP64 oracle directly: image
    within 1e-5, loss within 1e-5, and the gradient of that slot alone (the
    other slots' gates closed) within the gradient bar."""
    import oracle
    gpu_util.lib()
    scene, _, _ = synth.case_c1(n=1500)
    cams = _cams()
    rng = np.random.default_rng(6)
    targets = [rng.uniform(0, 1, (3, h, w)).astype(np.float32) for w, h in SIZES]
    order = [2, 1, 0]
    r, vid = _slots(scene, cams, order, compact=True, persistent=True)
    flat_t = torch.from_numpy(np.concatenate([t.ravel() for t in targets])).cuda()
    offs = torch.tensor(np.concatenate([[0], np.cumsum([t.size for t in targets])[:-1]]), dtype=torch.int64,
                        device="cuda")
    model = raster.GaussianModel.from_scene(scene)
    grad = torch.zeros_like(model.flat)
    gate = torch.tensor([0, 1, 0], dtype=torch.uint8, device="cuda")  # slot 1 holds view 1 (48x40)
    r.forward(model.c_params())
    r.compute_loss(flat_t, offs, vid, with_grad=True)
    r.backward(model.c_params(), model.c_grads(grad), view_gate=gate)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    v = order[1]
    w, h = SIZES[v]
    rc = oracle.RasterConfig()
    f = oracle.forward(scene, cams[v], rc, margin_rel=1e-4)
    off = r.views.pix_offsets[1]
    img = r.image[3 * off:3 * off + 3 * w * h].view(3, h, w).cpu().numpy()
    ok = ~f["margin"].astype(bool)[None].repeat(3, 0)
    assert f["margin"].mean() < 0.01
    assert np.abs(img - f["image"])[ok].max() <= 1e-5 * np.abs(f["image"]).max()
    L, dL = oracle.loss_and_grad(f["image"], targets[v])
    assert abs(float(r.loss[1].item()) - L) <= 1e-5 * L
    og = oracle.backward(scene, cams[v], rc, f, dL)
    gg = gpu_util.gpu_grads(model, grad)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert gpu_util.rel_err(gg[k], og[k]) < 1e-4, (k, gpu_util.rel_err(gg[k], og[k]))
        assert gpu_util.cosine(gg[k], og[k]) > 0.9999, k


def test_batched_loop_runs_and_gates():
    """Eager and graph forms of one batched iteration agree; over 20 graph
    iterations the gate counts 2 decisions per iteration and Adam steps at
    most once per iteration."""
    gpu_util.lib()
    scene, _, _ = synth.case_c1(n=1500)
    cams = _cams()
    rng = np.random.default_rng(5)
    targets = [torch.from_numpy(rng.uniform(0, 1, (3, h, w)).astype(np.float32)) for w, h in SIZES]
    seq = rng.integers(0, 3, size=60).astype(np.int32)
    one = []
    for graph in (False, True):
        model = raster.GaussianModel.from_scene(scene)
        loop = RefinementLoop(model, cams, targets, seq, gated=True, W=4, views_per_step=2)
        loop.step_graph() if graph else loop.step_eager()
        torch.cuda.synchronize()
        one.append(model.flat.cpu().numpy())
        if graph:
            for _ in range(19):
                loop.step_graph()
            torch.cuda.synchronize()
            assert int(loop.renderer.status.item()) == 0
            st = loop.gate.read()
            assert st["t"] == 40 and st["errors"] == 0
            steps = int(loop.adam.step_count.item())
            assert 2 <= steps <= 20  # warmup iterations always step
            assert np.isfinite(model.flat.cpu().numpy()).all()
        loop.close()
    assert gpu_util.rel_err(one[1], one[0]) < 1e-6


@pytest.mark.parametrize("coarse", [False, True])
def test_batched_loop_compact_persistent_equals_default(coarse):
    """The batched loop with per-view packed tile grids and persistent
    compositing (with tile lists, and with super-tile lists over the packed
    grids) takes the same decisions and steps as with largest-view slots,
    tile lists and a block per tile (parameters equal up to the order of
    float atomics)."""
    gpu_util.lib()
    scene, _, _ = synth.case_c1(n=1500)
    cams = _cams()
    rng = np.random.default_rng(5)
    targets = [torch.from_numpy(rng.uniform(0, 1, (3, h, w)).astype(np.float32)) for w, h in SIZES]
    seq = rng.integers(0, 3, size=60).astype(np.int32)
    out = []
    for compact in (False, True):
        model = raster.GaussianModel.from_scene(scene)
        st = raster.RasterSettings(persistent=compact, coarse_lists=compact and coarse)
        loop = RefinementLoop(model, cams, targets, seq, st, gated=True, W=4, views_per_step=3, log_capacity=16,
                              compact_tiles=compact, batch_lr_scale=True)
        for _ in range(12):
            loop.step_graph()
        torch.cuda.synchronize()
        assert int(loop.renderer.status.item()) == 0
        log = loop.read_log(12)
        out.append((model.flat.cpu().numpy(), log["g"], int(loop.adam.step_count.item())))
        loop.close()
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]
    assert gpu_util.rel_err(out[1][0], out[0][0]) < 1e-6


@pytest.mark.parametrize("gated", [False, True])
def test_per_view_steps_equal_an_explicit_sequence(gated):
    """Per-view optimizer steps of a batch: the raster adjoint of the opened
    views from the batch's forward pass, then for each opened view in slot
    order the projection adjoint of its 2D gradients fused with one Adam
    step (at the parameters as they stand).  Equal to the explicit sequence
    of those calls, and the step count advances once per opened view."""
    gpu_util.lib()
    scene, _, _ = synth.case_c1(n=1500)
    cams = _cams()
    rng = np.random.default_rng(9)
    targets = [torch.from_numpy(rng.uniform(0, 1, (3, h, w)).astype(np.float32)) for w, h in SIZES]
    seq = np.array([2, 0, 1] * 4, np.int32)
    model = raster.GaussianModel.from_scene(scene)
    loop = RefinementLoop(model, cams, targets, seq, gated=gated, W=0, views_per_step=3, per_view_steps=True,
                          compact_tiles=True)
    flat0 = model.flat.clone()
    loop.gate.decide(torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda"),
                     torch.ones(3, device="cuda"), loop.g, loop.any)  # every view gets a history
    loop.gate.update(torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda"), torch.ones(3, device="cuda") * 10)
    loop.step_eager()
    torch.cuda.synchronize()
    g = loop.g.cpu().numpy().copy() if gated else np.ones(3, np.uint8)
    assert int(loop.adam.step_count.item()) == int(g.sum())
    got = model.flat.clone()
    # the explicit sequence on a fresh copy of the same state
    model2 = raster.GaussianModel.from_scene(scene)
    model2.flat.copy_(flat0)
    adam2 = raster.AdamState(model2)
    r = loop.renderer
    r.forward(model2.c_params())
    r.compute_loss(loop.targets, loop.target_offsets, loop.view_ids, with_grad=True)
    gate = torch.from_numpy(g).cuda()
    r.raster_bwd(view_gate=gate)
    for k in range(3):
        if g[k]:
            one = torch.zeros(3, dtype=torch.uint8, device="cuda")
            one[k] = 1
            r.project_bwd_adam(model2, adam2, view_gate=one)
    torch.cuda.synchronize()
    assert int(adam2.step_count.item()) == int(g.sum())
    assert gpu_util.rel_err(got.cpu().numpy(), model2.flat.cpu().numpy()) < 1e-6
    loop.close()


def test_fused_and_unfused_loops_agree():
    """The loop's backward branch in its two forms (projection adjoint and Adam
    fused in one kernel; gradients stored, then the Adam kernel) gives the same
    parameters, step counts, decisions and logged norms over 12 graph
    iterations of a 2-view batched loop."""
    gpu_util.lib()
    scene, _, _ = synth.case_c1(n=1500)
    cams = _cams()
    rng = np.random.default_rng(7)
    targets = [torch.from_numpy(rng.uniform(0, 1, (3, h, w)).astype(np.float32)) for w, h in SIZES]
    seq = rng.integers(0, 3, size=40).astype(np.int32)
    res = []
    for fused in (False, True):
        model = raster.GaussianModel.from_scene(scene)
        loop = RefinementLoop(model, cams, targets, seq, gated=True, W=4, views_per_step=2, fused=fused,
                              log_capacity=12)
        for _ in range(12):
            loop.step_graph()
        torch.cuda.synchronize()
        log = loop.read_log(12)
        res.append((model.flat.cpu().numpy(), int(loop.adam.step_count.item()), log))
        loop.close()
    (p0, s0, l0), (p1, s1, l1) = res
    assert s0 == s1 and s0 >= 2
    assert np.array_equal(l0["g"], l1["g"])
    assert gpu_util.rel_err(p1, p0) < 1e-6
    np.testing.assert_allclose(l1["grad_sq"], l0["grad_sq"], rtol=1e-4)
    np.testing.assert_allclose(l1["update_sq"], l0["update_sq"], rtol=1e-4)


def test_autotune_picks_a_timed_candidate():
    from paper_2603_08997_gb300 import autotune
    gpu_util.lib()
    scene, _, _ = synth.case_c1(n=1500)
    cams = _cams()
    rng = np.random.default_rng(6)
    targets = [torch.from_numpy(rng.uniform(0, 1, (3, h, w)).astype(np.float32)).cuda() for w, h in SIZES]
    model = raster.GaussianModel.from_scene(scene)
    cands = ((8, 64, 1, 2), (16, 256, 1, 2), (32, 128, 2, 2))
    autotune._cache.clear()
    st, times = autotune.autotune(model, cams, targets, candidates=cands, views_per_step=3, reps=2)
    assert set(times) == set(cands) and all(np.isfinite(t) and t > 0 for t in times.values())
    assert (st.tile, st.batch, st.pixels_per_thread_fwd, st.pixels_per_thread) == min(times, key=times.get)
    st2, times2 = autotune.autotune(model, cams, targets, candidates=cands, views_per_step=3)
    assert times2 == {} and st2 == st  # cached
    autotune._cache.clear()


def test_host_targets_feed_equals_device_targets():
    """Targets fed from pinned host memory one iteration ahead (HostTargets)
    give the same per-iteration losses and decisions as device targets."""
    from paper_2603_08997_gb300.refine import HostTargets
    gpu_util.lib()
    scene, _, _ = synth.case_c1(n=1500)
    cams = [synth.camera_pinhole(64.0, 64.0, 32.0, 32.0, 64, 64) for _ in range(3)]
    for k, c in enumerate(cams):  # three poses: small rotations about y
        a = 0.05 * k
        c.R = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]], np.float32)
    rng = np.random.default_rng(8)
    tg = torch.from_numpy(rng.uniform(0, 1, (3, 3, 64, 64)).astype(np.float32))
    seq = rng.integers(0, 3, size=40).astype(np.int32)
    logs = []
    for host in (False, True):
        model = raster.GaussianModel.from_scene(scene)
        if host:
            slot = torch.empty((1, 3, 64, 64), dtype=torch.float32, device="cuda")
            loop = RefinementLoop(model, cams, slot, seq, gated=True, W=6, log_capacity=40)
            loop.target_offsets = torch.zeros(3, dtype=torch.int64, device="cuda")
            feeder = HostTargets(loop, tg.pin_memory(), seq)
            loop.capture()
            for _ in range(40):
                feeder.step()
        else:
            loop = RefinementLoop(model, cams, tg.cuda(), seq, gated=True, W=6, log_capacity=40)
            loop.capture()
            for _ in range(40):
                loop.step_graph()
        torch.cuda.synchronize()
        logs.append(loop.read_log(40))
        loop.close()
    assert np.array_equal(logs[0]["loss"], logs[1]["loss"])
    assert np.array_equal(logs[0]["g"], logs[1]["g"])


def test_choose_list_form_times_both_and_keeps_the_shape():
    """autotune.choose_list_form times both list forms on the workload and
    returns the faster one, the launch shape untouched."""
    from paper_2603_08997_gb300 import autotune
    gpu_util.lib()
    scene, _, _ = synth.case_c1(n=1500)
    cams = _cams()
    model = raster.GaussianModel.from_scene(scene)
    rng = np.random.default_rng(11)
    targets = [torch.from_numpy(rng.uniform(0, 1, (3, h, w)).astype(np.float32)).cuda() for w, h in SIZES]
    base = raster.RasterSettings(tile=8, batch=128)
    st, ms = autotune.choose_list_form(model, cams, targets, base, reps=2)
    assert set(ms) == {"tile", "coarse"} and all(0.0 < v < 1e3 for v in ms.values())
    assert st.coarse_lists == (ms["coarse"] < ms["tile"])
    assert (st.tile, st.batch) == (8, 128)
