"""Pins of the rasterizer oracle (Sec. 3, Eq. cov / proj / blend / alpha):
closed forms, brute force, tile-size invariance, an independent rotation /
Jacobian / SH reference, and the stable key sort."""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import Scene, camera_pinhole

RC = oracle.RasterConfig()


def _one(means, log_scales, quats, logits, rgbs):
    n = len(means)
    return Scene(np.array(means, np.float32).reshape(n, 3), np.array(log_scales, np.float32).reshape(n, 3),
                 np.array(quats, np.float32).reshape(n, 4), np.array(logits, np.float32).reshape(n),
                 synth.dc_from_rgb(np.array(rgbs, np.float64).reshape(n, 3)).reshape(n, 1, 3))


def test_single_isotropic_gaussian_closed_form():
    """On the optical axis at depth z with scale s: Sigma2D = ((f s/z)^2 + lowpass) I,
    so C(p) = c min(0.99, o exp(-|dp|^2 / (2 ((f s/z)^2 + lowpass))))."""
    f, z, s, logit = 40.0, 3.0, 0.05, 0.7
    cam = camera_pinhole(f, f, 16.0, 16.0, 32, 32)
    sc = _one([[0, 0, z]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [logit], [[0.2, 0.5, 0.9]])
    out = oracle.forward(sc, cam, RC)
    o = 1 / (1 + math.exp(-float(np.float32(logit))))
    s_eff = math.exp(float(np.float32(math.log(s))))  # the stored log-scale is float32
    var = (f * s_eff / z) ** 2 + RC.lowpass
    rgb = out["proj"]["rgb"][0]
    for (i, j) in [(16, 16), (15, 16), (20, 18), (10, 25), (16, 3)]:
        dx, dy = i + 0.5 - 16.0, j + 0.5 - 16.0
        a = min(RC.alpha_max, o * math.exp(-(dx * dx + dy * dy) / (2 * var)))
        want = rgb * a if a >= RC.alpha_min else np.zeros(3)
        np.testing.assert_allclose(out["image"][:, j, i], want, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rgb, [0.2, 0.5, 0.9], rtol=1e-6)


def test_two_gaussians_front_to_back():
    """C = c1 a1 + c2 a2 (1 - a1), T_final = (1 - a1)(1 - a2) for two overlapping Gaussians."""
    cam = camera_pinhole(40.0, 40.0, 16.0, 16.0, 32, 32)
    sc = _one([[0.01, 0, 2.0], [0, 0.02, 3.0]], [[math.log(0.08)] * 3, [math.log(0.1)] * 3],
              [[1, 0, 0, 0], [1, 0, 0, 0]], [0.3, 1.0], [[0.9, 0.1, 0.1], [0.1, 0.1, 0.9]])
    out = oracle.forward(sc, cam, RC)
    pr = out["proj"]
    i, j = 16, 16
    a = []
    for g in range(2):
        dx, dy = i + 0.5 - pr["mean2d"][g, 0], j + 0.5 - pr["mean2d"][g, 1]
        Q = pr["conic"][g]
        a.append(min(RC.alpha_max, pr["opacity"][g] * math.exp(-0.5 * (Q[0] * dx * dx + 2 * Q[1] * dx * dy + Q[2] * dy * dy))))
    want = pr["rgb"][0] * a[0] + pr["rgb"][1] * a[1] * (1 - a[0])
    np.testing.assert_allclose(out["image"][:, j, i], want, rtol=1e-12)
    assert abs(out["T_final"][j, i] - (1 - a[0]) * (1 - a[1])) < 1e-14


def test_projection_vs_independent_references():
    """Sigma from scipy's quaternion rotation; J from a finite-difference
    Jacobian of the pinhole map; Sigma2D = J W Sigma W^T J^T + lowpass I."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    sc, _ = synth.scene_tiny(20, seed=4, sh_degree=0)
    cam = synth.camera_look_at((0.3, -0.2, -1.0), (0.0, 0.0, 3.0), 32, 32, 60.0)
    pr = oracle.project(sc, cam, RC)
    R_c = cam.R.astype(np.float64)
    t_c = cam.t.astype(np.float64)
    # the camera reaches both sides as float32 numbers
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    for i in range(sc.n):
        if pr["touched"][i] == 0 or pr["flags"][i] & 3:
            continue
        q = sc.quats[i].astype(np.float64)
        R = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S = np.diag(np.exp(sc.log_scales[i].astype(np.float64)))
        Sigma = R @ S @ S.T @ R.T
        mu = sc.means[i].astype(np.float64)

        def proj(p):
            x = R_c @ p + t_c
            return np.array([fx * x[0] / x[2] + cx, fy * x[1] / x[2] + cy])

        np.testing.assert_allclose(pr["mean2d"][i], proj(mu), rtol=1e-12)
        h = 1e-6
        Jw = np.stack([(proj(mu + h * e) - proj(mu - h * e)) / (2 * h) for e in np.eye(3)], 1)  # = J W
        cov = Jw @ Sigma @ Jw.T + RC.lowpass * np.eye(2)
        np.testing.assert_allclose(pr["cov2d"][i], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-7, atol=1e-9)
        Q = np.linalg.inv(cov)
        np.testing.assert_allclose(pr["conic"][i], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-6, atol=1e-9)
        assert pr["depth"][i] == pytest.approx((R_c @ mu + t_c)[2], rel=1e-14)


def _real_sh_scipy(l, m, d):
    sp = pytest.importorskip("scipy.special")
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    am = abs(m)
    if hasattr(sp, "sph_harm_y"):
        Y = complex(sp.sph_harm_y(l, am, theta, phi))
    else:  # older scipy: sph_harm(m, n, azimuth, polar)
        Y = complex(sp.sph_harm(am, l, phi, theta))
    if m > 0:
        return math.sqrt(2) * Y.real
    if m < 0:
        return math.sqrt(2) * Y.imag
    return Y.real


def test_sh_basis_vs_scipy_and_textbook():
    rng = np.random.default_rng(0)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y, _ = oracle.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert Y[l * l + l + m] == pytest.approx(_real_sh_scipy(l, m, d), rel=1e-10, abs=1e-12)
        # textbook low orders (Condon-Shortley phase): Y00, Y1-1, Y10, Y11, Y2-2
        x, y, z = d
        assert Y[0] == pytest.approx(0.5 / math.sqrt(math.pi), rel=1e-14)
        assert Y[1] == pytest.approx(-math.sqrt(3 / (4 * math.pi)) * y, rel=1e-12, abs=1e-15)
        assert Y[2] == pytest.approx(math.sqrt(3 / (4 * math.pi)) * z, rel=1e-12, abs=1e-15)
        assert Y[3] == pytest.approx(-math.sqrt(3 / (4 * math.pi)) * x, rel=1e-12, abs=1e-15)
        assert Y[4] == pytest.approx(0.5 * math.sqrt(15 / math.pi) * x * y, rel=1e-12, abs=1e-15)


def test_sh_orthonormal():
    """Gauss-Legendre x uniform-azimuth quadrature of Y_i Y_j over the sphere = identity."""
    zs, wz = np.polynomial.legendre.leggauss(12)
    nphi = 16
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        for k in range(nphi):
            phi = 2 * math.pi * k / nphi
            r = math.sqrt(1 - z * z)
            Y, _ = oracle.sh_basis(3, np.array([r * math.cos(phi), r * math.sin(phi), z]))
            G += np.outer(Y, Y) * w * (2 * math.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_gradient_tangent_fd():
    rng = np.random.default_rng(3)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    _, dY = oracle.sh_basis(3, d)
    h = 1e-6
    for e in np.eye(3):
        def at(v):
            v = v / np.linalg.norm(v)
            return oracle.sh_basis(3, v)[0]
        fd = (at(d + h * e) - at(d - h * e)) / (2 * h)
        # analytic: d Y(v/|v|)/dv at |v| = 1 is (I - d d^T) grad
        an = (dY - np.outer(dY @ d, d)) @ e
        np.testing.assert_allclose(fd, an, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_tiled_equals_brute_force_c1(tile):
    scene, cam, _ = synth.case_c1()
    rc = oracle.RasterConfig(tile=tile)
    f = oracle.forward(scene, cam, rc)
    b = oracle.render_brute(f["proj"], cam, rc)
    assert np.array_equal(f["image"], b["image"])
    assert np.array_equal(f["T_final"], b["T_final"])


def test_rect_is_conservative():
    """Every (pixel, Gaussian) pair with alpha' >= 1/255 lies in the Gaussian's tile rectangle."""
    scene, cam, _ = synth.case_c1(n=300)
    pr = oracle.project(scene, cam, RC)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    px, py = xs + 0.5, ys + 0.5
    for g in range(scene.n):
        if pr["touched"][g] == 0:
            continue
        dx, dy = px - pr["mean2d"][g, 0], py - pr["mean2d"][g, 1]
        Q = pr["conic"][g]
        a = np.minimum(RC.alpha_max, pr["opacity"][g] * np.exp(-0.5 * (Q[0] * dx * dx + 2 * Q[1] * dx * dy + Q[2] * dy * dy)))
        jj, ii = np.nonzero(a >= RC.alpha_min)
        r = pr["rect"][g]
        assert ((ii // 16 >= r[0]) & (ii // 16 <= r[2]) & (jj // 16 >= r[1]) & (jj // 16 <= r[3])).all()


def test_bin_sort_vs_numpy_stable_argsort():
    scene, cam, _ = synth.case_c1()
    cams = [cam, synth.camera_pinhole(50.0, 50.0, 24.0, 20.0, 48, 40)]
    projs = [oracle.project(scene, c, RC) for c in cams]
    keys, vals, ranges, toff = oracle.bin_sort(projs, cams, 16)
    # emission order: view-major, index ascending, tiles row-major
    ek, ev = [], []
    for v, (pr, c) in enumerate(zip(projs, cams)):
        tx = (c.width + 15) // 16
        for i in range(scene.n):
            if pr["touched"][i] == 0:
                continue
            x0, y0, x1, y1 = pr["rect"][i]
            for ty in range(y0, y1 + 1):
                for t in range(x0, x1 + 1):
                    ek.append(((int(toff[v]) + ty * tx + t) << 32) | int(pr["depth_bits"][i]))
                    ev.append(i)
    ek = np.array(ek, np.uint64)
    order = np.argsort(ek, kind="stable")
    assert np.array_equal(keys, ek[order]) and np.array_equal(vals, np.array(ev, np.uint32)[order])
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    for t in range(ranges.shape[0]):
        hit = np.nonzero(tiles == t)[0]
        if len(hit) == 0:
            assert tuple(ranges[t]) == (0, 0)
        else:
            assert tuple(ranges[t]) == (hit[0], hit[-1] + 1)


def test_stop_rule_and_cutoff():
    """Eq. (blend) with both cut-offs on a stack of isotropic on-axis Gaussians
    whose alphas follow from the closed form: contributions stop before the
    Gaussian that would take T below 1e-4, alpha' is clamped at 0.99, and a
    pixel where alpha' < 1/255 receives nothing."""
    cam = camera_pinhole(40.0, 40.0, 16.0, 16.0, 32, 32)
    for logit, s, n in [(8.0, 2.0, 3), (1.4, 1.0, 8)]:
        zs = [2.0 + 0.1 * k for k in range(n)]
        sc = _one([[0, 0, z] for z in zs], [[math.log(s)] * 3] * n, [[1, 0, 0, 0]] * n, [logit] * n,
                  [[0.2 + 0.05 * k, 0.5, 0.7] for k in range(n)])
        out = oracle.forward(sc, cam, RC)
        o = 1 / (1 + math.exp(-float(np.float32(logit))))
        s_eff = math.exp(float(np.float32(math.log(s))))
        T, C, cnt = 1.0, np.zeros(3), 0
        for k, z in enumerate(zs):
            var = (40.0 * s_eff / z) ** 2 + RC.lowpass
            a = min(RC.alpha_max, o * math.exp(-0.5 * 0.5 / var))   # pixel (16,16): |dp|^2 = 0.5
            if a < RC.alpha_min:
                continue
            if T * (1 - a) < RC.t_min:
                break
            C += out["proj"]["rgb"][k] * a * T
            T *= 1 - a
            cnt += 1
        assert out["n_contrib"][16, 16] == cnt and cnt < n
        assert out["T_final"][16, 16] == pytest.approx(T, rel=1e-10)
        np.testing.assert_allclose(out["image"][:, 16, 16], C, rtol=1e-10)  # 1 - a amplifies rounding
    # far from a small Gaussian: nothing
    sc = _one([[0, 0, 3.0]], [[math.log(0.01)] * 3], [[1, 0, 0, 0]], [0.0], [[0.5, 0.5, 0.5]])
    out = oracle.forward(sc, cam, RC)
    assert out["n_contrib"][0, 0] == 0 and out["image"][:, 0, 0].max() == 0.0
