"""The per-warp marking of the compositing kernels skips a record when the
minimum of q(dp) = |U dp|^2 over a pixel block exceeds the support ellipse's
bound.  These host tests check, in float64, the closed form the kernels use
for that minimum (0 when the block contains the mean, else the least of the
four edges' clamped one-dimensional minima) against brute force over a dense
grid of the rectangle: it must never exceed the true minimum (a record would
be skipped wrongly) and it must equal it (else the test loses its effect)."""
import numpy as np


def rect_qmin(u00, u01, u11, dx0, dx1, dy0, dy1):
    """The closed form, restated from the kernels' description."""
    if dx0 <= 0 <= dx1 and dy0 <= 0 <= dy1:
        return 0.0
    sv = -u00 * u01 / (u01 * u01 + u11 * u11)  # minimising dy at dx = 1
    sh = -u01 / u00                            # minimising dx at dy = 1

    def q(dx, dy):
        z0, z1 = u00 * dx + u01 * dy, u11 * dy
        return z0 * z0 + z1 * z1

    cands = [q(dx0, min(max(sv * dx0, dy0), dy1)), q(dx1, min(max(sv * dx1, dy0), dy1)),
             q(min(max(sh * dy0, dx0), dx1), dy0), q(min(max(sh * dy1, dx0), dx1), dy1)]
    return min(cands)


def brute_qmin(u00, u01, u11, dx0, dx1, dy0, dy1, k=401):
    xs = np.linspace(dx0, dx1, k)
    ys = np.linspace(dy0, dy1, k)
    X, Y = np.meshgrid(xs, ys)
    z0, z1 = u00 * X + u01 * Y, u11 * Y
    return float((z0 * z0 + z1 * z1).min())


def test_closed_form_matches_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(400):
        # a screen-space covariance with sigma 0.5..20 px, aspect up to 40, any angle
        s1 = np.exp(rng.uniform(np.log(0.5), np.log(20.0)))
        s2 = s1 / rng.uniform(1.0, 40.0)
        th = rng.uniform(0, np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        cov = R @ np.diag([s1 * s1, s2 * s2]) @ R.T
        Q = np.linalg.inv(cov)
        L = np.linalg.cholesky(Q)  # Q = L L^T; U = L^T is upper triangular with Q = U^T U
        U = L.T
        u00, u01, u11 = U[0, 0], U[0, 1], U[1, 1]
        assert u00 > 0 and u11 > 0
        # an 8 x 4 or 8 x 8 block of pixel centres somewhere around the mean
        w, h = 7.0, float(rng.choice([3.0, 7.0]))
        dx0 = rng.uniform(-4 * s1 - w, 4 * s1)
        dy0 = rng.uniform(-4 * s1 - h, 4 * s1)
        cf = rect_qmin(u00, u01, u11, dx0, dx0 + w, dy0, dy0 + h)
        bf = brute_qmin(u00, u01, u11, dx0, dx0 + w, dy0, dy0 + h)
        # never above the true minimum (the sampled minimum is at least the true one)
        assert cf <= bf * (1 + 1e-12) + 1e-12
        # and equal to it up to the sampling step
        step = max(w, h) / 400
        grad_bound = 2 * np.sqrt(max(bf, 1e-30)) * np.linalg.norm(U, 2) * step + (np.linalg.norm(U, 2) * step) ** 2
        assert bf - cf <= grad_bound + 1e-9


def test_block_containing_the_mean_is_zero():
    assert rect_qmin(1.0, 0.3, 0.5, -1.0, 6.0, -2.0, 1.0) == 0.0


def test_axis_aligned_reduces_to_the_nearest_edge():
    # U diagonal: q = (u00 dx)^2 + (u11 dy)^2, least at the rectangle's point nearest the origin
    u00, u11 = 0.5, 2.0
    assert np.isclose(rect_qmin(u00, 0.0, u11, 3.0, 10.0, -1.0, 2.0), (u00 * 3.0) ** 2)
    assert np.isclose(rect_qmin(u00, 0.0, u11, 3.0, 10.0, 1.5, 2.0), (u00 * 3.0) ** 2 + (u11 * 1.5) ** 2)
