"""Seeded scene, camera and view-sequence generators.

Workload recipes (all numpy ``default_rng(seed)``, float32 arrays):

* C1, single-view parity: N=2,000 Gaussians with means uniform in
  [-2,2]x[-2,2]x[2,6] in front of an identity-pose pinhole camera
  (fx=fy=64, cx=cy=32, 64x64), log-scales N(-3,0.5), random unit quaternions,
  opacity logits N(0,1), SH degree 0 with colours U(0,1); target U(0,1).
* C2, single-view fwd+bwd+Adam: N=200,000 in the unit ball (radius U^(1/3)),
  SH degree 3 (DC colour U(0,1), higher bands N(0,0.05)), log-scales
  N(-4.5,0.7), opacity logits N(0,1.5); camera at (0,0,-3) looking at the
  origin, 980x545, 60 degree horizontal field of view; target = render of a
  perturbed copy plus N(0,0.01) noise.
* C3, refinement loop: ground truth = the C2 generator at N=3,000,000; start =
  a perturbed copy (C2 perturbation x0.2) that the caller first refines for
  5,000 always-backward iterations (pre_sequence, a stand-in for the
  densification phase, so the measured loop starts near its plateau as the
  paper's post-densification phase does); 200 cameras on a jittered ring at
  1297x840; 5,000 measured iterations with views drawn uniformly with
  replacement.
* C4: the C3 scene with 8 views per launch at resolutions drawn from
  {640x360, 980x545, 1297x840, 1600x1063}.
* C5: N=6,000,000, four 1920x1080 views.

These stand in for Mip-NeRF 360 / Deep Blending / Tanks&Temples scenes of the
paper's Sec. 4 (about 2.7M Gaussians per scene, Sec. 4.2), which are not
available here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

F32 = np.float32


def sh_coeff_count(degree: int) -> int:
    """Number of real SH basis functions up to ``degree``: (degree+1)^2."""
    return (degree + 1) ** 2


def dc_from_rgb(rgb: np.ndarray) -> np.ndarray:
    """Input encoding: the DC SH coefficient that yields colour ``rgb`` for a
    degree-0 scene, with colour = Y00 * f + 0.5 and Y00 = 1 / (2 sqrt(pi)).

    This is how the generator chooses coefficients; it is the usual 3DGS
    initialisation convention, not part of the method under test."""
    y00 = 0.5 / math.sqrt(math.pi)
    return ((rgb.astype(np.float64) - 0.5) / y00).astype(F32)


@dataclass
class Camera:
    """Pinhole camera. World -> camera: x_c = R @ x + t (x right, y down, z forward)."""
    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = 0.2

    def center(self) -> np.ndarray:
        """Camera centre in world coordinates (float64)."""
        R = self.R.astype(np.float64)
        return -R.T @ self.t.astype(np.float64)


@dataclass
class Scene:
    means: np.ndarray          # [N,3] f32
    log_scales: np.ndarray     # [N,3] f32
    quats: np.ndarray          # [N,4] f32, (w,x,y,z)
    opacity_logit: np.ndarray  # [N]   f32
    sh: np.ndarray             # [N,K,3] f32, K=(deg+1)^2
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def sh_degree(self) -> int:
        return int(round(math.sqrt(self.sh.shape[1]))) - 1

    def copy(self) -> "Scene":
        return Scene(self.means.copy(), self.log_scales.copy(), self.quats.copy(),
                     self.opacity_logit.copy(), self.sh.copy(), dict(self.extra))

    def flat(self) -> np.ndarray:
        """All parameters as one f32 vector in the group order
        means | log_scales | quats | opacity_logit | sh (each group row-major)."""
        return np.concatenate([self.means.ravel(), self.log_scales.ravel(), self.quats.ravel(),
                               self.opacity_logit.ravel(), self.sh.ravel()]).astype(F32)


def camera_pinhole(fx, fy, cx, cy, width, height, znear=0.2) -> Camera:
    """Identity-pose pinhole camera."""
    return Camera(np.eye(3, dtype=F32), np.zeros(3, F32), float(fx), float(fy), float(cx),
                  float(cy), int(width), int(height), float(znear))


def camera_look_at(pos, target, width, height, fovx_deg, up=(0.0, 1.0, 0.0), znear=0.2) -> Camera:
    """Camera at ``pos`` looking at ``target`` with world ``up`` shown upward in the
    image (image y points down). fx = fy = (W/2)/tan(fovx/2), principal point at
    the image centre."""
    pos = np.asarray(pos, np.float64)
    fwd = np.asarray(target, np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    y_c = -(up - fwd * np.dot(up, fwd))
    y_c /= np.linalg.norm(y_c)
    x_c = np.cross(y_c, fwd)
    R = np.stack([x_c, y_c, fwd])
    t = -R @ pos
    f = (width / 2.0) / math.tan(math.radians(fovx_deg) / 2.0)
    return Camera(R.astype(F32), t.astype(F32), f, f, width / 2.0, height / 2.0,
                  int(width), int(height), znear)


def ring_cameras(n_views: int, width: int, height: int, seed: int = 0,
                 fovx_deg: float = 60.0) -> list:
    """Jittered orbit ring: azimuth k*(360/n) deg + U(-0.5,0.5) deg, radius 3+N(0,0.05),
    height N(0,0.1), looking at the origin, up +y."""
    rng = np.random.default_rng(seed)
    step = 360.0 / n_views
    cams = []
    for k in range(n_views):
        az = math.radians(k * step + rng.uniform(-0.5, 0.5))
        r = 3.0 + rng.normal(0.0, 0.05)
        h = rng.normal(0.0, 0.1)
        pos = (r * math.sin(az), h, -r * math.cos(az))
        cams.append(camera_look_at(pos, (0.0, 0.0, 0.0), width, height, fovx_deg))
    return cams


def _unit_quats(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(F32)


def scene_cube(n: int, seed: int = 0) -> Scene:
    """C1 generator (camera frame = world frame, identity pose)."""
    rng = np.random.default_rng(seed)
    means = np.empty((n, 3), F32)
    means[:, 0:2] = rng.uniform(-2.0, 2.0, size=(n, 2))
    means[:, 2] = rng.uniform(2.0, 6.0, size=n)
    log_scales = rng.normal(-3.0, 0.5, size=(n, 3)).astype(F32)
    quats = _unit_quats(rng, n)
    opacity_logit = rng.normal(0.0, 1.0, size=n).astype(F32)
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    sh = dc_from_rgb(rgb).reshape(n, 1, 3)
    return Scene(means, log_scales, quats, opacity_logit, sh)


def scene_ball(n: int, seed: int = 0, sh_degree: int = 3, opacity_std: float = 1.5,
               log_scale_mean: float = -4.5, log_scale_std: float = 0.7) -> Scene:
    """C2/C3/C5 generator: means uniform in the unit ball."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.uniform(0.0, 1.0, size=(n, 1)) ** (1.0 / 3.0)
    means = (d * r).astype(F32)
    log_scales = rng.normal(log_scale_mean, log_scale_std, size=(n, 3)).astype(F32)
    quats = _unit_quats(rng, n)
    opacity_logit = rng.normal(0.0, opacity_std, size=n).astype(F32)
    K = sh_coeff_count(sh_degree)
    sh = np.empty((n, K, 3), F32)
    sh[:, 0, :] = dc_from_rgb(rng.uniform(0.0, 1.0, size=(n, 3)))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, size=(n, K - 1, 3))
    return Scene(means, log_scales, quats, opacity_logit, sh)


def perturb_scene(scene: Scene, seed: int, scale: float = 1.0) -> Scene:
    """Perturbed copy: means + N(0,0.01 s), DC + N(0,0.05 s), opacity logit + N(0,0.2 s),
    log-scales + N(0,0.1 s)."""
    rng = np.random.default_rng(seed)
    out = scene.copy()
    n = scene.n
    out.means = (scene.means + rng.normal(0, 0.01 * scale, size=(n, 3))).astype(F32)
    out.sh = scene.sh.copy()
    out.sh[:, 0, :] = (scene.sh[:, 0, :] + rng.normal(0, 0.05 * scale, size=(n, 3))).astype(F32)
    out.opacity_logit = (scene.opacity_logit + rng.normal(0, 0.2 * scale, size=n)).astype(F32)
    out.log_scales = (scene.log_scales + rng.normal(0, 0.1 * scale, size=(n, 3))).astype(F32)
    return out


def sparse_start(scene: Scene, n0: int, seed: int, perturb: float = 0.2, scale_boost: float = 1.44) -> Scene:
    """The start of a densification phase: a random subset of n0 of the
    scene's Gaussians (kept in index order), perturbed like perturb_scene x
    perturb, with scales multiplied by scale_boost so the sparser set still
    covers the volume (x1.44 ~ (3M / 1M)^(1/3) for a third of the Gaussians)."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(scene.n, size=n0, replace=False))
    sub = Scene(scene.means[idx].copy(), scene.log_scales[idx].copy(), scene.quats[idx].copy(),
                scene.opacity_logit[idx].copy(), scene.sh[idx].copy())
    out = perturb_scene(sub, seed + 1, perturb)
    out.log_scales = (out.log_scales + np.float32(math.log(scale_boost))).astype(F32)
    return out


def scene_tiny(n: int, seed: int, width: int = 32, height: int = 32, sh_degree: int = 1,
               depth=(2.0, 4.0), log_scale=(-2.6, 0.3)) -> tuple:
    """Small scene for brute-force and finite-difference checks: Gaussians spread over
    the view frustum of a 32x32 identity-pose camera (fx=fy=32)."""
    rng = np.random.default_rng(seed)
    cam = camera_pinhole(32.0 * width / 32, 32.0 * width / 32, width / 2.0, height / 2.0, width, height)
    z = rng.uniform(depth[0], depth[1], size=n)
    u = rng.uniform(0.1 * width, 0.9 * width, size=n)
    v = rng.uniform(0.1 * height, 0.9 * height, size=n)
    means = np.stack([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z], 1).astype(F32)
    log_scales = rng.normal(log_scale[0], log_scale[1], size=(n, 3)).astype(F32)
    quats = _unit_quats(rng, n)
    opacity_logit = rng.normal(0.0, 1.0, size=n).astype(F32)
    K = sh_coeff_count(sh_degree)
    sh = np.empty((n, K, 3), F32)
    sh[:, 0, :] = dc_from_rgb(rng.uniform(0.1, 0.9, size=(n, 3)))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.3, size=(n, K - 1, 3))
    return Scene(means, log_scales, quats, opacity_logit, sh), cam


def view_sequence(n_iters: int, n_views: int, seed: int = 0) -> np.ndarray:
    """Views drawn uniformly with replacement (the loop's sampling step, as input)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_views, size=n_iters).astype(np.int32)


# ---------------------------------------------------------------- workloads

def case_c1(seed: int = 0, n: int = 2000):
    scene = scene_cube(n, seed)
    cam = camera_pinhole(64.0, 64.0, 32.0, 32.0, 64, 64)
    target = np.random.default_rng(seed + 1).uniform(0.0, 1.0, size=(3, 64, 64)).astype(F32)
    return scene, cam, target


def case_c2(seed: int = 0, n: int = 200_000):
    """Returns (scene, perturbed copy used to render the target, camera, noise[3,H,W])."""
    scene = scene_ball(n, seed, sh_degree=3, opacity_std=1.5)
    target_scene = perturb_scene(scene, seed + 1, 1.0)
    cam = camera_look_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 980, 545, 60.0)
    noise = np.random.default_rng(seed + 2).normal(0.0, 0.01, size=(3, 545, 980)).astype(F32)
    return scene, target_scene, cam, noise


def case_c3(seed: int = 0, n: int = 3_000_000, n_views: int = 200, n_iters: int = 5000,
            width: int = 1297, height: int = 840, start_scale: float = 0.2):
    """Returns (ground-truth scene, start scene, cameras, view sequence)."""
    gt = scene_ball(n, seed, sh_degree=3, opacity_std=1.5)
    start = perturb_scene(gt, seed + 1, start_scale)
    cams = ring_cameras(n_views, width, height, seed + 2)
    seq = view_sequence(n_iters, n_views, seed)
    return gt, start, cams, seq


def pre_sequence(n_iters: int = 5000, n_views: int = 200, seed: int = 7) -> np.ndarray:
    """View sequence of the refinement that precedes the measured loop."""
    return view_sequence(n_iters, n_views, seed)


C4_RESOLUTIONS = ((640, 360), (980, 545), (1297, 840), (1600, 1063))


def case_c4(seed: int = 0, n_views_per_launch: int = 8, n_ring: int = 200):
    """Eight ring cameras per launch with resolutions drawn from C4_RESOLUTIONS."""
    rng = np.random.default_rng(seed + 3)
    picks = rng.choice(n_ring, size=n_views_per_launch, replace=False)
    res = rng.choice(len(C4_RESOLUTIONS), size=n_views_per_launch)
    ring = np.random.default_rng(seed + 2)
    cams = []
    base = ring_cameras(n_ring, 1297, 840, seed + 2)
    for p, r in zip(picks, res):
        w, h = C4_RESOLUTIONS[int(r)]
        c = base[int(p)]
        f = (w / 2.0) / math.tan(math.radians(60.0) / 2.0)
        cams.append(Camera(c.R.copy(), c.t.copy(), f, f, w / 2.0, h / 2.0, w, h, c.znear))
    del ring
    return cams, picks.astype(np.int32)


def case_c4_ring(seed: int = 0, n: int = 3_000_000, n_views: int = 200, n_iters: int = 500,
                 views_per_step: int = 8, start_scale: float = 0.2):
    """Batched workload: the C3 scenes, every ring camera with a resolution drawn
    from C4_RESOLUTIONS (60 degree horizontal field of view at its width), and
    a view sequence of n_iters * views_per_step draws.  Returns (ground-truth
    scene, start scene, cameras, view sequence)."""
    gt = scene_ball(n, seed, sh_degree=3, opacity_std=1.5)
    start = perturb_scene(gt, seed + 1, start_scale)
    rng = np.random.default_rng(seed + 3)
    res = rng.choice(len(C4_RESOLUTIONS), size=n_views)
    cams = []
    for c, r in zip(ring_cameras(n_views, 1297, 840, seed + 2), res):
        w, h = C4_RESOLUTIONS[int(r)]
        f = (w / 2.0) / math.tan(math.radians(60.0) / 2.0)
        cams.append(Camera(c.R.copy(), c.t.copy(), f, f, w / 2.0, h / 2.0, w, h, c.znear))
    seq = view_sequence(n_iters * views_per_step, n_views, seed)
    return gt, start, cams, seq


def case_c5(seed: int = 0, n: int = 6_000_000, n_views: int = 4):
    scene = scene_ball(n, seed, sh_degree=3, opacity_std=1.5)
    cams = ring_cameras(n_views, 1920, 1080, seed + 2)
    return scene, cams


def projected_records(n: int, width: int, height: int, seed: int = 0, tie_frac: float = 0.2,
                      sigma_range=(0.6, 6.0), aniso=(1.0, 8.0), cull_frac: float = 0.05) -> dict:
    """Random screen-space Gaussians, the input of the binning and compositing
    stages, for stage-wise parity tests.

    Returns float32 centres (mean2d, may lie outside the image), covariance
    eigen-structure (sigma1 >= sigma2 in pixels, angle theta), opacity, colour,
    depth (about tie_frac of them repeat another Gaussian's depth exactly), a
    pixel-space box [x0, x1] x [y0, y1] of half-width 3.5 sigma1 around the
    centre, and a culled flag for about cull_frac of them."""
    rng = np.random.default_rng(seed)
    mean2d = np.stack([rng.uniform(-0.1 * width, 1.1 * width, n), rng.uniform(-0.1 * height, 1.1 * height, n)], 1)
    s1 = np.exp(rng.uniform(np.log(sigma_range[0]), np.log(sigma_range[1]), n))
    s2 = s1 / rng.uniform(aniso[0], aniso[1], n)
    theta = rng.uniform(0.0, np.pi, n)
    opacity = rng.uniform(0.02, 1.0, n)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    depth = rng.uniform(0.5, 20.0, n).astype(F32)
    ties = rng.random(n) < tie_frac
    src = rng.integers(0, n, n)
    depth[ties] = depth[src[ties]]
    half = 3.5 * s1
    box = np.stack([mean2d[:, 0] - half, mean2d[:, 0] + half, mean2d[:, 1] - half, mean2d[:, 1] + half], 1)
    culled = rng.random(n) < cull_frac
    return dict(mean2d=mean2d.astype(F32), sigma1=s1.astype(F32), sigma2=s2.astype(F32), theta=theta.astype(F32),
                opacity=opacity.astype(F32), rgb=rgb.astype(F32), depth=depth, box=box.astype(F32), culled=culled)


def opaque_stack_records(n: int, width: int, height: int, clamp_at=(40, 230), seed: int = 0) -> dict:
    """A deep stack of screen-space Gaussians over a small image, for the
    adjoint's transmittance rebuild: every Gaussian covers the whole image,
    record i lies at depth 1 + i / 100 (so the list order is the index order);
    the records at positions `clamp_at` are wide (sigma 400 px) and nearly
    opaque (opacity U(0.997, 0.9995)), so alpha' reaches the 0.99 clamp at every
    pixel; the others have sigma 60 px and opacity U(0.006, 0.02).  Layout as
    projected_records."""
    rng = np.random.default_rng(seed)
    mean2d = np.stack([rng.uniform(0.3 * width, 0.7 * width, n), rng.uniform(0.3 * height, 0.7 * height, n)], 1)
    s1 = np.full(n, 60.0)
    opacity = rng.uniform(0.006, 0.02, n)
    for k in clamp_at:
        if k < n:
            s1[k] = 400.0
            opacity[k] = rng.uniform(0.997, 0.9995)
    s2 = s1 / rng.uniform(1.0, 1.5, n)
    theta = rng.uniform(0.0, np.pi, n)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    depth = (1.0 + np.arange(n) / 100.0).astype(F32)
    half = 3.5 * s1
    box = np.stack([mean2d[:, 0] - half, mean2d[:, 0] + half, mean2d[:, 1] - half, mean2d[:, 1] + half], 1)
    return dict(mean2d=mean2d.astype(F32), sigma1=s1.astype(F32), sigma2=s2.astype(F32), theta=theta.astype(F32),
                opacity=opacity.astype(F32), rgb=rgb.astype(F32), depth=depth, box=box.astype(F32),
                culled=np.zeros(n, bool))


def dl_dimage(width: int, height: int, seed: int = 0) -> np.ndarray:
    """A random upstream gradient dL/dimage [3,H,W] (a linear functional of the image)."""
    return np.random.default_rng(seed).normal(0.0, 1.0, (3, height, width)).astype(F32)
