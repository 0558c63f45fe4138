"""Seeded synthetic scenes and cameras.

This module only draws inputs. It holds none of the rendering method's
arithmetic, so both the CUDA path and the FP64 oracle can consume its output
without sharing any of the method.

The shapes follow the paper's scene representation (Sec. 3.1): per Gaussian a
mean (3), log-scales (3), a quaternion (w, x, y, z), an opacity logit and
spherical-harmonics coefficients (up to degree 3, 16 x 3 values). Cameras are
pinhole cameras in the OpenCV convention (+x right, +y down, +z forward) with
a row-major 4x4 world-to-camera matrix.

The distributions stand in for the trained Mip-NeRF360 / Tanks&Temples scenes
the paper measures on (Sec. 4.1), which are not available here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Inverse of the degree-0 real spherical-harmonic value 1/(2*sqrt(pi)); used
# only to turn a drawn final colour into the DC coefficient that produces it
# (colour = 0.5 + Y00 * k00, as in 3DGS).
_INV_Y00 = 2.0 * math.sqrt(math.pi)


@dataclasses.dataclass
class Scene:
    means: np.ndarray          # (N, 3) float32
    log_scales: np.ndarray     # (N, 3) float32
    quats: np.ndarray          # (N, 4) float32, (w, x, y, z), not necessarily unit
    opacity_logits: np.ndarray  # (N,) float32
    sh: np.ndarray             # (N, (deg+1)^2, 3) float32
    sh_degree: int
    filter_var: np.ndarray | None = None  # (N,) float32: 3D smoothing-filter variance, or None

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def _fv(self, f):
        return None if self.filter_var is None else f(self.filter_var)

    def astype(self, dtype) -> "Scene":
        return Scene(self.means.astype(dtype), self.log_scales.astype(dtype),
                     self.quats.astype(dtype), self.opacity_logits.astype(dtype),
                     self.sh.astype(dtype), self.sh_degree, self._fv(lambda v: v.astype(dtype)))

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity_logits[idx].copy(),
                     self.sh[idx].copy(), self.sh_degree, self._fv(lambda v: v[idx].copy()))

    def concat(self, other: "Scene") -> "Scene":
        assert other.sh_degree == self.sh_degree
        assert (self.filter_var is None) == (other.filter_var is None)
        return Scene(np.concatenate([self.means, other.means]),
                     np.concatenate([self.log_scales, other.log_scales]),
                     np.concatenate([self.quats, other.quats]),
                     np.concatenate([self.opacity_logits, other.opacity_logits]),
                     np.concatenate([self.sh, other.sh]), self.sh_degree,
                     self._fv(lambda v: np.concatenate([v, other.filter_var])))

    def with_filter(self, filter_var) -> "Scene":
        """The same Gaussians with a per-Gaussian 3D smoothing-filter variance."""
        return dataclasses.replace(self, filter_var=np.asarray(filter_var, dtype=self.means.dtype).reshape(-1))


@dataclasses.dataclass
class Camera:
    world_to_cam: np.ndarray   # (4, 4) float64, row-major, OpenCV axes
    fx: float
    fy: float
    cx: float
    cy: float
    z_near: float
    width: int
    height: int

    def rounded(self) -> "Camera":
        """The camera with every parameter rounded to float32, the precision
        the C ABI takes it in (so that a float64 consumer sees the same camera)."""
        f = lambda v: float(np.float32(v))
        return Camera(self.world_to_cam.astype(np.float32).astype(np.float64), f(self.fx), f(self.fy),
                      f(self.cx), f(self.cy), f(self.z_near), self.width, self.height)

    def crop(self, x0: int, y0: int, w: int, h: int) -> "Camera":
        """The same camera restricted to pixels [x0, x0+w) x [y0, y0+h)."""
        return Camera(self.world_to_cam.copy(), self.fx, self.fy,
                      self.cx - x0, self.cy - y0, self.z_near, w, h)


@dataclasses.dataclass
class Params:
    K: int = 8
    tau_alpha: float = 1.0 / 255.0
    tau_K: float = 0.05
    alpha_max: float = 0.999
    bg: tuple = (0.0, 0.0, 0.0)
    no_tail: bool = False  # inference without the tail: core over the background
    sorted_blend: bool = False  # mean-depth-sorted alpha blending ("w/o per-pixel HT")


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    # Normalised N(0, I4) 4-vectors are uniform on SO(3).
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    # QR of a Gaussian matrix with a sign fix gives a Haar-distributed rotation.
    out = np.empty((n, 3, 3))
    for i in range(n):
        a = rng.standard_normal((3, 3))
        q, r = np.linalg.qr(a)
        q = q * np.sign(np.diag(r))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        out[i] = q
    return out


def look_at(eye, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """World-to-camera matrix (OpenCV: +z forward, +y down) looking from eye at target."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    if abs(np.dot(f, up)) > 0.99 * np.linalg.norm(up):
        up = np.array([0.0, 0.0, 1.0]) if abs(f[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    x = np.cross(up, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])          # rows: camera axes in world coordinates
    M = np.eye(4)
    M[:3, :3] = R
    M[:3, 3] = -R @ eye
    return M


def identity_camera(width: int, height: int, f: float, z_near: float = 0.2) -> Camera:
    return Camera(np.eye(4), f, f, width / 2.0, height / 2.0, z_near, width, height)


def fov_camera(world_to_cam, width: int, height: int, vfov_deg: float = 60.0,
               z_near: float = 0.2) -> Camera:
    f = (height / 2.0) / math.tan(math.radians(vfov_deg) / 2.0)
    return Camera(np.asarray(world_to_cam, np.float64), f, f, width / 2.0, height / 2.0,
                  z_near, width, height)


# --------------------------------------------------------------------------
# Scene distributions
# --------------------------------------------------------------------------

def small_box_scene(n: int, seed: int, sh_degree: int = 0,
                    rng: np.random.Generator | None = None) -> Scene:
    """Means x, y ~ U[-1, 1], z ~ U[2, 4]; log-scales N(-2.5, 0.5); uniform
    rotations; logits N(0, 1); final degree-0 colour U[0, 1]^3 (higher bands,
    if requested, N(0, 0.05))."""
    rng = rng if rng is not None else np.random.Generator(np.random.PCG64(seed))
    means = np.empty((n, 3))
    means[:, 0:2] = rng.uniform(-1.0, 1.0, (n, 2))
    means[:, 2] = rng.uniform(2.0, 4.0, n)
    log_scales = rng.normal(-2.5, 0.5, (n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, n)
    nc = (sh_degree + 1) ** 2
    sh = np.zeros((n, nc, 3))
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    sh[:, 0, :] = (rgb - 0.5) * _INV_Y00
    if nc > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, (n, nc - 1, 3))
    return Scene(means.astype(np.float32), log_scales.astype(np.float32),
                 quats.astype(np.float32), logits.astype(np.float32),
                 sh.astype(np.float32), sh_degree)


def cluster_scene(n: int, seed: int, n_clusters: int = 64, sh_degree: int = 3,
                  rng: np.random.Generator | None = None) -> Scene:
    """Mixture of anisotropic clusters in a 20 m cube: centres U([-10, 10]^3),
    per-cluster per-axis std U[0.2, 2] under a random rotation, equal weights.
    Log-scales N(-4, 1); uniform rotations; logits N(0, 1.5); SH degree 3 with
    raw DC coefficients U[0, 1] and higher bands N(0, 0.05)."""
    rng = rng if rng is not None else np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(-10.0, 10.0, (n_clusters, 3))
    stds = rng.uniform(0.2, 2.0, (n_clusters, 3))
    rots = _random_rotations(rng, n_clusters)
    which = rng.integers(0, n_clusters, n)
    local = rng.standard_normal((n, 3)) * stds[which]
    means = centres[which] + np.einsum("nij,nj->ni", rots[which], local)
    log_scales = rng.normal(-4.0, 1.0, (n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, 1.5, n)
    nc = (sh_degree + 1) ** 2
    sh = np.empty((n, nc, 3))
    sh[:, 0, :] = rng.uniform(0.0, 1.0, (n, 3))
    if nc > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, (n, nc - 1, 3))
    return Scene(means.astype(np.float32), log_scales.astype(np.float32),
                 quats.astype(np.float32), logits.astype(np.float32),
                 sh.astype(np.float32), sh_degree)


# --------------------------------------------------------------------------
# The five workloads (sizes as stated for the paper's hot path)
# --------------------------------------------------------------------------

def config1():
    """64x64, f = 64, identity camera, 256 Gaussians, SH degree 0, K = 4,
    16x16 tiles, black background, seed 0."""
    scene = small_box_scene(256, seed=0)
    cam = identity_camera(64, 64, 64.0)
    return scene, cam, Params(K=4), (16, 16)


def config2_camera() -> Camera:
    # Camera at (0, 0, -15) looking down +z: 5 m outside the [-10, 10]^3 cube.
    return fov_camera(look_at((0.0, 0.0, -15.0), (0.0, 0.0, 0.0)), 1920, 1080, 60.0, 0.2)


def config2(n: int = 1_000_000, seed: int = 1):
    """1M clustered Gaussians, SH degree 3, one 1920x1080 view, 60 deg vertical
    FOV, near plane 0.2, K = 8."""
    return cluster_scene(n, seed=seed), config2_camera(), Params(K=8)


def config3(n: int = 500_000, seed: int = 2):
    """Training step: config-1 distribution, 1200x800, f = 1200, K = 8. The target
    image comes from the same Gaussians with means perturbed by N(0, 0.01) and
    logits by N(0, 0.1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scene = small_box_scene(n, seed, rng=rng)
    target = perturbed(scene, rng)
    cam = identity_camera(1200, 800, 1200.0)
    return scene, target, cam, Params(K=8)


def perturbed(scene: Scene, rng: np.random.Generator) -> Scene:
    """Target Gaussians of a training step: means + N(0, 0.01), logits + N(0, 0.1)."""
    n = scene.n
    return Scene(scene.means + rng.normal(0.0, 0.01, scene.means.shape).astype(np.float32),
                 scene.log_scales.copy(), scene.quats.copy(),
                 scene.opacity_logits + rng.normal(0.0, 0.1, n).astype(np.float32),
                 scene.sh.copy(), scene.sh_degree)


def filter_variance_from_cameras(means, cameras, scale: float = 0.2, margin: float = 0.15) -> np.ndarray:
    """Input recipe for the 3D smoothing filter (an input of the render, as a
    training loop would compute it from its cameras): the filter's standard
    deviation is `scale` times the smallest depth / focal length over the
    cameras that see the mean (in front of the near plane, projecting into
    the image widened by `margin` on each side); Gaussians seen by no camera
    take the largest variance. Returns float32 variances."""
    means = np.asarray(means, np.float64)
    best = np.full(means.shape[0], np.inf)
    for cam in cameras:
        M = np.asarray(cam.world_to_cam, np.float64)
        v = means @ M[:3, :3].T + M[:3, 3]
        z = v[:, 2]
        front = z > cam.z_near
        zs = np.where(front, z, 1.0)
        u = cam.fx * v[:, 0] / zs + cam.cx
        w = cam.fy * v[:, 1] / zs + cam.cy
        seen = front & (u >= -margin * cam.width) & (u <= (1 + margin) * cam.width) \
            & (w >= -margin * cam.height) & (w <= (1 + margin) * cam.height)
        best = np.where(seen, np.minimum(best, z / min(cam.fx, cam.fy)), best)
    var = (scale * best) ** 2
    seen_any = np.isfinite(var)
    var[~seen_any] = var[seen_any].max() if seen_any.any() else 0.0
    return var.astype(np.float32)


def config4_views(n_views: int = 32, seed: int = 3):
    """32 cameras on a 6 m sphere around (0, 0, 3) looking at it; W ~ U{320..1600},
    H ~ U{240..1064} independently; 60 deg vertical FOV."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    centre = np.array([0.0, 0.0, 3.0])
    cams = []
    for _ in range(n_views):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        eye = centre + 6.0 * d
        w = int(rng.integers(320, 1601))
        h = int(rng.integers(240, 1065))
        cams.append(fov_camera(look_at(eye, centre), w, h, 60.0, 0.2))
    return cams


def config4_scene(n: int = 3_000_000, seed: int = 3) -> Scene:
    return small_box_scene(n, seed)


def config4_multi_scene_sizes():
    return [50_000, 100_000, 250_000, 500_000, 750_000, 1_000_000, 1_500_000, 2_000_000]


def config4_multi(seed: int = 5, sizes=None):
    """Eight scenes of uneven size (config-1 distribution), one 1280x720 view
    each from a camera on the 6 m sphere around the box centre."""
    sizes = sizes if sizes is not None else config4_multi_scene_sizes()
    rng = np.random.Generator(np.random.PCG64(seed + 2000))
    centre = np.array([0.0, 0.0, 3.0])
    out = []
    for i, n in enumerate(sizes):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        cam = fov_camera(look_at(centre + 6.0 * d, centre), 1280, 720, 60.0, 0.2)
        out.append((small_box_scene(n, seed * 100 + i), cam))
    return out


def config5(n: int = 6_000_000, seed: int = 4, frac_flat: float = 0.05,
            frac_near: float = 0.01, frac_max_opacity: float = 0.01, o_max: float = 0.999):
    """Stress: config-2 distribution at 1920x1080 with 5% flat splats (one axis
    log-scale = ln 1e-7), 1% with the mean within one scale of the camera or of
    the near plane, opacities clipped to o <= 0.999 with 1% exactly at 0.999."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scene = cluster_scene(n, seed, rng=rng)
    cam = config2_camera()
    idx = rng.permutation(n)
    n_flat = int(round(frac_flat * n))
    n_near = int(round(frac_near * n))
    n_omax = int(round(frac_max_opacity * n))
    flat = idx[:n_flat]
    near = idx[n_flat:n_flat + n_near]
    omax = idx[n_flat + n_near:n_flat + n_near + n_omax]
    axis = rng.integers(0, 3, n_flat)
    scene.log_scales[flat, axis] = np.float32(math.log(1e-7))
    # Means near the camera centre or the near plane (in world space).
    Minv = np.linalg.inv(cam.world_to_cam)
    sc = np.exp(scene.log_scales[near].astype(np.float64)).max(axis=1)
    half = len(near) // 2
    z_view = np.concatenate([rng.uniform(-1.0, 1.0, half) * sc[:half],
                             cam.z_near + rng.uniform(-1.0, 1.0, len(near) - half) * sc[half:]])
    xy_view = rng.uniform(-0.5, 0.5, (len(near), 2)) * np.maximum(z_view, 0.05)[:, None]
    pv = np.concatenate([xy_view, z_view[:, None], np.ones((len(near), 1))], axis=1)
    scene.means[near] = (pv @ Minv.T)[:, :3].astype(np.float32)
    # Opacity clip: logit(0.999) as the maximum; 1% exactly at the maximum.
    lmax = np.float32(math.log(o_max / (1.0 - o_max)))
    scene.opacity_logits = np.minimum(scene.opacity_logits, lmax)
    scene.opacity_logits[omax] = lmax
    return scene, cam, Params(K=8)


def random_dl_dimage(shape, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 777))
    return rng.standard_normal(shape).astype(np.float32)
