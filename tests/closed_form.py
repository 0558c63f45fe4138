"""Independent closed forms used to pin the oracle.

Nothing here follows the paper's inversion-free route: each quantity is
computed the textbook way (world-space rays, inverse covariance, scipy
rotations), so that agreement with the oracle is evidence, not repetition.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial.transform import Rotation


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, np.float64)))


def rotation(q_wxyz):
    q = np.asarray(q_wxyz, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def camera_ray(cam, xs, ys):
    """World-space origin and (unnormalised) direction of the pixel ray."""
    M = np.asarray(cam.world_to_cam, np.float64)
    R, t = M[:3, :3], M[:3, 3]
    origin = -R.T @ t
    d_cam = np.array([(xs - cam.cx) / cam.fx, (ys - cam.cy) / cam.fy, 1.0])
    return origin, R.T @ d_cam


def min_mahalanobis_along_ray(mean, log_scales, quat, origin, direction):
    """min_t (x(t) - mu)^T Sigma^{-1} (x(t) - mu) for x(t) = origin + t direction,
    with Sigma = R S S R^T; returns (rho2_min, t_star)."""
    R = rotation(quat)
    s = np.exp(np.asarray(log_scales, np.float64))
    u0 = (R.T @ (origin - np.asarray(mean, np.float64))) / s
    v = (R.T @ direction) / s
    t_star = -np.dot(u0, v) / np.dot(v, v)
    rho2 = np.dot(u0, u0) - np.dot(u0, v) ** 2 / np.dot(v, v)
    return rho2, t_star


def fragment(scene, gid, cam, xs, ys):
    """(rho2, view-depth of the maximum, unclamped alpha, rgb_raw) via the
    inverse covariance, for non-degenerate Gaussians."""
    o_w, r_w = camera_ray(cam, xs, ys)
    rho2, t = min_mahalanobis_along_ray(scene.means[gid], scene.log_scales[gid],
                                        scene.quats[gid], o_w, r_w)
    x = o_w + t * r_w
    M = np.asarray(cam.world_to_cam, np.float64)
    z = (M @ np.append(x, 1.0))[2]
    o = sigmoid(scene.opacity_logits[gid])
    return rho2, z, o * math.exp(-0.5 * rho2)


def sh_real_from_complex(dirs, degree=3):
    """Real SH of 3DGS's ordering from scipy's complex Y_l^m (Condon-Shortley
    phase included): Y_{l,-|m|} = sqrt(2) Im Y_l^{|m|}, Y_{l,0} = Re Y_l^0,
    Y_{l,|m|} = sqrt(2) Re Y_l^{|m|}."""
    from scipy.special import sph_harm_y
    dirs = np.asarray(dirs, np.float64).reshape(-1, 3)
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    theta = np.arccos(np.clip(dirs[:, 2], -1, 1))
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    out = np.zeros((dirs.shape[0], 16))
    k = 0
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            Ylm = sph_harm_y(l, abs(m), theta, phi)
            if m < 0:
                out[:, k] = math.sqrt(2) * Ylm.imag
            elif m == 0:
                out[:, k] = Ylm.real
            else:
                out[:, k] = math.sqrt(2) * Ylm.real
            k += 1
    return out


def colour(scene, gid, cam, degree=None):
    """0.5 + sum_lm Y_lm(dir) k_lm (before the clamp) using scipy's SH."""
    deg = scene.sh_degree if degree is None else degree
    M = np.asarray(cam.world_to_cam, np.float64)
    centre = -M[:3, :3].T @ M[:3, 3]
    d = np.asarray(scene.means[gid], np.float64) - centre
    Y = sh_real_from_complex(d, 3)[0][: (deg + 1) ** 2]
    return 0.5 + Y @ np.asarray(scene.sh[gid], np.float64)


def sorted_alpha_blend(frags, bg):
    """Eq. (2) with background: frags = list of (z, gid, alpha, rgb), any order."""
    C = np.zeros(3)
    T = 1.0
    for z, gid, a, c in sorted(frags, key=lambda f: (f[0], f[1])):
        C += a * T * np.asarray(c)
        T *= 1.0 - a
    return C + T * np.asarray(bg, np.float64), T


def project(cam, pts_world):
    M = np.asarray(cam.world_to_cam, np.float64)
    P = (M[:3, :3] @ np.asarray(pts_world, np.float64).T).T + M[:3, 3]
    return np.stack([cam.fx * P[:, 0] / P[:, 2] + cam.cx, cam.fy * P[:, 1] / P[:, 2] + cam.cy], 1)
