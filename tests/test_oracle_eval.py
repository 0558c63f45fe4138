"""Pins for the oracle's ray-splat evaluation (Sec. 3.2, Eq. (9)-(13) and the
max-point depth of Sec. 3.3, Eq. (14)).

The paper states that rho^2 from the Pluecker form equals the minimum of the
Mahalanobis distance along the pixel ray, i.e. what inverse-based ray
approaches compute, and that degenerate splats need no special case. Each
test below checks the oracle against an independent computation of that
statement."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_08129_gb300 import scenes
from tests import closed_form as cf


def _cam(width=64, height=48, f=60.0, M=None):
    cam = scenes.identity_camera(width, height, f)
    if M is not None:
        cam.world_to_cam = np.asarray(M, np.float64)
    return cam


def _scene_from(means, log_scales, quats, logits, rgb=None, degree=0):
    n = len(means)
    sh = np.zeros((n, (degree + 1) ** 2, 3))
    if rgb is not None:
        sh[:, 0, :] = (np.asarray(rgb) - 0.5) * 2.0 * math.sqrt(math.pi)
    return scenes.Scene(np.asarray(means, np.float64), np.asarray(log_scales, np.float64),
                        np.asarray(quats, np.float64), np.asarray(logits, np.float64), sh, degree)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rho2_and_depth_match_inverse_covariance(seed):
    """rho^2 equals min_t of the Mahalanobis distance along the ray, and the
    depth is the view z of that minimiser (Sec. 3.2, 3.3)."""
    rng = np.random.default_rng(seed)
    n = 40
    scene = scenes.small_box_scene(n, seed=100 + seed, sh_degree=0).astype(np.float64)
    M = scenes.look_at(rng.uniform(-0.5, 0.5, 3) + [0, 0, -0.5], [0.1, -0.1, 3.0])
    cam = scenes.fov_camera(M, 80, 60, 55.0)
    sp = oracle.preprocess(scene, cam, scenes.Params())
    checked = 0
    for g in range(n):
        if not sp["valid"][g]:
            continue
        for _ in range(5):
            xs = sp["p"][g][0] + rng.uniform(-1.2, 1.2) * sp["h"][g][0]
            ys = sp["p"][g][1] + rng.uniform(-1.2, 1.2) * sp["h"][g][1]
            hit, rho2, z, a_raw, den, num = oracle.eval_pair(sp, g, xs, ys)
            ref_rho2, ref_z, ref_a = cf.fragment(scene, g, cam, xs, ys)
            assert hit
            assert rho2 == pytest.approx(ref_rho2, rel=1e-9, abs=1e-11)
            assert z == pytest.approx(ref_z, rel=1e-9)
            assert a_raw == pytest.approx(ref_a, rel=1e-9, abs=1e-14)
            checked += 1
    assert checked > 100


def test_rho2_matches_dense_ray_sampling():
    """Brute-force minimisation of the Gaussian along the ray (no closed form)."""
    scene = scenes.small_box_scene(6, seed=7).astype(np.float64)
    cam = _cam()
    sp = oracle.preprocess(scene, cam, scenes.Params())
    for g in range(6):
        xs, ys = sp["p"][g][0] + 0.3 * sp["h"][g][0], sp["p"][g][1] - 0.2 * sp["h"][g][1]
        hit, rho2, z, *_ = oracle.eval_pair(sp, g, xs, ys)
        o_w, r_w = cf.camera_ray(cam, xs, ys)
        R = cf.rotation(scene.quats[g])
        s = np.exp(scene.log_scales[g])
        ts = np.linspace(0.5, 8.0, 200001)
        X = o_w[None, :] + ts[:, None] * r_w[None, :]
        U = ((X - scene.means[g]) @ R) / s
        m2 = (U * U).sum(1)
        i = int(np.argmin(m2))
        assert 0 < i < len(ts) - 1
        assert rho2 == pytest.approx(m2[i], rel=1e-6, abs=1e-9)
        assert z == pytest.approx(X[i, 2], abs=1e-4)


def test_isotropic_sphere_on_axis():
    """Sphere of std sigma at distance D on the optical axis: the ray at angle
    theta passes at distance D sin(theta), so rho^2 = (D sin(theta)/sigma)^2."""
    D, sigma, f = 3.0, 0.1, 100.0
    scene = _scene_from([[0, 0, D]], [[math.log(sigma)] * 3], [[1, 0, 0, 0]], [2.0])
    cam = scenes.Camera(np.eye(4), f, f, 0.0, 0.0, 0.2, 64, 64)
    sp = oracle.preprocess(scene, cam, scenes.Params())
    for theta in [0.0, 0.005, 0.01, 0.02, 0.03]:
        xs = f * math.tan(theta)
        hit, rho2, z, *_ = oracle.eval_pair(sp, 0, xs, 0.0)
        assert rho2 == pytest.approx((D * math.sin(theta) / sigma) ** 2, rel=1e-10, abs=1e-12)
        # The closest point to the centre along the ray is at depth D cos^2(theta).
        assert z == pytest.approx(D * math.cos(theta) ** 2, rel=1e-10)


@pytest.mark.parametrize("sw", [1e-7, 0.0])
def test_flat_splat_equals_surfel(sw):
    """A Gaussian with one vanishing axis must reduce to 2D-surfel evaluation:
    intersect the ray with the splat plane and take (u/s_u)^2 + (v/s_v)^2
    (Sec. 3.2: degenerate splats need no special case)."""
    rng = np.random.default_rng(3)
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    su, sv = 0.15, 0.08
    ls = [math.log(su), math.log(sv), math.log(sw) if sw > 0 else -np.inf]
    mean = [0.1, -0.05, 2.5]
    scene = _scene_from([mean], [ls], [q], [1.0])
    cam = _cam(64, 64, 64.0)
    with np.errstate(divide="ignore"):
        sp = oracle.preprocess(scene, cam, scenes.Params())
    assert sp["valid"][0]
    R = cf.rotation(q)
    tu, tv, tw = R[:, 0], R[:, 1], R[:, 2]
    for xs, ys in [(33.1, 30.7), (36.0, 31.0), (30.2, 28.9), (sp["p"][0][0], sp["p"][0][1])]:
        hit, rho2, z, *_ = oracle.eval_pair(sp, 0, xs, ys)
        assert hit and np.isfinite(rho2) and np.isfinite(z)
        o_w, r_w = cf.camera_ray(cam, xs, ys)
        t = np.dot(np.asarray(mean) - o_w, tw) / np.dot(r_w, tw)
        x = o_w + t * r_w - mean
        ref = (np.dot(x, tu) / su) ** 2 + (np.dot(x, tv) / sv) ** 2
        assert rho2 == pytest.approx(ref, rel=1e-5, abs=1e-7)
        assert z == pytest.approx((o_w + t * r_w)[2], rel=1e-5)


def test_needle_and_point_are_finite():
    """Two or three vanishing axes still give finite or 'miss' results."""
    scene = _scene_from([[0.0, 0.0, 2.0], [0.05, 0.0, 2.0]],
                        [[math.log(0.1), -np.inf, -np.inf], [-np.inf] * 3],
                        [[1, 0, 0, 0], [0.9, 0.1, 0.3, 0.2]], [1.0, 1.0])
    cam = _cam(32, 32, 32.0)
    with np.errstate(divide="ignore"):
        sp = oracle.preprocess(scene, cam, scenes.Params())
        for g in range(2):
            for xs, ys in [(16.0, 16.0), (16.5, 15.2), (20.0, 16.0)]:
                hit, rho2, z, a, den, num = oracle.eval_pair(sp, g, xs, ys)
                assert not np.isnan(rho2)
                assert hit == (den != 0.0)


def test_edge_on_flat_splat_misses():
    """A ray inside the plane of a flat splat has a vanishing denominator:
    the ray misses (Sec. 3.2). q = (1/2, 1/2, 1/2, 1/2) is an exact cyclic
    permutation: t_u = y, t_v = z, t_w = x, so the flat splat lies in the
    plane x = 0, which contains the optical axis."""
    scene = _scene_from([[0.0, 0.0, 2.0]], [[math.log(0.2), math.log(0.2), -np.inf]],
                        [[0.5, 0.5, 0.5, 0.5]], [1.0])
    cam = scenes.Camera(np.eye(4), 50.0, 50.0, 0.0, 0.0, 0.2, 8, 8)
    with np.errstate(divide="ignore"):
        sp = oracle.preprocess(scene, cam, scenes.Params())
    for ys in [0.0, 1.0, -2.5]:
        hit, rho2, z, a, den, num = oracle.eval_pair(sp, 0, 0.0, ys)
        assert den == 0.0 and not hit
    hit, rho2, z, a, den, num = oracle.eval_pair(sp, 0, 0.5, 0.0)
    assert hit and den > 0
