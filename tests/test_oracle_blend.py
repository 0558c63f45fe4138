"""Pins for the oracle's hybrid-transparency compositing (Sec. 3.3,
Eq. (15)-(16); Sec. 4.2 for K and tau_K).

Fragments are recomputed here independently (inverse covariance, scipy
rotations) and composited by textbook rules in the special cases where the
hybrid formula must reduce to them."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2410_08129_gb300 import scenes
from tests import closed_form as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _independent_fragments(scene, cam, params, xs, ys):
    """(z, gid, alpha, rgb) for every Gaussian kept at a pixel, computed without
    the oracle (valid only for non-degenerate Gaussians in front of the camera)."""
    frags = []
    M = np.asarray(cam.world_to_cam)
    for g in range(scene.n):
        o = cf.sigmoid(scene.opacity_logits[g])
        rho_c = 2 * math.log(o / params.tau_alpha)
        if rho_c <= 0:
            continue
        # near cull: view-z extent of the cutoff ellipsoid
        R = cf.rotation(scene.quats[g])
        s = np.exp(scene.log_scales[g])
        A = M[:3, :3] @ R @ np.diag(s)
        zc = (M @ np.append(scene.means[g], 1))[2]
        if zc - math.sqrt(rho_c * (A[2] ** 2).sum()) <= cam.z_near:
            continue
        rho2, z, a_raw = cf.fragment(scene, g, cam, xs, ys)
        if rho2 <= rho_c:
            rgb = np.maximum(cf.colour(scene, g, cam), 0.0)
            frags.append((z, g, min(a_raw, params.alpha_max), rgb))
    return frags


def _scene(n, seed, degree=1):
    s = scenes.small_box_scene(n, seed=seed, sh_degree=degree).astype(np.float64)
    s.log_scales += 0.6  # overlap heavily at the small test resolution
    return s


@pytest.mark.parametrize("seed", [0, 1])
def test_k_at_least_fragments_is_sorted_alpha_blending(seed):
    """K >= |F| and tau_K = 0: Eq. (15) is Eq. (2) plus background."""
    scene = _scene(14, 30 + seed)
    cam = scenes.identity_camera(20, 16, 20.0)
    prm = scenes.Params(K=64, tau_K=0.0, bg=(0.2, 0.5, 0.9))
    img, d = oracle.render(scene, cam, prm, diagnostics=True)
    assert d["n_frag"].max() >= 5
    for j in range(cam.height):
        for i in range(cam.width):
            fr = _independent_fragments(scene, cam, prm, i + 0.5, j + 0.5)
            ref, T = cf.sorted_alpha_blend(fr, prm.bg)
            np.testing.assert_allclose(img[j, i], ref, rtol=1e-9, atol=1e-12)
            assert d["n_frag"][j, i] == len(fr)
            assert d["T_core"][j, i] == pytest.approx(T, rel=1e-9, abs=1e-15)


@pytest.mark.parametrize("K,tau_K", [(3, 0.05), (1, 0.1), (0, 0.05)])
def test_no_tail_is_sorted_blend_of_the_core(K, tau_K):
    """Inference without the tail (Sec. 4.4): the K nearest candidates
    (alpha >= tau_K, (z, gid) order) blended over the background, and
    nothing else contributes."""
    scene = _scene(14, 50 + K)
    cam = scenes.identity_camera(20, 16, 20.0)
    prm = scenes.Params(K=K, tau_K=tau_K, bg=(0.7, 0.2, 0.4), no_tail=True)
    img, d = oracle.render(scene, cam, prm, diagnostics=True)
    deep = 0
    for j in range(cam.height):
        for i in range(cam.width):
            fr = _independent_fragments(scene, cam, prm, i + 0.5, j + 0.5)
            cand = sorted((f for f in fr if f[2] >= tau_K), key=lambda f: (f[0], f[1]))
            ref, T = cf.sorted_alpha_blend(cand[:K], prm.bg)
            np.testing.assert_allclose(img[j, i], ref, rtol=1e-9, atol=1e-12)
            assert d["A_tail"][j, i] == 0.0 and d["T_tail"][j, i] == 1.0
            deep += len(fr) > K
    assert deep > 20  # pixels whose tail was dropped


def _mean_depth_blend(frags, zmean, bg, tmin=1e-4):
    """Eq. (2) over fragments in (mean depth, gid) order, stopping before the
    fragment that would take the transmittance below tmin."""
    C, T = np.zeros(3), 1.0
    for z, gid, a, c in sorted(frags, key=lambda f: (zmean[f[1]], f[1])):
        if T * (1.0 - a) < tmin:
            break
        C += a * T * np.asarray(c)
        T *= 1.0 - a
    return C + T * np.asarray(bg, np.float64), T


@pytest.mark.parametrize("boost", [0.0, 8.0])
def test_sorted_blend_uses_mean_depth_order_and_stops_early(boost):
    """Tab. 3 "w/o per-pixel HT": fragments ordered by their Gaussian's
    view-space mean depth (not the per-pixel depth), blended front to back;
    with opaque splats (boost) the early termination is exercised."""
    scene = _scene(16, 60 + int(boost))
    scene.opacity_logits += boost
    if boost:
        scene.log_scales += 1.0  # overlapping opaque splats end the blending early
    cam = scenes.identity_camera(20, 16, 20.0)
    prm = scenes.Params(K=4, bg=(0.3, 0.1, 0.6), sorted_blend=True)
    img, d = oracle.render(scene, cam, prm, diagnostics=True)
    M = np.asarray(cam.world_to_cam)
    zmean = (scene.means @ M[:3, :3].T + M[:3, 3])[:, 2]
    stopped = reordered = 0
    for j in range(cam.height):
        for i in range(cam.width):
            fr = _independent_fragments(scene, cam, prm, i + 0.5, j + 0.5)
            ref, T = _mean_depth_blend(fr, zmean, prm.bg)
            np.testing.assert_allclose(img[j, i], ref, rtol=1e-9, atol=1e-12)
            assert d["T_core"][j, i] == pytest.approx(T, rel=1e-9, abs=1e-15)
            used = int(d["n_core"][j, i])
            stopped += used < len(fr)
            by_pixel = [f[1] for f in sorted(fr, key=lambda f: (f[0], f[1]))]
            by_mean = [f[1] for f in sorted(fr, key=lambda f: (zmean[f[1]], f[1]))]
            reordered += by_pixel != by_mean
    assert reordered > 0
    if boost:
        assert stopped > 0


def test_sorted_blend_equals_hybrid_when_orders_agree():
    """Isotropic splats spread in depth and translucent: the point of maximum
    contribution on a ray is the centre's projection onto it, so here mean order =
    per-pixel order and nothing stops early; with K >= |F| and tau_K = 0 both
    blendings are Eq. (2)."""
    scene = _scene(10, 70)
    scene.means[:, 2] = 2.0 + 0.4 * np.arange(10)
    scene.log_scales[:] = math.log(0.3)
    scene.opacity_logits[:] = -1.0
    cam = scenes.identity_camera(20, 16, 20.0)
    a = oracle.render(scene, cam, scenes.Params(K=64, tau_K=0.0, bg=(0.2, 0.2, 0.2), sorted_blend=True))
    b = oracle.render(scene, cam, scenes.Params(K=64, tau_K=0.0, bg=(0.2, 0.2, 0.2)))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


def test_k_zero_is_order_independent_blend():
    """K = 0 (full OIT): C = (1 - prod(1 - a)) sum(a c)/sum(a) + prod(1 - a) bg."""
    scene = _scene(14, 40)
    cam = scenes.identity_camera(16, 16, 16.0)
    prm = scenes.Params(K=0, bg=(0.3, 0.1, 0.7))
    img = oracle.render(scene, cam, prm)
    for j in range(cam.height):
        for i in range(cam.width):
            fr = _independent_fragments(scene, cam, prm, i + 0.5, j + 0.5)
            if not fr:
                np.testing.assert_allclose(img[j, i], prm.bg, atol=1e-15)
                continue
            a = np.array([f[2] for f in fr])
            c = np.array([f[3] for f in fr])
            Tt = np.prod(1 - a)
            ref = (1 - Tt) * (a[:, None] * c).sum(0) / a.sum() + Tt * np.asarray(prm.bg)
            np.testing.assert_allclose(img[j, i], ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_equal_colour_tail_equals_sorted_blending(K):
    """When every fragment that can fall into the tail has the same colour, the
    tail term (1 - T_tail) c_tail + T_tail bg is exactly the sorted blend of
    those fragments, so Eq. (15) equals Eq. (2) for any K (tau_K = 0)."""
    n_front, n_back = 3, 12
    rng = np.random.default_rng(50 + K)
    front = _scene(n_front, 60 + K, degree=0)
    back = _scene(n_back, 70 + K, degree=0)
    front.means[:, 2] = rng.uniform(2.0, 2.3, n_front)
    back.means[:, 2] = rng.uniform(3.2, 4.0, n_back)
    back.sh[:, 0, :] = (np.array([0.9, 0.2, 0.4]) - 0.5) * 2 * math.sqrt(math.pi)
    front.log_scales[:] = math.log(0.35)  # front splats cover the image
    front.opacity_logits[:] = -1.5
    scene = front.concat(back)
    cam = scenes.identity_camera(12, 12, 12.0)
    prm = scenes.Params(K=K, tau_K=0.0, bg=(0.05, 0.6, 0.3))
    img, d = oracle.render(scene, cam, prm, diagnostics=True)
    n_tested = 0
    for j in range(cam.height):
        for i in range(cam.width):
            fr = _independent_fragments(scene, cam, prm, i + 0.5, j + 0.5)
            n_front_here = sum(1 for f in fr if f[1] < n_front)
            if n_front_here > K:
                continue  # a distinct colour would fall into the tail
            ref, _ = cf.sorted_alpha_blend(fr, prm.bg)
            np.testing.assert_allclose(img[j, i], ref, rtol=1e-9, atol=1e-12)
            n_tested += int(len(fr) > K)
    assert n_tested >= 10


def test_hand_worked_tau_k_case():
    """Golden hand-worked case (tests/golden/hand_cases.json, 'tau_K'):
    on-axis spheres, K = 1; the nearer fragment is below tau_K and goes to
    the tail behind the farther one (Sec. 4.2)."""
    with open(os.path.join(GOLDEN, "hand_cases.json")) as f:
        case = json.load(f)["tau_K"]
    logits = [math.log(a / (1 - a)) for a in case["opacities"]]
    n = len(logits)
    sh = np.zeros((n, 1, 3))
    sh[:, 0, :] = (np.asarray(case["colours"]) - 0.5) * 2 * math.sqrt(math.pi)
    scene = scenes.Scene(np.array([[0.0, 0.0, z] for z in case["depths"]]),
                         np.full((n, 3), math.log(case["sigma"])), np.tile([1.0, 0, 0, 0], (n, 1)),
                         np.array(logits), sh, 0)
    # cx = cy = 4.5 puts the centre of pixel (4, 4) on the optical axis, where rho^2 = 0.
    cam = scenes.Camera(np.eye(4), 20.0, 20.0, 4.5, 4.5, 0.2, 9, 9)
    prm = scenes.Params(K=case["K"], tau_K=case["tau_K"], bg=tuple(case["bg"]))
    img = oracle.render(scene, cam, prm)
    np.testing.assert_allclose(img[4, 4], case["expected_centre"], rtol=1e-12)


def test_single_tail_fragment_equals_sorted_blending():
    """With exactly one tail fragment, c_tail = c and T_tail = 1 - alpha, so the
    tail term is that fragment alpha-blended last (any K, tau_K = 0)."""
    scene = _scene(10, 80)
    cam = scenes.identity_camera(14, 14, 14.0)
    prm0 = scenes.Params(K=64, tau_K=0.0, bg=(0.4, 0.4, 0.1))
    _, d = oracle.render(scene, cam, prm0, diagnostics=True)
    nmax = int(d["n_frag"].max())
    assert nmax >= 3
    for K in range(1, nmax):
        prm = scenes.Params(K=K, tau_K=0.0, bg=prm0.bg)
        img, dk = oracle.render(scene, cam, prm, diagnostics=True)
        for j, i in zip(*np.nonzero(dk["n_frag"] == K + 1)):
            fr = _independent_fragments(scene, cam, prm, i + 0.5, j + 0.5)
            ref, _ = cf.sorted_alpha_blend(fr, prm.bg)
            np.testing.assert_allclose(img[j, i], ref, rtol=1e-9, atol=1e-12)


def test_alpha_clamp():
    """alpha = min(o e^{-rho^2/2}, alpha_max): an opaque sphere on the axis."""
    sh = np.zeros((1, 1, 3))
    sh[0, 0, :] = (np.array([0.8, 0.1, 0.3]) - 0.5) * 2 * math.sqrt(math.pi)
    scene = scenes.Scene(np.array([[0, 0, 3.0]]), np.full((1, 3), math.log(0.2)),
                         np.array([[1.0, 0, 0, 0]]), np.array([12.0]), sh, 0)
    cam = scenes.Camera(np.eye(4), 20.0, 20.0, 4.5, 4.5, 0.2, 9, 9)
    prm = scenes.Params(K=4, bg=(1.0, 1.0, 1.0))
    img = oracle.render(scene, cam, prm)
    a = prm.alpha_max
    np.testing.assert_allclose(img[4, 4], a * np.array([0.8, 0.1, 0.3]) + (1 - a) * 1.0, rtol=1e-12)


def test_permutation_invariance():
    """No global sort is needed (Sec. 4.3): shuffling the input leaves the
    image unchanged and maps core ids through the permutation."""
    scene = _scene(40, 90, degree=2)
    cam = scenes.identity_camera(24, 20, 24.0)
    prm = scenes.Params(K=3, bg=(0.1, 0.2, 0.3))
    img, d = oracle.render(scene, cam, prm, diagnostics=True)
    perm = np.random.default_rng(0).permutation(scene.n)
    img2, d2 = oracle.render(scene.subset(perm), cam, prm, diagnostics=True)
    np.testing.assert_allclose(img2, img, rtol=1e-12, atol=1e-14)
    core2 = np.where(d2["core_gid"] >= 0, perm[np.maximum(d2["core_gid"], 0)], -1)
    np.testing.assert_array_equal(core2, d["core_gid"])


def test_transmittance_bounds_and_finiteness():
    scene = _scene(60, 91, degree=3)
    # degenerate members: flat, needle, zero-size
    scene.log_scales[0, 2] = -np.inf
    scene.log_scales[1, 1:] = -np.inf
    scene.log_scales[2, 0] = math.log(1e-7)
    cam = scenes.identity_camera(24, 24, 24.0)
    prm = scenes.Params(K=4, bg=(0.5, 0.5, 0.5))
    with np.errstate(divide="ignore"):
        img, d = oracle.render(scene, cam, prm, diagnostics=True)
    assert np.isfinite(img).all()
    for k in ("T_core", "T_tail"):
        assert (d[k] >= 0).all() and (d[k] <= 1).all()
    assert (d["A_tail"] >= 0).all()
    assert (d["n_core"] <= prm.K).all() and (d["n_core"] <= d["n_frag"]).all()


def test_empty_scene_is_background():
    scene = _scene(5, 92)
    scene.means[:, 2] = -5.0  # all behind the camera
    cam = scenes.identity_camera(8, 8, 8.0)
    prm = scenes.Params(K=4, bg=(0.25, 0.5, 0.75))
    img = oracle.render(scene, cam, prm)
    np.testing.assert_allclose(img, np.broadcast_to(prm.bg, img.shape), atol=0)


def test_cutoff_is_inclusive_at_rho_c():
    """A fragment is kept iff rho^2 <= rho_c: probe an on-axis sphere just
    inside and just outside the cutoff radius."""
    D, sigma, f = 3.0, 0.1, 100.0
    scene = scenes.Scene(np.array([[0, 0, D]]), np.full((1, 3), math.log(sigma)),
                         np.array([[1.0, 0, 0, 0]]), np.array([0.5]), np.zeros((1, 1, 3)), 0)
    prm = scenes.Params()
    rho_c = 2 * math.log(cf.sigmoid(0.5) / prm.tau_alpha)
    for eps, kept in [(-1e-7, True), (1e-7, False)]:
        theta = math.asin(sigma * math.sqrt(rho_c * (1 + eps)) / D)
        # put the centre of pixel 0 at x = f tan(theta)
        cam = scenes.Camera(np.eye(4), f, f, 0.5 - f * math.tan(theta), 0.5, 0.2, 1, 1)
        _, d = oracle.render(scene, cam, scenes.Params(K=4), diagnostics=True)
        assert d["n_frag"][0, 0] == int(kept)
