"""Pin for the oracle's analytic backward (Sec. 3.3: per-pixel shared tail
partials; Sec. 3.2: the evaluation is additions, multiplications and one
division, so it is differentiable everywhere the discrete decisions hold).

FP64 central differences of the oracle's own forward (itself pinned in
test_oracle_eval/setup/blend) against its analytic gradient, on every
parameter whose perturbation leaves every discrete decision unchanged."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_08129_gb300 import scenes


def _signature(scene, cam, prm, win):
    img, d = oracle.render(scene, cam, prm, window=win, diagnostics=True)
    return img, (d["frag_hash"].tobytes(), d["core_gid"].tobytes(), d["n_frag"].tobytes())


def _fd_check(scene, cam, prm, win, seed, h=1e-6, max_params=None):
    x0, y0, w, hh = win
    g = np.random.default_rng(seed).standard_normal((hh, w, 3))
    an = oracle.render_backward(scene, cam, prm, g, window=win)
    _, sig0 = _signature(scene, cam, prm, win)
    fields = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    attr = {"opacity_logits": "opacity_logits"}
    n_cmp, n_skip = 0, 0
    worst = 0.0
    for name in fields:
        arr = getattr(scene, attr.get(name, name))
        flat = arr.reshape(-1)
        gan = an[name].reshape(-1)
        scale = max(np.abs(gan).max(), 1e-12)
        idx = range(flat.size) if max_params is None else \
            np.random.default_rng(seed + 1).choice(flat.size, min(flat.size, max_params), replace=False)
        for k in idx:
            old = flat[k]
            flat[k] = old + h
            ip, sp = _signature(scene, cam, prm, win)
            flat[k] = old - h
            im, sm = _signature(scene, cam, prm, win)
            flat[k] = old
            if sp != sig0 or sm != sig0:
                n_skip += 1
                continue
            fd = ((ip - im) * g).sum() / (2 * h)
            err = abs(fd - gan[k])
            worst = max(worst, err / (1e-6 * scale + 1e-5 * abs(gan[k])))
            assert err <= 1e-6 * scale + 1e-5 * abs(gan[k]), (name, k, fd, gan[k])
            n_cmp += 1
    return n_cmp, n_skip


@pytest.mark.parametrize("K,tau_K", [(2, 0.05), (0, 0.05), (64, 0.0)])
def test_analytic_gradient_matches_central_differences(K, tau_K):
    scene = scenes.small_box_scene(14, seed=200 + K, sh_degree=3).astype(np.float64)
    scene.log_scales += 0.7
    scene.sh[:, 1:, :] *= 8.0  # make the view dependence matter
    cam = scenes.fov_camera(scenes.look_at((0.2, -0.1, -0.3), (0.0, 0.1, 3.0)), 40, 30, 60.0)
    prm = scenes.Params(K=K, tau_K=tau_K, bg=(0.3, 0.6, 0.2))
    n_cmp, n_skip = _fd_check(scene, cam, prm, (12, 8, 16, 14), seed=K)
    assert n_cmp > 0.8 * (n_cmp + n_skip) and n_cmp > 500


@pytest.mark.parametrize("K", [2, 5])
def test_no_tail_gradient_matches_central_differences(K):
    scene = scenes.small_box_scene(14, seed=220 + K, sh_degree=1).astype(np.float64)
    scene.log_scales += 0.7
    cam = scenes.fov_camera(scenes.look_at((0.2, -0.1, -0.3), (0.0, 0.1, 3.0)), 40, 30, 60.0)
    prm = scenes.Params(K=K, tau_K=0.05, bg=(0.3, 0.6, 0.2), no_tail=True)
    n_cmp, n_skip = _fd_check(scene, cam, prm, (12, 8, 16, 14), seed=K)
    assert n_cmp > 0.8 * (n_cmp + n_skip) and n_cmp > 300


@pytest.mark.parametrize("boost", [0.0, 3.0])
def test_sorted_blend_gradient_matches_central_differences(boost):
    scene = scenes.small_box_scene(14, seed=230, sh_degree=1).astype(np.float64)
    scene.log_scales += 0.7
    scene.opacity_logits += boost
    cam = scenes.fov_camera(scenes.look_at((0.2, -0.1, -0.3), (0.0, 0.1, 3.0)), 40, 30, 60.0)
    prm = scenes.Params(K=4, bg=(0.3, 0.6, 0.2), sorted_blend=True)
    n_cmp, n_skip = _fd_check(scene, cam, prm, (12, 8, 16, 14), seed=int(boost))
    assert n_cmp > 0.7 * (n_cmp + n_skip) and n_cmp > 200


def test_gradient_zero_where_alpha_clamped_and_colour_clamped():
    """No gradient flows to the opacity where alpha = alpha_max, nor to SH
    coefficients of a channel clamped at zero."""
    sh = np.zeros((1, 1, 3))
    sh[0, 0, :] = (np.array([0.8, -0.3, 0.3]) - 0.5) * 2 * math.sqrt(math.pi)
    scene = scenes.Scene(np.array([[0, 0, 3.0]]), np.full((1, 3), math.log(0.01)),
                         np.array([[1.0, 0, 0, 0]]), np.array([12.0]), sh, 0)
    cam = scenes.Camera(np.eye(4), 20.0, 20.0, 0.5, 0.5, 0.2, 1, 1)  # single pixel on the axis
    prm = scenes.Params(K=4, bg=(1.0, 1.0, 1.0))
    an = oracle.render_backward(scene, cam, prm, np.ones((1, 1, 3)))
    assert an["opacity_logits"][0] == 0.0
    assert an["sh"][0, 0, 1] == 0.0 and an["sh"][0, 0, 0] != 0.0


def test_window_gradients_add_up():
    """The gradient of a full frame is the sum of the gradients of a split."""
    scene = scenes.small_box_scene(20, seed=300, sh_degree=1).astype(np.float64)
    scene.log_scales += 0.5
    cam = scenes.identity_camera(24, 16, 24.0)
    prm = scenes.Params(K=3, bg=(0.1, 0.1, 0.1))
    g = np.random.default_rng(1).standard_normal((16, 24, 3))
    full = oracle.render_backward(scene, cam, prm, g)
    a = oracle.render_backward(scene, cam, prm, g[:, :10], window=(0, 0, 10, 16))
    b = oracle.render_backward(scene, cam, prm, g[:, 10:], window=(10, 0, 14, 16))
    for k in full:
        np.testing.assert_allclose(full[k], a[k] + b[k], rtol=1e-10, atol=1e-12)


def _weights_sorted(frags):
    """Blending weights alpha_i T_i of a depth-sorted fragment list (Eq. (2))."""
    out, T = {}, 1.0
    for z, gid, a, c in sorted(frags, key=lambda f: (f[0], f[1])):
        out[gid] = max(out.get(gid, 0.0), a * T)
        T *= 1.0 - a
    return out


@pytest.mark.parametrize("K,tau_K", [(64, 0.0), (0, 0.05)])
def test_visibility_is_the_largest_blending_weight(K, tau_K):
    """With K >= |F| and tau_K = 0 the weights are those of sorted alpha
    blending; with K = 0 every fragment is in the tail and weighs
    (1 - prod(1 - a)) a_j / sum(a)."""
    from tests.test_oracle_blend import _independent_fragments
    scene = scenes.small_box_scene(12, seed=500 + K, sh_degree=0).astype(np.float64)
    scene.log_scales += 0.6
    cam = scenes.identity_camera(20, 16, 20.0)
    prm = scenes.Params(K=K, tau_K=tau_K)
    out = oracle.render_backward(scene, cam, prm, np.ones((16, 20, 3)), stats=True)
    want = np.zeros(scene.n)
    for j in range(cam.height):
        for i in range(cam.width):
            fr = _independent_fragments(scene, cam, prm, i + 0.5, j + 0.5)
            if K:
                w = _weights_sorted(fr)
            else:
                A = sum(f[2] for f in fr)
                Tt = float(np.prod([1.0 - f[2] for f in fr]))
                w = {f[1]: (1.0 - Tt) * f[2] / A for f in fr} if A > 0 else {}
            for gid, v in w.items():
                want[gid] = max(want[gid], v)
    assert want.max() > 0.1
    np.testing.assert_allclose(out["visibility"], want, rtol=1e-10, atol=1e-14)


def test_densification_statistic_is_half_distance_times_mean_gradient():
    scene = scenes.small_box_scene(30, seed=510, sh_degree=1).astype(np.float64)
    scene.log_scales += 0.4
    scene.means[:4, 0] += 20.0  # outside the view
    cam = scenes.fov_camera(scenes.look_at((0.3, -0.2, -0.5), (0.0, 0.0, 3.0)), 32, 24, 60.0)
    prm = scenes.Params(K=3)
    g = np.random.default_rng(3).standard_normal((24, 32, 3))
    out = oracle.render_backward(scene, cam, prm, g, stats=True)
    M = np.asarray(cam.world_to_cam)
    centre = -M[:3, :3].T @ M[:3, 3]
    dist = np.linalg.norm(scene.means - centre, axis=1)
    sp = oracle.preprocess(scene, cam, prm)
    covers = (sp["valid"] == 1) & (sp["rect"][:, 0] <= sp["rect"][:, 1]) & (sp["rect"][:, 2] <= sp["rect"][:, 3])
    assert 0 < covers.sum() < scene.n
    np.testing.assert_array_equal(out["densify_count"], covers.astype(float))
    want = np.where(covers, 0.5 * dist * np.linalg.norm(out["means"], axis=1), 0.0)
    np.testing.assert_allclose(out["densify_grad"], want, rtol=1e-12, atol=0)


def test_config3_crop_central_differences():
    """The training step's finite-difference check at its stated size: 64
    Gaussians of the training distribution (SH degree 3, view dependence
    boosted) seen through a 32x32 crop of the 1200x800, f = 1200 camera with
    the principal point shifted, K = 8. Every one of the 64 x 59 parameters
    (means, log-scales, quaternions, opacity logits, SH) is perturbed by
    h = 1e-6 both ways in FP64; parameters whose perturbation changes a
    discrete decision (fragment set, core membership or order) are skipped."""
    scene = scenes.small_box_scene(64, seed=2, sh_degree=3).astype(np.float64)
    scene.sh[:, 1:, :] *= 6.0
    scene.means[:, :2] *= 0.04
    cam = scenes.identity_camera(1200, 800, 1200.0).crop(584, 384, 32, 32)
    assert (cam.cx, cam.cy) == (16.0, 16.0) and (cam.width, cam.height) == (32, 32)
    prm = scenes.Params(K=8, bg=(0.1, 0.2, 0.3))
    img, d = oracle.render(scene, cam, prm, diagnostics=True)
    assert d["n_frag"].mean() > 8 and (d["n_frag"] > prm.K).mean() > 0.3  # core and tail both used
    n_cmp, n_skip = _fd_check(scene, cam, prm, (0, 0, 32, 32), seed=3)
    assert n_cmp + n_skip == 64 * 59
    assert n_cmp > 0.9 * (n_cmp + n_skip), (n_cmp, n_skip)
