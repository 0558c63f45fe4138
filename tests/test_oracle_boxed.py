"""The oracle's box-restricted window render equals its brute force.

``oracle.render(..., box_margin=m)`` tests a window's pixels only against the
Gaussians whose covered-pixel rectangle (from Sec. 3.2's tight box, itself
pinned by brute-force containment in ``test_oracle_setup.py``), grown by m
pixels, meets the window. It exists so that 128x128 crops of million-Gaussian
scenes finish in seconds. It must change nothing: image, every per-pixel
diagnostic and the near-decision flags (whose cutoff band extends just
outside the box) are compared bit for bit with the brute force, on the
stress distribution (flat splats, splats at the camera and the near plane,
opacities at the clamp) and on windows at the image's edges and corners."""
import numpy as np
import pytest

import oracle
from paper_2410_08129_gb300 import scenes

KEYS = ("n_frag", "n_core", "core_gid", "T_core", "T_tail", "A_tail", "c_tail", "ambiguous",
        "near_decision", "frag_hash", "amb_effect")


def _check(scene, cam, prm, win, subset=True):
    img0, d0 = oracle.render(scene, cam, prm, window=win, diagnostics=True)
    img1, d1 = oracle.render(scene, cam, prm, window=win, diagnostics=True, box_margin=2)
    assert np.array_equal(img0, img1)
    for k in KEYS:
        assert np.array_equal(d0[k], d1[k]), k
    assert 0 < d1["n_tested"] and (d1["n_tested"] < scene.n or not subset)
    return d0, d1["n_tested"]


@pytest.fixture(scope="module")
def stress():
    scene, cam, _ = scenes.config5(n=40_000, seed=9)
    return scene.astype(np.float64), cam.rounded()


@pytest.mark.parametrize("win", [(936, 516, 48, 48), (0, 0, 40, 24), (1880, 1056, 40, 24),
                                 (700, 0, 32, 16), (0, 600, 16, 32)])
@pytest.mark.parametrize("K", [4, 16])
def test_boxed_equals_brute_force_on_the_stress_distribution(stress, win, K):
    scene, cam = stress
    d, tested = _check(scene, cam, scenes.Params(K=K), win)
    assert d["n_frag"].max() > 0 or win[1] == 0


def test_boxed_keeps_the_cutoff_band():
    """A dense scene with a few dozen pixels in the cutoff band: the boxed
    render flags the same ones."""
    scene = scenes.small_box_scene(20000, seed=13, sh_degree=1).astype(np.float64)
    scene.log_scales += 0.6
    cam = scenes.identity_camera(64, 48, 60.0)
    d, _ = _check(scene, cam, scenes.Params(K=4), (8, 8, 40, 32), subset=False)
    assert (d["near_decision"] & oracle.AMB_CUTOFF != 0).sum() >= 20
    _check(scene, cam, scenes.Params(K=4, sorted_blend=True), (0, 0, 64, 48), subset=False)


def test_boxed_sees_a_band_pixel_outside_the_rectangle():
    """An isotropic splat whose cutoff lies 2e-6 (relative) inside rho^2 at
    pixel (40, 24): that pixel is rejected, so it lies outside the splat's
    covered rectangle, yet it is a near-decision. A window holding that
    pixel but none of the rectangle must still flag it. (Row 24's centre is
    on the splat's horizontal axis, so the box's right edge is the cutoff
    ellipse's own extreme and falls just short of that pixel's centre.)"""
    cam = scenes.Camera(np.eye(4), 60.0, 60.0, 32.0, 24.5, 0.2, 64, 48)
    c, sigma = np.array([0.0, 0.0, 3.0]), 0.3
    r = np.array([(40.5 - cam.cx) / cam.fx, (24.5 - cam.cy) / cam.fy, 1.0])
    r /= np.linalg.norm(r)
    rho2 = (c @ c - (c @ r) ** 2) / sigma ** 2
    o = (1 / 255) * np.exp(0.5 * rho2 * (1 - 2e-6))
    scene = scenes.Scene(c[None], np.full((1, 3), np.log(sigma)), np.array([[1.0, 0, 0, 0]]),
                         np.array([np.log(o / (1 - o))]), np.full((1, 1, 3), 1.0), 0)
    sp = oracle.preprocess(scene, cam, scenes.Params(K=4))
    assert sp["valid"][0] and sp["rect"][0][1] == 39
    win = (40, 16, 8, 16)
    img0, d0 = oracle.render(scene, cam, scenes.Params(K=4), window=win, diagnostics=True)
    img1, d1 = oracle.render(scene, cam, scenes.Params(K=4), window=win, diagnostics=True, box_margin=2)
    assert d0["near_decision"][24 - 16, 0] == oracle.AMB_CUTOFF
    for k in KEYS:
        assert np.array_equal(d0[k], d1[k]), k
    assert np.array_equal(img0, img1) and d1["n_tested"] == 1
