"""Pins for the 3D smoothing filter in the oracle. Sec. 4.2 applies the 3D
filter of Yu et al.: before rendering, every Gaussian is convolved with an
isotropic Gaussian of variance v (the filter's variance, an input per
Gaussian). The filtered Gaussian must be that convolution: its density is
checked against a numerical 3D quadrature of the convolution integral, its
per-ray rho^2 and alpha against the covariance Sigma + v I assembled as a
matrix, and its analytic gradient against central differences."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_08129_gb300 import scenes
from tests.closed_form import camera_ray, rotation, sigmoid
from tests.test_oracle_backward import _fd_check


def _scene(n, seed, degree=0):
    s = scenes.small_box_scene(n, seed=seed, sh_degree=degree).astype(np.float64)
    s.log_scales += 0.6
    return s


def _filter(scene, seed, lo=0.3, hi=3.0):
    """Variances between lo and hi times the squared smallest scale."""
    smin = np.exp(scene.log_scales).min(1)
    f = np.random.default_rng(seed).uniform(lo, hi, scene.n)
    return scene.with_filter(f * smin ** 2)


def _convolved_density(mu, log_s, q, logit, v, x, half=6.0, h=0.15):
    """o int G(y) N(x - y; 0, v I) dy by a tensor-product trapezoid rule in the
    Gaussian's own frame y = mu + R diag(s) u (the integrand is smooth there
    and negligible beyond |u| = half)."""
    R, s = rotation(q), np.exp(log_s)
    g = np.arange(-half, half + h / 2, h)
    U = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    Y = mu + (U * s) @ R.T
    d2 = ((x - Y) ** 2).sum(1)
    integrand = np.exp(-0.5 * (U ** 2).sum(1)) * np.exp(-0.5 * d2 / v) / (2 * math.pi * v) ** 1.5
    return sigmoid(logit) * integrand.sum() * h ** 3 * np.prod(s)


def test_filtered_density_is_the_convolution():
    scene = _filter(_scene(4, 11), 12)
    cam = scenes.identity_camera(32, 32, 32.0)
    sp = oracle.preprocess(scene, cam, scenes.Params(K=4))
    rng = np.random.default_rng(13)
    for i in range(scene.n):
        R = sp["R"][i]
        s1 = sp["s"][i]
        for _ in range(3):
            x = scene.means[i] + R @ (s1 * rng.uniform(-1.5, 1.5, 3))
            u = (R.T @ (x - scene.means[i])) / s1
            got = sp["o"][i] * math.exp(-0.5 * u @ u)
            ref = _convolved_density(scene.means[i], scene.log_scales[i], scene.quats[i],
                                     scene.opacity_logits[i], scene.filter_var[i], x)
            assert abs(got - ref) <= 1e-7 * max(ref, 1e-3), (i, got, ref)


def test_filtered_rho2_and_alpha_from_the_summed_covariance():
    """rho^2 of a pixel ray = min_t (x(t) - mu)^T (Sigma + v I)^{-1} (x(t) - mu)
    and alpha = o sqrt(det Sigma / det(Sigma + v I)) e^{-rho^2/2}, with the
    covariances assembled as matrices."""
    scene = _filter(_scene(6, 21), 22)
    cam = scenes.fov_camera(scenes.look_at((0.1, 0.2, -0.5), (0.0, 0.0, 3.0)), 48, 40, 60.0)
    sp = oracle.preprocess(scene, cam, scenes.Params(K=4))
    checked = 0
    for i in range(scene.n):
        if not sp["valid"][i]:
            continue
        R, s = rotation(scene.quats[i]), np.exp(scene.log_scales[i])
        Sig = R @ np.diag(s ** 2) @ R.T
        Sig_f = Sig + scene.filter_var[i] * np.eye(3)
        P = np.linalg.inv(Sig_f)
        x0, x1, y0, y1 = sp["rect"][i]
        for xs, ys in [((x0 + x1) / 2 + 0.5, (y0 + y1) / 2 + 0.5), (x0 + 1.5, (y0 + y1) / 2 + 0.5)]:
            o_w, r_w = camera_ray(cam, xs, ys)
            d0 = o_w - scene.means[i]
            t = -(d0 @ P @ r_w) / (r_w @ P @ r_w)
            e = d0 + t * r_w
            rho2 = e @ P @ e
            hit, rho2_o, z, araw, den, num = oracle.eval_pair(sp, i, xs, ys)
            assert hit
            assert abs(rho2_o - rho2) <= 1e-8 * max(1.0, rho2), (i, rho2_o, rho2)
            a_ref = sigmoid(scene.opacity_logits[i]) * math.sqrt(np.linalg.det(Sig) / np.linalg.det(Sig_f)) \
                * math.exp(-0.5 * rho2)
            assert abs(araw - a_ref) <= 1e-10, (i, araw, a_ref)
            checked += 1
    assert checked >= 6


def test_zero_variance_is_no_filter():
    scene = _scene(30, 31, degree=1)
    cam = scenes.identity_camera(40, 32, 40.0)
    prm = scenes.Params(K=3, bg=(0.2, 0.1, 0.4))
    plain, d0 = oracle.render(scene, cam, prm, diagnostics=True)
    zero = scene.with_filter(np.zeros(scene.n))
    filt, d1 = oracle.render(zero, cam, prm, diagnostics=True)
    assert np.array_equal(plain, filt)
    assert np.array_equal(d0["core_gid"], d1["core_gid"])
    g = np.random.default_rng(32).standard_normal((32, 40, 3))
    a, b = oracle.render_backward(scene, cam, prm, g), oracle.render_backward(zero, cam, prm, g)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_filter_widens_and_dims_each_splat():
    """With v > 0 every scale grows to sqrt(s^2 + v) and the peak opacity
    drops by prod s / sqrt(s^2 + v); the cutoff follows the filtered opacity."""
    scene = _filter(_scene(8, 41), 42)
    cam = scenes.identity_camera(32, 32, 32.0)
    prm = scenes.Params(K=4)
    sp = oracle.preprocess(scene, cam, prm)
    s = np.exp(scene.log_scales)
    v = scene.filter_var[:, None]
    np.testing.assert_allclose(sp["s"], np.sqrt(s * s + v), rtol=1e-14)
    np.testing.assert_allclose(sp["o"], sigmoid(scene.opacity_logits) * np.prod(s / np.sqrt(s * s + v), 1),
                               rtol=1e-13)
    np.testing.assert_allclose(sp["rho_c"], 2 * np.log(sp["o"] / prm.tau_alpha), rtol=1e-12)


@pytest.mark.parametrize("K", [2, 0])
def test_filtered_gradient_matches_central_differences(K):
    """The filter variance is an input (not differentiated); the gradient of
    every parameter goes through the filtered scales and opacity."""
    scene = _filter(scenes.small_box_scene(12, seed=400 + K, sh_degree=1).astype(np.float64), 401, 0.5, 4.0)
    scene.log_scales += 0.5
    cam = scenes.fov_camera(scenes.look_at((0.2, -0.1, -0.3), (0.0, 0.1, 3.0)), 40, 30, 60.0)
    prm = scenes.Params(K=K, bg=(0.3, 0.6, 0.2))
    n_cmp, n_skip = _fd_check(scene, cam, prm, (12, 8, 16, 14), seed=K)
    assert n_cmp > 0.8 * (n_cmp + n_skip) and n_cmp > 200
