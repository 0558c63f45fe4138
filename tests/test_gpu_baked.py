"""Baked inference (App. A): htgs_bake folds the activations (unit quaternion,
exp of the log-scales, sigmoid of the logit as 2 ln o) and the 3D filter into
one record per Gaussian that also holds its SH coefficients, and a forward
render of the baked scene reads those records instead of the raw parameters.
The records must be the definitions written out, and the render must equal
the raw scene's render bit for bit (and so the FP64 oracle's within the image
tolerance); the backward needs the raw parameters and rejects a baked scene."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import (FIELDS, BakedGaussians, BatchRenderer, GaussianTensors, Renderer,
                                             _c_grad)
from tests.gpu_util import image_parity

pytestmark = pytest.mark.gpu


def _scene(n, seed, degree, filt):
    s = scenes.small_box_scene(n, seed=seed, sh_degree=degree)
    s.quats = (s.quats * np.random.default_rng(seed).uniform(0.5, 2.0, (n, 1))).astype(np.float32)  # not unit
    if filt:
        smin = np.exp(s.log_scales.astype(np.float64)).min(1)
        s = s.with_filter((np.random.default_rng(seed + 1).uniform(0.2, 2.0, n) * smin ** 2).astype(np.float32))
    return s


@pytest.mark.parametrize("degree,filt", [(0, False), (1, True), (2, False), (3, True)])
def test_baked_records_are_the_activations(degree, filt):
    scene = _scene(777, 40 + degree, degree, filt)
    g = GaussianTensors.from_scene(scene)
    rec = g.bake().records.view(scene.n, B.baked_floats(degree)).cpu().numpy().astype(np.float64)
    q = scene.quats.astype(np.float64)
    s = np.exp(scene.log_scales.astype(np.float64))
    two_ln_o = -2.0 * np.log1p(np.exp(-scene.opacity_logits.astype(np.float64)))
    if filt:
        v = scene.filter_var.astype(np.float64)[:, None]
        two_ln_o -= np.log1p(v / s ** 2).sum(1)
        s = np.sqrt(s * s + v)
    np.testing.assert_allclose(rec[:, 0:4], q / np.linalg.norm(q, axis=1, keepdims=True), rtol=0, atol=1e-6)
    np.testing.assert_array_equal(rec[:, 4:7], scene.means.astype(np.float64))
    np.testing.assert_allclose(rec[:, 7], two_ln_o, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(rec[:, 8:11], s, rtol=2e-6)
    assert (rec[:, 11] == 0).all()
    nf = 3 * (degree + 1) ** 2
    np.testing.assert_array_equal(rec[:, 12:12 + nf], scene.sh.reshape(scene.n, -1).astype(np.float64))
    assert (rec[:, 12 + nf:] == 0).all()


@pytest.mark.parametrize("degree,filt,K", [(0, False, 4), (3, True, 8), (1, False, 0)])
def test_baked_render_equals_raw_render(degree, filt, K):
    scene = _scene(3000, 50 + degree, degree, filt)
    cam = scenes.fov_camera(scenes.look_at((0.2, -0.1, -0.4), (0.0, 0.0, 3.0)), 160, 120, 60.0).rounded()
    prm = scenes.Params(K=K, bg=(0.1, 0.4, 0.2))
    g = GaussianTensors.from_scene(scene)
    r = Renderer(cam, prm, scene.n)
    raw = r.forward(g).clone()
    baked = r.forward(g.bake()).clone()
    assert torch.equal(raw, baked)
    ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    # (Degree-3 colours reach a little above 1: higher bands are N(0, 0.05).)
    image_parity(baked.cpu().numpy(), ref, d, f"baked degree={degree} K={K}", max_colour=1.5)


def test_baked_scenes_in_a_batch():
    sc = [_scene(n, 60 + i, i % 4, i % 2 == 1) for i, n in enumerate([500, 2000, 800])]
    gs = [GaussianTensors.from_scene(s) for s in sc]
    cams = [scenes.fov_camera(scenes.look_at((0.1 * i, 0.0, -0.3), (0.0, 0.0, 3.0)), w, h, 55.0).rounded()
            for i, (w, h) in enumerate([(96, 64), (130, 77), (64, 160)])]
    prm = scenes.Params(K=8)
    raw = [im.clone() for im in BatchRenderer(gs, cams, prm, save=False).forward()]
    bk = [im.clone() for im in BatchRenderer([g.bake() for g in gs], cams, prm, save=False).forward()]
    for a, b in zip(raw, bk):
        assert torch.equal(a, b)


def test_backward_rejects_a_baked_scene():
    scene = _scene(200, 70, 1, False)
    cam = scenes.identity_camera(64, 48, 64.0).rounded()
    prm = scenes.Params(K=4)
    g = GaussianTensors.from_scene(scene)
    bg = g.bake()
    r = Renderer(cam, prm, scene.n)
    r.forward(bg)
    grads = {f: torch.zeros_like(getattr(g, f)) for f in FIELDS}
    dl = torch.ones(cam.height, cam.width, 3, device="cuda")
    st = B.htgs_render_backward(bg.c_struct(), cam, prm, r.launch, r.workspace, r.capacity, r.saved, dl,
                                _c_grad(grads))
    assert st == B.HTGS_ERR_INVALID_ARG
    # the raw scene still differentiates through the same buffers
    assert B.htgs_render_backward(g.c_struct(), cam, prm, r.launch, r.workspace, r.capacity, r.saved, dl,
                                  _c_grad(grads)) == B.HTGS_OK


def test_bake_rejects_bad_arguments():
    g = GaussianTensors.from_scene(_scene(64, 80, 2, False))
    bad = torch.empty(64 * B.baked_floats(2) + 1, dtype=torch.float32, device="cuda")[1:]  # 4-byte offset
    assert B.htgs_bake(g.c_struct(), bad) == B.HTGS_ERR_INVALID_ARG
    rec = g.bake()
    assert B.htgs_bake(rec.c_struct(), bad) == B.HTGS_ERR_INVALID_ARG  # baking a baked scene
