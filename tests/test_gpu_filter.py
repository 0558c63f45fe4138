"""GPU parity of the 3D smoothing filter (Sec. 4.2, the filter of Yu et al.)
through the C ABI against the FP64 oracle: forward image and core ids, and
the gradients (which flow through the filtered scales and opacity)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import FIELDS, BatchRenderer, GaussianTensors, Renderer
from tests.gpu_util import (assert_core_ids, assert_grad_close, gpu_render, image_parity,
                            grads_to_numpy, saved_planes)

pytestmark = pytest.mark.gpu


def _filtered(n, seed, cams, degree=1, scale=2.0):
    s = scenes.small_box_scene(n, seed=seed, sh_degree=degree)
    s.log_scales -= np.float32(0.8)  # small splats, so the filter matters
    return s.with_filter(scenes.filter_variance_from_cameras(s.means, cams, scale=scale))


def test_filtered_forward_matches_oracle():
    cam = scenes.identity_camera(96, 72, 90.0).rounded()
    scene = _filtered(800, 51, [cam])
    prm = scenes.Params(K=8, bg=(0.1, 0.3, 0.2))
    img, r, _ = gpu_render(scene, cam, prm)
    ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    image_parity(img, ref, d, "3D filter K=8")
    sv = saved_planes(r, cam, prm.K)
    assert assert_core_ids(sv, d, scene, cam, prm, label="3D filter K=8")["exact"] > 0.99
    # the filter changes the image (wider, dimmer splats)
    plain, _, _ = gpu_render(dataclasses.replace(scene, filter_var=None), cam, prm)
    assert np.abs(plain - img).max() > 1e-2


@pytest.mark.parametrize("K", [4, 0])
def test_filtered_gradients_match_oracle(K):
    cam = scenes.identity_camera(1200, 800, 1200.0).crop(584, 384, 32, 32).rounded()
    scene = scenes.small_box_scene(64, seed=52 + K, sh_degree=2)
    scene.means[:, :2] *= np.float32(0.04)
    scene.log_scales -= np.float32(0.5)
    scene = scene.with_filter(scenes.filter_variance_from_cameras(scene.means, [cam], scale=3.0))
    prm = scenes.Params(K=K, bg=(0.1, 0.2, 0.3))
    _, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    dl = np.random.default_rng(K).standard_normal((cam.height, cam.width, 3))
    dl[d["near_decision"] != 0] = 0.0
    dl = dl.astype(np.float32)
    ref = oracle.render_backward(scene.astype(np.float64), cam, prm, dl.astype(np.float64))
    g = GaussianTensors.from_scene(scene)
    r = Renderer(cam, prm, scene.n)
    r.forward(g)
    got = r.backward(g, torch.as_tensor(dl).cuda())
    torch.cuda.synchronize()
    assert_grad_close(grads_to_numpy(got), ref, label=f"3D filter K={K}")


def test_filtered_batch_equals_single_views():
    cams = [scenes.fov_camera(scenes.look_at((0.5 * i - 0.5, 0.2, -1.0), (0.0, 0.0, 3.0)), 80 + 16 * i, 60, 60.0)
            .rounded() for i in range(3)]
    scene = _filtered(3000, 53, cams)
    g = GaussianTensors.from_scene(scene)
    prm = scenes.Params(K=8)
    br = BatchRenderer([g] * 3, cams, prm)
    imgs = [im.clone() for im in br.forward()]
    dls = [torch.randn(im.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(i))
           for i, im in enumerate(imgs)]
    grads = br.backward(dls)
    want = {f: torch.zeros_like(getattr(g, f)) for f in FIELDS}
    for cam, img, dl in zip(cams, imgs, dls):
        r = Renderer(cam, prm, scene.n)
        ref = r.forward(g)
        assert float((img - ref).abs().max()) <= 1e-5
        single = r.backward(g, dl)
        for f in FIELDS:
            want[f] += single[f]
    torch.cuda.synchronize()
    for f in FIELDS:
        torch.testing.assert_close(grads[id(g)][f], want[f], rtol=1e-4, atol=1e-6 * float(want[f].abs().max()))
