"""GPU parity at the benchmark sizes (1M clustered Gaussians at 1920x1080;
6M-Gaussian stress scene with flat splats, near-camera splats and opacities
at the clamp), in the launch configuration the benchmark times, checked on
128x128 crops. The oracle tests each crop pixel against the Gaussians whose
FP64 box meets it, which equals its brute force (tests/test_oracle_boxed.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import GaussianTensors, Renderer
from tests.gpu_util import assert_core_ids, crop_parity, gpu_render, saved_planes

pytestmark = pytest.mark.gpu

# 128x128 crops of the 1920x1080 frame: the centre (about 50 fragments per
# pixel), a denser region (140) and an off-axis one (80).
CROPS_1080 = [(896, 476, 128, 128), (400, 700, 128, 128), (1500, 200, 128, 128)]
# Share of pixels the oracle marks ambiguous on these crops, measured on
# these exact inputs: 0.03-0.07% at K = 4, 0.03-0.10% at K = 8, 0.10-0.19%
# at K = 16 (depth ties in the core, cutoff decisions of fragments in front).
CAP_CFG2 = {4: 1e-3, 8: 0.0011, 16: 0.0019}
# 6M-Gaussian stress frame, 128x128 crops: centre (770 fragments per pixel)
# and a shallower one (250). Measured 0.04-0.06%, 0.11%, 0.19-0.26% and
# 0.22-0.38% at K = 4, 8, 16, 32 (depth ties in deep cores).
CROPS_STRESS = [(896, 476, 128, 128), (300, 300, 128, 128)]
CAP_CFG5 = {4: 1e-3, 8: 0.0011, 16: 0.0026, 32: 0.0039}


@pytest.fixture(scope="module")
def cfg2_scene():
    scene, cam, prm = scenes.config2()
    return scene, cam.rounded()


@pytest.mark.parametrize("K", [8, 4, 16])
def test_config2_crops(cfg2_scene, K):
    """1M clustered Gaussians at 1920x1080, rendered whole in the launch
    configuration of the benchmark; three 128x128 crops against the oracle:
    image and core ids on every pixel."""
    scene, cam = cfg2_scene
    prm = scenes.Params(K=K)
    img, r, g = gpu_render(scene, cam, prm)
    assert np.isfinite(img).all()
    sv = saved_planes(r, cam, K)
    for win in CROPS_1080:
        rep, ref, d = crop_parity(scene, cam, prm, win, img, f"config2 K={K} crop {win}", CAP_CFG2[K])
        assert_core_ids(sv, d, scene, cam, prm, window=win, label=f"config2 K={K} crop {win}")


def test_config2_counters_and_instances(cfg2_scene):
    scene, cam = cfg2_scene
    prm = scenes.Params(K=8)
    img, r, g = gpu_render(scene, cam, prm)
    c = B.htgs_get_counters(r.workspace)
    print("instances", r.last_instances, c)
    assert c["kept"] > 0 and c["box_pairs"] >= c["kept"] // 4
    assert r.last_instances > scene.n // 4


@pytest.fixture(scope="module")
def cfg5_scene():
    scene, cam, _ = scenes.config5()
    return scene, cam.rounded()


@pytest.mark.parametrize("K", [4, 8, 16, 32])
def test_config5_stress(cfg5_scene, K):
    """6M Gaussians at 1920x1080 with 5% flat splats, 1% at the camera or the
    near plane and 1% at the opacity clamp: render and backward are finite,
    and two 128x128 crops match the oracle (image and core ids)."""
    scene, cam = cfg5_scene
    prm = scenes.Params(K=K)
    g = GaussianTensors.from_scene(scene)
    r = Renderer(cam, prm, scene.n)
    img = r.forward(g)
    dl = torch.randn_like(img)
    grads = r.backward(g, dl)
    torch.cuda.synchronize()
    assert torch.isfinite(img).all()
    for k, v in grads.items():
        assert torch.isfinite(v).all(), k
    img_np = img.cpu().numpy().astype(np.float64)
    sv = saved_planes(r, cam, K)
    for win in CROPS_STRESS:
        rep, ref, d = crop_parity(scene, cam, prm, win, img_np, f"stress K={K} crop {win}", CAP_CFG5[K])
        assert_core_ids(sv, d, scene, cam, prm, window=win, label=f"stress K={K} crop {win}")
