"""Programmatic dependent launch: a render call launches its kernels so that
each one's CTAs may be scheduled while its predecessor finishes, every kernel
waiting for its predecessor before touching memory; a call that asks for
phase timing events launches them plainly. Both must give the same image
and saved state bit for bit, and the same gradients up to the order of the
adjoint's atomic accumulation."""
import numpy as np
import pytest
import torch

from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import GaussianTensors, Renderer

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K", [4, 8, 16])
def test_dependent_and_plain_launches_agree(K):
    scene = scenes.small_box_scene(20000, seed=11, sh_degree=2)
    cam = scenes.identity_camera(320, 208, 300.0).rounded()
    prm = scenes.Params(K=K, bg=(0.1, 0.2, 0.3))
    g = GaussianTensors.from_scene(scene)
    events = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for e in events:
        e.record()
    outs = []
    for launch in (B.c_launch((16, 16), 1), B.c_launch((16, 16), 1, 0, events)):
        r = Renderer(cam, prm, scene.n, launch=launch)
        img = r.forward(g, save=True)
        dl = torch.sin(torch.arange(img.numel(), device="cuda", dtype=torch.float32)).view_as(img) * 1e-2
        grads = r.backward(g, dl)
        torch.cuda.synchronize()
        assert r.status()[0] == B.HTGS_OK
        outs.append((img.cpu().numpy(), r.saved.cpu().numpy(), {k: v.cpu().numpy() for k, v in grads.items()}))
    (ia, sa, ga), (ib, sb, gb) = outs
    assert np.array_equal(ia, ib)
    assert np.array_equal(sa.view(np.uint32), sb.view(np.uint32))
    for k in ga:
        scale = max(float(np.abs(ga[k]).max()), 1e-30)
        assert np.abs(ga[k] - gb[k]).max() <= 1e-5 * scale, k


def test_staging_batch_sizes_agree():
    """The forward's staging batch (32, 64 or 128 records in three buffers,
    192 in two) changes only the schedule: the image and saved state are the
    same bit for bit."""
    scene = scenes.small_box_scene(20000, seed=12, sh_degree=1)
    cam = scenes.identity_camera(320, 208, 300.0).rounded()
    prm = scenes.Params(K=8, bg=(0.1, 0.2, 0.3))
    g = GaussianTensors.from_scene(scene)
    outs = []
    for batch in (128, 192, 64, 32):
        r = Renderer(cam, prm, scene.n, launch=B.c_launch((16, 16), 1, smem_batch=batch))
        img = r.forward(g, save=True)
        torch.cuda.synchronize()
        assert r.status()[0] == B.HTGS_OK
        outs.append((img.cpu().numpy(), r.saved.cpu().numpy().view(np.uint32)))
    for img, saved in outs[1:]:
        assert np.array_equal(img, outs[0][0])
        assert np.array_equal(saved, outs[0][1])
