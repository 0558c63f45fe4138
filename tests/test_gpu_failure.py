"""Failure detection without a GPU fault. The tile sort's decoupled
look-back waits for other blocks with an iteration limit; when the limit runs
out the kernel records HTGS_ERR_TIMEOUT in the workspace's status word and
carries on, and the blend skips its work. The test hook of htgs_launch makes
the first block of the first digit pass also wait for a word that nothing
writes: the wait must give up within its limit, the host must read the
status, and the context must stay usable, the next render on the same
buffers being exact."""
import time

import pytest
import torch

from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import GaussianTensors, Renderer

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [256, 20000])
def test_bounded_lookback_wait_reports_a_timeout(n):
    scene = scenes.small_box_scene(n, seed=90, sh_degree=1)
    cam = scenes.identity_camera(160, 120, 150.0).rounded()
    prm = scenes.Params(K=4)
    g = GaussianTensors.from_scene(scene)
    good = Renderer(cam, prm, scene.n).forward(g).clone()
    r = Renderer(cam, prm, scene.n, launch=B.c_launch((16, 16), test_lookback_stall=1))
    t0 = time.time()
    with pytest.raises(B.HTGSError) as e:
        r.forward(g)
    assert e.value.status == B.HTGS_ERR_TIMEOUT
    assert time.time() - t0 < 120
    # The status word is reset by the next render; with the hook off the
    # same workspace renders the same image as a fresh renderer.
    r.launch = B.c_launch((16, 16))
    assert torch.equal(r.forward(g), good)
