"""htgs_render_static: the forward render for callers that cannot allocate
device memory (a plugin inside a host application that owns the device heap,
or a real-time loop that must not allocate). Its scratch is a fixed-size
array inside the library, so the caller passes only inputs and outputs; the
result must equal the regular htgs_render (same tolerance as every other
image comparison), on two calls in a row that share the array.

This file is named to be collected last."""
import numpy as np
import pytest
import torch

from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import GaussianTensors, Renderer
from tests.gpu_util import IMAGE_TOL

pytestmark = pytest.mark.gpu


def test_static_scratch_render_matches_render_on_two_calls():
    scene, cam, prm, tile = scenes.config1()
    cam = cam.rounded()
    g = GaussianTensors.from_scene(scene)
    launch = B.c_launch(tile)
    ref = Renderer(cam, prm, scene.n, launch=launch).forward(g).clone()
    for call in range(2):
        img = torch.full_like(ref, float("nan"))
        st = B.htgs_render_static(g.c_struct(), cam, prm, launch, img)
        assert st == B.HTGS_OK, (call, B.htgs_status_string(st))
        torch.cuda.synchronize()
        assert torch.isfinite(img).all()
        err = float((img - ref).abs().max())
        assert err <= IMAGE_TOL, (call, err)


def test_static_scratch_rejects_scenes_beyond_its_size():
    scene, cam, prm, tile = scenes.config1()
    cam = cam.rounded()
    big = scenes.small_box_scene(400_000, seed=1)  # records alone exceed the array
    g = GaussianTensors.from_scene(big)
    img = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    st = B.htgs_render_static(g.c_struct(), cam, prm, B.c_launch(tile), img)
    assert st == B.HTGS_ERR_WORKSPACE, B.htgs_status_string(st)


def _static_ceiling(cam, prm, launch):
    """Largest Gaussian count whose instance-free workspace fits the static
    array (host arithmetic through htgs_workspace_size)."""
    lo, hi = 1, 1 << 24
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if B.htgs_workspace_size(mid, cam, prm, launch, 0)[0] <= B.HTGS_STATIC_SCRATCH_BYTES:
            lo = mid
        else:
            hi = mid
    return lo


def test_static_scratch_renders_a_scene_just_under_its_ceiling():
    """The stated limit holds: a scene 2000 Gaussians under the largest
    count whose workspace fits (its first 256 are the 64x64 test frame, the
    rest lie behind the camera and cover no tile) renders, and equals the
    frame rendered by htgs_render; one Gaussian over the limit is refused."""
    frame, cam, prm, tile = scenes.config1()
    cam = cam.rounded()
    launch = B.c_launch(tile)
    n_max = _static_ceiling(cam, prm, launch)
    assert 130_000 < n_max < 150_000  # about 240 bytes per Gaussian in 32 MiB
    hidden = scenes.small_box_scene(n_max - 2000 - frame.n, seed=5)
    hidden.means[:, 2] = np.float32(-3.0)
    scene = frame.concat(hidden)
    g = GaussianTensors.from_scene(scene)
    ref = Renderer(cam, prm, frame.n, launch=launch).forward(GaussianTensors.from_scene(frame)).clone()
    img = torch.full_like(ref, float("nan"))
    st = B.htgs_render_static(g.c_struct(), cam, prm, launch, img)
    assert st == B.HTGS_OK, B.htgs_status_string(st)
    assert torch.equal(img, ref)
    over = GaussianTensors.from_scene(frame.concat(scenes.small_box_scene(n_max + 1 - frame.n, seed=6)))
    st = B.htgs_render_static(over.c_struct(), cam, prm, launch, img)
    assert st == B.HTGS_ERR_WORKSPACE, B.htgs_status_string(st)
