"""The forward blend skips a warp's pixel block when an axis separates the
block from a record's cutoff ellipse (Sec. 3.2: the region rho^2 <= rho_c of
a splat on the image plane), a test added on top of the box test. It must be
conservative: skipping never changes which fragments are kept. Each launch
shape has its own blocks (8 x 4, 8 x 8, 8 x 16 pixels), so the kept-fragment
count and the image must be identical across shapes, and both agree with the
FP64 oracle, on a scene of needles, discs and sub-pixel splats in every
orientation (the shapes a box fits worst)."""
import numpy as np
import pytest

import oracle
from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from tests.gpu_util import gpu_render, image_parity

pytestmark = pytest.mark.gpu

SHAPES = [((16, 16), 1), ((16, 16), 2), ((16, 16), 4), ((32, 16), 1), ((32, 16), 2), ((16, 8), 1), ((8, 8), 2)]


def _thin_scene(n, seed):
    scene = scenes.small_box_scene(n, seed=seed, sh_degree=1)
    rng = np.random.default_rng(seed + 1)
    ls = rng.normal(-4.5, 0.5, (n, 3))
    rows = np.arange(n)
    long_axis = rng.integers(0, 3, n)
    ls[rows, long_axis] = rng.normal(-1.6, 0.4, n)                 # needles
    disc = rng.random(n) < 0.4
    ls[rows[disc], (long_axis[disc] + 1) % 3] = rng.normal(-1.8, 0.4, disc.sum())  # discs
    tiny = rng.random(n) < 0.15
    ls[tiny] = rng.normal(-6.0, 0.3, (tiny.sum(), 3))              # sub-pixel
    scene.log_scales = ls.astype(np.float32)
    scene.opacity_logits = (scene.opacity_logits + 1.5).astype(np.float32)
    return scene


@pytest.fixture(scope="module")
def thin():
    scene = _thin_scene(3000, seed=71)
    cam = scenes.identity_camera(256, 192, 256.0).rounded()
    prm = scenes.Params(K=4, bg=(0.2, 0.3, 0.1))
    runs = {}
    for tile, ppt in SHAPES:
        img, r, _ = gpu_render(scene, cam, prm, tile=tile, ppt=ppt, save=False)
        runs[(tile, ppt)] = (img, B.htgs_get_counters(r.workspace))
    return scene, cam, prm, runs


def test_kept_fragments_identical_across_launch_shapes(thin):
    scene, cam, prm, runs = thin
    kept = {k: c["kept"] for k, (_, c) in runs.items()}
    assert len(set(kept.values())) == 1, kept
    img0 = runs[SHAPES[0]][0]
    for k, (img, _) in runs.items():
        assert np.abs(img - img0).max() <= 1e-6, k


def test_thin_splats_match_the_oracle(thin):
    scene, cam, prm, runs = thin
    img, counters = runs[SHAPES[0]]
    ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    image_parity(img, ref, d, "thin splats")
    # Every fragment the oracle keeps is kept (up to cutoff decisions that
    # FP32 and FP64 take differently, a few per million).
    n_ref = int(d["n_frag"].sum())
    assert abs(counters["kept"] - n_ref) <= 1e-4 * n_ref + 10, (counters["kept"], n_ref)
