"""Split tiles. A tile whose instance list is longer than the chunk size is
processed by several CTAs; each leaves the sums over its fragments and its K
nearest candidates, and the last one to finish merges them in chunk order
(the core of Sec. 3.3 is the K nearest candidates of the whole list, and the
tail sums are plain sums). Image, core ids and gradients must match the FP64
oracle as for unsplit tiles, and the work items must cover every tile's list
exactly once."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from tests.gpu_util import (assert_core_ids, assert_grad_close, gpu_render, grads_to_numpy, image_parity,
                            saved_planes, workspace_view)

pytestmark = pytest.mark.gpu

MIN_CHUNK = 1024


def _dense(n=20000, seed=21, degree=1):
    """About 4000 instances per 16x16 tile: every tile is cut into chunks."""
    s = scenes.small_box_scene(n, seed=seed, sh_degree=degree)
    s.log_scales += np.float32(0.7)
    return s


def _camera():
    return scenes.identity_camera(96, 80, 80.0).rounded()


def _bucket(length):
    length = np.asarray(length, np.int64)
    out = np.full(length.shape, 63)
    nz = length > 0
    l = np.floor(np.log2(length[nz])).astype(np.int64)
    sub = np.where(l > 0, (length[nz] >> np.maximum(l - 1, 0)) & 1, 0)
    out[nz] = 62 - np.minimum(2 * l + sub, 62)
    return out


@pytest.fixture(scope="module")
def dense():
    scene, cam = _dense(), _camera()
    prm = scenes.Params(K=8, bg=(0.2, 0.1, 0.0))
    img, r, g = gpu_render(scene, cam, prm)
    ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    return scene, cam, prm, img, r, ref, d


def test_items_cover_every_tile_list_once(dense):
    scene, cam, prm, img, r, ref, d = dense
    lay = B.htgs_workspace_layout(scene.n, cam, prm, r.launch, r.capacity)
    n_items = int(workspace_view(r, lay.n_items, 1, torch.int32).item())
    items = workspace_view(r, lay.items, 4 * n_items, torch.int32).view(-1, 4).cpu().numpy().astype(np.int64)
    ranges = workspace_view(r, lay.ranges, 2 * lay.n_tiles, torch.int32).view(-1, 2).cpu().numpy()
    ranges = ranges.view(np.uint32).astype(np.int64)
    counts = ranges[:, 1] - ranges[:, 0]
    total = int(r.last_instances)
    chunk = max(MIN_CHUNK, -(-total // 2048), -(-2 * total // lay.slots))
    assert counts.sum() == total and n_items <= lay.max_items
    seen = {}
    lengths = []
    for t, k, m, slot0 in items:
        expect_m = -(-counts[t] // chunk) if counts[t] > chunk else 1
        assert m == expect_m, (t, m, expect_m)
        per = -(-counts[t] // m)
        a = min(ranges[t, 0] + k * per, ranges[t, 1])
        lengths.append(min(a + per, ranges[t, 1]) - a)
        seen.setdefault(t, []).append((k, slot0))
    assert sorted(seen) == list(range(lay.n_tiles))
    used = []
    for t, lst in seen.items():
        ks = sorted(k for k, _ in lst)
        m = len(ks)
        assert ks == list(range(m))
        if m > 1:
            slot0 = lst[0][1]
            assert all(s == slot0 for _, s in lst)
            used.append((slot0, slot0 + m))
    assert len(used) > 0, "the scene must split some tiles"
    used.sort()
    for (a0, a1), (b0, _) in zip(used, used[1:]):
        assert a1 <= b0
    assert used[-1][1] <= lay.slots
    # The longest chunks come first.
    assert np.all(np.diff(_bucket(lengths)) >= 0)


def test_split_image_parity(dense):
    scene, cam, prm, img, r, ref, d = dense
    # About 2000 fragments per pixel: the oracle marks 0.13% of the pixels
    # ambiguous (depth ties in the core, cutoff and tau_K decisions).
    image_parity(img, ref, d, "split tiles K=8", 0.0014)


def test_split_core_ids(dense):
    scene, cam, prm, img, r, ref, d = dense
    sv = saved_planes(r, cam, prm.K)
    assert_core_ids(sv, d, scene, cam, prm, label="split tiles K=8")


@pytest.mark.parametrize("K,tile,ppt", [(4, (16, 8), 2), (32, (16, 16), 1), (16, (8, 8), 2), (0, (16, 16), 4),
                                         (8, (32, 16), 2)])
def test_split_launch_shapes(K, tile, ppt):
    scene, cam = _dense(12000, seed=22, degree=0), _camera()
    prm = scenes.Params(K=K)
    img, r, _ = gpu_render(scene, cam, prm, tile=tile, ppt=ppt)
    ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    # Thousands of fragments per pixel put adjacent depths of a large core
    # and cutoff decisions within the oracle's margins on many pixels: it
    # marks 0.17, 0.99, 0.40, 0.16 and 0.16% ambiguous at K = 4, 32, 16, 0, 8.
    cap = {4: 0.0017, 32: 0.0099, 16: 0.0041, 0: 0.0016, 8: 0.0016}[K]
    image_parity(img, ref, d, f"split shapes K={K} {tile} ppt={ppt}", cap)
    if K:
        sv = saved_planes(r, cam, K)
        assert_core_ids(sv, d, scene, cam, prm, label=f"split shapes K={K}")


def test_split_deterministic(dense):
    scene, cam, prm, img, r, ref, d = dense
    again, _, _ = gpu_render(scene, cam, prm)
    assert np.array_equal(img, again)


def test_split_gradients():
    scene = _dense(9000, seed=23, degree=2)
    cam = _camera()
    prm = scenes.Params(K=8, bg=(0.1, 0.2, 0.3))
    _, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    dl = np.random.default_rng(5).standard_normal((cam.height, cam.width, 3))
    dl[d["near_decision"] != 0] = 0.0
    dl = dl.astype(np.float32)
    ref = oracle.render_backward(scene.astype(np.float64), cam, prm, dl.astype(np.float64))
    _, r, g = gpu_render(scene, cam, prm)
    lay = B.htgs_workspace_layout(scene.n, cam, prm, r.launch, r.capacity)
    n_items = int(workspace_view(r, lay.n_items, 1, torch.int32).item())
    assert n_items > lay.n_tiles, "the scene must split some tiles"
    grads = r.backward(g, torch.as_tensor(dl).cuda())
    torch.cuda.synchronize()
    assert_grad_close(grads_to_numpy(grads), ref, label="split tiles K=8")
