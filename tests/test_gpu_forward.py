"""GPU parity of the forward path through the C ABI against the FP64 oracle
(Sec. 3.2-3.3): image, per-pixel core ids, tile binning, launch-shape
invariance, determinism, edge cases and the overflow protocol."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import GaussianTensors, Renderer
from tests.gpu_util import assert_core_ids, gpu_render, image_parity, saved_planes, workspace_view

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg1():
    scene, cam, prm, tile = scenes.config1()
    cam = cam.rounded()
    img, r, g = gpu_render(scene, cam, prm, tile=tile)
    ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    return scene, cam, prm, tile, img, r, g, ref, d


def test_config1_image_parity(cfg1):
    scene, cam, prm, tile, img, r, g, ref, d = cfg1
    image_parity(img, ref, d, "config1 K=4")


def test_config1_core_ids_match(cfg1):
    """The K-core (ids in depth order) is integer work: identical on every
    pixel without a near-decision, valid within the margins on the others."""
    scene, cam, prm, tile, img, r, g, ref, d = cfg1
    sv = saved_planes(r, cam, prm.K)
    assert assert_core_ids(sv, d, scene, cam, prm, label="config1")["exact"] > 0.99
    ok = d["ambiguous"] == 0
    # T_core per pixel (FP32 vs FP64)
    assert np.abs(sv["T_core"][ok] - d["T_core"][ok]).max() <= 1e-5


def _gpu_tile_lists(r, scene_n, cam, prm):
    """Per-tile record lists of the last render, and the records' tile rectangles."""
    lay = B.htgs_workspace_layout(scene_n, cam, prm, r.launch, r.capacity)
    rect = workspace_view(r, lay.rect, 2 * scene_n, torch.int32).view(scene_n, 2).cpu().numpy().view(np.uint32)
    ranges = workspace_view(r, lay.ranges, 2 * lay.n_tiles, torch.int32).view(-1, 2).cpu().numpy()
    total = int(r.last_instances)
    vals = workspace_view(r, lay.sorted_vals, max(total, 1), torch.int32).cpu().numpy()[:total]
    lists = [vals[a:b] if b > a else vals[:0] for a, b in ranges]
    return lists, rect, lay


def test_config1_binning_matches_oracle(cfg1):
    """Tile lists (Sec. 4.3). With the whole-rectangle cover they equal the
    oracle's binning of the GPU's own rectangles bit for bit. With the
    default ellipse cover each list is the rectangle list with some records
    left out, in the same (ascending gid) order, and no record is left out of
    a tile holding a pixel that the FP64 oracle puts clearly inside its cutoff
    (rho^2 below rho_c by more than the near-decision margin 4e-6 max(1, rho_c)).
    The oracle's covered pixel rectangle lies inside the GPU's tiles."""
    scene, cam, prm, tile, img, r, g, ref, d = cfg1
    tw, th = tile
    n = scene.n
    r_rect = Renderer(cam, prm, n, launch=B.c_launch(tile, tile_cover=B.COVER_RECT))
    img_rect = r_rect.forward(g)
    lists_rect, rect, lay = _gpu_tile_lists(r_rect, n, cam, prm)
    tx0, tx1 = rect[:, 0] & 0xFFFF, rect[:, 0] >> 16
    ty0, ty1 = rect[:, 1] & 0xFFFF, rect[:, 1] >> 16
    empty = tx0 > tx1
    prect = np.stack([tx0 * tw, (tx1 + 1) * tw - 1, ty0 * th, (ty1 + 1) * th - 1], 1).astype(np.int64)
    prect[:, 1] = np.minimum(prect[:, 1], cam.width - 1)
    prect[:, 3] = np.minimum(prect[:, 3], cam.height - 1)
    prect[empty] = [0, -1, 0, -1]
    counts, olists = oracle.bin_tiles(prect, cam.width, cam.height, tw, th)
    assert r_rect.last_instances == int(counts.sum())
    off = 0
    for t in range(lay.n_tiles):
        c = int(counts[t])
        np.testing.assert_array_equal(lists_rect[t], olists[off:off + c])
        off += c
    # Ellipse cover (the render of the fixture): ordered sub-lists.
    lists, rect_e, _ = _gpu_tile_lists(r, n, cam, prm)
    np.testing.assert_array_equal(rect_e, rect)
    assert 0 < r.last_instances <= r_rect.last_instances
    for t in range(lay.n_tiles):
        assert np.all(np.diff(lists[t]) > 0)
        assert np.isin(lists[t], lists_rect[t]).all()
    assert np.array_equal(img, img_rect.cpu().numpy().astype(np.float64))
    # Tiles with a pixel clearly inside the cutoff keep the record.
    sp = oracle.preprocess(scene.astype(np.float64), cam, prm)
    members = [set(map(int, l)) for l in lists]
    tiles_x = lay.tiles_x
    needed = 0
    for gi in np.flatnonzero(sp["valid"]):
        x0, x1, y0, y1 = sp["rect"][gi]
        if x0 > x1 or y0 > y1:
            continue
        assert not empty[gi]
        assert tx0[gi] * tw <= x0 and x1 <= (tx1[gi] + 1) * tw - 1
        assert ty0[gi] * th <= y0 and y1 <= (ty1[gi] + 1) * th - 1
        rc = float(sp["rho_c"][gi])
        tiles = set()
        for y in range(y0, y1 + 1):
            for x in range(x0, x1 + 1):
                t = (y // th) * tiles_x + x // tw
                if t in tiles:
                    continue
                hit, rho2, *_ = oracle.eval_pair(sp, int(gi), x + 0.5, y + 0.5)
                if hit and rho2 <= rc - 4e-6 * max(1.0, rc):
                    tiles.add(t)
        for t in tiles:
            assert int(gi) in members[t], (int(gi), t)
        needed += len(tiles)
    print("COVER config1", {"instances_rect": int(r_rect.last_instances), "instances_ellipse": int(r.last_instances),
                            "tiles_with_inside_pixels": needed})
    assert needed <= r.last_instances


@pytest.mark.parametrize("tile,ppt", [((16, 16), 1), ((16, 16), 4), ((32, 16), 1), ((32, 16), 2), ((16, 8), 2),
                                      ((8, 8), 1), ((8, 8), 2)])
def test_launch_shapes_agree(cfg1, tile, ppt):
    """Tile shape and pixels per thread are tuning knobs: the per-pixel
    arithmetic and the (gid-ascending) traversal order do not change."""
    scene, cam, prm, _, img, *_ = cfg1
    img2, *_ = gpu_render(scene, cam, prm, tile=tile, ppt=ppt)
    assert np.abs(img2 - img).max() <= 1e-6


@pytest.mark.parametrize("batch", [32, 128, 192])
def test_smem_batch_sizes_agree(batch):
    """The records staged per shared-memory batch change only the staging:
    the traversal order and arithmetic are the same, so the image is
    bit-identical (including tiles split into chunks)."""
    scene = scenes.small_box_scene(9000, seed=41, sh_degree=1)
    scene.log_scales += np.float32(0.7)
    cam = scenes.identity_camera(96, 80, 80.0).rounded()
    prm = scenes.Params(K=8)
    ref, *_ = gpu_render(scene, cam, prm)
    g = GaussianTensors.from_scene(scene)
    r = Renderer(cam, prm, scene.n, launch=B.c_launch((16, 16), 1, smem_batch=batch))
    img = r.forward(g).cpu().numpy().astype(np.float64)
    assert np.array_equal(img, ref)


def test_deterministic(cfg1):
    scene, cam, prm, tile, img, r, g, *_ = cfg1
    a = r.forward(g).cpu().numpy()
    b = r.forward(g).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("K", [0, 1, 8, 16, 32])
def test_k_values(K):
    scene = scenes.small_box_scene(300, seed=5, sh_degree=1)
    scene.log_scales += np.float32(0.4)
    cam = scenes.identity_camera(80, 56, 70.0).rounded()
    prm = scenes.Params(K=K, bg=(0.2, 0.3, 0.4))
    img, r, g = gpu_render(scene, cam, prm)
    ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    image_parity(img, ref, d, f"k_values K={K}")
    if K:
        assert_core_ids(saved_planes(r, cam, K), d, scene, cam, prm, label=f"k_values K={K}")


@pytest.mark.parametrize("K", [4, 16])
def test_no_tail_matches_oracle(K):
    """Inference without the tail: the core over the background."""
    scene = scenes.small_box_scene(300, seed=5, sh_degree=1)
    scene.log_scales += np.float32(0.4)
    cam = scenes.identity_camera(80, 56, 70.0).rounded()
    prm = scenes.Params(K=K, bg=(0.2, 0.3, 0.4), no_tail=True)
    img, r, g = gpu_render(scene, cam, prm)
    ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    image_parity(img, ref, d, f"no_tail K={K}")
    sv = saved_planes(r, cam, K)
    assert assert_core_ids(sv, d, scene, cam, prm, label=f"no_tail K={K}")["exact"] > 0.99
    assert np.all(sv["A_tail"] == 0.0)
    with_tail, *_ = gpu_render(scene, cam, scenes.Params(K=K, bg=(0.2, 0.3, 0.4)))
    assert np.abs(with_tail - img).max() > 1e-3


def test_core_ties_broken_by_gid():
    """Exact depth ties (duplicated Gaussians give bit-equal depths in FP32
    and FP64): the core is the K smallest (depth, gid) pairs. Gid order B, B,
    A with A nearer and K = 2 must give (A, first B), also after A evicts a
    tied entry; then a scene where every Gaussian appears three times."""
    base = scenes.small_box_scene(2, seed=31)
    base.means[:] = [[0.0, 0.0, 3.0], [0.0, 0.0, 2.5]]
    base.log_scales[:] = np.float32(-1.5)
    base.opacity_logits[:] = np.float32(0.0)
    tri = base.subset(np.array([0, 0, 1, 0]))          # gids: B B A B
    cam = scenes.identity_camera(32, 32, 40.0).rounded()
    prm = scenes.Params(K=2)
    img, r, g = gpu_render(tri, cam, prm)
    sv = saved_planes(r, cam, 2)
    _, d = oracle.render(tri.astype(np.float64), cam, prm, diagnostics=True)
    both = d["n_core"] == 2
    assert both.sum() > 0
    np.testing.assert_array_equal(sv["core_gid"][both], np.broadcast_to([2, 0], (int(both.sum()), 2)))
    np.testing.assert_array_equal(sv["core_gid"][both], d["core_gid"][both])

    scene = scenes.small_box_scene(40, seed=32, sh_degree=1)
    scene.log_scales += np.float32(0.5)
    order = np.random.default_rng(33).permutation(np.repeat(np.arange(40), 3))
    dup = scene.subset(order)
    cam = scenes.identity_camera(64, 48, 60.0).rounded()
    for K in (2, 4, 8):
        prm = scenes.Params(K=K)
        img, r, g = gpu_render(dup, cam, prm)
        sv = saved_planes(r, cam, K)
        _, d = oracle.render(dup.astype(np.float64), cam, prm, diagnostics=True)
        ok = d["ambiguous"] == 0
        np.testing.assert_array_equal(sv["n_core"][ok], d["n_core"][ok])
        np.testing.assert_array_equal(sv["core_gid"][ok], d["core_gid"][ok])


def test_ragged_image_and_big_splats():
    """Image sizes that are not tile multiples; splats much larger than a tile."""
    scene = scenes.small_box_scene(60, seed=6, sh_degree=2)
    scene.log_scales += np.float32(1.0)
    cam = scenes.Camera(scenes.look_at((0.1, 0.2, -0.4), (0, 0, 3)), 75.0, 70.0, 50.3, 17.9, 0.2, 101, 37).rounded()
    prm = scenes.Params(K=4, bg=(1.0, 0.5, 0.0))
    for tile in [(16, 16), (32, 16), (16, 8), (8, 8)]:
        img, r, g = gpu_render(scene, cam, prm, tile=tile)
        ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
        image_parity(img, ref, d, f"ragged {tile}")


def test_empty_and_culled_scenes():
    cam = scenes.identity_camera(40, 24, 30.0).rounded()
    prm = scenes.Params(K=4, bg=(0.25, 0.5, 0.75))
    empty = scenes.small_box_scene(0, seed=1)
    img, *_ = gpu_render(empty, cam, prm)
    assert np.array_equal(img, np.broadcast_to(np.float32(prm.bg), img.shape).astype(np.float64))
    behind = scenes.small_box_scene(50, seed=2)
    behind.means[:, 2] = -3.0
    img, r, _ = gpu_render(behind, cam, prm)
    assert r.last_instances == 0
    np.testing.assert_allclose(img, np.broadcast_to(prm.bg, img.shape), atol=1e-7)


def test_overflow_is_reported_and_recovered():
    scene, cam, prm, tile = scenes.config1()
    cam = cam.rounded()
    g = GaussianTensors.from_scene(scene)
    r = Renderer(cam, prm, scene.n, launch=B.c_launch(tile), capacity=16)
    img = r.image_buffer()
    st = B.htgs_render(g.c_struct(), cam, prm, r.launch, r.workspace, r.capacity, r.saved, img)
    assert st == B.HTGS_OK
    dev, inst = B.htgs_get_error(r.workspace)
    assert dev == B.HTGS_ERR_OVERFLOW and inst > 16
    img2 = r.forward(g)           # grows the workspace and re-renders
    assert r.last_instances == inst
    ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
    image_parity(img2.cpu().numpy(), ref, d, "overflow recovered")


def test_invalid_arguments_rejected():
    scene, cam, prm, tile = scenes.config1()
    g = GaussianTensors.from_scene(scene)
    r = Renderer(cam, prm, scene.n, launch=B.c_launch(tile))
    img = r.image_buffer()
    bad = scenes.Params(K=33)
    with pytest.raises(B.HTGSError):
        B.htgs_workspace_size(scene.n, cam, bad, r.launch, 100)
    small = r.workspace[:1024]
    assert B.htgs_render(g.c_struct(), cam, prm, r.launch, small, r.capacity, None, img) == B.HTGS_ERR_WORKSPACE
    assert B.htgs_render(g.c_struct(), cam, prm, B.c_launch((32, 32)), r.workspace, r.capacity, None,
                         img) == B.HTGS_ERR_NOT_SUPPORTED
