"""The two tile-binning paths (Sec. 4.3: instances keyed by the tile id
alone) build the same lists. The stable counting sort by tile (computed from
the records' tile rectangles, for one view) and the stable LSD radix sort of
(tile key, record) pairs (the default) must give identical tile ranges,
identical record lists (records in emission order within each tile) and
therefore bit-identical images: for small and ragged views, mean-depth
emission order (sorted blending), the training distribution and the 1080p
frame at four tile shapes."""
import numpy as np
import pytest
import torch

from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import BatchRenderer, GaussianTensors, Renderer
from tests.gpu_util import workspace_view

pytestmark = pytest.mark.gpu


def _lists(r, scene_n, cam, prm):
    """(start, count) per tile, with start set to -1 for empty tiles (whose
    range only needs to be empty), and the record lists."""
    lay = B.htgs_workspace_layout(scene_n, cam, prm, r.launch, r.capacity)
    total = int(r.last_instances)
    ranges = workspace_view(r, lay.ranges, 2 * lay.n_tiles, torch.int32).view(-1, 2).cpu().numpy().astype(np.int64)
    count = ranges[:, 1] - ranges[:, 0]
    start = np.where(count > 0, ranges[:, 0], -1)
    vals = workspace_view(r, lay.sorted_vals, total, torch.int32).cpu().numpy()
    return np.stack([start, count], 1), vals


def _render_both(scene, cam, prm, tile=(16, 16)):
    g = GaussianTensors.from_scene(scene)
    out = {}
    for mode in (B.BINNING_RADIX, B.BINNING_COUNTING):
        r = Renderer(cam, prm, scene.n, launch=B.c_launch(tile, binning=mode))
        img = r.forward(g).clone()
        torch.cuda.synchronize()
        out[mode] = (img, *_lists(r, scene.n, cam, prm), r.last_instances)
    return out


@pytest.mark.parametrize("case", ["config1", "box_16x8", "sorted", "training_32x16", "empty_rows"])
def test_counting_sort_equals_radix_sort(case):
    tile = (16, 16)
    if case == "config1":
        scene, cam, prm, tile = scenes.config1()
    elif case == "box_16x8":
        scene = scenes.small_box_scene(5000, seed=101, sh_degree=1)
        cam, prm, tile = scenes.identity_camera(200, 150, 180.0), scenes.Params(K=8), (16, 8)
    elif case == "sorted":
        scene = scenes.small_box_scene(5000, seed=102, sh_degree=1)
        cam, prm = scenes.identity_camera(160, 120, 150.0), scenes.Params(K=8, sorted_blend=True)
    elif case == "training_32x16":
        scene, _, cam, prm = scenes.config3(n=60_000)
        tile = (32, 16)
    else:  # most records cover nothing; ragged image
        scene = scenes.small_box_scene(9000, seed=103, sh_degree=0)
        scene.means[: 8000, 0] += np.float32(50.0)
        cam, prm = scenes.identity_camera(123, 77, 110.0), scenes.Params(K=4)
    cam = cam.rounded()
    out = _render_both(scene, cam, prm, tile)
    (ia, ra, va, na), (ib, rb, vb, nb) = out[B.BINNING_RADIX], out[B.BINNING_COUNTING]
    assert na == nb > 0
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(va, vb)
    assert torch.equal(ia, ib)


@pytest.mark.parametrize("tile", [(16, 16), (32, 16), (16, 8), (8, 8)])
def test_counting_sort_on_the_headline_frame(tile):
    """1M clustered Gaussians at 1920x1080 (16x16 tiles: 8160 tiles and 3.5M
    instances, in 4 bands of 17 tile rows and 245 blocks of 4096 records;
    8x8: 32400 tiles in 17 bands, 62 blocks of 16384 records). Also prints
    the blend time after each binning path (the lists are the same, so the
    blend must take the same time)."""
    scene, cam, prm = scenes.config2()
    cam = cam.rounded()
    g = GaussianTensors.from_scene(scene)
    out, times = {}, {}
    for mode in (B.BINNING_RADIX, B.BINNING_COUNTING):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        for e in ev:
            e.record()  # torch reads only events it has recorded once
        r = Renderer(cam, prm, scene.n, launch=B.c_launch(tile, 0, 0, ev, binning=mode))
        img = r.forward(g).clone()
        t = []
        for _ in range(10):
            r.forward(g, image=img, save=False, check=False)
            torch.cuda.synchronize()
            t.append((ev[2].elapsed_time(ev[3]), ev[4].elapsed_time(ev[5])))
        times[mode] = np.median(np.array(t), axis=0)
        out[mode] = (img, *_lists(r, scene.n, cam, prm), r.last_instances)
    print("BINNING", tile, {("radix", "counting")[m - 1]: [round(float(x), 4) for x in v] for m, v in times.items()})
    (ia, ra, va, na), (ib, rb, vb, nb) = out[B.BINNING_RADIX], out[B.BINNING_COUNTING]
    assert na == nb > 2_000_000
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(va, vb)
    assert torch.equal(ia, ib)


def test_batch_views_equal_counting_sorted_single_views():
    """Each view of a batch (radix sort) equals the same view rendered alone
    with the counting sort (up to the summation
    order of tiles the batch splits differently: its chunk size depends on
    the batch's instance total)."""
    scene = scenes.small_box_scene(4000, seed=104, sh_degree=1)
    g = GaussianTensors.from_scene(scene)
    other = GaussianTensors.from_scene(scenes.small_box_scene(1500, seed=105, sh_degree=1))
    cams = [scenes.fov_camera(scenes.look_at((0.5 * i - 1.0, 0.2, -1.0), (0.0, 0.0, 3.0)), w, h, 60.0).rounded()
            for i, (w, h) in enumerate([(96, 64), (150, 90), (64, 64), (201, 133)])]
    prm = scenes.Params(K=8)
    views = [g, g, other, g]
    imgs = [im.clone() for im in BatchRenderer(views, cams, prm).forward()]
    for s, cam, img in zip(views, cams, imgs):
        one = Renderer(cam, prm, s.n, launch=B.c_launch((16, 16), binning=B.BINNING_COUNTING)).forward(s)
        assert float((one - img).abs().max()) <= 1e-6


def test_counting_sort_overflow_is_reported_and_recovered():
    scene, cam, prm, tile = scenes.config1()
    cam = cam.rounded()
    g = GaussianTensors.from_scene(scene)
    r = Renderer(cam, prm, scene.n, launch=B.c_launch(tile, binning=B.BINNING_COUNTING), capacity=16)
    img = r.image_buffer()
    st = B.htgs_render(g.c_struct(), cam, prm, r.launch, r.workspace, r.capacity, r.saved, img)
    assert st == B.HTGS_OK
    dev, inst = B.htgs_get_error(r.workspace)
    assert dev == B.HTGS_ERR_OVERFLOW and inst > 16
    img2 = r.forward(g)
    ref = Renderer(cam, prm, scene.n, launch=B.c_launch(tile, binning=B.BINNING_RADIX)).forward(g)
    assert r.last_instances == inst and torch.equal(img2, ref)


def test_counting_sort_needs_a_single_view_with_rows_that_fit():
    """The counting sort serves one view whose tile rows fit a band (2048
    tiles): a 20000-pixel-wide view at 8x8 tiles (2500 per row) and a batch
    of two views are refused when it is requested (the default radix sort
    takes them)."""
    prm = scenes.Params(K=8)
    wide = scenes.identity_camera(20000, 64, 900.0)
    with pytest.raises(B.HTGSError):
        B.htgs_workspace_size(1000, wide, prm, B.c_launch((8, 8), binning=B.BINNING_COUNTING), 10000)
    B.htgs_workspace_size(1000, wide, prm, B.c_launch((8, 8)), 10000)
    g = GaussianTensors.from_scene(scenes.small_box_scene(100, seed=1))
    cams = [scenes.identity_camera(64, 48, 60.0).rounded()] * 2
    br = BatchRenderer([g, g], cams, prm)
    with pytest.raises(B.HTGSError):
        B.htgs_batch_workspace_size(br.views(), prm, B.c_launch((16, 16), binning=B.BINNING_COUNTING), 10000)
