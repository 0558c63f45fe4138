"""Tile cover (Sec. 4.3: a Gaussian is binned into the tiles it can reach).
By default a record goes, per tile row of its bounding rectangle, to the span
of tiles its cutoff ellipse reaches; htgs_launch.tile_cover = 1 bins it into
every tile of the rectangle. The ellipse holds every pixel with
rho^2 <= rho_c, so the tiles left out hold no fragment of the record: the
box-pixel, kept and admitted fragment counts are identical, every list is the
rectangle list with records left out (same order), and the image is the same
(bit for bit where no tile list is cut into chunks; the cut depends on the
list lengths, and chunk merging only reorders float sums). Scenes: needles,
discs and sub-pixel splats in every orientation, splats over the image edge,
large splats, sorted blending, the 3D filter, the training distribution, the
1080p frame, and a batch of views; gradients agree as well."""
import numpy as np
import pytest
import torch

from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import BatchRenderer, GaussianTensors, Renderer
from tests.gpu_util import workspace_view
from tests.test_gpu_cull import _thin_scene

pytestmark = pytest.mark.gpu


def _lists(r, n, cam, prm):
    lay = B.htgs_workspace_layout(n, cam, prm, r.launch, r.capacity)
    ranges = workspace_view(r, lay.ranges, 2 * lay.n_tiles, torch.int32).view(-1, 2).cpu().numpy()
    total = int(r.last_instances)
    vals = workspace_view(r, lay.sorted_vals, max(total, 1), torch.int32).cpu().numpy()[:total]
    return [vals[a:b] if b > a else vals[:0] for a, b in ranges]


def _subsequence(y, x):
    """y is x with some entries left out, in the same order."""
    pos = {int(v): i for i, v in enumerate(x)}
    idx = [pos.get(int(v), -1) for v in y]
    return all(i >= 0 for i in idx) and all(b > a for a, b in zip(idx, idx[1:]))


def _both(scene, cam, prm, tile, binning=B.BINNING_AUTO):
    g = GaussianTensors.from_scene(scene)
    out = {}
    for cover in (B.COVER_RECT, B.COVER_ELLIPSE):
        r = Renderer(cam, prm, scene.n, launch=B.c_launch(tile, binning=binning, tile_cover=cover))
        img = r.forward(g).clone()
        torch.cuda.synchronize()
        assert B.htgs_get_error(r.workspace)[0] == B.HTGS_OK
        out[cover] = (img, B.htgs_get_counters(r.workspace), _lists(r, scene.n, cam, prm), int(r.last_instances))
    return out


# Counts that do not depend on how a tile's list is cut into chunks (the core
# insertions do: every chunk starts its partial core empty).
INVARIANT = ("box_pairs", "kept", "admitted")


def _same_fragments(ca, cb):
    return all(ca[k] == cb[k] for k in INVARIANT)


def _check(out, label):
    (ia, ca, la, na), (ib, cb, lb, nb) = out[B.COVER_RECT], out[B.COVER_ELLIPSE]
    assert _same_fragments(ca, cb), (ca, cb)
    assert 0 < nb <= na
    for t, (x, y) in enumerate(zip(la, lb)):
        assert _subsequence(y, x), t
    diff = float((ia - ib).abs().max())
    print("COVER", label, {"instances_rect": na, "instances_ellipse": nb, "removed": round(1 - nb / na, 4),
                           "kept": cb["kept"], "max_image_diff": diff})
    return diff


def _scene_case(case):
    if case == "thin_8x8":
        scene = _thin_scene(4000, seed=81)
        return scene, scenes.identity_camera(256, 192, 256.0), scenes.Params(K=4, bg=(0.2, 0.3, 0.1)), (8, 8)
    if case == "thin_32x16":
        scene = _thin_scene(4000, seed=82)
        return scene, scenes.identity_camera(301, 173, 230.0), scenes.Params(K=8), (32, 16)
    if case == "edges_16x16":  # splats across every image border, some centred outside
        scene = scenes.small_box_scene(6000, seed=83, sh_degree=1)
        scene.means[:, :2] *= np.float32(1.6)
        return scene, scenes.identity_camera(160, 120, 140.0), scenes.Params(K=8), (16, 16)
    if case == "large_16x8":  # splats covering dozens of tiles
        scene = scenes.small_box_scene(1500, seed=84, sh_degree=0)
        scene.log_scales += np.float32(1.3)
        return scene, scenes.identity_camera(200, 150, 180.0), scenes.Params(K=8), (16, 8)
    if case == "sorted":
        scene = _thin_scene(3000, seed=85)
        return scene, scenes.identity_camera(200, 150, 200.0), scenes.Params(K=8, sorted_blend=True), (16, 16)
    if case == "filter":
        scene = _thin_scene(3000, seed=86)
        cam = scenes.identity_camera(200, 150, 200.0)
        scene = scene.with_filter(scenes.filter_variance_from_cameras(scene.means, [cam], scale=3.0))
        return scene, cam, scenes.Params(K=8), (16, 16)
    if case == "training_32x16":
        scene, _, cam, prm = scenes.config3(n=40_000)
        return scene, cam, prm, (32, 16)
    raise KeyError(case)


@pytest.mark.parametrize("case", ["thin_8x8", "thin_32x16", "edges_16x16", "large_16x8", "sorted", "filter",
                                  "training_32x16"])
def test_ellipse_cover_drops_only_empty_tiles(case):
    scene, cam, prm, tile = _scene_case(case)
    cam = cam.rounded()
    out = _both(scene, cam, prm, tile)
    diff = _check(out, case)
    assert diff <= 1e-6


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_ellipse_cover_on_the_headline_frame(tile):
    """1M clustered Gaussians at 1920x1080: identical fragment counts and
    image, and the binning and blend times of both covers."""
    scene, cam, prm = scenes.config2()
    cam = cam.rounded()
    g = GaussianTensors.from_scene(scene)
    res, times = {}, {}
    for cover in (B.COVER_RECT, B.COVER_ELLIPSE):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        for e in ev:
            e.record()  # torch reads only events it has recorded once
        r = Renderer(cam, prm, scene.n, launch=B.c_launch(tile, 0, 0, ev, tile_cover=cover))
        img = r.forward(g).clone()
        t = []
        for _ in range(10):
            r.forward(g, image=img, save=False, check=False)
            torch.cuda.synchronize()
            t.append((ev[2].elapsed_time(ev[3]), ev[4].elapsed_time(ev[5])))
        times[cover] = [round(float(x), 4) for x in np.median(np.array(t), axis=0)]
        res[cover] = (img, B.htgs_get_counters(r.workspace), None, int(r.last_instances))
    (ia, ca, _, na), (ib, cb, _, nb) = res[B.COVER_RECT], res[B.COVER_ELLIPSE]
    print("COVER 1080p", tile, {"instances_rect": na, "instances_ellipse": nb, "removed": round(1 - nb / na, 4),
                                "binning_blend_ms_rect": times[B.COVER_RECT],
                                "binning_blend_ms_ellipse": times[B.COVER_ELLIPSE]})
    assert _same_fragments(ca, cb), (ca, cb)
    assert nb < na
    assert float((ia - ib).abs().max()) <= 1e-6


def test_counting_sort_with_either_cover():
    """The counting sort enumerates the same covers as the radix sort."""
    scene = _thin_scene(4000, seed=87)
    cam, prm = scenes.identity_camera(256, 192, 256.0).rounded(), scenes.Params(K=8)
    for cover in (B.COVER_RECT, B.COVER_ELLIPSE):
        g = GaussianTensors.from_scene(scene)
        imgs, lists = [], []
        for binning in (B.BINNING_RADIX, B.BINNING_COUNTING):
            r = Renderer(cam, prm, scene.n, launch=B.c_launch((16, 16), binning=binning, tile_cover=cover))
            imgs.append(r.forward(g).clone())
            lists.append(_lists(r, scene.n, cam, prm))
        assert torch.equal(imgs[0], imgs[1])
        for x, y in zip(*lists):
            np.testing.assert_array_equal(x, y)


def test_gradients_with_either_cover():
    """The adjoint walks the same lists: gradients agree up to the order of
    the atomic reductions."""
    scene = _thin_scene(2500, seed=88)
    cam, prm = scenes.identity_camera(160, 128, 160.0).rounded(), scenes.Params(K=8)
    g = GaussianTensors.from_scene(scene)
    dl = torch.randn(cam.height, cam.width, 3, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    grads = {}
    for name, cover in (("rect", B.COVER_RECT), ("rect_again", B.COVER_RECT), ("ellipse", B.COVER_ELLIPSE)):
        r = Renderer(cam, prm, scene.n, launch=B.c_launch((16, 16), tile_cover=cover))
        r.forward(g)
        grads[name] = {k: v.clone() for k, v in r.backward(g, dl).items()}

    def rel(x, y):
        a, b = x.double(), y.double()
        return (float((a - b).norm() / (a.norm() + 1e-30)), float((a - b).abs().max() / (a.abs().max() + 1e-30)))

    out = {}
    for k in grads["rect"]:
        rel_norm, rel_max = rel(grads["rect"][k], grads["ellipse"][k])
        out[k] = {"covers": (rel_norm, rel_max), "same_cover_rerun": rel(grads["rect"][k], grads["rect_again"][k])}
        # float32 atomics summed in another order (tens of thousands of terms
        # per Gaussian, with cancellation)
        assert rel_norm <= 1e-5 and rel_max <= 1e-4, (k, rel_norm, rel_max)
    print("COVER gradients", out)


def test_batch_with_either_cover():
    scene = _thin_scene(3000, seed=89)
    other = _thin_scene(1200, seed=90)
    g, h = GaussianTensors.from_scene(scene), GaussianTensors.from_scene(other)
    cams = [scenes.fov_camera(scenes.look_at((0.4 * i - 0.6, 0.1, -1.0), (0.0, 0.0, 3.0)), w, hh, 60.0).rounded()
            for i, (w, hh) in enumerate([(128, 96), (150, 90), (96, 96), (201, 133)])]
    prm = scenes.Params(K=8)
    views = [g, h, g, h]
    out = {}
    for cover in (B.COVER_RECT, B.COVER_ELLIPSE):
        br = BatchRenderer(views, cams, prm, launch=B.c_launch((16, 16), tile_cover=cover))
        out[cover] = ([im.clone() for im in br.forward()], int(br.last_instances))
    assert out[B.COVER_ELLIPSE][1] < out[B.COVER_RECT][1]
    for a, b in zip(out[B.COVER_RECT][0], out[B.COVER_ELLIPSE][0]):
        assert float((a - b).abs().max()) <= 1e-6
