"""The batched form: many views of uneven resolution, of one scene or of
several scenes of uneven size, in one launch per phase (persistent blend over
a (view, tile) queue), capturable in a CUDA graph. Each view's result must
equal rendering it alone, and the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import FIELDS, BatchRenderer, GaussianTensors, Renderer
from tests.gpu_util import image_parity

pytestmark = pytest.mark.gpu

SIZES = [(80, 60), (123, 77), (64, 64), (200, 150), (33, 47)]


def _cameras(sizes, seed=0):
    rng = np.random.default_rng(seed)
    cams = []
    for w, h in sizes:
        d = rng.standard_normal(3)
        d[2] = -abs(d[2]) - 1.0
        d /= np.linalg.norm(d)
        eye = np.array([0.0, 0.0, 3.0]) + 4.5 * d
        cams.append(scenes.fov_camera(scenes.look_at(eye, (0.0, 0.0, 3.0)), w, h, 60.0).rounded())
    return cams


def _scene(n, seed, degree=1):
    s = scenes.small_box_scene(n, seed=seed, sh_degree=degree)
    s.log_scales -= np.float32(0.5)
    return s


def test_batch_of_views_equals_single_renders():
    scene = _scene(3000, 1)
    g = GaussianTensors.from_scene(scene)
    cams = _cameras(SIZES)
    prm = scenes.Params(K=8, bg=(0.1, 0.2, 0.3))
    br = BatchRenderer([g] * len(cams), cams, prm)
    imgs = [im.clone() for im in br.forward()]
    for cam, img in zip(cams, imgs):
        ref = Renderer(cam, prm, scene.n).forward(g)
        assert float((img - ref).abs().max()) <= 1e-6


def test_batch_of_scenes_equals_single_renders():
    sc = [_scene(n, 10 + i, degree=i % 4) for i, n in enumerate([100, 1000, 5000])]
    gs = [GaussianTensors.from_scene(s) for s in sc]
    cams = _cameras(SIZES[:3], seed=1)
    prm = scenes.Params(K=4)
    br = BatchRenderer(gs, cams, prm, launch=B.c_launch((16, 8), 2))
    imgs = [im.clone() for im in br.forward()]
    for g, cam, img in zip(gs, cams, imgs):
        ref = Renderer(cam, prm, g.n, launch=B.c_launch((16, 8), 2)).forward(g)
        assert float((img - ref).abs().max()) <= 1e-6


def test_batch_view_matches_oracle():
    scene = _scene(1500, 2, degree=2)
    g = GaussianTensors.from_scene(scene)
    cams = _cameras(SIZES[:4], seed=2)
    prm = scenes.Params(K=8, bg=(0.3, 0.3, 0.3))
    imgs = BatchRenderer([g] * len(cams), cams, prm).forward()
    for cam, img in zip(cams, imgs):
        ref, d = oracle.render(scene.astype(np.float64), cam, prm, diagnostics=True)
        image_parity(img.cpu().numpy(), ref, d, f"batch view {cam.width}x{cam.height}")


def test_batch_backward_sums_views_of_one_scene():
    scene = _scene(2000, 3, degree=1)
    g = GaussianTensors.from_scene(scene)
    other = GaussianTensors.from_scene(_scene(700, 4, degree=1))
    cams = _cameras(SIZES[:4], seed=3)
    prm = scenes.Params(K=8)
    views = [g, g, other, g]
    br = BatchRenderer(views, cams, prm)
    br.forward()
    gen = torch.Generator(device="cuda").manual_seed(0)
    dls = [torch.randn(im.shape, device="cuda", generator=gen) for im in br.images]
    grads = br.backward(dls)
    torch.cuda.synchronize()
    want = {f: torch.zeros_like(getattr(g, f)) for f in FIELDS}
    for cam, dl, s in zip(cams, dls, views):
        r = Renderer(cam, prm, s.n)
        r.forward(s)
        single = r.backward(s, dl)
        if s is g:
            for f in FIELDS:
                want[f] += single[f]
        else:
            # Accumulators are atomic float sums over tiles: equal up to summation order.
            for f in FIELDS:
                torch.testing.assert_close(grads[id(other)][f], single[f], rtol=1e-5,
                                           atol=1e-6 * float(single[f].abs().max()))
    for f in FIELDS:
        torch.testing.assert_close(grads[id(g)][f], want[f], rtol=1e-4, atol=1e-6 * float(want[f].abs().max()))


def test_batch_captured_in_cuda_graph():
    scene = _scene(2000, 5)
    g = GaussianTensors.from_scene(scene)
    cams = _cameras(SIZES, seed=4)
    prm = scenes.Params(K=8)
    br = BatchRenderer([g] * len(cams), cams, prm)
    eager = [im.clone() for im in br.forward(check=True)]
    views = br.views()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        br.forward(check=False, views=views)   # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    for im in br.images:
        im.zero_()
    with torch.cuda.graph(graph, stream=stream):
        br.forward(check=False, views=views)
    graph.replay()
    torch.cuda.synchronize()
    st, _ = B.htgs_get_error(br.workspace)
    assert st == B.HTGS_OK
    for a, b in zip(eager, br.images):
        assert torch.equal(a, b)


@pytest.mark.parametrize("n_views,size,tile", [(1, (3840, 2160), (8, 8)), (3, (3840, 2160), (8, 8)),
                                               (2, (64, 48), (16, 16))])
def test_sorted_tile_lists(n_views, size, tile):
    """The radix sort splits the tile-key bits evenly into the fewest passes
    of at most 9 bits: 129,600 tiles of one 4K view at 8x8 take 2 passes of
    9 bits, three such views (388,800 tiles) 3 passes of 7 bits, 24 tiles one
    pass. Sorted keys are non-decreasing, each tile's records ascending (a
    stable sort of the gid-ordered emission) and the ranges delimit them."""
    scene = _scene(3000, 7)
    g = GaussianTensors.from_scene(scene)
    cams = [scenes.fov_camera(scenes.look_at((0.3 * i, 0.0, 0.0), (0.0, 0.0, 3.0)), size[0], size[1], 60.0).rounded()
            for i in range(n_views)]
    prm = scenes.Params(K=4)
    br = BatchRenderer([g] * n_views, cams, prm, launch=B.c_launch(tile, 1))
    br.forward()
    torch.cuda.synchronize()
    lay = B.htgs_batch_workspace_layout(br.views(), prm, br.launch, br.capacity)
    total = int(br.last_instances)
    ws = br.workspace
    keys = ws[lay.sorted_keys: lay.sorted_keys + 4 * total].view(torch.int32).cpu().numpy().astype(np.int64)
    vals = ws[lay.sorted_vals: lay.sorted_vals + 4 * total].view(torch.int32).cpu().numpy().astype(np.int64)
    ranges = ws[lay.ranges: lay.ranges + 8 * lay.n_tiles].view(torch.int32).view(-1, 2).cpu().numpy()
    assert total > 0 and keys.min() >= 0 and keys.max() < lay.n_tiles
    assert np.all(np.diff(keys) >= 0)
    same = np.diff(keys) == 0
    assert np.all(np.diff(vals)[same] > 0)
    starts = np.flatnonzero(np.r_[True, ~same])
    ends = np.r_[starts[1:], total]
    np.testing.assert_array_equal(ranges[keys[starts], 0], starts)
    np.testing.assert_array_equal(ranges[keys[starts], 1], ends)
    # every record of a view appears at most once per tile and belongs to the tile's view
    tiles_per_view = [((c.width + tile[0] - 1) // tile[0]) * ((c.height + tile[1] - 1) // tile[1]) for c in cams]
    view_of_key = np.searchsorted(np.cumsum(tiles_per_view), keys, side="right")
    np.testing.assert_array_equal(vals // scene.n, view_of_key)
    for k, (cam, img) in enumerate(zip(cams, br.images)):
        r = Renderer(cam, prm, scene.n, launch=B.c_launch(tile, 1))
        ref = r.forward(g)
        assert float((img - ref).abs().max()) <= 1e-5


def test_batch_training_step_captured_in_cuda_graph():
    """The whole batched training step in one CUDA graph: the batched
    forward, the per-view L1 loss and its gradient, the batched backward.
    Two scenes share the batch: a 2000-Gaussian scene seen by five views of
    uneven size and a 64-Gaussian scene seen only by a 32x32 crop of the
    1200x800 training camera. The replay equals an eager run of the same
    calls (images and upstream gradients bit for bit; losses and parameter
    gradients up to the order of their atomic sums), and the small scene's
    gradient equals the FP64 oracle's for the upstream gradient the loss
    produced (Sec. 3.3)."""
    import oracle
    from tests.gpu_util import assert_grad_close, grads_to_numpy
    big = _scene(2000, 8)
    small = scenes.small_box_scene(64, seed=2, sh_degree=1)
    small.means[:, :2] *= np.float32(0.04)
    gb, gs = GaussianTensors.from_scene(big), GaussianTensors.from_scene(small)
    crop = scenes.identity_camera(1200, 800, 1200.0).crop(584, 384, 32, 32).rounded()
    cams = _cameras(SIZES, seed=8) + [crop]
    views = [gb] * len(SIZES) + [gs]
    prm = scenes.Params(K=8, bg=(0.1, 0.2, 0.3))
    rng = np.random.Generator(np.random.PCG64(9))
    tb = GaussianTensors.from_scene(scenes.perturbed(big, rng))
    ts = GaussianTensors.from_scene(scenes.perturbed(small, rng))
    targets = [t.clone() for t in BatchRenderer([tb] * len(SIZES) + [ts], cams, prm).forward()]
    br = BatchRenderer(views, cams, prm)
    br.forward(check=True)  # sizes the instance capacity
    dls = [torch.empty_like(im) for im in br.images]
    losses = torch.zeros(len(cams), dtype=torch.float32, device="cuda")
    grads = br.gradient_buffers()
    vf, vb = br.views(), br.views(dl_dimages=dls, grads=grads)

    def step():
        B._check(B.htgs_render_batch(vf, prm, br.launch, br.workspace, br.capacity), "htgs_render_batch")
        for k in range(len(cams)):
            B._check(B.htgs_l1_loss_grad(br.images[k], targets[k], dls[k], losses[k:k + 1]), "l1")
        B._check(B.htgs_render_batch_backward(vb, prm, br.launch, br.workspace, br.capacity),
                 "htgs_render_batch_backward")

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager_img = [im.clone() for im in br.images]
    eager_dl = [d.clone() for d in dls]
    eager_loss = losses.clone()
    eager_grads = {k: {f: v.clone() for f, v in gd.items()} for k, gd in grads.items()}
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        step()
    for t in br.images + dls + [losses] + [v for gd in grads.values() for v in gd.values()]:
        t.zero_()
    graph.replay()
    torch.cuda.synchronize()
    st, _ = B.htgs_get_error(br.workspace)
    assert st == B.HTGS_OK
    for a, b in zip(eager_img, br.images):
        assert torch.equal(a, b)
    for a, b in zip(eager_dl, dls):
        assert torch.equal(a, b)
    # (the loss adds block partial sums atomically: equal up to summation order)
    torch.testing.assert_close(losses, eager_loss, rtol=1e-6, atol=0.0)
    assert float(losses.min()) > 0
    for key, gd in grads.items():
        for f in FIELDS:
            torch.testing.assert_close(gd[f], eager_grads[key][f], rtol=1e-5,
                                       atol=1e-6 * float(eager_grads[key][f].abs().max()))
    # The small scene's gradient against the oracle, for the upstream
    # gradient the captured loss wrote (its near-decision pixels, where FP32
    # and FP64 may choose differently, must not exist in this view).
    _, d = oracle.render(small.astype(np.float64), crop, prm, diagnostics=True)
    assert not d["near_decision"].any()
    dl = dls[-1].cpu().numpy().astype(np.float64)
    ref = oracle.render_backward(small.astype(np.float64), crop, prm, dl)
    assert_grad_close(grads_to_numpy(grads[id(gs)]), ref, label="graph-captured step, small scene")
