"""Workspace management and the torch.autograd.Function over the C ABI.

PyTorch provides device memory and the stream; every step of the render and
of its adjoint runs in libhtgs (hand-written sm_103a kernels).
"""
from __future__ import annotations

import dataclasses

import torch

from . import binding as B

FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")
# Optional training statistics written by the backward (one float per Gaussian).
STATS = ("visibility", "densify_grad", "densify_count")


def _c_grad(grads, stats=None) -> B.GaussiansGrad:
    """htgs_gaussians_grad of gradient tensors and optional statistic tensors
    (see htgs_gaussians_grad: visibility is max-combined, the densification
    sums are added to, so the caller initialises them)."""
    ptrs = [B._ptr(grads[f]).value for f in FIELDS]
    for k in STATS:
        t = (stats or {}).get(k)
        if t is not None and (t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous()):
            raise ValueError(f"{k} must be a contiguous float32 CUDA tensor")
        ptrs.append(B._ptr(t).value if t is not None else None)
    return B.GaussiansGrad(*ptrs)


def _grown_capacity(needed: int, current: int) -> int:
    """Instance capacity after an overflow: 25% headroom, at most the ABI's limit."""
    if needed > B.HTGS_MAX_CAPACITY:
        raise B.HTGSError(B.HTGS_ERR_OVERFLOW, f"{needed} tile instances exceed the {B.HTGS_MAX_CAPACITY} limit; "
                          "split the views over several batches")
    return min(max(int(needed * 1.25) + 1024, current), B.HTGS_MAX_CAPACITY)


@dataclasses.dataclass
class GaussianTensors:
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh: torch.Tensor
    sh_degree: int
    filter_var: torch.Tensor | None = None  # 3D smoothing-filter variance per Gaussian (not trained)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_scene(scene, device="cuda") -> "GaussianTensors":
        def t(a):
            return torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
        fv = getattr(scene, "filter_var", None)
        return GaussianTensors(t(scene.means), t(scene.log_scales), t(scene.quats),
                               t(scene.opacity_logits), t(scene.sh), int(scene.sh_degree),
                               t(fv) if fv is not None else None)

    def c_struct(self) -> B.Gaussians:
        return B.c_gaussians(self.means, self.log_scales, self.quats, self.opacity_logits, self.sh,
                             self.sh_degree, self.filter_var)

    def tensors(self):
        return [getattr(self, f) for f in FIELDS]

    def bake(self, stream=None) -> "BakedGaussians":
        """The scene with its activations (and the 3D filter) folded in, every
        coefficient of a Gaussian in one record (htgs_bake, App. A): renders
        identically, forward only."""
        rec = torch.empty(self.n * B.baked_floats(self.sh_degree), dtype=torch.float32, device=self.means.device)
        B._check(B.htgs_bake(self.c_struct(), rec, stream), "htgs_bake")
        return BakedGaussians(rec, self.n, self.sh_degree)


@dataclasses.dataclass
class BakedGaussians:
    """Baked records of a scene (see GaussianTensors.bake); accepted wherever
    a forward render takes a scene."""
    records: torch.Tensor
    n: int
    sh_degree: int

    def c_struct(self) -> B.Gaussians:
        return B.c_baked(self.records, self.n, self.sh_degree)


class Renderer:
    """Owns the caller-side buffers of one (camera, K, launch) configuration:
    the workspace (binning, sort, records, gradient accumulators) and the
    per-pixel state saved for the backward."""

    def __init__(self, camera, params, n, launch=None, capacity=None, device="cuda"):
        self.camera = camera
        self.params = params
        self.n = int(n)
        self.launch = launch if launch is not None else B.c_launch()
        self.device = torch.device(device)
        self.capacity = int(capacity) if capacity else max(8 * self.n, 1 << 16)
        self.workspace = None
        self.saved = None
        self._alloc()

    def _alloc(self):
        fwd, saved = B.htgs_workspace_size(self.n, self.camera, self.params, self.launch, self.capacity)
        # 256-byte aligned by the caching allocator.
        self.workspace = torch.empty(max(fwd, 256), dtype=torch.uint8, device=self.device)
        self.saved = torch.empty(max(saved // 4, 1), dtype=torch.float32, device=self.device)

    def grow(self, needed: int):
        self.capacity = _grown_capacity(needed, self.capacity)
        self._alloc()

    def image_buffer(self):
        return torch.empty((self.camera.height, self.camera.width, 3), dtype=torch.float32,
                           device=self.device)

    def forward(self, g: GaussianTensors, image=None, save=True, check=True, stream=None):
        """Renders into `image` (allocated when None). With check=True the
        stream is synchronised once to read the device status; on an
        instance overflow the workspace grows and the render is repeated."""
        if image is None:
            image = self.image_buffer()
        cg = g.c_struct()
        for _ in range(4):
            st = B.htgs_render(cg, self.camera, self.params, self.launch, self.workspace, self.capacity,
                               self.saved if save else None, image, stream)
            B._check(st, "htgs_render")
            if not check:
                return image
            dev_status, inst = B.htgs_get_error(self.workspace, stream)
            if dev_status == B.HTGS_ERR_OVERFLOW:
                self.grow(inst)
                continue
            B._check(dev_status, "htgs_render (device)")
            self.last_instances = inst
            return image
        raise B.HTGSError(B.HTGS_ERR_OVERFLOW, "htgs_render")

    def backward(self, g: GaussianTensors, dl_dimage: torch.Tensor, grads=None, stream=None, stats=None):
        """stats: optional dict of float32 (N,) tensors keyed by STATS."""
        dl = dl_dimage.contiguous()
        if dl.dtype != torch.float32 or tuple(dl.shape) != (self.camera.height, self.camera.width, 3):
            raise ValueError("dl_dimage must be float32 of shape (H, W, 3)")
        if grads is None:
            grads = {f: torch.empty_like(getattr(g, f)) for f in FIELDS}
        cgrad = _c_grad(grads, stats)
        st = B.htgs_render_backward(g.c_struct(), self.camera, self.params, self.launch, self.workspace,
                                    self.capacity, self.saved, dl, cgrad, stream)
        B._check(st, "htgs_render_backward")
        return grads

    def status(self, stream=None):
        return B.htgs_get_error(self.workspace, stream)


class RenderFunction(torch.autograd.Function):
    """image = render(means, log_scales, quats, opacity_logits, sh); the
    backward calls htgs_render_backward on the saved per-pixel state."""

    @staticmethod
    def forward(ctx, renderer: Renderer, sh_degree: int, filter_var, means, log_scales, quats, opacity_logits, sh):
        g = GaussianTensors(means.contiguous(), log_scales.contiguous(), quats.contiguous(),
                            opacity_logits.contiguous(), sh.contiguous(), sh_degree, filter_var)
        image = renderer.forward(g, save=True, check=True)
        ctx.renderer = renderer
        ctx.g = g
        return image

    @staticmethod
    def backward(ctx, dl_dimage):
        grads = ctx.renderer.backward(ctx.g, dl_dimage)
        return (None, None, None) + tuple(grads[f] for f in FIELDS)


def render(g: GaussianTensors, renderer: Renderer):
    """Differentiable render of one view (hybrid transparency, Eq. (15))."""
    return RenderFunction.apply(renderer, g.sh_degree, g.filter_var, g.means, g.log_scales, g.quats,
                                g.opacity_logits, g.sh)


class BatchRenderer:
    """Buffers of one batch of views (htgs_render_batch): the workspace and,
    per view, the image and the saved state. Views that share a scene pass
    the same GaussianTensors object; their gradients are summed."""

    def __init__(self, scenes, cameras, params, launch=None, capacity=None, device="cuda", save=True):
        assert len(scenes) == len(cameras) and 1 <= len(cameras) <= B.HTGS_MAX_VIEWS
        self.scenes = list(scenes)
        self.cameras = list(cameras)
        self.params = params
        self.launch = launch if launch is not None else B.c_launch()
        self.device = torch.device(device)
        self.save = save
        n_rec = sum(s.n for s in self.scenes)
        self.capacity = int(capacity) if capacity else max(8 * n_rec, 1 << 16)
        self.images = [torch.empty((c.height, c.width, 3), dtype=torch.float32, device=self.device)
                       for c in self.cameras]
        K = int(params.K)
        self.saved = [torch.empty(((7 + K) * c.width * c.height,), dtype=torch.float32, device=self.device)
                      for c in self.cameras] if save else None
        self._structs = {}
        self._alloc()

    def _struct(self, g):
        key = id(g)
        if key not in self._structs:
            self._structs[key] = g.c_struct()
        return self._structs[key]

    def views(self, dl_dimages=None, grads=None, stats=None):
        gs = [self._struct(s) for s in self.scenes]
        cg = None
        if grads is not None:
            cg = [_c_grad(grads[id(s)], (stats or {}).get(id(s))) for s in self.scenes]
        return B.c_views(gs, self.cameras, self.images, self.saved, dl_dimages, cg)

    def _alloc(self):
        nbytes = B.htgs_batch_workspace_size(self.views(), self.params, self.launch, self.capacity)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)

    def forward(self, check=True, stream=None, views=None):
        views = views if views is not None else self.views()
        for _ in range(4):
            B._check(B.htgs_render_batch(views, self.params, self.launch, self.workspace, self.capacity, stream),
                     "htgs_render_batch")
            if not check:
                return self.images
            st, inst = B.htgs_get_error(self.workspace, stream)
            if st == B.HTGS_ERR_OVERFLOW:
                self.capacity = _grown_capacity(inst, self.capacity)
                self._alloc()
                continue
            B._check(st, "htgs_render_batch (device)")
            self.last_instances = inst
            return self.images
        raise B.HTGSError(B.HTGS_ERR_OVERFLOW, "htgs_render_batch")

    def gradient_buffers(self):
        """One set of gradient tensors per distinct scene (keyed by id)."""
        out = {}
        for s in self.scenes:
            if id(s) not in out:
                out[id(s)] = {f: torch.empty_like(getattr(s, f)) for f in FIELDS}
        return out

    def backward(self, dl_dimages, grads=None, stream=None, stats=None):
        """stats: optional {id(scene): {statistic: float32 (N,) tensor}}."""
        if grads is None:
            grads = self.gradient_buffers()
        dls = [d.contiguous() for d in dl_dimages]
        views = self.views(dl_dimages=dls, grads=grads, stats=stats)
        B._check(B.htgs_render_batch_backward(views, self.params, self.launch, self.workspace, self.capacity,
                                              stream), "htgs_render_batch_backward")
        return grads
