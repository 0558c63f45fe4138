"""Thin ctypes binding over the C ABI of include/htgs.h.

The functions named like the C entry points (htgs_render, ...) only marshal
arguments: torch tensors become device pointers, scenes.Camera / Params
become the C structs, and torch's current CUDA stream is passed through.
Every step of the render path runs in the CUDA library; if the library is
missing the first call raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

HTGS_OK = 0
HTGS_ERR_INVALID_ARG = 1
HTGS_ERR_WORKSPACE = 2
HTGS_ERR_OVERFLOW = 3
HTGS_ERR_CUDA = 4
HTGS_ERR_TIMEOUT = 5
HTGS_ERR_NOT_SUPPORTED = 6
HTGS_ERR_INTERNAL = 7
HTGS_MAX_K = 32
HTGS_MAX_CAPACITY = (1 << 31) - 1
HTGS_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


class Gaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacity_logits", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("filter_var", ctypes.c_void_p), ("baked", ctypes.c_void_p)]


def baked_floats(sh_degree: int) -> int:
    """Floats per baked Gaussian (HTGS_BAKED_FLOATS)."""
    return 4 * ((12 + 3 * (sh_degree + 1) ** 2 + 3) // 4)


class GaussiansGrad(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacity_logits", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("visibility", ctypes.c_void_p),
                ("densify_grad", ctypes.c_void_p), ("densify_count", ctypes.c_void_p)]


class Camera(ctypes.Structure):
    _fields_ = [("world_to_cam", ctypes.c_float * 16), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("z_near", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("tau_alpha", ctypes.c_float), ("tau_K", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("bg", ctypes.c_float * 3), ("no_tail", ctypes.c_int32),
                ("sorted_blend", ctypes.c_int32)]


class Launch(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("px_per_thread", ctypes.c_int32), ("depth_bits", ctypes.c_int32),
                ("smem_batch", ctypes.c_int32), ("events", ctypes.c_void_p * 6),
                ("test_lookback_stall", ctypes.c_int32), ("binning", ctypes.c_int32),
                ("tile_cover", ctypes.c_int32)]


class Layout(ctypes.Structure):
    _fields_ = [("rec", ctypes.c_uint64), ("rect", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("sorted_keys", ctypes.c_uint64), ("sorted_vals", ctypes.c_uint64),
                ("ranges", ctypes.c_uint64), ("acc", ctypes.c_uint64), ("n_tiles", ctypes.c_int32),
                ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32), ("tile_bits", ctypes.c_int32),
                ("items", ctypes.c_uint64), ("n_items", ctypes.c_uint64), ("partials", ctypes.c_uint64),
                ("max_items", ctypes.c_int32),
                ("slots", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libhtgs.so (building it first if it is absent). Raises when the
    library cannot be built or loaded: there is no other implementation."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                path = _build.build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            L.htgs_workspace_size.argtypes = [ctypes.c_int64, P(Camera), P(Params), P(Launch),
                                              ctypes.c_int64, P(ctypes.c_size_t), P(ctypes.c_size_t)]
            L.htgs_render.argtypes = [P(Gaussians), P(Camera), P(Params), P(Launch), ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
            L.htgs_render_backward.argtypes = [P(Gaussians), P(Camera), P(Params), P(Launch),
                                               ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64,
                                               ctypes.c_void_p, ctypes.c_void_p, P(GaussiansGrad),
                                               ctypes.c_void_p]
            L.htgs_get_error.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                         P(ctypes.c_int32), P(ctypes.c_int64)]
            L.htgs_get_counters.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                             ctypes.c_void_p]
            L.htgs_workspace_layout.argtypes = [ctypes.c_int64, P(Camera), P(Params), P(Launch),
                                                ctypes.c_int64, P(Layout)]
            L.htgs_l1_loss_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.htgs_l1_loss_grad.restype = ctypes.c_int32
            L.htgs_render_static.argtypes = [P(Gaussians), P(Camera), P(Params), P(Launch), ctypes.c_void_p,
                                             ctypes.c_void_p]
            L.htgs_render_static.restype = ctypes.c_int32
            L.htgs_bake.argtypes = [P(Gaussians), ctypes.c_void_p, ctypes.c_void_p]
            L.htgs_fma_probe.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         P(ctypes.c_int64)]
            L.htgs_fma_probe.restype = ctypes.c_int32
            L.htgs_bake.restype = ctypes.c_int32
            L.htgs_status_string.argtypes = [ctypes.c_int32]
            L.htgs_status_string.restype = ctypes.c_char_p
            for f in ("htgs_workspace_size", "htgs_render", "htgs_render_backward", "htgs_get_error",
                      "htgs_workspace_layout", "htgs_get_counters"):
                getattr(L, f).restype = ctypes.c_int32
            _lib = L
    return _lib


class HTGSError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {htgs_status_string(status)} ({status})")
        self.status = status


def _check(status: int, what: str):
    if status != HTGS_OK:
        raise HTGSError(status, what)


def c_camera(cam) -> Camera:
    c = Camera()
    M = np.asarray(cam.world_to_cam, np.float64).reshape(16)
    for i in range(16):
        c.world_to_cam[i] = float(M[i])
    c.fx, c.fy, c.cx, c.cy, c.z_near = (float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy),
                                        float(cam.z_near))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def c_params(p) -> Params:
    q = Params()
    q.K = int(p.K)
    q.tau_alpha, q.tau_K, q.alpha_max = float(p.tau_alpha), float(p.tau_K), float(p.alpha_max)
    for i in range(3):
        q.bg[i] = float(p.bg[i])
    q.no_tail = 1 if getattr(p, "no_tail", False) else 0
    q.sorted_blend = 1 if getattr(p, "sorted_blend", False) else 0
    return q


BINNING_AUTO, BINNING_RADIX, BINNING_COUNTING = 0, 1, 2
# htgs_launch.tile_cover: the tiles of the rectangle the cutoff ellipse reaches
# (row by row), or every tile of the rectangle.
COVER_ELLIPSE, COVER_RECT = 0, 1


def c_launch(tile=(16, 16), px_per_thread=0, depth_bits=0, events=None, smem_batch=0,
             test_lookback_stall=0, binning=BINNING_AUTO, tile_cover=COVER_ELLIPSE) -> Launch:
    """events: up to 6 torch.cuda.Event(enable_timing=True) (or None) recorded
    around the render phases, see htgs_launch in include/htgs.h."""
    L = Launch(int(tile[0]), int(tile[1]), int(px_per_thread), int(depth_bits), int(smem_batch))
    L.test_lookback_stall = int(test_lookback_stall)
    L.binning = int(binning)
    L.tile_cover = int(tile_cover)
    for i, e in enumerate(events or []):
        L.events[i] = e.cuda_event if e is not None else None
    return L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def c_gaussians(means, log_scales, quats, logits, sh, sh_degree, filter_var=None) -> Gaussians:
    for t in (means, log_scales, quats, logits, sh) + ((filter_var,) if filter_var is not None else ()):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("Gaussian parameters must be contiguous float32 CUDA tensors")
    if filter_var is not None and filter_var.numel() != means.shape[0]:
        raise ValueError("filter_var needs one variance per Gaussian")
    return Gaussians(_ptr(means).value, _ptr(log_scales).value, _ptr(quats).value, _ptr(logits).value,
                     _ptr(sh).value, int(means.shape[0]), int(sh_degree),
                     _ptr(filter_var).value if filter_var is not None else None, None)


def c_baked(baked, n, sh_degree) -> Gaussians:
    """A baked scene: n records of baked_floats(sh_degree) floats (htgs_bake)."""
    if baked.dtype != torch.float32 or not baked.is_cuda or not baked.is_contiguous():
        raise ValueError("baked records must be a contiguous float32 CUDA tensor")
    if baked.numel() != n * baked_floats(sh_degree):
        raise ValueError("baked records have the wrong size for n and sh_degree")
    return Gaussians(None, None, None, None, None, int(n), int(sh_degree), None, _ptr(baked).value)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# -- entry points with the C names -------------------------------------------

def htgs_status_string(status: int) -> str:
    return lib().htgs_status_string(int(status)).decode()


def htgs_workspace_size(n, cam, params, launch, capacity):
    fwd = ctypes.c_size_t()
    saved = ctypes.c_size_t()
    st = lib().htgs_workspace_size(int(n), ctypes.byref(c_camera(cam)), ctypes.byref(c_params(params)),
                                   ctypes.byref(launch) if launch is not None else None, int(capacity),
                                   ctypes.byref(fwd), ctypes.byref(saved))
    _check(st, "htgs_workspace_size")
    return int(fwd.value), int(saved.value)


def htgs_workspace_layout(n, cam, params, launch, capacity) -> Layout:
    out = Layout()
    st = lib().htgs_workspace_layout(int(n), ctypes.byref(c_camera(cam)), ctypes.byref(c_params(params)),
                                     ctypes.byref(launch) if launch is not None else None, int(capacity),
                                     ctypes.byref(out))
    _check(st, "htgs_workspace_layout")
    return out


def htgs_render(gaussians: Gaussians, cam, params, launch, workspace, capacity, saved, image, stream=None):
    st = lib().htgs_render(ctypes.byref(gaussians), ctypes.byref(c_camera(cam)), ctypes.byref(c_params(params)),
                           ctypes.byref(launch) if launch is not None else None,
                           _ptr(workspace), workspace.numel() * workspace.element_size(), int(capacity),
                           _ptr(saved) if saved is not None else None, _ptr(image), _stream(stream))
    return int(st)


def htgs_render_backward(gaussians: Gaussians, cam, params, launch, workspace, capacity, saved, dl_dimage,
                         grads: GaussiansGrad, stream=None):
    st = lib().htgs_render_backward(ctypes.byref(gaussians), ctypes.byref(c_camera(cam)),
                                    ctypes.byref(c_params(params)),
                                    ctypes.byref(launch) if launch is not None else None, _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), int(capacity), _ptr(saved),
                                    _ptr(dl_dimage), ctypes.byref(grads), _stream(stream))
    return int(st)


def htgs_get_error(workspace, stream=None):
    status = ctypes.c_int32()
    inst = ctypes.c_int64()
    st = lib().htgs_get_error(_ptr(workspace), workspace.numel() * workspace.element_size(),
                              _stream(stream), ctypes.byref(status), ctypes.byref(inst))
    _check(st, "htgs_get_error")
    return int(status.value), int(inst.value)


def htgs_get_counters(workspace, stream=None):
    out = (ctypes.c_uint64 * 4)()
    st = lib().htgs_get_counters(_ptr(workspace), workspace.numel() * workspace.element_size(),
                                 _stream(stream), out)
    _check(st, "htgs_get_counters")
    return dict(box_pairs=int(out[0]), kept=int(out[1]), admitted=int(out[2]), inserted=int(out[3]))


def htgs_fma_probe(blocks, iters, out, stream=None):
    """Launches the FP32 FMA-chain probe; returns the FMAs per launch."""
    n = ctypes.c_int64(0)
    _check(lib().htgs_fma_probe(int(blocks), int(iters), _ptr(out), _stream(stream), ctypes.byref(n)),
           "htgs_fma_probe")
    return int(n.value)


def htgs_l1_loss_grad(image, target, dl_dimage, loss, stream=None):
    st = lib().htgs_l1_loss_grad(_ptr(image), _ptr(target), int(image.numel()), _ptr(dl_dimage), _ptr(loss),
                                 _stream(stream))
    return int(st)


def htgs_bake(gaussians: Gaussians, baked, stream=None):
    """Bakes raw parameters into records (App. A); returns the status."""
    return int(lib().htgs_bake(ctypes.byref(gaussians), _ptr(baked), _stream(stream)))


def htgs_render_static(gaussians: Gaussians, cam, params, launch, image, stream=None):
    """Forward render whose scratch lives in the library's own fixed-size
    device array: for callers that cannot allocate device memory. Returns the
    status (synchronises the stream)."""
    st = lib().htgs_render_static(ctypes.byref(gaussians), ctypes.byref(c_camera(cam)),
                                  ctypes.byref(c_params(params)),
                                  ctypes.byref(launch) if launch is not None else None, _ptr(image),
                                  _stream(stream))
    return int(st)


# -- batched form --------------------------------------------------------------

HTGS_MAX_VIEWS = 64


class View(ctypes.Structure):
    _fields_ = [("gaussians", ctypes.POINTER(Gaussians)), ("camera", Camera), ("image", ctypes.c_void_p),
                ("saved", ctypes.c_void_p), ("dl_dimage", ctypes.c_void_p),
                ("grads", ctypes.POINTER(GaussiansGrad))]


def c_views(gaussians_structs, cams, images, saved=None, dl_dimages=None, grads=None):
    """Array of htgs_view; the referenced structs are kept alive on the array."""
    n = len(cams)
    arr = (View * n)()
    keep = []
    for i in range(n):
        g = gaussians_structs[i]
        keep.append(g)
        arr[i].gaussians = ctypes.pointer(g)
        arr[i].camera = c_camera(cams[i])
        arr[i].image = _ptr(images[i]) if images is not None and images[i] is not None else None
        arr[i].saved = _ptr(saved[i]) if saved is not None and saved[i] is not None else None
        arr[i].dl_dimage = _ptr(dl_dimages[i]) if dl_dimages is not None else None
        if grads is not None:
            keep.append(grads[i])
            arr[i].grads = ctypes.pointer(grads[i])
    arr._keep = keep
    return arr


def _batch_lib():
    L = lib()
    if not hasattr(L, "_batch_ready"):
        P = ctypes.POINTER
        L.htgs_batch_workspace_size.argtypes = [ctypes.c_int32, P(View), P(Params), P(Launch), ctypes.c_int64,
                                                P(ctypes.c_size_t)]
        L.htgs_batch_workspace_size.restype = ctypes.c_int32
        L.htgs_batch_workspace_layout.argtypes = [ctypes.c_int32, P(View), P(Params), P(Launch), ctypes.c_int64,
                                                  P(Layout)]
        L.htgs_batch_workspace_layout.restype = ctypes.c_int32
        for f in ("htgs_render_batch", "htgs_render_batch_backward"):
            getattr(L, f).argtypes = [ctypes.c_int32, P(View), P(Params), P(Launch), ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.c_int64, ctypes.c_void_p]
            getattr(L, f).restype = ctypes.c_int32
        L._batch_ready = True
    return L


def htgs_batch_workspace_layout(views, params, launch, capacity) -> Layout:
    out = Layout()
    st = _batch_lib().htgs_batch_workspace_layout(len(views), views, ctypes.byref(c_params(params)),
                                                  ctypes.byref(launch) if launch is not None else None,
                                                  int(capacity), ctypes.byref(out))
    _check(st, "htgs_batch_workspace_layout")
    return out


def htgs_batch_workspace_size(views, params, launch, capacity):
    out = ctypes.c_size_t()
    st = _batch_lib().htgs_batch_workspace_size(len(views), views, ctypes.byref(c_params(params)),
                                                ctypes.byref(launch) if launch is not None else None,
                                                int(capacity), ctypes.byref(out))
    _check(st, "htgs_batch_workspace_size")
    return int(out.value)


def htgs_render_batch(views, params, launch, workspace, capacity, stream=None):
    return int(_batch_lib().htgs_render_batch(len(views), views, ctypes.byref(c_params(params)),
                                              ctypes.byref(launch) if launch is not None else None,
                                              _ptr(workspace), workspace.numel() * workspace.element_size(),
                                              int(capacity), _stream(stream)))


def htgs_render_batch_backward(views, params, launch, workspace, capacity, stream=None):
    return int(_batch_lib().htgs_render_batch_backward(len(views), views, ctypes.byref(c_params(params)),
                                                       ctypes.byref(launch) if launch is not None else None,
                                                       _ptr(workspace),
                                                       workspace.numel() * workspace.element_size(),
                                                       int(capacity), _stream(stream)))
