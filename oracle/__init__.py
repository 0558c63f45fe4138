"""FP64 CPU oracle for perspective-correct Gaussian splatting with hybrid
transparency (arXiv 2410.08129, Sec. 3.2-3.3).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module; the product path never
does. It wraps ``htgs_oracle.c`` (plain C, double precision, brute force over
every Gaussian for every pixel) through ctypes and shares no code with the
CUDA path.

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  preprocess    -- pinned (bounding box vs brute force and sampled silhouettes,
                   colour vs independent SH, culls vs closed forms)
  eval_pair     -- pinned (closed-form inverse-covariance minimum along the ray,
                   dense ray sampling, on-axis sphere, flat-splat surfel limit)
  render        -- pinned (K >= n with tau_K = 0 equals sorted alpha blending,
                   K = 0 equals the order-independent closed form, equal-colour
                   tails, hand-worked tau_K case, permutation invariance,
                   transmittance bounds, degenerate finiteness)
  render_backward -- pinned (FP64 central finite differences of render)
  sh_basis      -- pinned (quadrature orthonormality, complex-SH identities)
  bin           -- pinned (brute-force tile/rectangle overlap)
  3D filter     -- pinned (density against a quadrature of the convolution
                   integral, rho^2 and alpha from the summed covariance, zero
                   variance is no filter, gradient by central differences)
  no-tail and mean-depth-sorted blending -- pinned (the core's sorted blend
                   over the background; an independent per-pixel blend in
                   mean-depth order with early termination, equal to the
                   hybrid blend when the orders agree; central differences)
  training statistics -- pinned (largest blending weight against a per-pixel
                   recomputation; half distance times the mean gradient norm)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "htgs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhtgs_oracle.so")

_lib = None
_lock = threading.Lock()

AMB_CUTOFF, AMB_TAUK, AMB_AMAX, AMB_CORE_EDGE, AMB_CORE_TIE, AMB_DEN = 1, 2, 4, 8, 16, 32
AMB_TERM, AMB_ORDER = 64, 128


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no GPU involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-Wall", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Gaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("logits", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("filter_var", ctypes.c_void_p)]


class _Camera(ctypes.Structure):
    _fields_ = [("world_to_cam", ctypes.c_double * 16), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("z_near", ctypes.c_double), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class _Params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("tau_alpha", ctypes.c_double), ("tau_K", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("bg", ctypes.c_double * 3), ("no_tail", ctypes.c_int32),
                ("sorted_blend", ctypes.c_int32)]


class _Window(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_int32), ("y0", ctypes.c_int32), ("w", ctypes.c_int32),
                ("h", ctypes.c_int32)]


class _Splat(ctypes.Structure):
    _fields_ = [("valid", ctypes.c_int32), ("cull_reason", ctypes.c_int32),
                ("cull_margin", ctypes.c_double), ("o", ctypes.c_double), ("rho_c", ctypes.c_double),
                ("s", ctypes.c_double * 3), ("q", ctypes.c_double * 4),
                ("R", ctypes.c_double * 9), ("MT", ctypes.c_double * 16),
                ("r1", ctypes.c_double * 4), ("r2", ctypes.c_double * 4), ("r4", ctypes.c_double * 4),
                ("p", ctypes.c_double * 2), ("h", ctypes.c_double * 2),
                ("rect", ctypes.c_int32 * 4),
                ("dir", ctypes.c_double * 3), ("dist", ctypes.c_double),
                ("rgb_raw", ctypes.c_double * 3), ("rgb", ctypes.c_double * 3),
                ("o_raw", ctypes.c_double), ("s_raw", ctypes.c_double * 3), ("filter_var", ctypes.c_double)]


class _Diag(ctypes.Structure):
    _fields_ = [("n_frag", ctypes.c_void_p), ("n_core", ctypes.c_void_p),
                ("core_gid", ctypes.c_void_p), ("T_core", ctypes.c_void_p),
                ("T_tail", ctypes.c_void_p), ("A_tail", ctypes.c_void_p),
                ("c_tail", ctypes.c_void_p), ("ambiguous", ctypes.c_void_p),
                ("frag_hash", ctypes.c_void_p), ("near_decision", ctypes.c_void_p),
                ("amb_effect", ctypes.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            P = ctypes.POINTER
            lib.og_preprocess.argtypes = [P(_Gaussians), P(_Camera), P(_Params), ctypes.c_void_p]
            lib.og_render.argtypes = [P(_Gaussians), P(_Camera), P(_Params), P(_Window),
                                      ctypes.c_void_p, P(_Diag)]
            lib.og_render_boxed.argtypes = [P(_Gaussians), P(_Camera), P(_Params), P(_Window),
                                            ctypes.c_int32, ctypes.c_void_p, P(_Diag),
                                            P(ctypes.c_int64)]
            lib.og_render_splats.argtypes = [ctypes.c_void_p, ctypes.c_int64, P(_Camera), P(_Params),
                                             P(_Window), ctypes.c_void_p, P(_Diag)]
            lib.og_render_backward.argtypes = [P(_Gaussians), P(_Camera), P(_Params), P(_Window),
                                               ctypes.c_void_p] + [ctypes.c_void_p] * 8
            lib.og_eval_pair.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_void_p]
            lib.og_sh_basis.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.og_sh_basis.restype = None
            lib.og_bin.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
            lib.og_bin.restype = ctypes.c_int64
            lib.og_set_threads.argtypes = [ctypes.c_int]
            lib.og_set_threads.restype = None
            lib.og_get_threads.restype = ctypes.c_int
            lib.og_splat_size.restype = ctypes.c_int
            assert lib.og_splat_size() == ctypes.sizeof(_Splat), "splat struct layout mismatch"
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    _load().og_set_threads(int(n))


def get_threads() -> int:
    return int(_load().og_get_threads())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Keep:
    """Holds the float64 copies alive while C uses their pointers."""

    def __init__(self, scene):
        self.means = _f64(scene.means)
        self.log_scales = _f64(scene.log_scales)
        self.quats = _f64(scene.quats)
        self.logits = _f64(scene.opacity_logits)
        self.sh = _f64(scene.sh)
        fv = getattr(scene, "filter_var", None)
        self.filter_var = _f64(fv) if fv is not None else None
        self.g = _Gaussians(self.means.ctypes.data, self.log_scales.ctypes.data,
                            self.quats.ctypes.data, self.logits.ctypes.data, self.sh.ctypes.data,
                            self.means.shape[0], int(scene.sh_degree),
                            self.filter_var.ctypes.data if self.filter_var is not None else None)


def _camera(cam) -> _Camera:
    c = _Camera()
    M = np.asarray(cam.world_to_cam, np.float64).reshape(16)
    for i in range(16):
        c.world_to_cam[i] = float(M[i])
    c.fx, c.fy, c.cx, c.cy, c.z_near = map(float, (cam.fx, cam.fy, cam.cx, cam.cy, cam.z_near))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def _params(p) -> _Params:
    q = _Params()
    q.K = int(p.K)
    q.tau_alpha, q.tau_K, q.alpha_max = float(p.tau_alpha), float(p.tau_K), float(p.alpha_max)
    for i in range(3):
        q.bg[i] = float(p.bg[i])
    q.no_tail = 1 if getattr(p, "no_tail", False) else 0
    q.sorted_blend = 1 if getattr(p, "sorted_blend", False) else 0
    return q


def _window(cam, window):
    if window is None:
        window = (0, 0, cam.width, cam.height)
    x0, y0, w, h = map(int, window)
    return _Window(x0, y0, w, h), (x0, y0, w, h)


SPLAT_DTYPE = np.dtype([("valid", np.int32), ("cull_reason", np.int32), ("cull_margin", np.float64),
                        ("o", np.float64), ("rho_c", np.float64), ("s", np.float64, 3),
                        ("q", np.float64, 4), ("R", np.float64, (3, 3)), ("MT", np.float64, (4, 4)),
                        ("r1", np.float64, 4), ("r2", np.float64, 4), ("r4", np.float64, 4),
                        ("p", np.float64, 2), ("h", np.float64, 2), ("rect", np.int32, 4),
                        ("dir", np.float64, 3), ("dist", np.float64),
                        ("rgb_raw", np.float64, 3), ("rgb", np.float64, 3), ("o_raw", np.float64),
                        ("s_raw", np.float64, 3), ("filter_var", np.float64)], align=True)


def preprocess(scene, cam, params) -> np.ndarray:
    """Per-Gaussian setup (Sec. 3.2): opacity, cutoff, T' rows, bounding box,
    covered pixel rectangle and colour, as a structured array."""
    lib = _load()
    assert SPLAT_DTYPE.itemsize == ctypes.sizeof(_Splat)
    keep = _Keep(scene)
    out = np.zeros(scene.means.shape[0], dtype=SPLAT_DTYPE)
    c, p = _camera(cam), _params(params)
    rc = lib.og_preprocess(ctypes.byref(keep.g), ctypes.byref(c), ctypes.byref(p), out.ctypes.data)
    if rc:
        raise RuntimeError(f"og_preprocess failed ({rc})")
    return out


def eval_pair(splats: np.ndarray, gid: int, xs: float, ys: float):
    """(hit, rho2, z, unclamped alpha, den, num) for one Gaussian and one screen point."""
    lib = _load()
    out = np.zeros(5)
    sp = np.ascontiguousarray(splats[gid:gid + 1])
    hit = lib.og_eval_pair(sp.ctypes.data, float(xs), float(ys), out.ctypes.data)
    return bool(hit), out[0], out[1], out[2], out[3], out[4]


def render(scene, cam, params, window=None, diagnostics: bool = False, box_margin=None):
    """Brute-force FP64 render of a pixel window; returns the (h, w, 3) image,
    plus a dict of per-pixel diagnostics when requested.

    With ``box_margin`` (pixels) only the Gaussians whose FP64 covered-pixel
    rectangle (Sec. 3.2's tight box), grown by that margin, meets the window
    are tested against its pixels; every other pair lies outside the box and
    is rejected by the brute force as well, so the result is the same (the
    tests check this). The diagnostics then also hold ``n_tested``, the
    number of Gaussians tested.

    Diagnostics per pixel: fragment count, core size and ids (depth order),
    T_core, T_tail, A_tail, c_tail, ``near_decision`` (bits of every decision
    within rounding of its threshold), ``ambiguous`` (those whose flip alone
    moves the colour by more than 2e-5) and ``amb_effect`` (the sum over the
    near-decisions of the largest channel move that flipping each one alone
    makes: a per-pixel bound, to first order, on how far a result that takes
    any of them the other way can lie from this one)."""
    lib = _load()
    keep = _Keep(scene)
    c, p = _camera(cam), _params(params)
    win, (x0, y0, w, h) = _window(cam, window)
    img = np.zeros((h, w, 3), np.float64)
    diag = None
    d = {}
    if diagnostics:
        K = max(int(params.K), 1)
        d = dict(n_frag=np.zeros((h, w), np.int32), n_core=np.zeros((h, w), np.int32),
                 core_gid=np.zeros((h, w, K), np.int32), T_core=np.zeros((h, w)),
                 T_tail=np.zeros((h, w)), A_tail=np.zeros((h, w)), c_tail=np.zeros((h, w, 3)),
                 ambiguous=np.zeros((h, w), np.int32), frag_hash=np.zeros((h, w), np.uint64),
                 near_decision=np.zeros((h, w), np.int32), amb_effect=np.zeros((h, w)))
        diag = _Diag(*[d[k].ctypes.data for k in ("n_frag", "n_core", "core_gid", "T_core",
                                                   "T_tail", "A_tail", "c_tail", "ambiguous",
                                                   "frag_hash", "near_decision", "amb_effect")])
    dptr = ctypes.byref(diag) if diag is not None else None
    if box_margin is None:
        rc = lib.og_render(ctypes.byref(keep.g), ctypes.byref(c), ctypes.byref(p), ctypes.byref(win),
                           img.ctypes.data, dptr)
    else:
        tested = ctypes.c_int64(0)
        rc = lib.og_render_boxed(ctypes.byref(keep.g), ctypes.byref(c), ctypes.byref(p),
                                 ctypes.byref(win), int(box_margin), img.ctypes.data, dptr,
                                 ctypes.byref(tested))
        d["n_tested"] = int(tested.value)
    if rc:
        raise RuntimeError(f"og_render failed ({rc})")
    if diagnostics:
        if int(params.K) == 0:
            d["core_gid"] = d["core_gid"][:, :, :0]
        return img, d
    return img


def render_backward(scene, cam, params, dl_dimage, window=None, stats: bool = False):
    """Analytic FP64 gradient of sum(dl_dimage * render(...)) over the window.
    Returns a dict with means, log_scales, quats, opacity_logits and sh; with
    stats=True also the training statistics of the render: visibility (the
    largest blending weight of each Gaussian over the window's pixels),
    densify_grad (|dL/dmean| times half the distance to the camera, for
    Gaussians covering pixels of the view) and densify_count (1 for those)."""
    lib = _load()
    keep = _Keep(scene)
    c, p = _camera(cam), _params(params)
    win, (x0, y0, w, h) = _window(cam, window)
    g = _f64(dl_dimage).reshape(h, w, 3)
    n = scene.means.shape[0]
    out = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacity_logits=np.zeros(n), sh=np.zeros(scene.sh.shape))
    if stats:
        out.update(visibility=np.zeros(n), densify_grad=np.zeros(n), densify_count=np.zeros(n))
    ptr = lambda k: out[k].ctypes.data if stats else None
    rc = lib.og_render_backward(ctypes.byref(keep.g), ctypes.byref(c), ctypes.byref(p),
                                ctypes.byref(win), g.ctypes.data, out["means"].ctypes.data,
                                out["log_scales"].ctypes.data, out["quats"].ctypes.data,
                                out["opacity_logits"].ctypes.data, out["sh"].ctypes.data,
                                ptr("visibility"), ptr("densify_grad"), ptr("densify_count"))
    if rc:
        raise RuntimeError(f"og_render_backward failed ({rc})")
    return out


def sh_basis(dirs: np.ndarray, degree: int = 3):
    """Real SH values (16 per direction, zero above `degree`) and their
    gradients with respect to the (unnormalised) direction components."""
    lib = _load()
    dirs = _f64(dirs).reshape(-1, 3)
    Y = np.zeros((dirs.shape[0], 16))
    dY = np.zeros((dirs.shape[0], 16, 3))
    for i in range(dirs.shape[0]):
        d = np.ascontiguousarray(dirs[i])
        y = np.zeros(16)
        dy = np.zeros((16, 3))
        lib.og_sh_basis(d.ctypes.data, int(degree), y.ctypes.data, dy.ctypes.data)
        Y[i], dY[i] = y, dy
    return Y, dY


def bin_tiles(rects: np.ndarray, width: int, height: int, tile_w: int, tile_h: int):
    """Per-tile instance counts and gid lists (ascending gid within a tile) for
    inclusive pixel rectangles (x_min, x_max, y_min, y_max)."""
    lib = _load()
    rects = np.ascontiguousarray(rects, dtype=np.int32).reshape(-1, 4)
    tx = (width + tile_w - 1) // tile_w
    ty = (height + tile_h - 1) // tile_h
    counts = np.zeros(tx * ty, np.int64)
    total = lib.og_bin(rects.ctypes.data, rects.shape[0], width, height, tile_w, tile_h,
                       counts.ctypes.data, None)
    lists = np.zeros(max(total, 1), np.int32)
    lib.og_bin(rects.ctypes.data, rects.shape[0], width, height, tile_w, tile_h,
               counts.ctypes.data, lists.ctypes.data)
    return counts, lists[:total]
