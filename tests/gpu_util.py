"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300 import scenes
from paper_2410_08129_gb300.renderer import FIELDS, GaussianTensors, Renderer

# Per-channel tolerance of the image (FP32 path vs FP64 oracle).
IMAGE_TOL = 2e-4
# Largest share of pixels on which a near-decision (cutoff, tau_K, depth tie)
# could flip between FP32 and FP64 and move the colour by more than 2e-5;
# those pixels are excluded from the element-by-element comparison.
MAX_AMBIGUOUS = 0.03


def gpu_render(scene, cam, params, tile=(16, 16), ppt=0, capacity=None, save=True):
    assert cam_is_f32(cam), "round the camera with Camera.rounded() so both sides see the same one"
    g = GaussianTensors.from_scene(scene)
    r = Renderer(cam, params, scene.n, launch=B.c_launch(tile, ppt), capacity=capacity)
    img = r.forward(g, save=save)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64), r, g


def cam_is_f32(cam):
    vals = list(np.asarray(cam.world_to_cam, np.float64).ravel()) + [cam.fx, cam.fy, cam.cx, cam.cy, cam.z_near]
    return all(float(np.float32(v)) == float(v) for v in vals)


def saved_planes(r: Renderer, cam, K):
    npix = cam.width * cam.height
    s = r.saved[: (7 + K) * npix].view(7 + K, cam.height, cam.width)
    out = {
        "n_core": s[0].view(torch.int32).cpu().numpy(),
        "T_core": s[1].cpu().numpy(),
        "P": s[2].cpu().numpy(),
        "A_tail": s[3].cpu().numpy(),
        "c_tail": s[4:7].permute(1, 2, 0).cpu().numpy(),
        "core_gid": s[7:7 + K].view(torch.int32).permute(1, 2, 0).cpu().numpy() if K else
        np.zeros((cam.height, cam.width, 0), np.int32),
    }
    return out


# Near-decisions that can change the core's ids without moving the colour
# beyond the tolerance: two core depths within the oracle's tie margin, the
# K-th and (K+1)-th depths, alpha at tau_K. On such pixels more than one core
# list is correct. (A fragment at the cutoff has alpha = tau_alpha < tau_K
# and is never a core candidate.)
CORE_NEAR = oracle.AMB_CORE_TIE | oracle.AMB_CORE_EDGE | oracle.AMB_TAUK


def assert_core_ids(sv, d):
    """The core (integer work) equals the oracle's, ids in depth order, on
    every pixel without an ambiguity and without a near-decision that could
    change it; where the only such decision is a depth tie inside the core
    (the order of nearly equal depths), both lists hold the same ids. Returns
    the fraction of pixels compared exactly."""
    amb = d["ambiguous"] != 0
    near = d["near_decision"] & CORE_NEAR
    ok = ~amb & (near == 0)
    np.testing.assert_array_equal(sv["n_core"][ok], d["n_core"][ok])
    np.testing.assert_array_equal(sv["core_gid"][ok], d["core_gid"][ok])
    tie = ~amb & (near == oracle.AMB_CORE_TIE)
    np.testing.assert_array_equal(sv["n_core"][tie], d["n_core"][tie])
    np.testing.assert_array_equal(np.sort(sv["core_gid"][tie], -1), np.sort(d["core_gid"][tie], -1))
    return float(ok.mean())


def workspace_view(r: Renderer, offset, count, dtype):
    itemsize = torch.tensor([], dtype=dtype).element_size()
    return r.workspace[offset: offset + count * itemsize].view(dtype)


def compare_images(img, ref, amb, tol=IMAGE_TOL):
    """Returns (max error on unambiguous pixels, ambiguous fraction, max error on ambiguous pixels)."""
    err = np.abs(img - ref).max(-1)
    ok = amb == 0
    e_ok = float(err[ok].max()) if ok.any() else 0.0
    e_amb = float(err[~ok].max()) if (~ok).any() else 0.0
    return e_ok, float((~ok).mean()), e_amb


def crop_compare(scene, cam, params, window, img_full, sp=None):
    x0, y0, w, h = window
    ref, d = oracle.render(scene.astype(np.float64), cam, params, window=window, diagnostics=True)
    sub = img_full[y0:y0 + h, x0:x0 + w]
    return compare_images(sub, ref, d["ambiguous"]), ref, d


def grads_to_numpy(grads):
    return {f: grads[f].detach().cpu().numpy().astype(np.float64) for f in FIELDS}


def assert_grad_close(g, ref, rel_norm=1e-3, rel_elem=1e-3, floor=1e-2, names=FIELDS):
    """Per tensor: ||g - ref|| <= rel_norm ||ref||, and elementwise
    |g - ref| <= rel_elem * max(|ref|, floor * max|ref|) (+ a floor for
    all-zero tensors). The elementwise floor reflects FP32 accumulation: an
    element is a sum over pixels whose terms can be as large as the tensor's
    largest entry and cancel, so its absolute error scales with max|ref|,
    not with its own (possibly tiny) value."""
    report = {}
    for f in names:
        a, b = g[f].reshape(-1), ref[f].reshape(-1)
        nb = np.linalg.norm(b)
        mx = np.abs(b).max() if b.size else 0.0
        if nb == 0:
            assert np.abs(a).max() <= 1e-6, (f, np.abs(a).max())
            continue
        rn = np.linalg.norm(a - b) / nb
        bound = rel_elem * np.maximum(np.abs(b), floor * mx) + 1e-9
        worst = float(np.max(np.abs(a - b) / bound))
        report[f] = (rn, worst)
        k = int(np.argmax(np.abs(a - b) / bound))
        detail = dict(field=f, rel_norm=rn, worst=worst, index=k, got=float(a[k]), want=float(b[k]), max_abs=mx)
        assert rn <= rel_norm, detail
        assert worst <= 1.0, detail
    return report
