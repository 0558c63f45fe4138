"""Pins for the oracle's per-Gaussian setup (Sec. 3.1 and Sec. 3.2): the tight
perspective bounding box, the opacity-aware cutoff, the near-plane cull, the
spherical-harmonics colour and the tile binning."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2410_08129_gb300 import scenes
from tests import closed_form as cf


def _all_pixels(cam):
    ii, jj = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    return ii.ravel(), jj.ravel()


@pytest.mark.parametrize("which", ["box", "cluster"])
def test_bbox_contains_every_covered_pixel(which):
    """Brute force: every pixel whose ray passes within the cutoff (rho^2 <= rho_c)
    lies inside [p - h, p + h] and inside the covered pixel rectangle."""
    if which == "box":
        scene = scenes.small_box_scene(60, seed=11).astype(np.float64)
        cam = scenes.identity_camera(64, 64, 64.0)
    else:
        scene = scenes.cluster_scene(400, seed=12, sh_degree=0).astype(np.float64)
        scene.log_scales += 2.0  # make them big enough to cover several pixels
        cam = scenes.fov_camera(scenes.look_at((0, 0, -15), (0, 0, 0)), 96, 64, 60.0)
    sp = oracle.preprocess(scene, cam, scenes.Params())
    I, J = _all_pixels(cam)
    n_checked = 0
    for g in np.flatnonzero(sp["valid"]):
        x0, x1, y0, y1 = sp["rect"][g]
        px, py = sp["p"][g]
        hx, hy = sp["h"][g]
        # Only test the pixels near the box (the rest is far outside by construction).
        sel = (I + 0.5 > px - hx - 3) & (I + 0.5 < px + hx + 3) & (J + 0.5 > py - hy - 3) & (J + 0.5 < py + hy + 3)
        for i, j in zip(I[sel], J[sel]):
            hit, rho2, *_ = oracle.eval_pair(sp, int(g), i + 0.5, j + 0.5)
            if hit and rho2 <= sp["rho_c"][g]:
                assert px - hx - 1e-9 <= i + 0.5 <= px + hx + 1e-9
                assert py - hy - 1e-9 <= j + 0.5 <= py + hy + 1e-9
                assert x0 <= i <= x1 and y0 <= j <= y1
                n_checked += 1
    assert n_checked > 200


def test_bbox_is_tight_against_sampled_silhouette():
    """p +- h equal the extremes of the projected cutoff ellipsoid, found by
    projecting dense samples of its surface (no dual quadrics involved)."""
    scene = scenes.small_box_scene(20, seed=13).astype(np.float64)
    cam = scenes.fov_camera(scenes.look_at((0.3, -0.2, -0.5), (0, 0, 3)), 64, 64, 60.0)
    sp = oracle.preprocess(scene, cam, scenes.Params())
    rng = np.random.default_rng(0)
    u = rng.standard_normal((400000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    for g in np.flatnonzero(sp["valid"])[:10]:
        R = cf.rotation(scene.quats[g])
        s = np.exp(scene.log_scales[g])
        pts = scene.means[g] + math.sqrt(sp["rho_c"][g]) * (u * s) @ R.T
        xy = cf.project(cam, pts)
        lo, hi = xy.min(0), xy.max(0)
        p, h = sp["p"][g], sp["h"][g]
        for a in range(2):
            tol = 2e-3 * h[a] + 1e-6
            assert p[a] - h[a] == pytest.approx(lo[a], abs=tol)
            assert p[a] + h[a] == pytest.approx(hi[a], abs=tol)
            # the samples never leave the box
            assert lo[a] >= p[a] - h[a] - 1e-9 and hi[a] <= p[a] + h[a] + 1e-9


def test_bbox_on_axis_sphere_closed_form():
    """Sphere of std sigma on the axis at distance D with cutoff radius
    r = sigma sqrt(rho_c): half extent f r / sqrt(D^2 - r^2) (the tangent cone)."""
    D, sigma, f = 3.0, 0.1, 100.0
    logit = 1.3
    scene = scenes.Scene(np.array([[0.0, 0.0, D]]), np.full((1, 3), math.log(sigma)),
                         np.array([[1.0, 0, 0, 0]]), np.array([logit]), np.zeros((1, 1, 3)), 0)
    cam = scenes.Camera(np.eye(4), f, f, 10.0, 20.0, 0.2, 64, 64)
    prm = scenes.Params()
    sp = oracle.preprocess(scene, cam, prm)
    o = cf.sigmoid(logit)
    rho_c = 2 * math.log(o / prm.tau_alpha)
    assert sp["o"][0] == pytest.approx(o, rel=1e-15)
    assert sp["rho_c"][0] == pytest.approx(rho_c, rel=1e-14)
    r = sigma * math.sqrt(rho_c)
    h = f * r / math.sqrt(D * D - r * r)
    assert sp["p"][0] == pytest.approx([10.0, 20.0], abs=1e-12)
    assert sp["h"][0] == pytest.approx([h, h], rel=1e-12)
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")) as f:
        golden = json.load(f)["bbox_on_axis_sphere"]
    assert sp["h"][0][0] == pytest.approx(golden["expected_h"], abs=1e-6)


def test_culls():
    """rho_c <= 0 (o <= tau_alpha) culls; a cutoff ellipsoid that reaches the
    near plane culls; one that stays in front is kept."""
    prm = scenes.Params()
    lt = math.log(prm.tau_alpha / (1 - prm.tau_alpha))  # sigmoid(lt) = tau_alpha
    sigma = 0.1
    zn = 0.2
    # Near-plane geometry: extent along z is sigma*sqrt(rho_c) for an isotropic sphere.
    o = cf.sigmoid(0.0)
    r = sigma * math.sqrt(2 * math.log(o / prm.tau_alpha))
    means = np.array([[0, 0, 2.0], [0, 0, 2.0], [0, 0, zn + r - 1e-6], [0, 0, zn + r + 1e-6]])
    logits = np.array([lt - 1e-6, lt + 1e-3, 0.0, 0.0])
    scene = scenes.Scene(means, np.full((4, 3), math.log(sigma)), np.tile([1.0, 0, 0, 0], (4, 1)),
                         logits, np.zeros((4, 1, 3)), 0)
    cam = scenes.identity_camera(32, 32, 32.0, z_near=zn)
    sp = oracle.preprocess(scene, cam, prm)
    assert list(sp["valid"]) == [0, 1, 0, 1]
    assert list(sp["cull_reason"]) == [1, 0, 2, 0]


def test_sh_orthonormal_by_quadrature():
    """Gauss-Legendre x uniform-phi quadrature of Y_i Y_j over the sphere is
    the identity (degree <= 3 products are integrated exactly)."""
    nt, nphi = 16, 32
    x, w = np.polynomial.legendre.leggauss(nt)
    phi = np.arange(nphi) * 2 * math.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct * ct)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    weights = (np.repeat(w, nphi) * 2 * math.pi / nphi)
    Y, _ = oracle.sh_basis(dirs, 3)
    G = (Y * weights[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_matches_complex_sph_harm():
    """The 3DGS ordering and signs: real SH from scipy's complex Y_l^m."""
    rng = np.random.default_rng(5)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y, dY = oracle.sh_basis(d, 3)
    np.testing.assert_allclose(Y, cf.sh_real_from_complex(d), atol=1e-12)
    # Gradients by central differences of the polynomial basis.
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        Yp, _ = oracle.sh_basis(d + e, 3)
        Ym, _ = oracle.sh_basis(d - e, 3)
        np.testing.assert_allclose(dY[:, :, j], (Yp - Ym) / (2 * h), atol=1e-7)


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_colour_matches_independent_sh(degree):
    scene = scenes.cluster_scene(50, seed=21, sh_degree=degree).astype(np.float64)
    scene.sh *= 3.0  # large enough that some channels clamp at zero
    scene.sh[:, 0, :] -= 3.0
    cam = scenes.config2_camera()
    sp = oracle.preprocess(scene, cam, scenes.Params())
    clamped = 0
    for g in range(50):
        raw = cf.colour(scene, g, cam)
        np.testing.assert_allclose(sp["rgb_raw"][g], raw, atol=1e-12)
        np.testing.assert_allclose(sp["rgb"][g], np.maximum(raw, 0.0), atol=1e-12)
        clamped += int((raw < 0).sum())
    assert clamped > 0


def test_degree0_is_flat_colour():
    scene, cam, prm, _ = scenes.config1()
    s64 = scene.astype(np.float64)
    sp = oracle.preprocess(s64, cam, prm)
    np.testing.assert_allclose(sp["rgb"], 0.5 + s64.sh[:, 0, :] / (2 * math.sqrt(math.pi)), atol=1e-14)


def test_bin_matches_brute_force_overlap():
    """Tile lists are the tiles overlapping the pixel rectangle, gid ascending."""
    rng = np.random.default_rng(8)
    W, H, tw, th = 70, 45, 16, 8
    n = 300
    x0 = rng.integers(-5, W, n)
    y0 = rng.integers(-5, H, n)
    rects = np.stack([np.maximum(x0, 0), np.minimum(x0 + rng.integers(-2, 30, n), W - 1),
                      np.maximum(y0, 0), np.minimum(y0 + rng.integers(-2, 20, n), H - 1)], 1)
    counts, lists = oracle.bin_tiles(rects, W, H, tw, th)
    tx, ty = -(-W // tw), -(-H // th)
    off = 0
    for t in range(tx * ty):
        ti, tj = t % tx, t // tx
        px0, px1, py0, py1 = ti * tw, ti * tw + tw - 1, tj * th, tj * th + th - 1
        expect = [g for g in range(n) if rects[g, 0] <= rects[g, 1] and rects[g, 2] <= rects[g, 3]
                  and rects[g, 0] <= px1 and rects[g, 1] >= px0 and rects[g, 2] <= py1 and rects[g, 3] >= py0]
        assert counts[t] == len(expect)
        assert list(lists[off:off + counts[t]]) == expect
        off += counts[t]
    assert off == len(lists)
