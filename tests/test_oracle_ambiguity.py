"""Pins for the oracle's near-decision and ambiguity classification.

The oracle marks, per pixel, every discrete decision of Sec. 3.2-3.3 that
single precision may take the other way (``near_decision``): the cutoff
rho^2 <= rho_c, core admission alpha >= tau_K (Sec. 4.2), the alpha clamp,
and the depth order at the K-th/(K+1)-th candidate and inside the core. It
then flips each one alone, re-blends the pixel, and marks as ``ambiguous``
those whose flip moves the colour by more than 2e-5; ``amb_effect`` sums the
moves. These choose which pixels the GPU parity tests hold to a per-pixel
bound instead of the plain tolerance, so a wrong flag (for instance one that
marks every pixel holding any fragment near the cutoff) would hide errors.

Every case is built from isotropic Gaussians whose rho^2, alpha and depth at
a pixel follow in closed form from the ray geometry (distance of the centre
from the ray over sigma; the maximum sits at the foot of the perpendicular),
computed here without the oracle. The expected flags and colour moves are
derived from those values and from the compositing rule of Eq. (15)."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_08129_gb300 import scenes
from tests import closed_form as cf

TAU_A = 1.0 / 255.0
W = H = 16
FX = 16.0
CX = CY = 8.5   # the ray through pixel (8, 8) is the optical axis
CUT_REL, TAUK_ABS, AMAX_ABS, DEPTH_REL, EFFECT = 4e-6, 2e-6, 1e-6, 1e-6, 2e-5
Y00 = 0.5 / math.sqrt(math.pi)


def _camera():
    return scenes.Camera(np.eye(4), FX, FX, CX, CY, 0.2, W, H)


def _logit(o):
    return math.log(o / (1.0 - o))


def _scene(spheres):
    """spheres: list of (centre, sigma, opacity, rgb) -> a degree-0 Scene."""
    n = len(spheres)
    means = np.array([s[0] for s in spheres], np.float64).reshape(n, 3)
    log_scales = np.repeat(np.log([[s[1]] for s in spheres]), 3, axis=1)
    quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    logits = np.array([_logit(s[2]) for s in spheres])
    sh = np.array([[(np.asarray(s[3], np.float64) - 0.5) / Y00] for s in spheres])
    return scenes.Scene(means, log_scales, quats, logits, sh, 0)


def _ray(i, j):
    r = np.array([(i + 0.5 - CX) / FX, (j + 0.5 - CY) / FX, 1.0])
    return r / np.linalg.norm(r)


def _rho2_z(centre, sigma, i, j):
    """rho^2 and view depth of the maximum for an isotropic Gaussian."""
    c = np.asarray(centre, np.float64)
    r = _ray(i, j)
    t = c @ r
    return (c @ c - t * t) / sigma ** 2, t * r[2]


def _render(spheres, **kw):
    prm = scenes.Params(**{"K": 4, "bg": (0.0, 0.0, 0.0), **kw})
    img, d = oracle.render(_scene(spheres), _camera(), prm, diagnostics=True)
    return img, d, prm


def _opacity_for_cutoff(rho_c):
    return TAU_A * math.exp(0.5 * rho_c)


def _band_pixels(centre, sigma, rho_c):
    """Pixels whose rho^2 lies within the oracle's cutoff band, and the
    smallest relative distance to the band's edges over all pixels (so that
    a case can check it does not sit on an edge itself)."""
    hit, edge = set(), np.inf
    for j in range(H):
        for i in range(W):
            r2, _ = _rho2_z(centre, sigma, i, j)
            dist = abs(r2 - rho_c) / max(1.0, rho_c)
            edge = min(edge, abs(dist - CUT_REL) / CUT_REL)
            if dist <= CUT_REL:
                hit.add((i, j))
    return hit, edge


def _flagged(mask):
    jj, ii = np.nonzero(mask)
    return set(zip(ii.tolist(), jj.tolist()))


@pytest.mark.parametrize("side", [+1, -1])
def test_cutoff_band_flags_exactly_the_band(side):
    """rho_c placed 2e-6 (relative) above or below rho^2 at pixel (10, 8):
    the four symmetric pixels carry the cutoff bit and no other pixel does;
    the fragment there has alpha ~ tau_alpha, so keeping or dropping it
    moves the colour by alpha * c (> 2e-5): ambiguous, with that move as the
    pixel's budget. A kept fragment is counted, a rejected one is not."""
    centre, sigma, rgb = (0.0, 0.0, 3.0), 0.3, (1.0, 0.5, 0.2)
    r2p, _ = _rho2_z(centre, sigma, 10, 8)
    rho_c = r2p * (1 + side * 2e-6)
    o = _opacity_for_cutoff(rho_c)
    band, edge = _band_pixels(centre, sigma, rho_c)
    assert edge > 0.2
    assert band == {(10, 8), (6, 8), (8, 10), (8, 6)}
    img, d, _ = _render([(centre, sigma, o, rgb)])
    assert _flagged(d["near_decision"] != 0) == band
    assert np.all(d["near_decision"][d["near_decision"] != 0] == oracle.AMB_CUTOFF)
    assert _flagged(d["ambiguous"] != 0) == band
    assert np.all(d["ambiguous"][d["ambiguous"] != 0] == oracle.AMB_CUTOFF)
    alpha = o * math.exp(-0.5 * r2p)
    assert alpha == pytest.approx(TAU_A, rel=1e-4)
    for (i, j) in band:
        assert d["amb_effect"][j, i] == pytest.approx(alpha * max(rgb), rel=1e-9)
        assert d["n_frag"][j, i] == (1 if side > 0 else 0)
    assert np.all(d["amb_effect"][d["near_decision"] == 0] == 0.0)


@pytest.mark.parametrize("rel", [1e-5, -1e-5, 1e-4])
def test_cutoff_just_outside_the_band_is_not_flagged(rel):
    """rho_c 1e-5 or 1e-4 (relative) away from rho^2 at pixel (10, 8): the
    band (4e-6) does not reach it and no pixel is flagged."""
    centre, sigma = (0.0, 0.0, 3.0), 0.3
    r2p, _ = _rho2_z(centre, sigma, 10, 8)
    rho_c = r2p * (1 + rel)
    band, edge = _band_pixels(centre, sigma, rho_c)
    assert not band and edge > 0.2
    img, d, _ = _render([(centre, sigma, _opacity_for_cutoff(rho_c), (1.0, 0.5, 0.2))])
    assert not d["near_decision"].any() and not d["ambiguous"].any()
    assert d["n_frag"][8, 10] == (1 if rel > 0 else 0)


def test_cutoff_band_without_colour_move_is_not_ambiguous():
    """The same band with the splat's colour equal to the background: the
    decision is near (flagged) but neither side moves the colour."""
    centre, sigma, rgb = (0.0, 0.0, 3.0), 0.3, (0.25, 0.5, 0.75)
    r2p, _ = _rho2_z(centre, sigma, 10, 8)
    o = _opacity_for_cutoff(r2p * (1 + 2e-6))
    img, d, _ = _render([(centre, sigma, o, rgb)], bg=rgb)
    assert _flagged(d["near_decision"] != 0) == {(10, 8), (6, 8), (8, 10), (8, 6)}
    assert not d["ambiguous"].any()
    assert d["amb_effect"].max() < 1e-12


def test_fragment_away_from_the_cutoff_is_not_flagged():
    """A splat whose cutoff lies between pixel rings (no pixel within 1e-3
    of it) leaves every pixel unflagged, although many pixels hold its
    faint fragments (alpha within a factor 2 of tau_alpha)."""
    centre, sigma = (0.0, 0.0, 3.0), 0.3
    r2a, _ = _rho2_z(centre, sigma, 10, 8)
    r2b, _ = _rho2_z(centre, sigma, 11, 8)
    rho_c = 0.5 * (r2a + r2b)
    o = _opacity_for_cutoff(rho_c)
    img, d, _ = _render([(centre, sigma, o, (1.0, 1.0, 1.0))])
    faint = [(i, j) for j in range(H) for i in range(W)
             if 0.5 * rho_c <= _rho2_z(centre, sigma, i, j)[0] <= rho_c]
    assert len(faint) >= 8
    assert not d["near_decision"].any() and not d["ambiguous"].any()


def test_tau_k_flag_and_its_effect():
    """alpha = tau_K + 1e-6 at the centre pixel. Alone, core or tail give the
    same colour (a single fragment over the background), so the pixel is
    near but not ambiguous. With an opaque-ish splat behind it and K = 1,
    the front splat decides which of the two is the core: the flip moves
    the colour and the budget equals the difference of the two
    compositions of Eq. (15)."""
    tau_K = 0.05
    front = ((0.0, 0.0, 3.0), 0.3, tau_K + 1e-6, (1.0, 0.0, 0.0))
    img, d, _ = _render([front], K=1, tau_K=tau_K)
    assert _flagged(d["near_decision"] != 0) == {(8, 8)}
    assert d["near_decision"][8, 8] == oracle.AMB_TAUK
    assert not d["ambiguous"].any() and d["amb_effect"][8, 8] < 1e-12

    back_a, back_c = 0.6, np.array([0.0, 0.0, 1.0])
    back = ((0.0, 0.0, 4.0), 0.3, back_a, tuple(back_c))
    img, d, _ = _render([front, back], K=1, tau_K=tau_K)
    assert d["near_decision"][8, 8] == oracle.AMB_TAUK
    assert d["ambiguous"][8, 8] == oracle.AMB_TAUK
    a, ca = front[2], np.array(front[3])
    # core = front, tail = back (one tail fragment composites like Eq. (2))
    c_front = a * ca + (1 - a) * back_a * back_c
    # front forced into the tail: core = back, tail = front
    c_back = back_a * back_c + (1 - back_a) * a * ca
    np.testing.assert_allclose(img[8, 8], c_front, rtol=1e-9, atol=1e-12)
    assert d["amb_effect"][8, 8] == pytest.approx(np.abs(c_front - c_back).max(), rel=1e-6)


def test_alpha_clamp_is_near_but_never_ambiguous():
    """o e^{-rho^2/2} = alpha_max + 5e-7 at the centre pixel: the clamp is a
    near-decision (it changes the gradient), but alpha = min(., alpha_max)
    is continuous, so the colour cannot move and the pixel is not ambiguous."""
    img, d, prm = _render([((0.0, 0.0, 3.0), 0.3, 0.999 + 5e-7, (1.0, 1.0, 1.0))])
    assert _flagged(d["near_decision"] != 0) == {(8, 8)}
    assert d["near_decision"][8, 8] == oracle.AMB_AMAX
    assert not d["ambiguous"].any()
    np.testing.assert_allclose(img[8, 8], prm.alpha_max, rtol=1e-12)


@pytest.mark.parametrize("same_colour", [False, True])
def test_core_edge_tie(same_colour):
    """K = 1 and two splats whose depths differ by 4e-7 (relative) on every
    ray: wherever both are core candidates the K-th and (K+1)-th candidate
    depths are within the oracle's 1e-6 margin (edge bit). Swapping them
    moves the colour by alpha_A alpha_B (c_A - c_B), zero for equal colours."""
    ca = np.array([1.0, 0.2, 0.0])
    cb = ca if same_colour else np.array([0.0, 0.4, 1.0])
    A = ((0.0, 0.0, 3.0), 0.3, 0.5, tuple(ca))
    Bs = ((0.0, 0.0, 3.0 * (1 + 4e-7)), 0.3, 0.45, tuple(cb))
    img, d, prm = _render([A, Bs], K=1)
    both = set()
    for j in range(H):
        for i in range(W):
            ra, za = _rho2_z(A[0], A[1], i, j)
            rb, zb = _rho2_z(Bs[0], Bs[1], i, j)
            aa, ab = A[2] * math.exp(-0.5 * ra), Bs[2] * math.exp(-0.5 * rb)
            assert abs(zb - za) / za == pytest.approx(4e-7, rel=1e-3)
            if aa >= prm.tau_K and ab >= prm.tau_K:
                both.add((i, j))
                expect = aa * ab * np.abs(ca - cb).max()
                assert d["amb_effect"][j, i] == pytest.approx(expect, rel=1e-6, abs=1e-15)
    assert len(both) >= 5
    assert _flagged(d["near_decision"] & oracle.AMB_CORE_EDGE) == both
    assert not (d["near_decision"] & ~oracle.AMB_CORE_EDGE).any()
    amb = _flagged(d["ambiguous"] != 0)
    assert amb == (set() if same_colour else both)


def test_core_tie_inside_the_core_and_clear_gaps():
    """K = 2: two near-equal depths inside the core (tie bit, moving the
    colour by alpha_A alpha_B (c_A - c_B) as the colour behind them is shared),
    a third splat far behind (no edge bit: its depth is 30% away)."""
    ca, cb, cc = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0])
    A = ((0.0, 0.0, 3.0), 0.3, 0.5, tuple(ca))
    Bs = ((0.0, 0.0, 3.0 * (1 + 3e-7)), 0.3, 0.4, tuple(cb))
    C = ((0.0, 0.0, 4.0), 0.3, 0.7, tuple(cc))
    img, d, _ = _render([A, Bs, C], K=2)
    assert d["near_decision"][8, 8] == oracle.AMB_CORE_TIE
    assert d["ambiguous"][8, 8] == oracle.AMB_CORE_TIE
    assert d["amb_effect"][8, 8] == pytest.approx(0.5 * 0.4 * 1.0, rel=1e-6)
    # Core (depth order) is A then B; the tail is C.
    assert list(d["core_gid"][8, 8]) == [0, 1]
    # A 1e-5 gap is outside the margin: nothing is flagged.
    B2 = ((0.0, 0.0, 3.0 * (1 + 1e-5)), 0.3, 0.4, tuple(cb))
    img, d, _ = _render([A, B2, C], K=2)
    assert not d["near_decision"].any() and not d["ambiguous"].any()


def test_random_scene_flags_only_real_events():
    """A generic scene: every near-decision bit the oracle sets (or not) is
    recomputed here from the inverse-covariance fragments of every pixel.
    With no event within the margins, no pixel may be flagged."""
    scene = scenes.small_box_scene(24, seed=77, sh_degree=0).astype(np.float64)
    scene.log_scales += 0.6
    cam = scenes.identity_camera(20, 16, 20.0)
    prm = scenes.Params(K=3)
    img, d = oracle.render(scene, cam, prm, diagnostics=True)
    M = np.asarray(cam.world_to_cam)
    deep = 0
    for j in range(cam.height):
        for i in range(cam.width):
            bits = 0
            cand = []
            nfr = 0
            for g in range(scene.n):
                o = float(cf.sigmoid(scene.opacity_logits[g]))
                rho_c = 2 * math.log(o / prm.tau_alpha)
                if rho_c <= 0:
                    continue
                R = cf.rotation(scene.quats[g])
                A = M[:3, :3] @ R @ np.diag(np.exp(scene.log_scales[g]))
                zc = (M @ np.append(scene.means[g], 1))[2]
                if zc - math.sqrt(rho_c * (A[2] ** 2).sum()) <= cam.z_near:
                    continue
                rho2, z, a_raw = cf.fragment(scene, g, cam, i + 0.5, j + 0.5)
                if abs(rho2 - rho_c) <= CUT_REL * max(1.0, rho_c):
                    bits |= oracle.AMB_CUTOFF
                if rho2 > rho_c:
                    continue
                nfr += 1
                alpha = min(a_raw, prm.alpha_max)
                if abs(alpha - prm.tau_K) <= TAUK_ABS:
                    bits |= oracle.AMB_TAUK
                if abs(a_raw - prm.alpha_max) <= AMAX_ABS:
                    bits |= oracle.AMB_AMAX
                if alpha >= prm.tau_K:
                    cand.append((z, g))
            cand.sort()
            K = prm.K
            if len(cand) > K and abs(cand[K][0] - cand[K - 1][0]) <= DEPTH_REL * abs(cand[K - 1][0]):
                bits |= oracle.AMB_CORE_EDGE
            for a, b in zip(cand[:K], cand[1:K]):
                if abs(b[0] - a[0]) <= DEPTH_REL * abs(a[0]):
                    bits |= oracle.AMB_CORE_TIE
            deep += nfr > K
            assert d["n_frag"][j, i] == nfr
            assert d["near_decision"][j, i] == bits, (i, j)
            assert d["ambiguous"][j, i] & ~bits == 0
    assert deep >= 20
    assert not d["near_decision"].any()  # a generic scene has no event within the margins


def test_sorted_blend_order_flip():
    """Mean-depth-sorted blending (Tab. 3 variant): two splats whose mean
    depths differ by 4e-7 (relative). Their order is a near-decision; the
    swap moves the colour by alpha_A alpha_B (c_A - c_B)."""
    ca, cb = np.array([1.0, 0.3, 0.0]), np.array([0.0, 0.3, 1.0])
    A = ((0.0, 0.0, 3.0), 0.3, 0.5, tuple(ca))
    Bs = ((0.0, 0.0, 3.0 * (1 + 4e-7)), 0.3, 0.6, tuple(cb))
    img, d, _ = _render([A, Bs], sorted_blend=True)
    assert d["near_decision"][8, 8] & oracle.AMB_ORDER
    assert d["ambiguous"][8, 8] == oracle.AMB_ORDER
    assert d["amb_effect"][8, 8] == pytest.approx(0.5 * 0.6 * 1.0, rel=1e-6)
    np.testing.assert_allclose(img[8, 8], 0.5 * ca + 0.5 * 0.6 * cb, rtol=1e-9)


@pytest.mark.parametrize("inside", [True, False])
def test_sorted_blend_termination_flip(inside):
    """Early termination: with alpha_A = 0.99 in front, the second splat's
    alpha puts T (1 - alpha_B) 3e-7 (relative) above or below the 1e-4 stop
    threshold. Blending it or not moves the colour by 0.01 alpha_B c_B; the
    pixel is flagged, and its budget is that move."""
    aa = 0.99
    ab = 1.0 - 0.01 * (1 + (3e-7 if inside else -3e-7))
    ca, cb = np.array([0.2, 0.2, 0.2]), np.array([1.0, 0.5, 0.0])
    A = ((0.0, 0.0, 3.0), 0.3, aa, tuple(ca))
    Bs = ((0.0, 0.0, 3.5), 0.3, ab, tuple(cb))
    img, d, _ = _render([A, Bs], sorted_blend=True)
    assert d["near_decision"][8, 8] & oracle.AMB_TERM
    assert d["ambiguous"][8, 8] == oracle.AMB_TERM
    assert d["amb_effect"][8, 8] == pytest.approx(0.01 * ab * 1.0, rel=1e-6)
    expect = aa * ca + ((1 - aa) * ab * cb if inside else 0.0)
    np.testing.assert_allclose(img[8, 8], expect, rtol=1e-9, atol=1e-15)
    assert d["n_core"][8, 8] == (2 if inside else 1)
