"""Pins of the oracle's forward pass (preprocess, lists, blending) against
closed forms, numbers the paper prints and library routines.

Each test names the passage of Faster-GS (arXiv 2602.09999) it pins."""
import json
import math
import os

import numpy as np
import pytest

from _util import Y00, axis_camera, iso_gaussians, make_params
from paper_2602_09999_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def _render(oracle, cam, params, **kw):
    return oracle.render(cam, params, **kw)


# --------------------------------------------------------------------------
# P1: one isotropic Gaussian on the optical axis (Eq. 1-3, Sec. 3.2 bounds)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("W,H,depth,sigma,o", [(33, 33, 4.0, 0.1, 0.7), (64, 48, 3.0, 0.05, 0.3),
                                               (40, 37, 6.0, 0.3, 0.95)])
def test_p1_isotropic_closed_form(oracle_mod, W, H, depth, sigma, o):
    cam = axis_camera(W, H)
    dc = np.array([[0.3, -0.5, 0.7]])
    p = iso_gaussians([depth], [sigma], [o], dc)
    pre, lists, out = _render(oracle_mod, cam, p)
    f = cam.fx
    s2d = (f * sigma / depth) ** 2                 # Sigma2D = (f sigma / d)^2 I
    shat = s2d + 0.3                               # dilation
    assert pre["xy"][0] == pytest.approx([cam.cx, cam.cy], abs=1e-12)
    assert pre["conic"][0] == pytest.approx([1 / shat, 0.0, 1 / shat], rel=1e-12, abs=1e-15)
    assert pre["aux"][0, 2] == pytest.approx(s2d * s2d, rel=1e-12)        # det Sigma2D
    o64 = 1.0 / (1.0 + math.exp(-float(np.log(o / (1 - o)))))
    k = 2.0 * math.log(255.0 * o64)
    ext = math.sqrt(k * shat)
    assert pre["aux"][0, 5] == pytest.approx(ext, rel=1e-12)
    rgb = np.maximum(Y00 * dc[0] + 0.5, 0.0)
    assert pre["rgb"][0] == pytest.approx(rgb, rel=1e-14)
    # image: alpha = o exp(-r^2 / (2 shat)), contributes iff >= 1/255
    u = np.arange(W) + 0.5
    v = np.arange(H) + 0.5
    r2 = (u[None, :] - cam.cx) ** 2 + (v[:, None] - cam.cy) ** 2
    a = o64 * np.exp(-0.5 * r2 / shat)
    a = np.where(a >= 1 / 255, np.minimum(a, 0.99), 0.0)
    np.testing.assert_allclose(out["image"], a[None] * rgb[:, None, None], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["T_final"], 1.0 - a, rtol=1e-12, atol=1e-15)
    # tiles: those whose box of pixel centres meets the disk of radius ext
    tx, ty = cam.tiles
    expect = []
    for t in range(tx * ty):
        x0, y0 = (t % tx) * 16 + 0.5, (t // tx) * 16 + 0.5
        x1, y1 = min(x0 + 15, W - 0.5), min(y0 + 15, H - 0.5)
        dx = max(x0 - cam.cx, 0.0, cam.cx - x1)
        dy = max(y0 - cam.cy, 0.0, cam.cy - y1)
        if dx * dx + dy * dy <= ext * ext:
            expect.append(t)
    assert sorted(lists["tile"].tolist()) == expect


def test_golden_truncation_radii(oracle_mod):
    """Sec. 2.1 / Sec. 3.2 print ~3.33 sigma for tau = 1/255 at o ~ 1; Suppl.
    C prints ~3.03 sigma where o / tau = 100.  The oracle's opacity-aware
    half-extent divided by the dilated std must reproduce both."""
    gold = json.load(open(GOLDEN))
    cam = axis_camera(65, 65)
    for o, key in [(1.0 - 1e-12, "truncation_sigma_tau_255"),
                   (100.0 / 255.0, "truncation_sigma_tau_100")]:
        p = iso_gaussians([4.0], [0.2], [o], [[0.5, 0.5, 0.5]])
        pre = oracle_mod.preprocess(cam, p)
        shat = (cam.fx * 0.2 / 4.0) ** 2 + 0.3
        ratio = pre["aux"][0, 5] / math.sqrt(shat)
        assert round(ratio, gold[key]["digits"]) == gold[key]["value"], key
    assert gold["tau_alpha"]["value"] == pytest.approx(1 / 255)


# --------------------------------------------------------------------------
# P3: two and three overlapping Gaussians written out by hand (Eq. 4)
# --------------------------------------------------------------------------
def _hand_blend(cam, gs):
    """gs: list of (depth, sigma, o, rgb) in front-to-back order."""
    W, H = cam.width, cam.height
    u = np.arange(W) + 0.5
    v = np.arange(H) + 0.5
    r2 = (u[None, :] - cam.cx) ** 2 + (v[:, None] - cam.cy) ** 2
    C = np.zeros((3, H, W))
    T = np.ones((H, W))
    for d, s, o, c in gs:
        shat = (cam.fx * s / d) ** 2 + 0.3
        a = o * np.exp(-0.5 * r2 / shat)
        a = np.where(a >= 1 / 255, np.minimum(a, 0.99), 0.0)
        C += (a * T)[None] * np.asarray(c)[:, None, None]
        T = T * (1 - a)
    return C, T


def test_p3_overlapping_by_hand(oracle_mod):
    cam = axis_camera(41, 41)
    dcs = np.array([[0.9, -0.2, 0.1], [-0.4, 0.8, 0.3], [0.2, 0.2, -0.9]])
    rgbs = np.maximum(Y00 * dcs + 0.5, 0)
    depths, sigmas, ops = [3.0, 4.0, 5.0], [0.08, 0.15, 0.3], [0.6, 0.5, 0.8]
    for count in (2, 3):
        p = iso_gaussians(depths[:count], sigmas[:count], ops[:count], dcs[:count])
        _, _, out = _render(oracle_mod, cam, p)
        C, T = _hand_blend(cam, [(depths[i], sigmas[i], ops[i], rgbs[i]) for i in range(count)])
        np.testing.assert_allclose(out["image"], C, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(out["T_final"], T, rtol=1e-12, atol=1e-14)
    # swapping depths swaps the blending order
    d2 = [5.0, 4.0, 3.0]
    p = iso_gaussians(d2, sigmas, ops, dcs)
    _, _, out = _render(oracle_mod, cam, p)
    C, _ = _hand_blend(cam, [(d2[i], sigmas[i], ops[i], rgbs[i]) for i in (2, 1, 0)])
    np.testing.assert_allclose(out["image"], C, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# P4: clamp, cutoff and early stop (Suppl. B.1)
# --------------------------------------------------------------------------
def test_p4_alpha_clamp(oracle_mod):
    cam = axis_camera(33, 33)   # odd size: the axis hits pixel (16,16) at its centre
    dc = [[0.4, 0.1, -0.3]]
    p = iso_gaussians([4.0], [0.5], [1 - 1e-5], dc)
    _, _, out = _render(oracle_mod, cam, p)
    rgb = Y00 * np.asarray(dc[0]) + 0.5
    np.testing.assert_allclose(out["image"][:, 16, 16], 0.99 * rgb, rtol=1e-14)
    assert out["T_final"][16, 16] == pytest.approx(0.01, rel=1e-12)


@pytest.mark.parametrize("factor,expect_visible", [(0.999, False), (1.001, True)])
def test_p4_alpha_cutoff(oracle_mod, factor, expect_visible):
    """A Gaussian whose alpha peaks just below / above 1/255 at the nearest
    pixel centre contributes nothing / something."""
    cam = axis_camera(33, 33)
    # det(Sigma2D) well above 1e-6; o just above 1/255 so that the offset r
    # stays below half a pixel and pixel (16, 16) is the nearest centre
    depth, sigma, o = 4.0, 0.02, 0.005
    shat = (cam.fx * sigma / depth) ** 2 + 0.3
    # offset r in pixels so that o exp(-r^2/(2 shat)) = factor / 255
    r = math.sqrt(2 * shat * math.log(255 * o / factor))
    assert r < 0.5
    off = r * depth / cam.fx
    p = iso_gaussians([depth], [sigma], [o], [[0.5, 0.5, 0.5]], offsets=[[off, 0.0]])
    _, _, out = _render(oracle_mod, cam, p)
    assert (out["image"].max() > 0) == expect_visible


def test_p4_early_stop(oracle_mod):
    """Opaque stack at one pixel: T_j = 0.2^j; the 6th entry would take T to
    6.4e-5 < 1e-4, so it is not blended and blending stops (check before
    blend); T_final = 0.2^5 >= 1e-4 and n_contrib = 5."""
    cam = axis_camera(33, 33)
    n = 8
    depths = 3.0 + 0.1 * np.arange(n)
    dcs = np.random.default_rng(0).uniform(-1, 1, (n, 3))
    p = iso_gaussians(depths, [0.3] * n, [0.8] * n, dcs)
    _, lists, out = _render(oracle_mod, cam, p)
    rgb = np.maximum(Y00 * dcs + 0.5, 0)
    expect = sum(0.8 * 0.2 ** j * rgb[j] for j in range(5))
    np.testing.assert_allclose(out["image"][:, 16, 16], expect, rtol=1e-12)
    assert out["T_final"][16, 16] == pytest.approx(0.2 ** 5, rel=1e-12)
    assert out["n_contrib"][16, 16] == 5
    assert out["last_gid"][16, 16] == 4
    assert out["T_final"].min() >= 1e-4


# --------------------------------------------------------------------------
# SH: orthonormality by quadrature (P2), library comparison, derivative
# --------------------------------------------------------------------------
def test_p2_sh_orthonormal_by_quadrature(oracle_mod):
    xg, wg = np.polynomial.legendre.leggauss(12)            # cos(theta) nodes
    phis = np.arange(24) * 2 * np.pi / 24
    G = np.zeros((16, 16))
    for ct, w in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            Y = oracle_mod.sh_basis([st * math.cos(ph), st * math.sin(ph), ct])
            G += w * (2 * np.pi / 24) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_matches_scipy_condon_shortley(oracle_mod):
    """Real SH built from scipy's complex Y_l^m (which includes the
    Condon-Shortley phase): m > 0 -> sqrt2 Re Y_l^m, m < 0 -> sqrt2 Im Y_l^|m|."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(5)
    for _ in range(20):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = oracle_mod.sh_basis(d)
        for l in range(4):
            for m in range(-l, l + 1):
                c = complex(sp.sph_harm_y(l, abs(m), theta, phi))
                ref = c.real if m == 0 else (math.sqrt(2) * (c.real if m > 0 else c.imag))
                assert Y[l * l + l + m] == pytest.approx(ref, abs=1e-12), (l, m)


def test_sh_gradient_matches_finite_differences(oracle_mod):
    rng = np.random.default_rng(6)
    for _ in range(10):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        _, dY = oracle_mod.sh_basis(d, with_grad=True)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = (oracle_mod.sh_basis(d + e) - oracle_mod.sh_basis(d - e)) / (2 * h)
            np.testing.assert_allclose(dY[:, a], fd, atol=1e-8)


def test_p2_sh_degree0_colour_view_independent(oracle_mod):
    p = scenes.tiny_scene(200, seed=3)
    p["sh_rest"][:] = 0
    cams = scenes.orbit_cameras(3, 64, 64, radius=4.0)
    for deg in (0, 3):
        for cam in cams:
            pre = oracle_mod.preprocess(cam, p, sh_degree=deg)
            expect = np.maximum(p["sh_dc"].astype(np.float64) * Y00 + 0.5, 0)
            np.testing.assert_allclose(pre["rgb"], expect, rtol=1e-14)


# --------------------------------------------------------------------------
# P14 + Eq. 2: EWA covariance against a numerical Jacobian of the pinhole
# projection and scipy's quaternion rotation; Cauchy-Binet determinant
# --------------------------------------------------------------------------
def test_p14_ewa_against_numerical_projection(oracle_mod):
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(7)
    cam = scenes.orbit_cameras(1, 320, 240, radius=5.0, seed=9)[0]
    n = 50
    p = make_params(rng.uniform(-1, 1, (n, 3)), rng.normal(-2.5, 0.8, (n, 3)),
                    rng.standard_normal((n, 4)), rng.normal(0, 1, n),
                    rng.uniform(0, 1, (n, 3)), dtype=np.float64)
    pre = oracle_mod.preprocess(cam, p)
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)

    def proj(x):
        c = R @ x + t
        return np.array([cam.fx * c[0] / c[2] + cam.cx, cam.fy * c[1] / c[2] + cam.cy])

    for i in range(n):
        mu = p["means"][i]
        h = 1e-6
        Jn = np.stack([(proj(mu + h * e) - proj(mu - h * e)) / (2 * h) for e in np.eye(3)], 1)
        q = p["quats"][i]
        Rq = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy: scalar last
        S = np.diag(np.exp(p["log_scales"][i]))
        Sig = Rq @ S @ S @ Rq.T
        S2 = Jn @ Sig @ Jn.T
        np.testing.assert_allclose(pre["xy"][i], proj(mu), rtol=1e-12)
        assert pre["aux"][i, 2] == pytest.approx(np.linalg.det(S2), rel=1e-6)
        conic = np.linalg.inv(S2 + 0.3 * np.eye(2))
        np.testing.assert_allclose(pre["conic"][i], [conic[0, 0], conic[0, 1], conic[1, 1]],
                                   rtol=1e-6, atol=1e-12)
        assert pre["depth"][i] == pytest.approx((R @ mu + t)[2], rel=1e-14)


def test_degenerate_gaussians_are_skipped(oracle_mod):
    """Suppl. B.1: |q| < 1e-4 or |Sigma2D| < 1e-6 -> not rendered; behind
    the near plane -> not rendered."""
    cam = axis_camera(33, 33)
    p = iso_gaussians([4.0, 4.0, 0.1, 4.0], [0.2, 1e-5, 0.2, 0.2], [0.5] * 4, [[0.5] * 3] * 4)
    p["quats"][3] = [5e-5, 0, 0, 0]
    pre = oracle_mod.preprocess(cam, p)
    assert pre["visible"].tolist() == [True, False, False, False]
    assert pre["aux"][1, 2] < 1e-6
