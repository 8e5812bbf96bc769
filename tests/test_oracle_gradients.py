"""Pins of the oracle's analytic backward (the exact adjoint of the blend and
of the preprocessing) against central finite differences of its own forward
(P12) and the dot-product test (P13).  Scenes are chosen away from the kinks
of the method: every threshold decision has a relative margin above 1e-3,
no colour channel is clamped, opacities stay below 0.9."""
import numpy as np
import pytest

from paper_2602_09999_gb300 import scenes

NAMES = ("means", "log_scales", "quats", "opacity", "sh_dc", "sh_rest")


def _clean_scene(oracle, n, W, H, seed0=0, depth_spread=1.0):
    """First seeded scene whose decisions all have margin > 1e-3."""
    m = oracle.Margins(rel=1e-3, px=1e-3, t_rel=1e-3, depth_rel=1e-3)
    for seed in range(seed0, seed0 + 200):
        p = scenes.small_scene(n, seed, spread=0.6, log_scale_mean=-2.2, log_scale_std=0.3,
                               opacity_mean=0.0, opacity_std=0.8)
        p = {k: v.astype(np.float64) for k, v in p.items()}
        p["opacity"] = np.minimum(p["opacity"], 2.0)        # o <= 0.88
        cam = scenes.look_at((0.3, -0.2, 4.0), (0.0, 0.0, 0.0), W, H)
        pre, lists, out = oracle.render(cam, p, margins=m)
        vis = pre["visible"]
        if vis.sum() < n or out["ambiguous"].any() or pre["clamped"][vis].any():
            continue
        if np.any(lists["flags"] & oracle.IMARGINAL):
            continue
        return p, cam
    pytest.skip("no clean scene found")


def _image(oracle, cam, p, bg):
    _, _, out = oracle.render(cam, p, bg=bg)
    return out["image"]


def _loss(oracle, cams, p, targets, lam, bg):
    tot = 0.0
    for cam, t in zip(cams, targets):
        L, _ = oracle.loss(_image(oracle, cam, p, bg), t, lam)
        tot += L / len(cams)
    return tot


@pytest.mark.parametrize("n,lam,bg", [(1, 0.2, (0.0, 0.0, 0.0)), (4, 0.2, (0.2, 0.5, 0.9)),
                                      (8, 0.0, (0.0, 0.0, 0.0))])
def test_p12_directional_finite_differences(oracle_mod, n, lam, bg):
    p, cam = _clean_scene(oracle_mod, n, 32, 32, seed0=10 * n)
    tgt = scenes.target_image(32, 32, view=n)
    loss, _, grads, _, _ = oracle_mod.train_step([cam], p, [tgt], lam=lam, bg=bg)
    rng = np.random.default_rng(n)
    for name in NAMES:
        v = rng.standard_normal(p[name].shape)
        h = 1e-6 * max(1.0, float(np.abs(p[name]).max()))
        pp = dict(p)
        pp[name] = p[name] + h * v
        Lp = _loss(oracle_mod, [cam], pp, [tgt], lam, bg)
        pp[name] = p[name] - h * v
        Lm = _loss(oracle_mod, [cam], pp, [tgt], lam, bg)
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(grads[name] * v))
        assert an == pytest.approx(fd, rel=2e-5, abs=1e-12), name


def test_p12_elementwise_finite_differences(oracle_mod):
    """Every scalar parameter of 2 Gaussians, two views (gradients summed,
    loss averaged over the batch)."""
    p, cam = _clean_scene(oracle_mod, 2, 24, 24, seed0=300)
    cam2 = scenes.look_at((-0.4, 0.3, 3.5), (0.0, 0.0, 0.0), 24, 24)
    tgts = [scenes.target_image(24, 24, view=v) for v in (7, 8)]
    _, _, grads, _, _ = oracle_mod.train_step([cam, cam2], p, tgts, lam=0.2)
    for name in NAMES:
        flat = p[name].reshape(-1)
        g = grads[name].reshape(-1)
        for j in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[j]))
            pp = dict(p)
            x = flat.copy()
            x[j] += h
            pp[name] = x.reshape(p[name].shape)
            Lp = _loss(oracle_mod, [cam, cam2], pp, tgts, 0.2, (0, 0, 0))
            x[j] -= 2 * h
            pp[name] = x.reshape(p[name].shape)
            Lm = _loss(oracle_mod, [cam, cam2], pp, tgts, 0.2, (0, 0, 0))
            fd = (Lp - Lm) / (2 * h)
            assert g[j] == pytest.approx(fd, rel=1e-4, abs=1e-10), (name, j)


def test_p13_dot_product_test(oracle_mod):
    """<J v, w> = <v, J^T w> for the image map theta -> image: J v by central
    differences, J^T w by the analytic backward with dL/dimage = w."""
    p, cam = _clean_scene(oracle_mod, 6, 32, 32, seed0=500)
    bg = (0.1, 0.3, 0.6)
    rng = np.random.default_rng(42)
    w = rng.standard_normal((3, 32, 32))
    pre, lists, _ = oracle_mod.render(cam, p, bg=bg)
    sg = oracle_mod.blend_backward(cam, pre, lists, w, bg)
    JTw = oracle_mod.preprocess_backward(cam, p, sg)
    v = {k: rng.standard_normal(p[k].shape) for k in NAMES}
    h = 1e-6
    pp = {k: p[k] + h * v[k] for k in NAMES}
    Ip = _image(oracle_mod, cam, pp, bg)
    pm = {k: p[k] - h * v[k] for k in NAMES}
    Im = _image(oracle_mod, cam, pm, bg)
    Jv = (Ip - Im) / (2 * h)
    lhs = float(np.sum(Jv * w))
    rhs = sum(float(np.sum(JTw[k] * v[k])) for k in NAMES)
    assert lhs == pytest.approx(rhs, rel=1e-6)


def test_clamped_alpha_has_no_geometry_gradient(oracle_mod):
    """Suppl. B.1 clamp: where min(0.99, o G) is active, alpha does not
    depend on o or on the geometry (reading R11: the exact derivative)."""
    from _util import axis_camera, iso_gaussians
    cam = axis_camera(1, 1)
    cam.cx = cam.cy = 0.5
    p = iso_gaussians([4.0], [0.5], [1 - 1e-6], [[0.3, 0.2, 0.1]])
    pre, lists, out = oracle_mod.render(cam, p)
    sg = oracle_mod.blend_backward(cam, pre, lists, np.ones((3, 1, 1)))
    assert sg["opacity"][0] == 0 and not sg["xy"].any() and not sg["conic"].any()
    assert sg["rgb"][0] == pytest.approx([0.99] * 3)
