"""Pins of the oracle's dynamic (4D) Gaussians: the linear-velocity form of
the conditional Gaussian (Sec. 3.4).  A view at time t sees the mean
mu + v (t - t0) and the opacity times exp(-(t - t0)^2 / (2 sigma_t^2)).

P15 (the static limit), the closed form of the temporal factor at one
standard deviation, the conditional mean against a static Gaussian moved
there, and central finite differences of the loss for every group,
velocity and temporal centre included."""
import numpy as np
import pytest

from paper_2602_09999_gb300 import scenes

STATIC = ("means", "log_scales", "quats", "opacity", "sh_dc", "sh_rest")
ALL = STATIC + ("velocity", "t0")


def _f64(p):
    return {k: (np.asarray(v, np.float64) if k != "sigma_t" else v) for k, v in p.items()}


def _dynamic(p, seed, time, v_std=0.05, sigma_t=0.125, spread=0.15):
    """Velocities N(0, v_std), temporal centres within `spread` of `time`."""
    rng = np.random.default_rng(seed)
    n = p["means"].shape[0]
    q = dict(p)
    q["velocity"] = rng.normal(0.0, v_std, (n, 3))
    q["t0"] = time + rng.uniform(-spread, spread, n)
    q["sigma_t"] = sigma_t
    return q


def test_p15_static_limit(oracle_mod):
    """v = 0 and t = t0: image, loss and every static gradient equal the
    static Gaussians' bit for bit, and dL/dv = dL/dt0 = 0."""
    p = _f64(scenes.small_scene(40, seed=3, spread=0.6))
    cam = scenes.look_at((0.3, -0.2, 4.0), (0.0, 0.0, 0.0), 48, 40)
    cam.time = 0.375                            # exact in float32
    n = p["means"].shape[0]
    q = dict(p, velocity=np.zeros((n, 3)), t0=np.full(n, 0.375), sigma_t=0.1)
    tgt = scenes.target_image(48, 40, view=1)
    Ls, imgs_s, gs, _, _ = oracle_mod.train_step([cam], p, [tgt])
    Ld, imgs_d, gd, _, _ = oracle_mod.train_step([cam], q, [tgt])
    assert Ls == Ld
    np.testing.assert_array_equal(imgs_s[0], imgs_d[0])
    for k in STATIC:
        np.testing.assert_array_equal(gs[k], gd[k])
    assert not np.any(gd["velocity"]) and not np.any(gd["t0"])


def test_temporal_factor_at_one_standard_deviation(oracle_mod):
    """t - t0 = sigma_t (all exact in binary): o(t) = sigmoid(w) e^(-1/2)."""
    p = _f64(scenes.small_scene(16, seed=4, spread=0.5))
    cam = scenes.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 32, 32)
    cam.time = 0.5
    n = p["means"].shape[0]
    q = dict(p, velocity=np.zeros((n, 3)), t0=np.full(n, 0.375), sigma_t=0.125)
    pre = oracle_mod.preprocess(cam, q)
    sig = 1.0 / (1.0 + np.exp(-p["opacity"]))
    ok = pre["status"] & 4 != 0
    np.testing.assert_allclose(pre["opacity"][ok], sig[ok] * np.exp(-0.5), rtol=1e-14)


def test_conditional_mean_equals_a_moved_static_gaussian(oracle_mod):
    """The dynamic Gaussian at time t projects, sorts and blends like a static
    Gaussian placed at mu + v (t - t0) with the scaled opacity logit."""
    p = _f64(scenes.small_scene(30, seed=5, spread=0.6))
    cam = scenes.look_at((0.2, 0.1, 4.0), (0.0, 0.0, 0.0), 40, 36)
    cam.time = 0.5
    n = p["means"].shape[0]
    rng = np.random.default_rng(6)
    q = dict(p, velocity=rng.normal(0.0, 0.4, (n, 3)), t0=np.full(n, 0.25), sigma_t=1e6)
    moved = dict(p, means=p["means"] + q["velocity"] * 0.25)
    pd, _, od = oracle_mod.render(cam, q)
    ps, _, os_ = oracle_mod.render(cam, moved)
    np.testing.assert_allclose(pd["xy"], ps["xy"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(od["image"], os_["image"], rtol=0, atol=1e-12)


def _clean_dynamic_scene(oracle, n, W, H, time, seed0):
    m = oracle.Margins(rel=1e-3, px=1e-3, t_rel=1e-3, depth_rel=1e-3)
    for seed in range(seed0, seed0 + 200):
        p = scenes.small_scene(n, seed, spread=0.6, log_scale_mean=-2.2, log_scale_std=0.3,
                               opacity_mean=0.0, opacity_std=0.8)
        p = _f64(p)
        p["opacity"] = np.minimum(p["opacity"], 2.0)
        q = _dynamic(p, seed, time)
        cam = scenes.look_at((0.3, -0.2, 4.0), (0.0, 0.0, 0.0), W, H)
        cam.time = time
        pre, lists, out = oracle.render(cam, q, margins=m)
        vis = pre["visible"]
        if vis.sum() < n or out["ambiguous"].any() or pre["clamped"][vis].any():
            continue
        if np.any(lists["flags"] & oracle.IMARGINAL):
            continue
        return q, cam
    pytest.skip("no clean scene found")


def _loss(oracle, cams, p, targets, lam):
    tot = 0.0
    for cam, t in zip(cams, targets):
        _, _, out = oracle.render(cam, p)
        L, _ = oracle.loss(out["image"], t, lam)
        tot += L / len(cams)
    return tot


@pytest.mark.parametrize("n", [1, 5])
def test_dynamic_directional_finite_differences(oracle_mod, n):
    q, cam = _clean_dynamic_scene(oracle_mod, n, 32, 32, 0.5, seed0=40 * n)
    tgt = scenes.target_image(32, 32, view=n)
    _, _, grads, _, _ = oracle_mod.train_step([cam], q, [tgt], lam=0.2)
    rng = np.random.default_rng(n)
    for name in ALL:
        v = rng.standard_normal(np.shape(q[name]))
        h = 1e-6 * max(1.0, float(np.abs(q[name]).max()))
        pp = dict(q)
        pp[name] = q[name] + h * v
        Lp = _loss(oracle_mod, [cam], pp, [tgt], 0.2)
        pp[name] = q[name] - h * v
        Lm = _loss(oracle_mod, [cam], pp, [tgt], 0.2)
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(grads[name] * v))
        assert an == pytest.approx(fd, rel=2e-5, abs=1e-12), name


def test_dynamic_elementwise_finite_differences_two_times(oracle_mod):
    """Velocity and temporal centre of 2 Gaussians, element by element, seen
    by two views at different times (gradients summed over the batch)."""
    q, cam = _clean_dynamic_scene(oracle_mod, 2, 24, 24, 0.5, seed0=700)
    cam2 = scenes.look_at((-0.4, 0.3, 3.5), (0.0, 0.0, 0.0), 24, 24)
    cam2.time = 0.55
    tgts = [scenes.target_image(24, 24, view=v) for v in (3, 4)]
    _, _, grads, _, _ = oracle_mod.train_step([cam, cam2], q, tgts, lam=0.2)
    for name in ("velocity", "t0", "means", "opacity"):
        flat = np.asarray(q[name]).reshape(-1)
        g = grads[name].reshape(-1)
        for j in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[j]))
            pp = dict(q)
            x = flat.copy()
            x[j] += h
            pp[name] = x.reshape(np.shape(q[name]))
            Lp = _loss(oracle_mod, [cam, cam2], pp, tgts, 0.2)
            x[j] -= 2 * h
            pp[name] = x.reshape(np.shape(q[name]))
            Lm = _loss(oracle_mod, [cam, cam2], pp, tgts, 0.2)
            fd = (Lp - Lm) / (2 * h)
            assert g[j] == pytest.approx(fd, rel=1e-4, abs=1e-10), (name, j)
