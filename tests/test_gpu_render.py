"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs: per-Gaussian screen state, tile lists (bit-exact after
removing decisions float32 may take either way), images, final
transmittance and last contributor (against the oracle's result where every
float32 decision is determined, else against one of the results of the
pixel's admissible decision paths; colour within 2e-4), loss, gradients
(relative L2 1e-3 per tensor), Adam and the full step, single and batched
uneven views."""
import dataclasses
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_util import (GRAD_REL_L2, IMAGE_TOL, ambiguity_masks, compare_lists,  # noqa: E402
                      gpu_forward, gpu_grads, gpu_pixel_state, grad_errors, ill_conditioned, image_check,
                      oracle_forward, oracle_grads, rel_l2)
from paper_2602_09999_gb300 import binding as B  # noqa: E402
from paper_2602_09999_gb300 import scenes  # noqa: E402
from paper_2602_09999_gb300 import train as T  # noqa: E402

GROUPS = T.GROUPS


def _scene_cases():
    return [
        ("tiny256", scenes.tiny_scene(10_000, seed=0), [scenes.tiny_camera(256, 256)]),
        ("ragged", scenes.tiny_scene(6_000, seed=1), [scenes.tiny_camera(250, 183)]),
        ("orbit_small", scenes.outdoor_scene(40_000, seed=2),
         scenes.orbit_cameras(1, 203, 131, radius=6.0, seed=5)),
    ]


@pytest.fixture(scope="module", params=_scene_cases(), ids=lambda c: c[0])
def case(request, oracle_mod):
    name, params, cams = request.param
    rast, views, t, images = gpu_forward(params, cams)
    pres, lists, outs = oracle_forward(params, cams)
    return dict(name=name, params=params, cams=cams, rast=rast, views=views, t=t, images=images,
                pres=pres, lists=lists, outs=outs)


def test_screen_state_matches_oracle(case):
    scr = case["rast"].screen().cpu().numpy()
    rendered = case["rast"].rendered().cpu().numpy()
    for v, pre in enumerate(case["pres"]):
        s = scr[v]
        bits = s[:, 11].view(np.uint32)
        gvis = rendered[v]
        assert np.all((bits[gvis] & 8) != 0)
        keep_any = np.zeros(pre["xy"].shape[0], bool)
        li = case["lists"][v]
        keep_any[li["gid"][(li["flags"] & oracle.KEEP) != 0]] = True
        sure = ~pre["marginal"]
        marg_g = np.zeros_like(keep_any)
        marg_g[li["gid"][(li["flags"] & oracle.IMARGINAL) != 0]] = True
        sure &= ~marg_g
        np.testing.assert_array_equal(gvis[sure], keep_any[sure])
        m = gvis & keep_any
        assert m.sum() > 100
        np.testing.assert_allclose(s[m, 0:2], pre["xy"][m], atol=2e-3, rtol=0)
        # the conic in eigen form: eigenvalues lb >= ls and the major-axis direction
        ca, cb, cc = (pre["conic"][m, i] for i in range(3))
        half = np.sqrt(0.25 * (ca - cc) ** 2 + cb ** 2)
        lb_o, ls_o = 0.5 * (ca + cc) + half, (ca * cc - cb * cb) / (0.5 * (ca + cc) + half)
        np.testing.assert_allclose(s[m, 2], lb_o, rtol=1e-5)
        np.testing.assert_allclose(s[m, 3], ls_o, rtol=1e-5)
        c, sn = s[m, 4].astype(np.float64), s[m, 5].astype(np.float64)
        np.testing.assert_allclose(c * c + sn * sn, 1.0, atol=1e-6)
        lb, ls = s[m, 2].astype(np.float64), s[m, 3].astype(np.float64)
        conic_g = np.stack([ls * c * c + lb * sn * sn, (ls - lb) * sn * c, ls * sn * sn + lb * c * c], 1)
        cmax = np.maximum(np.abs(ca), np.abs(cc))[:, None]
        assert np.all(np.abs(conic_g - pre["conic"][m]) <= 1e-5 * cmax + 1e-7)
        np.testing.assert_allclose(s[m, 6], pre["opacity"][m], rtol=2e-6)
        np.testing.assert_allclose(s[m, 7], pre["depth"][m], rtol=2e-6)
        np.testing.assert_allclose(s[m, 8:11], pre["rgb"][m], atol=2e-5)
        clamp_g = np.stack([(bits[m] >> c) & 1 for c in range(3)], 1)
        np.testing.assert_array_equal(clamp_g, pre["clamped"][m])


def test_tile_lists_bit_exact(case):
    compared, excluded = compare_lists(case["rast"], case["views"], case["pres"], case["lists"])
    assert compared == case["rast"].layout.total_tiles
    total = sum(li["gid"].size for li in case["lists"])
    assert excluded <= 0.01 * total


def test_images_within_tolerance(case):
    """Every pixel: colour, final transmittance and last blended Gaussian
    equal to the oracle's (colour within 2e-4, T within 5e-5) where every
    float32 decision is determined, else jointly equal to one of the FP64
    results of the pixel's admissible decision paths; pixels whose paths
    overflow (held to the allowance bound instead) stay below 1e-4 of the
    pixels."""
    imgs = case["views"].split(case["images"])
    states = gpu_pixel_state(case["rast"], case["views"])
    npx = allow = paths = 0
    for v, out in enumerate(case["outs"]):
        T, last = states[v]
        r = image_check(imgs[v].cpu().numpy(), out, T=T, last=last)
        assert r.bad == 0, (case["name"], v, r)
        assert r.excluded == 0, (case["name"], v, r)
        npx += r.pixels
        allow += r.allowance_pixels
        paths += r.path_pixels
        print(f"{case['name']} view {v}: {r.summary()}")
    assert allow <= 1e-4 * npx, (case["name"], allow, npx)


def test_forward_is_deterministic(case):
    images2 = torch.zeros_like(case["images"])
    case["rast"].forward(T.params_struct(case["t"]), 3, (0.0, 0.0, 0.0), images2)
    torch.cuda.synchronize()
    assert torch.equal(images2, case["images"])


# --------------------------------------------------------------------------
# loss (synthetic images: inputs never come from either side's output)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("sizes,lam", [([(64, 64)], 0.2), ([(37, 53)], 0.2),
                                       ([(40, 30), (17, 33), (64, 48)], 0.2),
                                       ([(100, 60)], 0.0), ([(33, 20)], 1.0)])
def test_loss_matches_oracle(sizes, lam):
    rng = np.random.default_rng(len(sizes) * 100 + sizes[0][0])
    cams = [scenes.look_at((0, 0, 4), (0, 0, 0), w, h) for w, h in sizes]
    imgs = [rng.uniform(0, 1.2, (3, h, w)).astype(np.float32) for w, h in sizes]
    tgts = [rng.uniform(0, 1, (3, h, w)).astype(np.float32) for w, h in sizes]
    views = T.Views(cams)
    rast = T.Rasterizer(10, views, 16)
    im = views.concat([torch.from_numpy(i) for i in imgs]).cuda()
    tg = views.concat([torch.from_numpy(i) for i in tgts]).cuda()
    loss = torch.zeros(1, device="cuda")
    dl = torch.zeros_like(im)
    rast.loss(im, tg, lam, loss, dl)
    torch.cuda.synchronize()
    B_ = len(sizes)
    Lo, grads = 0.0, []
    for i, t in zip(imgs, tgts):
        L, g = oracle.loss(i.astype(np.float64), t.astype(np.float64), lam, grad_scale=1.0 / B_)
        Lo += L / B_
        grads.append(g)
    assert float(loss.item()) == pytest.approx(Lo, rel=2e-6, abs=1e-7)
    for v, g in enumerate(views.split(dl)):
        gg = g.cpu().numpy()
        scale = np.abs(grads[v]).max()
        assert np.abs(gg - grads[v]).max() <= 2e-5 * scale + 1e-12


def test_loss_finite_where_the_covariance_term_vanishes():
    """Images anticorrelated with their targets, so that the SSIM term
    2 cov + C2 passes through zero over many windows: the loss and dL/dC
    stay finite (the SSIM partials are never divided by that term), no
    flag is set, and both match the oracle."""
    rng = np.random.default_rng(77)
    W, H = 640, 480
    cams = [scenes.look_at((0, 0, 4), (0, 0, 0), W, H)]
    tgt = rng.uniform(0.0, 0.1, (3, H, W)).astype(np.float32)
    # cov(x, y) = -k var(y): with var(y) ~ 8.3e-4, k ~ 0.54 puts 2 cov + C2 near 0
    k = rng.uniform(0.3, 0.8, (3, H, W)).astype(np.float32)
    img = (0.5 - k * tgt).astype(np.float32)
    views = T.Views(cams)
    rast = T.Rasterizer(10, views, 16)
    im = views.concat([torch.from_numpy(img)]).cuda()
    tg = views.concat([torch.from_numpy(tgt)]).cuda()
    loss = torch.zeros(1, device="cuda")
    dl = torch.zeros_like(im)
    rast.loss(im, tg, 0.2, loss, dl)
    torch.cuda.synchronize()
    assert torch.isfinite(dl).all() and np.isfinite(float(loss.item()))
    assert rast.error()[0] == 0
    Lo, go = oracle.loss(img.astype(np.float64), tgt.astype(np.float64), 0.2)
    assert float(loss.item()) == pytest.approx(Lo, rel=2e-6, abs=1e-7)
    gg = views.split(dl)[0].cpu().numpy()
    assert np.abs(gg - go).max() <= 2e-5 * np.abs(go).max() + 1e-12


# --------------------------------------------------------------------------
# backward: gradients through the C ABI vs the oracle's exact adjoint.
# dL/dC is zeroed, on both sides, on pixels where decisions float32 may take
# the other way can move the value beyond the image tolerance or flip the
# sign of the L1 term (gpu_util.gradient_mask); Gaussians whose footprint
# dwarfs the view (ill-conditioned sums) are left out of the relative L2.
# --------------------------------------------------------------------------
def _check_grads(params, cams, targets, bg=(0.0, 0.0, 0.0), deg=3, lam=0.2):
    masks = ambiguity_masks(cams, params, deg, bg, targets=targets)
    Lg, gg, _ = gpu_grads(params, cams, targets, masks, lam, bg, deg)
    Lo, go = oracle_grads(cams, params, targets, masks, lam, bg, deg)
    assert Lg == pytest.approx(Lo, rel=1e-5)
    bad = ill_conditioned(cams, params)
    errs = grad_errors(gg, go, bad)
    print({k: f"{v:.2e}" for k, v in errs.items()}, "masked px", int(sum(m.sum() for m in masks)),
          "ill-conditioned", int(bad.sum()))
    for k, e in errs.items():
        assert e <= GRAD_REL_L2, (k, e)


@pytest.mark.parametrize("name,n,size,bg,deg", [("tiny", 4000, (128, 96), (0, 0, 0), 3),
                                                ("bg", 3000, (96, 96), (0.2, 0.5, 0.9), 3),
                                                ("deg1", 3000, (80, 64), (0, 0, 0), 1)])
def test_gradients_match_oracle(oracle_mod, name, n, size, bg, deg):
    params = scenes.tiny_scene(n, seed=20 + n)
    cams = [scenes.tiny_camera(*size)]
    targets = [scenes.target_image(*size, view=3)]
    _check_grads(params, cams, targets, bg, deg)


def test_gradients_match_oracle_anisotropic_scene(oracle_mod):
    """Outdoor-shaped scene: strongly anisotropic Gaussians of many sizes,
    near-plane splats among them."""
    params = scenes.outdoor_scene(20_000, seed=81)
    cams = scenes.orbit_cameras(2, 140, 100, radius=6.0, seed=8)
    targets = [scenes.target_image(140, 100, view=i) for i in range(2)]
    _check_grads(params, cams, targets)


def test_batched_uneven_views_match_oracle(oracle_mod):
    params = scenes.tiny_scene(5000, seed=31)
    sizes = [(120, 90), (77, 101), (64, 64)]
    cams = [scenes.look_at((0.5 * i, 0.3, 4.0), (0, 0, 0), w, h) for i, (w, h) in enumerate(sizes)]
    targets = [scenes.target_image(w, h, view=i) for i, (w, h) in enumerate(sizes)]
    _check_grads(params, cams, targets)


# --------------------------------------------------------------------------
# Adam
# --------------------------------------------------------------------------
def _adam_inputs(n, seed):
    rng = np.random.default_rng(seed)
    shapes = {"means": (n, 3), "log_scales": (n, 3), "quats": (n, 4), "opacity": (n,),
              "sh_dc": (n, 3), "sh_rest": (n, 15, 3)}
    p = {k: rng.standard_normal(s).astype(np.float32) for k, s in shapes.items()}
    g = {k: (rng.standard_normal(s) * 10.0 ** rng.uniform(-7, 0, s)).astype(np.float32)
         for k, s in shapes.items()}
    for k in g:
        g[k].reshape(-1)[::13] = 0.0
    m = {k: (0.1 * rng.standard_normal(s)).astype(np.float32) for k, s in shapes.items()}
    v = {k: (0.01 * rng.random(s)).astype(np.float32) for k, s in shapes.items()}
    return p, g, m, v


@pytest.mark.parametrize("n,step,device_state", [(1001, 1, False), (4096, 7, False),
                                                 (777, 3, True)])
def test_adam_matches_oracle(oracle_mod, n, step, device_state):
    p, g, m, v = _adam_inputs(n, n + step)
    lr = T.DEFAULT_LR
    tp = {k: torch.from_numpy(p[k].copy()).cuda() for k in GROUPS}
    tg = {k: torch.from_numpy(g[k].copy()).cuda() for k in GROUPS}
    tm = {k: torch.from_numpy(m[k].copy()).cuda() for k in GROUPS}
    tv = {k: torch.from_numpy(v[k].copy()).cuda() for k in GROUPS}
    s = torch.cuda.current_stream().cuda_stream
    ps, gs, ms, vs = (T.params_struct(x) for x in (tp, tg, tm, tv))
    if device_state:
        st = B.fgs_adam_state()
        for i in range(6):
            st.lr[i] = lr[i]
        st.beta1, st.beta2, st.eps, st.step = 0.9, 0.999, 1e-15, step - 1
        import ctypes
        buf = torch.frombuffer(bytearray(ctypes.string_at(ctypes.addressof(st), ctypes.sizeof(st))),
                               dtype=torch.uint8).cuda()
        B.fgs_adam_step_device(ps, gs, ms, vs, buf.data_ptr(), s)
    else:
        B.fgs_adam_step(ps, gs, ms, vs, lr, 0.9, 0.999, 1e-15, step, s)
    torch.cuda.synchronize()
    for i, k in enumerate(GROUPS):
        po = p[k].astype(np.float64).copy()
        mo = m[k].astype(np.float64).copy()
        vo = v[k].astype(np.float64).copy()
        oracle.adam(po.reshape(-1), g[k].astype(np.float64).reshape(-1), mo.reshape(-1),
                    vo.reshape(-1), lr[i], step)
        du_g = tp[k].cpu().numpy().astype(np.float64) - p[k]
        du_o = po - p[k]
        # update error relative to the learning rate, plus float32 rounding of p
        assert np.abs(du_g - du_o).max() <= 1e-5 * lr[i] + 2.4e-7 * np.abs(p[k]).max(), k
        # moments: float32 rounding of the inputs' magnitudes (m may cancel)
        ulp = 2.0 ** -24
        m_tol = 4 * ulp * (np.abs(m[k]) + np.abs(g[k])) + 1e-6 * np.abs(mo)
        assert np.all(np.abs(tm[k].cpu().numpy() - mo) <= m_tol), k
        v_tol = 4 * ulp * (np.abs(v[k]) + g[k].astype(np.float64) ** 2) + 1e-6 * np.abs(vo)
        assert np.all(np.abs(tv[k].cpu().numpy() - vo) <= v_tol), k


# --------------------------------------------------------------------------
# full step and graph capture
# --------------------------------------------------------------------------
def test_full_step_matches_oracle(oracle_mod):
    params = scenes.tiny_scene(3000, seed=41)
    cams = [scenes.tiny_camera(96, 80)]
    targets = [scenes.target_image(96, 80, view=9)]
    tr = T.Trainer(params, cams, k_max=200_000)
    tr.set_targets(targets)
    tr.step()
    torch.cuda.synchronize()
    Lo, _, go, newp, _ = oracle.train_step(cams, params, targets)
    assert float(tr.loss.item()) == pytest.approx(Lo, rel=1e-5)
    assert tr.adam_step_count() == 1
    for i, k in enumerate(GROUPS):
        got = tr.params[k].cpu().numpy().astype(np.float64)
        g = go[k]
        rms = np.sqrt(np.mean(g * g)) if np.any(g) else 0.0
        robust = np.abs(g) > 1e-2 * rms
        # first Adam step moves each element by ~lr * sign(g)
        err = np.abs(got - newp[k])
        assert err[robust].max() <= 1e-3 * T.DEFAULT_LR[i] + 2.4e-7 * np.abs(newp[k]).max(), k
        still = g == 0
        np.testing.assert_array_equal(got[still], np.asarray(params[k], np.float64)[still])


@pytest.mark.parametrize("sh_dt,m_dt", [("f32", "f32"), ("bf16", "bf16"), ("f16", "f16"),
                                         ("bf16", "f32")])
def test_fused_backward_adam_matches_separate(oracle_mod, sh_dt, m_dt):
    """fgs_render_backward_adam equals fgs_render_backward followed by
    fgs_adam_step_device: the gradients up to atomic-add order, and its
    update exactly the Adam step of the gradients it used (every Gaussian,
    invisible ones included)."""
    dts = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
    params = scenes.outdoor_scene(20_000, seed=81)
    cams = scenes.orbit_cameras(2, 160, 120, radius=6.0, seed=4)
    targets = [scenes.target_image(160, 120, view=i) for i in range(2)]
    kw = dict(k_max=400_000, sh_dtype=dts[sh_dt], moment_dtype=dts[m_dt])
    sep = T.Trainer(params, cams, fused_adam=False, **kw)
    fus = T.Trainer(params, cams, fused_adam=True, store_grads=True, **kw)
    ref = T.Trainer(params, cams, fused_adam=False, **kw)   # Adam of the fused gradients
    assert fus.fused_adam and not sep.fused_adam
    for tr in (sep, fus):
        tr.set_targets(targets)
        tr.step()
    torch.cuda.synchronize()
    assert fus.adam_step_count() == sep.adam_step_count() == 1
    assert torch.equal(fus.images, sep.images)
    bad = ill_conditioned(cams, params)
    for k in GROUPS:
        a, b = fus.grads[k].cpu().numpy(), sep.grads[k].cpu().numpy()
        assert np.any(b != 0), k
        assert rel_l2(a[~bad], b[~bad]) < 1e-5, k
    for k in GROUPS:
        ref.grads[k].copy_(fus.grads[k])
    B.fgs_adam_step_device(ref.p_s, ref.g_s, ref.m_s, ref.v_s, ref.adam_state.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for i, k in enumerate(GROUPS):
        for got, want in ((fus.params[k], ref.params[k]), (fus.exp_avg[k], ref.exp_avg[k]),
                          (fus.exp_avg_sq[k], ref.exp_avg_sq[k])):
            g64, w64 = got.double().cpu().numpy(), want.double().cpu().numpy()
            # same arithmetic; allow one unit of the storage type for contraction choices
            eps = torch.finfo(got.dtype).eps
            assert np.all(np.abs(g64 - w64) <= eps * np.abs(w64) + 1e-30), k
        # zero-gradient (invisible) Gaussians are part of the comparison (Sec. 3.3)
        zero = (fus.grads[k].reshape(fus.n, -1) == 0).all(dim=1).cpu().numpy()
        assert zero.any()


@pytest.mark.parametrize("dt", ["f32", "f16"])
def test_fused_adam_nonzero_moments(dt):
    """With nonzero moments, the fused backward + Adam update equals the
    separate Adam step of the same gradients bit for bit (both take the
    same roundings), zero-gradient Gaussians included: whole blocks of 128
    culled by opacity, the ragged last block, a block seen only by the
    second camera (which looks away from the scene), and a block with a
    single rendered Gaussian."""
    dts = {"f32": torch.float32, "f16": torch.float16}
    n = 20_000                                      # 156 full blocks + 32
    params = scenes.outdoor_scene(n, seed=85)
    op, mu = params["opacity"].copy(), params["means"].copy()
    culled = np.zeros(n, bool)
    for b in (3, 10, 11, 12, 13, 14):
        culled[128 * b:128 * (b + 1)] = True
    culled[128 * 156:] = True                       # the ragged last block
    culled[128 * 40 + 1:128 * 41] = True            # all but one Gaussian of block 40
    op[culled] = -8.0                               # sigmoid < 1/255
    mu[128 * 40] = (0.05, 0.02, 4.0)                # ... in front of the first camera
    op[128 * 40] = 2.0
    rng = np.random.default_rng(3)                  # block 20: seen by the second camera only
    mu[128 * 20:128 * 21] = np.c_[rng.uniform(-0.3, 0.3, (128, 2)), np.full(128, 12.0)]
    op[128 * 20:128 * 21] = 2.0
    params = dict(params, opacity=op, means=mu)
    cams = [scenes.look_at((0.0, 0.0, 6.0), (0.0, 0.0, 0.0), 128, 96),
            scenes.look_at((0.0, 0.0, 10.0), (0.0, 0.0, 20.0), 96, 128)]
    targets = [scenes.target_image(c.width, c.height, view=i) for i, c in enumerate(cams)]
    kw = dict(k_max=400_000, sh_dtype=dts[dt], moment_dtype=dts[dt])
    fus = T.Trainer(params, cams, fused_adam=True, store_grads=True, **kw)
    ref = T.Trainer(params, cams, fused_adam=False, **kw)
    assert fus.fused_adam
    g = torch.Generator(device="cpu").manual_seed(4)
    for k in GROUPS:
        m = (torch.rand(fus.exp_avg[k].shape, generator=g) - 0.5) * 1e-2
        v = torch.rand(fus.exp_avg_sq[k].shape, generator=g) * 1e-4 + 1e-6
        for tr in (fus, ref):
            tr.exp_avg[k].copy_(m)
            tr.exp_avg_sq[k].copy_(v)
    fus.set_targets(targets)
    before = {k: fus.params[k].clone() for k in GROUPS}
    fus.step()
    torch.cuda.synchronize()
    for k in GROUPS:
        ref.grads[k].copy_(fus.grads[k])
    B.fgs_adam_step_device(ref.p_s, ref.g_s, ref.m_s, ref.v_s, ref.adam_state.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    gm = fus.grads["means"].cpu().numpy()
    dark = np.zeros(n, bool)                        # blocks with nothing rendered
    for b in (3, 10, 11, 12, 13, 14, 156):
        dark[128 * b:128 * (b + 1)] = True
    assert not np.any(gm[dark])
    assert np.any(gm[128 * 20:128 * 21]) and np.any(gm[128 * 40:128 * 41])
    for k in GROUPS:
        moved = (fus.params[k].reshape(n, -1) != before[k].reshape(n, -1)).any(dim=1).cpu().numpy()
        assert moved[dark].mean() > 0.99, k         # nonzero moments move them too
        for got, want in ((fus.params[k], ref.params[k]), (fus.exp_avg[k], ref.exp_avg[k]),
                          (fus.exp_avg_sq[k], ref.exp_avg_sq[k])):
            diff = (got != want).reshape(n, -1).any(dim=1).cpu().numpy()
            assert not diff.any(), (k, np.flatnonzero(diff)[:8])


def test_graph_replay_matches_eager():
    params = scenes.tiny_scene(4000, seed=51)
    cams = [scenes.tiny_camera(128, 128)]
    targets = [scenes.target_image(128, 128, view=1)]
    a = T.Trainer(params, cams, k_max=300_000)
    b = T.Trainer(params, cams, k_max=300_000)
    a.set_targets(targets)
    b.set_targets(targets)
    b.capture(warmup=1)           # one eager warm-up step inside capture()
    a.step()                      # keep the two trainers in step
    for _ in range(3):
        a.step()
        b.replay()
    torch.cuda.synchronize()
    assert a.adam_step_count() == b.adam_step_count() == 4
    assert float(a.loss.item()) == pytest.approx(float(b.loss.item()), rel=1e-4)
    for k in GROUPS:
        assert rel_l2(b.params[k].cpu().numpy(), a.params[k].cpu().numpy()) < 1e-4, k
    # forward alone is deterministic: replaying the same state gives the same image
    a.forward_only()
    img1 = a.images.clone()
    a.forward_only()
    assert torch.equal(img1, a.images)


# --------------------------------------------------------------------------
# launch configurations change speed only
# --------------------------------------------------------------------------
def test_blend_configurations_agree(oracle_mod):
    """Every blend launch configuration renders the same image bit for bit
    (per-pixel arithmetic does not depend on it) and meets the gradient
    parity bar against the oracle (only the order of float32 additions in the
    per-Gaussian sums differs)."""
    params = scenes.outdoor_scene(30_000, seed=71)
    cams = scenes.orbit_cameras(2, 150, 111, radius=6.0, seed=3)
    targets = [scenes.target_image(150, 111, view=i) for i in range(2)]
    bad = ill_conditioned(cams, params)
    masks = ambiguity_masks(cams, params, targets=targets)
    Lo, go = oracle_grads(cams, params, targets, masks)
    ref_img = None
    from paper_2602_09999_gb300 import tune
    # and backward pairs of their own (forward pair, schedule, backward pair)
    mixed = [(2, 128, B.FGS_SCHEDULE_QUEUE, 4, 128), (4, 64, B.FGS_SCHEDULE_GRID, 1, 256),
             (1, 256, B.FGS_SCHEDULE_QUEUE, 2, 256)]
    for cfg in tune.all_choices() + mixed:
        L, gg, rast = gpu_grads(params, cams, targets, masks, tuning=cfg)
        Tf, nc = (x.clone() for x in rast.per_pixel())
        if ref_img is None:
            ref_img = (Tf, nc)
        assert torch.equal(Tf, ref_img[0]) and torch.equal(nc, ref_img[1]), cfg
        assert L == pytest.approx(Lo, rel=1e-5), cfg
        for k, e in grad_errors(gg, go, bad).items():
            assert e <= GRAD_REL_L2, (cfg, k, e)


def _length_bucket(c):
    """Quarter-octave bucket of a list length, longest first (empty last)."""
    c = int(c)
    if c == 0:
        return 129
    e = c.bit_length() - 1
    m = (c >> (e - 2)) & 3 if e >= 2 else (c << (2 - e)) & 3
    return 128 - (4 * e + m)


def test_tile_queue_order_reset_and_repeat(oracle_mod):
    """The work queue holds every tile once, in non-increasing quarter-octave
    buckets of list length; its counters are zero after every blend launch
    (the last CTA out resets them), so a second backward over the same
    forward gives the same gradients up to atomic-add order."""
    params = scenes.outdoor_scene(20_000, seed=73)
    cams = [scenes.Camera(R=c.R, t=c.t, fx=c.fx / 8, fy=c.fy / 8, cx=c.cx / 8, cy=c.cy / 8,
                          width=c.width // 8, height=c.height // 8, near=c.near, cam_pos=c.cam_pos)
            for c in scenes.uneven_cameras()]
    rast, views, t, images = gpu_forward(params, cams)
    assert rast.layout.tuning.blend_schedule == B.FGS_SCHEDULE_QUEUE
    tiles = rast.layout.total_tiles
    q = rast.slot(B.FGS_WS_TILE_QUEUE, torch.int32).cpu().numpy()
    assert np.all(q[:4] == 0)
    order = q[4:4 + tiles]
    assert sorted(order.tolist()) == list(range(tiles))
    ranges = rast.slot(B.FGS_WS_RANGES, torch.int32).cpu().numpy().reshape(-1, 2)[:tiles]
    buckets = [_length_bucket(ranges[i, 1] - ranges[i, 0]) for i in order]
    assert all(a <= b for a, b in zip(buckets, buckets[1:]))
    targets = views.concat([torch.from_numpy(scenes.target_image(c.width, c.height, view=i))
                            for i, c in enumerate(cams)]).cuda()
    loss = torch.zeros(1, device="cuda")
    dl = torch.zeros_like(images)
    rast.loss(images, targets, 0.2, loss, dl)
    runs = []
    for _ in range(2):
        grads = {k: torch.zeros(t[k].shape, device="cuda") for k in GROUPS}
        rast.backward(T.params_struct(t), 3, (0.0, 0.0, 0.0), dl, T.params_struct(grads))
        torch.cuda.synchronize()
        assert np.all(rast.slot(B.FGS_WS_TILE_QUEUE, torch.int32)[:4].cpu().numpy() == 0)
        runs.append({k: v.cpu().numpy() for k, v in grads.items()})
    # atomic-add order differs between the runs; Gaussians whose footprint
    # dwarfs the image sum cancelling terms in any order (as in the parity tests)
    bad = ill_conditioned(cams, params)
    for k in GROUPS:
        assert np.any(runs[0][k] != 0), k
        assert rel_l2(runs[1][k][~bad], runs[0][k][~bad]) < 1e-5, k


def test_autotuner_picks_a_supported_configuration(tmp_path, monkeypatch):
    from paper_2602_09999_gb300 import tune
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tuning.json"))
    params = scenes.tiny_scene(5000, seed=72)
    tr = T.Trainer(params, [scenes.tiny_camera(128, 96)], k_max=200_000)
    choice, ms = tune.autotune(tr, reps=1)
    assert tuple(choice[:2]) in B.BLEND_CONFIGS and choice[2] in B.BLEND_SCHEDULES
    assert tuple(choice[3:5]) == (0, 0) or tuple(choice[3:5]) in B.BLEND_CONFIGS
    assert tuple(choice[5:7]) == (0, 0) or all(d in B.SORT_DIGIT_BITS for d in choice[5:7])
    assert choice[7] in B.DUPLICATE_ORDERS
    # every choice, then the backward's other pairs, then the forward's, then
    # the sort digit widths, then the split duplication order
    assert len(ms) == (len(B.BLEND_CONFIGS) * len(B.BLEND_SCHEDULES) + 2 * (len(B.BLEND_CONFIGS) - 1)
                       + len(B.SORT_DIGIT_BITS) ** 2 - 1 + 1)
    again, _ = tune.autotune(tr)           # cached
    assert tuple(again) == tuple(choice)


@pytest.mark.parametrize("digits", [(11, 8), (8, 11), (11, 11)])
def test_sort_digit_widths_give_the_same_lists(digits):
    """The radix digit width of either sort changes speed only: the sorted
    tile lists, ranges, image and per-pixel state are bit-identical to the
    8-bit sorts' (the two-view batch has 12 tile-id bits: two passes at
    either width; a single small view, 6 bits, one)."""
    from paper_2602_09999_gb300 import tune
    params = scenes.outdoor_scene(60_000, seed=31)
    for cams in (scenes.orbit_cameras(2, 640, 480, radius=6.0, seed=32),
                 [scenes.tiny_camera(100, 70)]):
        rast, views, t, images = gpu_forward(params, cams)
        ref = [x.clone() for x in rast.sorted_lists()] + [images.clone()] + [x.clone() for x in rast.per_pixel()]
        tune.apply(rast.layout, (2, 128, 0, 0, 0) + digits)
        images2 = torch.zeros_like(images)
        rast.forward(T.params_struct(t), 3, (0.0, 0.0, 0.0), images2)
        torch.cuda.synchronize()
        got = list(rast.sorted_lists()) + [images2] + list(rast.per_pixel())
        K = min(rast.error()[1], rast.k_max)
        for a, b, name in zip(ref, got, ("keys", "vals", "ranges", "image", "T", "n_contrib")):
            if name in ("keys", "vals"):
                a, b = a[:K], b[:K]
            assert torch.equal(a, b), (digits, name)


def test_duplicate_orders_give_the_same_lists():
    """The duplication order changes speed only: the split order (consecutive
    entries per warp, the large rectangles listed and culled one warp per
    entry by a second kernel) emits the instances the strided order does, so
    the sorted lists, ranges, image and per-pixel state are bit-identical: on
    a two-view batch, on a close view where many rectangles are large (the
    list must not be empty), and when the instances overflow k_max (the kept
    prefix is the same)."""
    from paper_2602_09999_gb300 import tune
    outdoor = scenes.outdoor_scene(60_000, seed=31)
    cases = [(outdoor, scenes.orbit_cameras(2, 640, 480, radius=6.0, seed=32), None, False),
             (scenes.small_scene(20_000, seed=33, log_scale_mean=-1.5), [scenes.tiny_camera(320, 240)], None,
              True),
             (outdoor, scenes.orbit_cameras(1, 640, 480, radius=6.0, seed=34), 20_000, False)]
    for params, cams, k_max, many_big in cases:
        rast, views, t, images = gpu_forward(params, cams, k_max=k_max)
        flags, inst = rast.error()
        assert bool(flags & B.FGS_FLAG_CAPACITY) == (k_max is not None)
        ref = [x.clone() for x in rast.sorted_lists()] + [images.clone()] + [x.clone() for x in rast.per_pixel()]
        tune.apply(rast.layout, (2, 128, 0, 0, 0, 0, 0, B.FGS_DUPLICATE_SPLIT))
        images2 = torch.zeros_like(images)
        rast.forward(T.params_struct(t), 3, (0.0, 0.0, 0.0), images2)
        torch.cuda.synchronize()
        # the workspace header's third counter: the split order's list length
        n_big = int(rast.ws[24:28].view(torch.int32).item())
        if many_big:
            assert n_big > 100, n_big
        got = list(rast.sorted_lists()) + [images2] + list(rast.per_pixel())
        K = min(inst, rast.k_max)
        for a, b, name in zip(ref, got, ("keys", "vals", "ranges", "image", "T", "n_contrib")):
            if name in ("keys", "vals"):
                a, b = a[:K], b[:K]
            assert torch.equal(a, b), (len(cams), k_max, name)


def test_unsupported_configuration_is_rejected():
    params = scenes.tiny_scene(100, seed=73)
    rast, views, t, images = gpu_forward(params, [scenes.tiny_camera(32, 32)])
    rast.layout.tuning.blend_pixels_per_thread = 3
    with pytest.raises(B.FGSError) as e:
        rast.forward(T.params_struct(t), 3, (0, 0, 0), images)
    assert e.value.code == -9
    rast.layout.tuning.blend_pixels_per_thread = 2
    rast.layout.tuning.backward_pixels_per_thread = 4
    rast.layout.tuning.backward_batch = 32       # not a supported pair
    with pytest.raises(B.FGSError) as e:
        rast.forward(T.params_struct(t), 3, (0, 0, 0), images)
    assert e.value.code == -9


# --------------------------------------------------------------------------
# host-detected errors and the capacity flag
# --------------------------------------------------------------------------
def test_capacity_overflow_sets_flag_without_fault():
    params = scenes.tiny_scene(5000, seed=61)
    cams = [scenes.tiny_camera(128, 128)]
    rast, views, t, images = gpu_forward(params, cams, k_max=1000)
    flags, inst = rast.error(clear=True)
    assert flags & B.FGS_FLAG_CAPACITY and inst > 1000
    flags2, _ = rast.error()
    assert flags2 == 0


def test_host_errors_are_reported():
    params = scenes.tiny_scene(100, seed=62)
    cams = [scenes.tiny_camera(32, 32)]
    rast, views, t, images = gpu_forward(params, cams)
    ps = T.params_struct(t)
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(B.FGSError) as e:
        B.fgs_render_forward(rast.ws.data_ptr(), rast.layout, ps, 4, views.host,
                             views.device.data_ptr(), (0, 0, 0), images.data_ptr(), s)
    assert e.value.code == -3
    with pytest.raises(B.FGSError) as e:
        B.fgs_render_forward(rast.ws.data_ptr() + 16, rast.layout, ps, 3, views.host,
                             views.device.data_ptr(), (0, 0, 0), images.data_ptr(), s)
    assert e.value.code == -8
    other = B.fgs_workspace_size(101, views.host, 1, rast.k_max)
    with pytest.raises(B.FGSError) as e:
        B.fgs_render_forward(rast.ws.data_ptr(), other, ps, 3, views.host,
                             views.device.data_ptr(), (0, 0, 0), images.data_ptr(), s)
    assert e.value.code == -2
    with pytest.raises(B.FGSError) as e:
        B.fgs_render_forward(rast.ws.data_ptr(), rast.layout, ps, 3, views.host, None, (0, 0, 0),
                             images.data_ptr(), s)
    assert e.value.code == -1
