"""Reduced-storage variant: SH coefficients and Adam moments in bf16 or fp16,
blending, conics and gradient accumulation in float32.

The oracle reads the same quantised SH values (promoted exactly to FP64), so
images and gradients keep the float32 bars.  For Adam, the oracle's FP64
update of the quantised inputs, rounded back to the storage type, must match
the GPU within one unit in the last place of that type (an fp16 second
moment is stored as sqrt(v))."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_util import (GRAD_REL_L2, ambiguity_masks, gpu_pixel_state, grad_errors,  # noqa: E402
                      ill_conditioned, image_check, oracle_grads)
from paper_2602_09999_gb300 import binding as B  # noqa: E402
from paper_2602_09999_gb300 import scenes  # noqa: E402
from paper_2602_09999_gb300 import train as T  # noqa: E402

GROUPS = T.GROUPS
DTYPES = {"bf16": torch.bfloat16, "fp16": torch.float16}


def quantised(params, dt):
    q = dict(params)
    for k in ("sh_dc", "sh_rest"):
        q[k] = torch.from_numpy(np.asarray(params[k])).to(dt).to(torch.float32).numpy()
    return q


def crop_cameras(cams, size=64):
    """Cameras whose size x size image is the centre crop of each view."""
    out = []
    for c in cams:
        dx, dy = (c.width - size) // 2, (c.height - size) // 2
        out.append(scenes.Camera(R=c.R, t=c.t, fx=c.fx, fy=c.fy, cx=c.cx - dx, cy=c.cy - dy,
                                 width=size, height=size, near=c.near, cam_pos=c.cam_pos))
    return out


@pytest.mark.parametrize("name,n", [("bf16", 60_000), ("fp16", 60_000), ("bf16", 3_000_000),
                                    ("fp16", 3_000_000)])
def test_reduced_storage_render_and_gradients(oracle_mod, name, n):
    """The precision variant: the outdoor scene, four uneven views (1237x822,
    960x640, 1600x1064, 640x426) each as its 64x64 centre crop.  Prints per
    image PSNR and max abs error and per tensor the relative L2 error."""
    dt = DTYPES[name]
    params = scenes.outdoor_scene(n, seed=91 if n < 1_000_000 else 0)
    cams = crop_cameras(scenes.uneven_cameras())
    targets = [scenes.target_image(64, 64, view=i) for i in range(len(cams))]
    q = quantised(params, dt)
    masks = ambiguity_masks(cams, q, targets=targets)
    tr = T.Trainer(params, cams, k_max=max(600_000, 4 * n), sh_dtype=dt, moment_dtype=dt)
    tr.set_targets(targets)
    tr.rast.forward(tr.p_s, 3, tr.bg, tr.images)
    tr.rast.loss(tr.images, tr.targets, tr.lam, tr.loss, tr.dl)
    for v, m in enumerate(masks):
        tr.views.split(tr.dl)[v][:, torch.from_numpy(m).cuda()] = 0.0
    tr.rast.backward(tr.p_s, 3, tr.bg, tr.dl, tr.g_s)
    torch.cuda.synchronize()
    Lo, go = oracle_grads(cams, q, targets, masks)
    assert float(tr.loss.item()) == pytest.approx(Lo, rel=1e-5)
    report = []
    checks = []
    states = gpu_pixel_state(tr.rast, tr.views)
    for v, img in enumerate(tr.views.split(tr.images)):
        _, _, out = oracle.render(cams[v], q, margins=oracle.FP32_MARGINS)
        g = img.cpu().numpy().astype(np.float64)
        r = image_check(g, out, T=states[v][0], last=states[v][1])
        checks.append(r)
        d = g - out["image"]
        mse = float(np.mean(d ** 2))
        psnr = 10 * np.log10(1.0 / mse) if mse > 0 else float("inf")
        report.append(f"view{v}: psnr {psnr:.1f} dB, max abs {np.abs(d).max():.2e}; {r.summary()}")
    bad = ill_conditioned(cams, q)
    errs = grad_errors({k: tr.grads[k].cpu().numpy() for k in GROUPS}, go, bad)
    raw = grad_errors({k: tr.grads[k].cpu().numpy() for k in GROUPS}, go, None)
    print(f"\n[{name}, n={n}] " + "; ".join(report))
    print(f"[{name}, n={n}] grad rel L2 " + ", ".join(f"{k} {e:.2e}" for k, e in errs.items()) +
          f" ({int(bad.sum())} ill-conditioned Gaussians excluded; with them: " +
          ", ".join(f"{k} {e:.2e}" for k, e in raw.items()) + ")")
    for r in checks:
        assert r.bad == 0 and r.excluded == 0, (name, r)
    assert sum(r.allowance_pixels for r in checks) <= 1e-4 * sum(r.pixels for r in checks)
    for k, e in errs.items():
        assert e <= GRAD_REL_L2, (name, k, e)


def _ulp(x, dt):
    """Spacing of the storage type at |x| (bf16: 8-bit, fp16: 11-bit mantissa)."""
    x = np.abs(np.asarray(x, np.float64))
    mant = 8 if dt == torch.bfloat16 else 11
    e = np.floor(np.log2(np.maximum(x, 1e-30)))
    if dt == torch.float16:
        e = np.maximum(e, -14.0)
    return 2.0 ** (e - (mant - 1))


@pytest.mark.parametrize("name", ["bf16", "fp16"])
def test_reduced_storage_adam(oracle_mod, name):
    dt = DTYPES[name]
    n, step = 2000, 3
    rng = np.random.default_rng(5)
    shapes = {"means": (n, 3), "log_scales": (n, 3), "quats": (n, 4), "opacity": (n,),
              "sh_dc": (n, 3), "sh_rest": (n, 15, 3)}
    p = {k: rng.uniform(-1, 1, s).astype(np.float32) for k, s in shapes.items()}
    g = {k: (rng.standard_normal(s) * 10.0 ** rng.uniform(-4, -1, s)).astype(np.float32)
         for k, s in shapes.items()}
    m = {k: (1e-2 * rng.standard_normal(s)).astype(np.float32) for k, s in shapes.items()}
    v = {k: (1e-4 * rng.random(s) + 1e-6).astype(np.float32) for k, s in shapes.items()}
    tp = {k: torch.from_numpy(p[k]).cuda().to(dt if k in ("sh_dc", "sh_rest") else torch.float32)
          for k in GROUPS}
    tg = {k: torch.from_numpy(g[k]).cuda() for k in GROUPS}
    tm = {k: torch.from_numpy(m[k]).cuda().to(dt) for k in GROUPS}
    if dt == torch.float16:
        tv = {k: torch.from_numpy(np.sqrt(v[k])).cuda().to(dt) for k in GROUPS}
    else:
        tv = {k: torch.from_numpy(v[k]).cuda().to(dt) for k in GROUPS}
    # the values the GPU actually starts from
    p0 = {k: tp[k].float().cpu().numpy().astype(np.float64) for k in GROUPS}
    m0 = {k: tm[k].float().cpu().numpy().astype(np.float64) for k in GROUPS}
    v0 = {k: (tv[k].float().cpu().numpy().astype(np.float64) ** 2 if dt == torch.float16
              else tv[k].float().cpu().numpy().astype(np.float64)) for k in GROUPS}
    lr = T.DEFAULT_LR
    B.fgs_adam_step(T.params_struct(tp), T.params_struct(tg), T.params_struct(tm),
                    T.params_struct(tv), lr, 0.9, 0.999, 1e-15, step,
                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for i, k in enumerate(GROUPS):
        po, mo, vo = p0[k].copy(), m0[k].copy(), v0[k].copy()
        oracle.adam(po.reshape(-1), g[k].astype(np.float64).reshape(-1), mo.reshape(-1),
                    vo.reshape(-1), lr[i], step)
        got_p = tp[k].float().cpu().numpy()
        pdt = dt if k in ("sh_dc", "sh_rest") else None
        if pdt is None:
            assert np.abs(got_p - po).max() <= 1e-5 * lr[i] + 2.4e-7 * np.abs(po).max(), k
        else:
            assert np.all(np.abs(got_p - po) <= _ulp(po, pdt) * 1.01 + 1e-5 * lr[i]), k
        got_m = tm[k].float().cpu().numpy()
        assert np.all(np.abs(got_m - mo) <= _ulp(mo, dt) * 1.01 + 1e-12), k
        got_s = tv[k].float().cpu().numpy()
        if dt == torch.float16:
            ref_s = np.sqrt(vo)
            assert np.all(np.abs(got_s - ref_s) <= _ulp(ref_s, dt) * 1.01), k
        else:
            assert np.all(np.abs(got_s - vo) <= _ulp(vo, dt) * 1.01 + 1e-30), k


@pytest.mark.parametrize("name", ["bf16", "fp16"])
def test_vanishing_second_moment_keeps_parameters_bounded(name):
    """Gradients of 8e-7: their fp16 sqrt(v) (2.5e-8) rounds to zero while
    m = 8e-8 still fits.  Where the stored second moment vanishes the stored
    first moment is zero too, so the 40 steps of zero gradient that follow
    move no parameter by more than Adam's own bound (|step| <= about 7.3 lr
    with b1 = 0.9, b2 = 0.999); without that rule they would divide m by
    eps = 1e-15.  bf16 keeps both moments (its exponent range is float32's)."""
    dt = DTYPES[name]
    n = 4096
    rng = np.random.default_rng(8)
    shapes = {"means": (n, 3), "log_scales": (n, 3), "quats": (n, 4), "opacity": (n,),
              "sh_dc": (n, 3), "sh_rest": (n, 15, 3)}
    tp = {k: torch.from_numpy(rng.uniform(-1, 1, s).astype(np.float32)).cuda()
          .to(dt if k in ("sh_dc", "sh_rest") else torch.float32) for k, s in shapes.items()}
    p0 = {k: tp[k].float().clone() for k in GROUPS}
    sign = {k: np.where(rng.random(s) < 0.5, -1.0, 1.0) for k, s in shapes.items()}
    tg = {k: torch.from_numpy((8e-7 * sign[k]).astype(np.float32)).cuda() for k in GROUPS}
    tm = {k: torch.zeros(s, device="cuda", dtype=dt) for k, s in shapes.items()}
    tv = {k: torch.zeros(s, device="cuda", dtype=dt) for k, s in shapes.items()}
    lr = T.DEFAULT_LR
    stream = torch.cuda.current_stream().cuda_stream
    args = [T.params_struct(tp), T.params_struct(tg), T.params_struct(tm), T.params_struct(tv)]
    B.fgs_adam_step(*args, lr, 0.9, 0.999, 1e-15, 1, stream)
    torch.cuda.synchronize()
    vanished = 0
    for k in GROUPS:
        gone = tv[k] == 0
        vanished += int(gone.sum())
        assert torch.all(tm[k][gone] == 0), k
    if dt == torch.float16:
        assert vanished == sum(int(np.prod(s)) for s in shapes.values())
    else:
        assert vanished == 0
    for k in GROUPS:
        tg[k].zero_()
    for step in range(2, 42):
        B.fgs_adam_step(*args, lr, 0.9, 0.999, 1e-15, step, stream)
    torch.cuda.synchronize()
    for i, k in enumerate(GROUPS):
        moved = (tp[k].float() - p0[k]).abs().max().item()
        assert torch.isfinite(tp[k].float()).all(), k
        assert moved <= 41 * 7.3 * lr[i] + 2e-2, (k, moved)
