"""Dynamic (4D) Gaussians on the GPU, through the C ABI, against the FP64
oracle: the linear-velocity form of the conditional Gaussian (Sec. 3.4),
views of uneven sizes at different times in one batched call.  Lists
bit-exact, images on the oracle's admissible decision paths, the loss, every
gradient tensor (velocity and temporal centre included) within 1e-3
relative L2, the static limit bit for bit, and the fused Adam step over all
eight groups."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import (GRAD_REL_L2, ambiguity_masks, compare_lists, gpu_forward,  # noqa: E402
                      gpu_grads, gpu_pixel_state, grad_errors, ill_conditioned, image_check, oracle_forward,
                      oracle_grads, rel_l2)
from paper_2602_09999_gb300 import binding as B  # noqa: E402
from paper_2602_09999_gb300 import scenes  # noqa: E402
from paper_2602_09999_gb300 import train as T  # noqa: E402

SIZES = [(200, 200), (176, 144), (240, 160)]


def _scene(n=60_000, seed=11):
    return scenes.dynamic_scene(n, seed=seed), scenes.dynamic_cameras(3, seed=12, sizes=SIZES)


def test_dynamic_forward_matches_oracle(oracle_mod):
    p, cams = _scene()
    assert len({c.time for c in cams}) > 1
    rast, views, t, images = gpu_forward(p, cams)
    pres, lists, outs = oracle_forward(p, cams)
    compared, excluded = compare_lists(rast, views, pres, lists)
    assert compared == rast.layout.total_tiles
    assert excluded <= 0.01 * sum(li["gid"].size for li in lists)
    states = gpu_pixel_state(rast, views)
    for v, img in enumerate(views.split(images)):
        T_, last = states[v]
        r = image_check(img.cpu().numpy(), outs[v], T=T_, last=last)
        print(f"view {v}: {r.summary()}")
        assert r.bad == 0 and r.excluded == 0, (v, r)
        assert r.allowance_pixels <= 1e-4 * r.pixels, (v, r)


def test_dynamic_gradients_match_oracle(oracle_mod):
    p, cams = _scene()
    targets = [scenes.target_image(c.width, c.height, view=i) for i, c in enumerate(cams)]
    masks = ambiguity_masks(cams, p, targets=targets)
    Lg, gg, _ = gpu_grads(p, cams, targets, masks)
    Lo, go = oracle_grads(cams, p, targets, masks)
    assert Lg == pytest.approx(Lo, rel=1e-5)
    bad = ill_conditioned(cams, p)
    errs = grad_errors(gg, go, bad)
    print({k: f"{e:.2e}" for k, e in errs.items()}, "ill-conditioned", int(bad.sum()))
    assert set(errs) == set(T.GROUPS + T.MOTION_GROUPS)
    for k, e in errs.items():
        assert e <= GRAD_REL_L2, (k, e)


def test_dynamic_static_limit_on_gpu():
    """v = 0 and t0 = the views' time: the same image bit for bit as the
    static Gaussians, and zero velocity and t0 gradients (P15)."""
    p, cams = _scene(20_000, seed=13)
    for c in cams:
        c.time = 0.375
    q = dict(p, velocity=np.zeros_like(p["velocity"]), t0=np.full_like(p["t0"], 0.375))
    static = {k: p[k] for k in T.GROUPS}
    _, views_s, _, img_s = gpu_forward(static, cams)
    _, views_d, _, img_d = gpu_forward(q, cams)
    assert torch.equal(img_s, img_d)
    targets = [scenes.target_image(c.width, c.height, view=i) for i, c in enumerate(cams)]
    _, gd, _ = gpu_grads(q, cams, targets)
    assert not np.any(gd["velocity"]) and not np.any(gd["t0"])


def test_dynamic_fused_adam_matches_separate():
    """The fused backward + Adam over eight groups equals the separate calls:
    the gradients up to atomic-add order, its update exactly the Adam step of
    the gradients it used."""
    p, cams = _scene(30_000, seed=14)
    targets = [scenes.target_image(c.width, c.height, view=i) for i, c in enumerate(cams)]
    sep = T.Trainer(p, cams, k_max=2_000_000, fused_adam=False)
    fus = T.Trainer(p, cams, k_max=2_000_000, fused_adam=True, store_grads=True)
    ref = T.Trainer(p, cams, k_max=2_000_000, fused_adam=False)
    assert fus.groups == T.GROUPS + T.MOTION_GROUPS
    for tr in (sep, fus):
        tr.set_targets(targets)
        tr.step()
    torch.cuda.synchronize()
    assert torch.equal(fus.images, sep.images)
    bad = ill_conditioned(cams, p)
    for k in fus.groups:
        a, b = fus.grads[k].cpu().numpy(), sep.grads[k].cpu().numpy()
        assert np.any(b != 0), k
        assert rel_l2(a[~bad], b[~bad]) < 1e-5, k
    for k in fus.groups:
        ref.grads[k].copy_(fus.grads[k])
    B.fgs_adam_step_device(ref.p_s, ref.g_s, ref.m_s, ref.v_s, ref.adam_state.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for k in fus.groups:
        for got, want in ((fus.params[k], ref.params[k]), (fus.exp_avg[k], ref.exp_avg[k]),
                          (fus.exp_avg_sq[k], ref.exp_avg_sq[k])):
            g64, w64 = got.double().cpu().numpy(), want.double().cpu().numpy()
            eps = torch.finfo(got.dtype).eps
            assert np.all(np.abs(g64 - w64) <= eps * np.abs(w64) + 1e-30), k
