"""The hand-written adjoint behind torch.autograd (train.RasterizeFn),
through the C ABI: its forward equals the rasterizer's bit for bit; the
gradients autograd returns for L = sum(w * image), with seeded per-pixel
weights w, match the FP64 oracle's exact adjoint for dL/dC = w within 1e-3
relative L2 per tensor (w zeroed on the pixels where float32 decisions may
go the other way, on both sides); and a float32 central difference of L
along a random direction agrees with the gradient on a scene without such
decisions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_util import GRAD_REL_L2, ambiguity_masks, grad_errors, ill_conditioned  # noqa: E402
from paper_2602_09999_gb300 import scenes  # noqa: E402
from paper_2602_09999_gb300 import train as T  # noqa: E402


def _leaves(params):
    t = T.to_device_params(params)
    return {k: t[k].clone().requires_grad_(True) for k in T.GROUPS}


def _render(rast, leaves, bg=(0.0, 0.0, 0.0)):
    return T.RasterizeFn.apply(rast, 3, bg, *[leaves[k] for k in T.GROUPS])


def test_autograd_matches_rasterizer_and_oracle():
    params = scenes.outdoor_scene(20_000, seed=33)
    cams = [scenes.orbit_cameras(2, 120, 96, radius=6.0, seed=4)[0],
            scenes.orbit_cameras(2, 88, 110, radius=6.0, seed=4)[1]]
    bg = (0.1, 0.2, 0.3)
    views = T.Views(cams)
    rast = T.Rasterizer(20_000, views, k_max=2_000_000)
    leaves = _leaves(params)
    images = _render(rast, leaves, bg)
    # the same forward through the plain call
    ref = torch.empty_like(images)
    rast.forward(T.params_struct({k: v.detach() for k, v in leaves.items()}), 3, bg, ref)
    torch.cuda.synchronize()
    assert torch.equal(images.detach(), ref)
    # L = sum(w * image), w seeded, zero where a float32 decision can move the value
    rng = np.random.default_rng(5)
    masks = ambiguity_masks(cams, params, 3, bg)
    ws = []
    for c, m in zip(cams, masks):
        w = rng.uniform(-1.0, 1.0, (3, c.height, c.width))
        w[:, m] = 0.0
        ws.append(w)
    w_dev = views.concat([torch.from_numpy(w.astype(np.float32)) for w in ws]).cuda()
    (images * w_dev).sum().backward()
    torch.cuda.synchronize()
    go = oracle.zero_grads(params)
    for cam, w in zip(cams, ws):
        pre, lists, out = oracle.render(cam, params, 3, bg)
        sg = oracle.blend_backward(cam, pre, lists, w, bg)
        oracle.preprocess_backward(cam, params, sg, 3, go)
    gg = {k: leaves[k].grad.cpu().numpy() for k in T.GROUPS}
    errs = grad_errors(gg, go, ill_conditioned(cams, params))
    print({k: f"{e:.2e}" for k, e in errs.items()})
    for k, e in errs.items():
        assert e <= GRAD_REL_L2, (k, e)


def test_autograd_directional_difference():
    """float32 central difference of sum(w * image) along a random direction
    of every tensor at once, on a scene of large soft Gaussians (no decision
    near a threshold), against the autograd gradient."""
    m = oracle.Margins(rel=1e-3, px=1e-3, t_rel=1e-3, depth_rel=1e-3)
    cam = scenes.look_at((0.3, -0.2, 4.0), (0.0, 0.0, 0.0), 40, 32)
    for seed in range(60, 160):
        p = scenes.small_scene(6, seed, spread=0.6, log_scale_mean=-2.0, log_scale_std=0.2,
                               opacity_mean=0.0, opacity_std=0.5)
        pre, lists, out = oracle.render(cam, p, 3, (0.0, 0.0, 0.0), m)
        if pre["visible"].all() and not out["ambiguous"].any() and not np.any(lists["flags"] & oracle.IMARGINAL):
            break
    else:
        pytest.skip("no clean scene found")
    views = T.Views([cam])
    rast = T.Rasterizer(6, views, k_max=10_000)
    w = torch.from_numpy(np.random.default_rng(1).uniform(0.5, 1.0, 3 * 40 * 32).astype(np.float32)).cuda()
    leaves = _leaves(p)
    (_render(rast, leaves) * w).sum().backward()
    rng = np.random.default_rng(2)
    dirs = {k: torch.from_numpy(rng.standard_normal(tuple(leaves[k].shape)).astype(np.float32)).cuda()
            for k in T.GROUPS}
    an = sum(float((leaves[k].grad * dirs[k]).sum()) for k in T.GROUPS)

    def L(sign, h):
        with torch.no_grad():
            q = {k: (leaves[k] + sign * h * dirs[k]).contiguous() for k in T.GROUPS}
            img = torch.empty(3 * 40 * 32, device="cuda")
            rast.forward(T.params_struct(q), 3, (0.0, 0.0, 0.0), img)
            return float((img.double() * w.double()).sum())

    h = 1e-3
    fd = (L(1, h) - L(-1, h)) / (2 * h)
    assert an == pytest.approx(fd, rel=2e-2, abs=1e-3)
