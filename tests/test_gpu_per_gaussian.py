"""The per-Gaussian blend backward (Sec. 3.2 "Per-Gaussian Backward", after
Mallick et al.: buckets of 32 list entries, one warp per bucket, the blend
replayed front to back from the (T, C) the forward stores in front of every
bucket) through the C ABI, against the FP64 oracle: every gradient tensor
within 1e-3 relative L2 on the scenes of the per-pixel tests, a batch of
uneven views and the full-size bench scene; the forward unchanged bit for
bit by the stored states; the same gradients as the per-pixel order up to
float32 rounding; and a fused, graph-captured training step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_util import (GRAD_REL_L2, ambiguity_masks, gpu_forward, gpu_grads, grad_errors,  # noqa: E402
                      gradient_mask, ill_conditioned, oracle_grads, rel_l2)
from paper_2602_09999_gb300 import binding as B  # noqa: E402
from paper_2602_09999_gb300 import scenes  # noqa: E402
from paper_2602_09999_gb300 import train as T  # noqa: E402
from paper_2602_09999_gb300 import tune  # noqa: E402


def _check(params, cams, targets, bg=(0.0, 0.0, 0.0), deg=3, tuning=None):
    masks = ambiguity_masks(cams, params, deg, bg, targets=targets)
    Lg, gg, rast = gpu_grads(params, cams, targets, masks, 0.2, bg, deg, tuning=tuning,
                             per_gaussian=True)
    assert rast.layout.tuning.blend_backward == B.FGS_BACKWARD_PER_GAUSSIAN
    Lo, go = oracle_grads(cams, params, targets, masks, 0.2, bg, deg)
    assert Lg == pytest.approx(Lo, rel=1e-5)
    bad = ill_conditioned(cams, params)
    errs = grad_errors(gg, go, bad)
    print({k: f"{v:.2e}" for k, v in errs.items()}, "ill-conditioned", int(bad.sum()))
    for k, e in errs.items():
        assert e <= GRAD_REL_L2, (k, e)
    return gg


@pytest.mark.parametrize("name,n,size,bg,deg", [("tiny", 4000, (128, 96), (0, 0, 0), 3),
                                                ("bg", 3000, (96, 96), (0.2, 0.5, 0.9), 3),
                                                ("deg1", 3000, (80, 64), (0, 0, 0), 1),
                                                ("ragged", 6000, (250, 183), (0, 0, 0), 3)])
def test_per_gaussian_gradients_match_oracle(oracle_mod, name, n, size, bg, deg):
    params = scenes.tiny_scene(n, seed=20 + n)
    cams = [scenes.tiny_camera(*size)]
    targets = [scenes.target_image(*size, view=3)]
    _check(params, cams, targets, bg, deg)


def test_per_gaussian_anisotropic_batch_and_configs(oracle_mod):
    """Outdoor-shaped scene, two uneven views in one call, every blend
    launch configuration (the forward stores the states in each)."""
    params = scenes.outdoor_scene(20_000, seed=81)
    cams = [scenes.orbit_cameras(2, 140, 100, radius=6.0, seed=8)[0],
            scenes.orbit_cameras(2, 96, 130, radius=6.0, seed=8)[1]]
    targets = [scenes.target_image(c.width, c.height, view=i) for i, c in enumerate(cams)]
    for cfg in tune.all_choices():
        _check(params, cams, targets, tuning=cfg)


def test_forward_unchanged_and_orders_agree():
    """Storing the bucket states leaves the forward bit for bit; the two
    backward orders give the same gradients up to float32 rounding."""
    params = scenes.outdoor_scene(40_000, seed=2)
    cams = scenes.orbit_cameras(2, 203, 131, radius=6.0, seed=5)
    *_, img_a = gpu_forward(params, cams)
    *_, img_b = gpu_forward(params, cams, per_gaussian=True)
    assert torch.equal(img_a, img_b)
    targets = [scenes.target_image(203, 131, view=i) for i in range(2)]
    La, ga, _ = gpu_grads(params, cams, targets)
    Lb, gb, _ = gpu_grads(params, cams, targets, per_gaussian=True)
    assert La == Lb
    bad = ill_conditioned(cams, params)
    for k in T.GROUPS:
        assert rel_l2(gb[k][~bad], ga[k][~bad]) < 1e-4, k


def test_per_gaussian_full_size(oracle_mod):
    """The bench scene (3M Gaussians in z-order, one 1237x822 view): every
    gradient tensor against the oracle."""
    p = scenes.outdoor_scene(3_000_000, seed=0)
    order = oracle.morton_order(p["means"]).astype(np.int64)
    scene = {k: np.ascontiguousarray(v[order]) for k, v in p.items()}
    cams = [scenes.orbit_cameras(100, 1237, 822, radius=6.0, seed=1)[7]]
    targets = [scenes.target_image(1237, 822, view=0)]
    pre, lists, out = oracle.render(cams[0], scene, 3, (0.0, 0.0, 0.0), oracle.FP32_MARGINS)
    m = gradient_mask(out, targets[0])
    L, dL = oracle.loss(out["image"], targets[0], 0.2)
    dL[:, m] = 0.0
    go = oracle.zero_grads(scene)
    sg = oracle.blend_backward(cams[0], pre, lists, dL)
    oracle.preprocess_backward(cams[0], scene, sg, 3, go)
    Lg, gg, _ = gpu_grads(scene, cams, targets, [m], k_max=8_000_000, per_gaussian=True)
    assert Lg == pytest.approx(L, rel=1e-5)
    bad = ill_conditioned(cams, scene)
    errs = grad_errors(gg, go, bad)
    print({k: f"{v:.2e}" for k, v in errs.items()}, "ill-conditioned", int(bad.sum()))
    for k, e in errs.items():
        assert e <= GRAD_REL_L2, (k, e)


def test_per_gaussian_graph_step_matches_per_pixel():
    """A fused, graph-captured training step with the per-Gaussian backward:
    the images of its forward equal the per-pixel trainer's, and its stored
    gradients agree with them up to float32 rounding."""
    p = scenes.outdoor_scene(30_000, seed=14)
    cams = scenes.orbit_cameras(2, 160, 120, radius=6.0, seed=6)
    targets = [scenes.target_image(160, 120, view=i) for i in range(2)]
    trs = [T.Trainer(p, cams, k_max=2_000_000, store_grads=True, per_gaussian=pg) for pg in (False, True)]
    for tr in trs:
        tr.set_targets(targets)
        tr.step()                 # eager step: loads every kernel
    torch.cuda.synchronize()
    trs = [T.Trainer(p, cams, k_max=2_000_000, store_grads=True, per_gaussian=pg) for pg in (False, True)]
    for tr in trs:
        tr.set_targets(targets)
        tr.capture(warmup=0)
        tr.replay()
    torch.cuda.synchronize()
    assert torch.equal(trs[0].images, trs[1].images)
    bad = ill_conditioned(cams, p)
    for k in T.GROUPS:
        a, b = trs[1].grads[k].cpu().numpy(), trs[0].grads[k].cpu().numpy()
        assert rel_l2(a[~bad], b[~bad]) < 1e-4, k
