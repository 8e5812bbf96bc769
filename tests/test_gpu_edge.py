"""Edge cases of the CUDA path, through the C ABI, against the FP64 oracle:
a scene with nothing rendered (behind the camera, outside the view, below
the opacity cutoff), one Gaussian, the largest batch (16 views of uneven
sizes), images one pixel wide or high, degenerate Gaussians mixed into a
scene (zero quaternion, vanishing and huge scales, opacity at the cutoff
and at the clamp), and zero instance capacity."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_util import (GRAD_REL_L2, ambiguity_masks, compare_lists, gpu_forward, gpu_grads,  # noqa: E402
                      gpu_pixel_state, grad_errors, ill_conditioned, image_check, oracle_forward,
                      oracle_grads)
from paper_2602_09999_gb300 import binding as B  # noqa: E402
from paper_2602_09999_gb300 import scenes  # noqa: E402
from paper_2602_09999_gb300 import train as T  # noqa: E402

BG = (0.25, 0.5, 0.75)


def _images_match(params, cams, bg=(0.0, 0.0, 0.0)):
    rast, views, t, images = gpu_forward(params, cams, bg=bg)
    pres, lists, outs = oracle_forward(params, cams, bg=bg)
    compare_lists(rast, views, pres, lists)
    states = gpu_pixel_state(rast, views)
    for v, img in enumerate(views.split(images)):
        T_, last = states[v]
        r = image_check(img.cpu().numpy(), outs[v], T=T_, last=last)
        assert r.bad == 0 and r.excluded == 0, (v, r)
        assert r.allowance_pixels <= 1e-4 * r.pixels, (v, r)
    return rast, views, images, outs


def _grads_match(params, cams, bg=(0.0, 0.0, 0.0)):
    targets = [scenes.target_image(c.width, c.height, view=i) for i, c in enumerate(cams)]
    masks = ambiguity_masks(cams, params, 3, bg, targets=targets)
    Lg, gg, _ = gpu_grads(params, cams, targets, masks, 0.2, bg)
    Lo, go = oracle_grads(cams, params, targets, masks, 0.2, bg)
    assert Lg == pytest.approx(Lo, rel=1e-5)
    errs = grad_errors(gg, go, ill_conditioned(cams, params))
    for k, e in errs.items():
        assert e <= GRAD_REL_L2, (k, e)
    return gg, go


def test_nothing_rendered():
    """Behind the camera, outside the view, or below 1/255: the image is the
    background exactly, T = 1 everywhere, no instances, zero gradients, and
    a fused Adam step leaves every parameter unchanged."""
    p = scenes.tiny_scene(3000, seed=2)
    cam = scenes.tiny_camera(70, 50)            # at z = 4 looking at -z
    means = p["means"].copy()
    third = len(means) // 3
    means[:third, 2] = 6.0                      # behind the camera
    means[third:2 * third, 0] = 50.0            # far outside the view
    p = dict(p, means=means)
    p["opacity"] = p["opacity"].copy()
    p["opacity"][2 * third:] = -8.0             # sigmoid < 1/255
    rast, views, t, images = gpu_forward(p, [cam], bg=BG)
    flags, inst = rast.error()
    assert flags == 0 and inst == 0
    img = images.cpu().numpy().reshape(3, 50, 70)
    for ch in range(3):
        assert np.all(img[ch] == np.float32(BG[ch]))
    T_final, n_contrib = rast.per_pixel()
    assert torch.all(T_final == 1.0) and torch.all(n_contrib == 0)
    tr = T.Trainer(p, [cam], k_max=10_000, bg=BG, store_grads=True)
    tr.set_targets([scenes.target_image(70, 50, view=0)])
    before = {k: tr.params[k].clone() for k in tr.groups}
    tr.step()
    torch.cuda.synchronize()
    for k in tr.groups:
        assert not torch.any(tr.grads[k]), k
        assert torch.equal(tr.params[k], before[k]), k


def test_one_gaussian():
    """One anisotropic Gaussian near the axis (with an SH tint and a
    background); and an isotropic one, whose rotation cannot matter: its
    quaternion gradient is zero up to float32 rounding."""
    p = scenes.tiny_scene(1, seed=3)
    p["means"] = np.array([[0.05, -0.03, 0.0]], np.float32)
    p["log_scales"] = np.array([[-2.0, -2.6, -1.8]], np.float32)
    p["opacity"] = np.full(1, 1.5, np.float32)
    cams = [scenes.tiny_camera(48, 40)]
    _images_match(p, cams, bg=BG)
    _grads_match(p, cams, bg=BG)
    iso = dict(p, log_scales=np.full((1, 3), -2.0, np.float32))
    targets = [scenes.target_image(48, 40, view=0)]
    _, gg, _ = gpu_grads(iso, cams, targets, None, 0.2, BG)
    assert np.abs(gg["quats"]).max() <= 1e-6 * np.abs(gg["means"]).max()


def test_sixteen_uneven_views():
    """The largest batch: 16 views of uneven sizes (from 1x1 to 80x64) in one
    call; every image and the summed gradients against the oracle."""
    p = scenes.tiny_scene(4000, seed=5)
    rng = np.random.default_rng(6)
    cams = []
    for v in range(B.FGS_MAX_VIEWS):
        w, h = (1, 1) if v == 0 else (int(rng.integers(8, 81)), int(rng.integers(1, 65)))
        ang = 2 * np.pi * v / B.FGS_MAX_VIEWS
        cams.append(scenes.look_at((4 * np.sin(ang), 0.5, 4 * np.cos(ang)), (0, 0, 0), w, h))
    _images_match(p, cams)
    _grads_match(p, cams)
    with pytest.raises(B.FGSError) as e:        # one view more than the ABI takes
        B.fgs_workspace_size(4000, B.camera_array(cams + cams[:1]), 17, 1000)
    assert e.value.code == -7


@pytest.mark.parametrize("size", [(1, 300), (300, 1), (17, 1), (1, 1)])
def test_one_pixel_wide_or_high(size):
    """The focal length of a 300-pixel view, so the strip is a slice of an
    ordinary image."""
    p = scenes.tiny_scene(3000, seed=7)
    w, h = size
    fx = 300 / (2 * np.tan(np.radians(30.0)))
    fov = 2 * np.degrees(np.arctan(w / (2 * fx)))
    cams = [scenes.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), w, h, fov_x_deg=fov)]
    _images_match(p, cams)
    _grads_match(p, cams)


def test_degenerate_gaussians_in_a_scene():
    """Zero quaternions, scales of e^-30 (a vanishing footprint) and e^1 (one
    covering the view), opacity logits at the 1/255 cutoff and far above the
    0.99 clamp, mixed into an ordinary scene."""
    p = scenes.tiny_scene(3000, seed=8)
    q, ls, op = p["quats"].copy(), p["log_scales"].copy(), p["opacity"].copy()
    q[0:20] = 0.0
    ls[20:40] = -30.0
    ls[40:42] = 1.0
    op[42:60] = np.float32(np.log(1.0 / 254.0))   # o at the 1/255 cutoff
    op[60:80] = 20.0                              # clamped to 0.99 near the centre
    p = dict(p, quats=q, log_scales=ls, opacity=op)
    cams = [scenes.tiny_camera(96, 72)]
    _images_match(p, cams)
    gg, go = _grads_match(p, cams)
    # Gaussians that cannot render (no rotation, no footprint) get no gradient
    for k in T.GROUPS:
        assert not np.any(gg[k][0:40]) and not np.any(go[k][0:40]), k


def test_zero_capacity_flags_and_renders_background():
    """k_max = 0: every instance is dropped; the capacity flag is set, the
    image is the background, nothing faults."""
    p = scenes.tiny_scene(2000, seed=9)
    rast, views, t, images = gpu_forward(p, [scenes.tiny_camera(64, 48)], k_max=0, bg=BG)
    flags, inst = rast.error()
    assert flags & B.FGS_FLAG_CAPACITY and inst > 0
    img = images.cpu().numpy().reshape(3, 48, 64)
    for ch in range(3):
        assert np.all(img[ch] == np.float32(BG[ch]))


def test_nonfinite_flag_from_loss_and_fused_adam():
    """Non-finite values put into the inputs on the host set the sticky
    FGS_FLAG_NONFINITE, read through fgs_get_error, without a device fault:
    a NaN target pixel (the loss and dL/dC), then a NaN parameter of a
    Gaussian outside the view (its fused Adam update).  A clean step sets
    nothing, and clearing the flags resets them."""
    p = scenes.tiny_scene(2000, seed=11)
    cam = scenes.tiny_camera(64, 48)
    target = scenes.target_image(64, 48, view=0)
    tr = T.Trainer(p, [cam], k_max=100_000)
    tr.set_targets([target])
    tr.step()
    flags, _ = tr.rast.error()
    assert flags == 0
    bad = target.copy()
    bad[1, 20, 30] = np.nan
    tr.set_targets([bad])
    tr.step()
    flags, _ = tr.rast.error(clear=True)
    assert flags & B.FGS_FLAG_NONFINITE and not flags & B.FGS_FLAG_CAPACITY
    assert not np.isfinite(float(tr.loss.item()))
    assert B.fgs_flag_string(B.FGS_FLAG_NONFINITE) != "unknown flag"
    assert tr.rast.error()[0] == 0
    # the loss is clean again; an invisible Gaussian's NaN reaches only Adam
    tr2 = T.Trainer(p, [cam], k_max=100_000)
    tr2.set_targets([target])
    with torch.no_grad():
        tr2.params["means"][0] = torch.tensor([0.0, 0.0, 9.0])   # behind the camera at z = 4
        tr2.params["log_scales"][0, 1] = float("nan")
    tr2.step()
    torch.cuda.synchronize()
    assert np.isfinite(float(tr2.loss.item()))
    flags, _ = tr2.rast.error()
    assert flags & B.FGS_FLAG_NONFINITE
    assert torch.isfinite(tr2.params["log_scales"][1:]).all()
