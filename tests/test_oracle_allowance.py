"""Pins of the oracle's allowance: the bound on how far a float32 evaluation
of the blend (Eq. 3-4, Suppl. B.1) may move a pixel where one of its
decisions sits within float32 error of its threshold.

A stack of isotropic Gaussians on the axis, with sigma proportional to depth,
so that every splat has the same footprint and each entry's alpha at a
chosen pixel is its opacity times one known factor.  Pairs of scenes take a
decision both ways by a perturbation inside its error bound; the change of
the pixel between them must stay within the allowance the oracle reports
for either scene.  Case B is the one a fixed margin on the stop test misses:
an entry with alpha at 1/255 taken the other way scales every later T by
1 - 1/255, and moves a stop test 0.2 % from its threshold."""
import math

import numpy as np
import pytest

from _util import Y00, axis_camera, iso_gaussians

PX, PY = 17, 16                 # pixel centre (17.5, 16.5): 1 px from the axis
T_MIN = 1e-4
A_MIN = 1.0 / 255.0


def _stack(cam, alphas, dcs, sigma0=0.3, d0=3.0):
    """Gaussians at depths d0 + 0.1 j with sigma_j / depth_j fixed; alphas are
    the wanted values at pixel (PX, PY)."""
    n = len(alphas)
    depths = d0 + 0.1 * np.arange(n)
    sig = sigma0 * depths / d0
    shat = (cam.fx * sigma0 / d0) ** 2 + 0.3          # dilated variance in px^2
    dx = PX + 0.5 - cam.cx
    G = math.exp(-0.5 * dx * dx / shat)
    return iso_gaussians(depths, sig, np.asarray(alphas) / G, dcs)


def _pixel(oracle, cam, p):
    _, _, out = oracle.render(cam, p, 3, (0.0, 0.0, 0.0), oracle.FP32_MARGINS)
    return out["image"][:, PY, PX], out, out["allowance"][PY, PX]


def _colours(n, bright):
    dc = np.full((n, 3), 0.2)
    dc[bright] = 2.0
    return dc


def _check_pair(oracle, cam, pa, pb):
    va, oa, alla = _pixel(oracle, cam, pa)
    vb, ob, allb = _pixel(oracle, cam, pb)
    diff = float(np.abs(va - vb).max())
    assert oa["n_contrib"][PY, PX] != ob["n_contrib"][PY, PX]       # the stop moved
    for out, allow in ((oa, alla), (ob, allb)):
        assert not out["hard"][PY, PX]
        assert out["ambiguous"][PY, PX]
        assert diff <= allow, (diff, allow)
    return diff, alla, allb


@pytest.mark.parametrize("side", [1, -1])
def test_stop_test_at_threshold_is_bounded(oracle_mod, side):
    """Case A: five entries at alpha 0.8 (T = 0.2^5), the sixth tested at
    1e-4 (1 -+ 5e-5): stopped before it in one scene, blended in the other.
    The difference is alpha_6 T_5 c_6."""
    cam = axis_camera(33, 33)
    T5 = 0.2 ** 5
    a6 = lambda d: 1.0 - T_MIN * (1.0 + d) / T5                    # noqa: E731
    base = [0.8] * 5
    pa = _stack(cam, base + [a6(-side * 5e-5), 0.8, 0.8], _colours(8, 5))
    pb = _stack(cam, base + [a6(side * 5e-5), 0.8, 0.8], _colours(8, 5))
    diff, alla, allb = _check_pair(oracle_mod, cam, pa, pb)
    c6 = Y00 * 2.0 + 0.5
    assert diff == pytest.approx(a6(0.0) * T5 * c6, rel=1e-3)
    # the bound is of the size of the light left at the stop, not larger
    assert max(alla, allb) <= 2.0 * T5 * c6


def test_flipped_low_alpha_moves_the_stop(oracle_mod):
    """Case B: a front entry at alpha = 1/255 (1 +- 1e-7), blended in one
    scene and not in the other; the seventh entry's test is 0.2 % below the
    threshold when the front entry is blended and 0.19 % above when not."""
    cam = axis_camera(33, 33)
    T6 = (1.0 - A_MIN) * 0.2 ** 5
    a7 = 1.0 - T_MIN * (1.0 - 2e-3) / T6
    tail = [0.8] * 5 + [a7, 0.8, 0.8]
    dcs = _colours(9, 6)
    pa = _stack(cam, [A_MIN * (1 + 1e-7)] + tail, dcs)
    pb = _stack(cam, [A_MIN * (1 - 1e-7)] + tail, dcs)
    diff, alla, allb = _check_pair(oracle_mod, cam, pa, pb)
    # the front entry's own first-order effect, alpha_0 |c_0 - R| with R the
    # normalised colour behind it, is far below the change: the moved stop
    # makes up the rest
    va, _, _ = _pixel(oracle_mod, cam, pa)
    c0 = Y00 * 0.2 + 0.5
    a0 = A_MIN * (1 + 1e-7)
    R = (va - a0 * c0) / (1.0 - a0)
    front = a0 * float(np.abs(c0 - R).max())
    assert front < 0.05 * diff
    assert diff > 1e-4


def test_exact_decisions_have_no_allowance(oracle_mod):
    """Without margins every decision is exact: no allowance and no flags,
    but at the pixel whose centre is the means' projection, where the
    exponent is exactly zero (the boundary of the power > 0 skip)."""
    cam = axis_camera(33, 33)
    T5 = 0.2 ** 5
    p = _stack(cam, [0.8] * 5 + [1.0 - T_MIN / T5 * (1 - 5e-5), 0.8], _colours(7, 5))
    _, _, out = oracle_mod.render(cam, p)
    on_mean = np.zeros((33, 33), bool)
    on_mean[16, 16] = True
    assert out["ambiguous"][16, 16]
    assert not out["allowance"][~on_mean].any()
    assert not out["hard"].any() and not out["ambiguous"][~on_mean].any()
