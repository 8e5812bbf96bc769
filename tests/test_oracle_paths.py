"""Pins of the oracle's admissible decision paths (orc_blend_paths): the
results a float32 evaluation of the blend (Eq. 3-4 with the Suppl. B.1
clamp and early stop) may reach at a pixel where a decision sits within
float32 error of its threshold.

The scenes are stacks of isotropic Gaussians on the optical axis with sigma
proportional to depth (every splat has the same footprint), so each entry's
alpha at one chosen pixel is its opacity times one known factor.  The
expected results are written out from Eq. 4 for each order and subset of
the entries: C = sum_i alpha_i T_i c_i with T_i = prod_{j<i} (1 - alpha_j),
stopping before the first entry whose T (1 - alpha) would fall below 1e-4.
The admissible set must not depend on which side of the threshold FP64
itself falls."""
import itertools
import math

import numpy as np
import pytest

from _util import Y00, axis_camera, iso_gaussians

PX, PY = 17, 16                 # pixel centre (17.5, 16.5): 1 px from the axis
T_MIN = 1e-4
A_MIN = 1.0 / 255.0


def _stack(cam, alphas, dcs, depths=None, sigma0=0.3, d0=3.0):
    """Gaussians at depths d0 + 0.1 j (or the given depths) with
    sigma / depth fixed; alphas are the values wanted at pixel (PX, PY)."""
    n = len(alphas)
    depths = d0 + 0.1 * np.arange(n) if depths is None else np.asarray(depths, np.float64)
    sig = sigma0 * depths / d0
    shat = (cam.fx * sigma0 / d0) ** 2 + 0.3          # dilated variance in px^2
    dx = PX + 0.5 - cam.cx
    G = math.exp(-0.5 * dx * dx / shat)
    return iso_gaussians(depths, sig, np.asarray(alphas) / G, dcs)


def _blend(alphas, colours):
    """Eq. 4 front to back over the given entries with the early stop:
    returns (C, T, index of the last blended entry or -1)."""
    T, C, last = 1.0, np.zeros(3), -1
    for i, (a, c) in enumerate(zip(alphas, colours)):
        if T * (1.0 - a) < T_MIN:
            break
        C = C + a * T * np.asarray(c)
        T *= 1.0 - a
        last = i
    return C, T, last


def _results(oracle, cam, p, margins=None):
    """The pixel's admissible results as a sorted list of (C, T, last gid)."""
    margins = oracle.FP32_MARGINS if margins is None else margins
    _, _, out = oracle.render(cam, p, 3, (0.0, 0.0, 0.0), margins)
    st = out["status"][PY, PX]
    if st == 0:
        return st, [(out["image"][:, PY, PX], out["T_final"][PY, PX], out["last_gid"][PY, PX])], out
    sel = out["path_pix"] == PY * cam.width + PX
    vals = out["path_val"][sel]
    return st, [(v[:3], v[3], int(v[4])) for v in vals], out


def _same_set(got, want, tol):
    assert len(got) == len(want), (len(got), len(want))
    key = lambda r: (round(float(r[1]), 9), tuple(np.round(r[0], 9)))   # noqa: E731
    for g, w in zip(sorted(got, key=key), sorted(want, key=key)):
        assert np.abs(np.asarray(g[0]) - np.asarray(w[0])).max() <= tol, (g, w)
        assert abs(g[1] - w[1]) <= tol, (g, w)
        assert g[2] == w[2], (g, w)


def _colour(dc):
    return Y00 * np.asarray(dc, np.float64) + 0.5


@pytest.mark.parametrize("side", [1, -1])
def test_stop_at_threshold_gives_both_results(oracle_mod, side):
    """Five entries at alpha 0.8 (T = 0.2^5), the sixth tested at 1e-4
    (1 -+ 5e-5): the results are the walk stopped before the sixth entry
    and the walk that blends it (then stops before the seventh), whichever
    side FP64 takes."""
    cam = axis_camera(33, 33)
    T5 = 0.2 ** 5
    a6 = 1.0 - T_MIN * (1.0 - side * 5e-5) / T5
    alphas = [0.8] * 5 + [a6, 0.8, 0.8]
    dcs = np.full((8, 3), 0.2)
    dcs[5] = 2.0
    st, got, _ = _results(oracle_mod, cam, _stack(cam, alphas, dcs))
    assert st == 1
    cols = _colour(dcs)
    stop5 = _blend(alphas[:5], cols[:5])
    C6 = stop5[0] + a6 * T5 * cols[5]
    want = [stop5, (C6, T5 * (1 - a6), 5)]
    _same_set(got, want, 1e-12)


def test_flipped_low_alpha_gives_both_walks(oracle_mod):
    """A front entry at alpha = 1/255 (1 +- 1e-7), blended or not; the
    seventh entry's stop test is decided (0.2 % from its threshold) in
    each branch, but differently: two results, the same for both scenes."""
    cam = axis_camera(33, 33)
    T6 = (1.0 - A_MIN) * 0.2 ** 5
    a7 = 1.0 - T_MIN * (1.0 - 2e-3) / T6
    tail = [0.8] * 5 + [a7, 0.8, 0.8]
    dcs = np.full((9, 3), 0.2)
    dcs[6] = 2.0
    cols = _colour(dcs)
    sets = []
    for d in (1e-7, -1e-7):
        a0 = A_MIN * (1 + d)
        st, got, _ = _results(oracle_mod, cam, _stack(cam, [a0] + tail, dcs))
        assert st == 1
        with_front = _blend([a0] + tail, cols)
        C, T, last = _blend(tail, cols[1:])
        without = (C, T, last + 1)
        assert with_front[2] == 5 and without[2] == 6       # the stop moved by one entry
        _same_set(got, [with_front, without], 1e-12)
        sets.append(got)
    _same_set(sets[0], sets[1], 1e-8)


@pytest.mark.parametrize("rel", [0.0, 1e-7])
def test_tied_depths_give_both_orders(oracle_mod, rel):
    """Two entries whose depths are equal, or 1e-7 apart (within float32
    resolution), with different colours and alphas: both orders are
    admissible; an entry in front of them is blended in both."""
    cam = axis_camera(33, 33)
    d = np.array([3.0, 3.5, 3.5 * (1 + rel)])
    alphas = [0.3, 0.5, 0.7]
    dcs = np.array([[0.1, 0.1, 0.1], [2.0, 0.0, 0.0], [0.0, 0.0, 2.0]])
    st, got, _ = _results(oracle_mod, cam, _stack(cam, alphas, dcs, depths=d))
    assert st == 1
    cols = _colour(dcs)
    a = _blend(alphas, cols)
    b = _blend([alphas[0], alphas[2], alphas[1]], cols[[0, 2, 1]])
    b = (b[0], b[1], 1)                                     # last blended: Gaussian 1
    _same_set(got, [a, b], 1e-12)
    assert np.abs(a[0] - b[0]).max() > 0.01                 # the orders really differ


def test_every_subset_of_uncertain_entries(oracle_mod):
    """Five entries at alpha = 1/255 exactly (each blend decision uncertain)
    in front of an opaque-ish one: the results are the 32 subsets blended;
    seven such entries (128 subsets) overflow the 64 results enumerated."""
    cam = axis_camera(33, 33)
    rng = np.random.default_rng(3)
    for k, want_status in ((5, 1), (7, 2)):
        alphas = [A_MIN] * k + [0.6]
        dcs = rng.uniform(0.0, 2.0, (k + 1, 3))
        st, got, _ = _results(oracle_mod, cam, _stack(cam, alphas, dcs))
        assert st == want_status
        if want_status == 2:
            continue
        cols = _colour(dcs)
        want = []
        for mask in itertools.product([0, 1], repeat=k):
            idx = [i for i in range(k) if mask[i]] + [k]
            C, T, _ = _blend([alphas[i] for i in idx], cols[idx])
            want.append((C, T, k))
        _same_set(got, want, 1e-12)


def test_no_margins_one_result(oracle_mod):
    """Without margins every decision is FP64's: one result per pixel, but at
    the pixel whose centre is the means' projection, where the exponent of
    all seven entries is exactly zero (the boundary of the power > 0 skip):
    2^7 subsets, more than the 64 results enumerated."""
    cam = axis_camera(33, 33)
    T5 = 0.2 ** 5
    p = _stack(cam, [0.8] * 5 + [1.0 - T_MIN / T5 * (1 - 5e-5), 0.8], np.full((7, 3), 0.4))
    _, _, out = oracle_mod.render(cam, p, paths=True)
    st = out["status"].copy()
    assert st[16, 16] == 2
    st[16, 16] = 0
    assert not st.any()


def test_fp64_result_is_admissible_on_a_random_scene(oracle_mod):
    """On a random scene: the FP64 walk is among every multi-result pixel's
    results (exactly), a pixel with one result has no allowance, and no
    pixel overflows."""
    from paper_2602_09999_gb300 import scenes
    p = scenes.outdoor_scene(60_000, seed=4)
    cam = scenes.orbit_cameras(1, 160, 120, radius=6.0, seed=5)[0]
    _, _, out = oracle_mod.render(cam, p, 3, (0.1, 0.2, 0.3), oracle_mod.FP32_MARGINS)
    st = out["status"]
    assert (st == 1).sum() > 10 and not (st == 2).any()
    assert not out["allowance"][st == 0].any()
    pix, val = out["path_pix"], out["path_val"]
    flat = out["image"].reshape(3, -1)
    hit = np.all(val[:, :3] == flat[:, pix].T, axis=1) & (val[:, 3] == out["T_final"].reshape(-1)[pix])
    found = np.zeros(flat.shape[1], bool)
    np.logical_or.at(found, pix, hit)
    assert found[(st == 1).reshape(-1)].all()
