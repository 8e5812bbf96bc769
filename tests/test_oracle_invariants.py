"""Invariants of the oracle (P5-P9): transmittance bounds, empty scenes,
permutation and tie handling, culling neutrality and the sorted lists."""
import numpy as np
import pytest

from _util import axis_camera, iso_gaussians
from paper_2602_09999_gb300 import scenes


@pytest.fixture(scope="module")
def tiny(oracle_mod):
    p = scenes.tiny_scene(3000, seed=11)
    cam = scenes.tiny_camera(96, 80)
    pre, lists, out = oracle_mod.render(cam, p)
    return p, cam, pre, lists, out


def test_p5_transmittance_monotone_and_bounded(oracle_mod, tiny):
    """T is non-increasing along each list and stays in [1e-4, 1]."""
    p, cam, pre, lists, out = tiny
    assert out["T_final"].min() >= 1e-4 and out["T_final"].max() <= 1.0
    rng = lists["ranges"]
    maxlen = int((rng[:, 1] - rng[:, 0]).max())
    prev = np.ones_like(out["T_final"])
    for j in list(range(0, maxlen, max(1, maxlen // 25))) + [maxlen]:
        cut = lists.copy()
        cut["ranges"] = np.ascontiguousarray(
            np.stack([rng[:, 0], np.minimum(rng[:, 1], rng[:, 0] + j)], 1))
        o = oracle_mod.blend_forward(cam, pre, cut)
        assert np.all(o["T_final"] <= prev + 0.0)
        assert o["T_final"].min() >= 1e-4
        prev = o["T_final"]
    np.testing.assert_array_equal(prev, out["T_final"])


def test_p6_transparent_scene_renders_background(oracle_mod):
    p = scenes.tiny_scene(500, seed=2)
    p["opacity"][:] = -30.0
    cam = scenes.tiny_camera(48, 48)
    bg = (0.2, 0.5, 0.9)
    tgt = scenes.target_image(48, 48)
    loss, images, grads, _, _ = oracle_mod.train_step([cam], p, [tgt], bg=bg)
    np.testing.assert_array_equal(images[0], np.broadcast_to(np.array(bg)[:, None, None],
                                                             images[0].shape))
    for k, g in grads.items():
        assert not np.any(g), k


def test_p7_permutation_invariance_without_ties(oracle_mod, tiny):
    p, cam, pre, lists, out = tiny
    assert np.unique(pre["depth"][pre["visible"]]).size == pre["visible"].sum()
    perm = np.random.default_rng(3).permutation(p["means"].shape[0])
    q = {k: v[perm] for k, v in p.items()}
    _, _, out2 = oracle_mod.render(cam, q)
    np.testing.assert_array_equal(out2["image"], out["image"])
    np.testing.assert_array_equal(out2["T_final"], out["T_final"])


def test_p7_depth_ties_resolved_by_index(oracle_mod):
    """Two Gaussians at exactly the same depth: the lower index blends first
    (stable sort over index-ordered emission)."""
    cam = axis_camera(33, 33)
    dc = np.array([[0.9, 0.0, 0.0], [0.0, 0.0, 0.9]])
    p = iso_gaussians([4.0, 4.0], [0.2, 0.3], [0.6, 0.7], dc)
    _, _, out = oracle_mod.render(cam, p)
    rgb = np.maximum(dc * (0.5 / np.sqrt(np.pi)) + 0.5, 0)
    # at the centre pixel both alphas equal the opacities
    expect = 0.6 * rgb[0] + 0.4 * 0.7 * rgb[1]
    np.testing.assert_allclose(out["image"][:, 16, 16], expect, rtol=1e-13)
    q = {k: v[::-1].copy() for k, v in p.items()}
    _, _, out2 = oracle_mod.render(cam, q)
    expect2 = 0.7 * rgb[1] + 0.3 * 0.6 * rgb[0]
    np.testing.assert_allclose(out2["image"][:, 16, 16], expect2, rtol=1e-13)


def test_p7_planted_ties_match_index_order(oracle_mod):
    """With many planted ties the tile render equals the brute-force render
    whose single list is ordered by (depth, index)."""
    p = scenes.tiny_scene(1500, seed=4)
    p["means"][1::2] = p["means"][0::2]          # pairs with identical depth
    cam = scenes.tiny_camera(64, 64)
    pre, lists, out = oracle_mod.render(cam, p)
    br = oracle_mod.blend_brute(cam, pre)
    np.testing.assert_allclose(out["image"], br["image"], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(out["last_gid"], br["last_gid"])


def test_p8_culling_neutral_and_brute_twin(oracle_mod, tiny):
    """Sec. 3.2: tight bounds and tile culling do not change the image.
    Culling on == culling off == tile-free brute force."""
    p, cam, pre, lists, out = tiny
    pre2, lists2, out2 = oracle_mod.render(cam, p, margins=oracle_mod.Margins(tile_culling=0))
    assert lists2["gid"].size > lists["gid"].size
    np.testing.assert_array_equal(out2["image"], out["image"])
    np.testing.assert_array_equal(out2["last_gid"], out["last_gid"])
    br = oracle_mod.blend_brute(cam, pre)
    np.testing.assert_allclose(br["image"], out["image"], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(br["last_gid"], out["last_gid"])


def test_p8_kept_tiles_cover_every_contributing_pixel(oracle_mod):
    """Every (Gaussian, tile) pair with a pixel where o G >= 1/255 is kept,
    and every kept tile lies inside the rectangle."""
    p = scenes.tiny_scene(800, seed=8)
    cam = scenes.tiny_camera(80, 64)
    pre, lists, _ = oracle_mod.render(cam, p)
    W, H = cam.width, cam.height
    tx, _ = cam.tiles
    u = np.arange(W) + 0.5
    v = np.arange(H) + 0.5
    kept = set(zip(lists["gid"].tolist(), lists["tile"].tolist()))
    for g in np.nonzero(pre["visible"])[0]:
        a, b, c = pre["conic"][g]
        dx = u[None, :] - pre["xy"][g, 0]
        dy = v[:, None] - pre["xy"][g, 1]
        oG = pre["opacity"][g] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
        ys, xs = np.nonzero(oG >= 1 / 255)
        need = set(((ys // 16) * tx + (xs // 16)).tolist())
        have = {t for (gg, t) in kept if gg == g}
        assert need <= have, g
        r = pre["rect"][g]
        for t in have:
            assert r[0] // 16 <= t % tx <= r[2] // 16 and r[1] // 16 <= t // tx <= r[3] // 16


def test_p9_lists_equal_lexicographic_sort(oracle_mod, tiny):
    """Sorted lists equal Python's sorted() over (tile, depth, index)."""
    p, cam, pre, lists, out = tiny
    keys = sorted(zip(lists["tile"].tolist(), pre["depth"][lists["gid"]].tolist(),
                      lists["gid"].tolist()))
    assert [k[0] for k in keys] == lists["tile"].tolist()
    assert [k[2] for k in keys] == lists["gid"].tolist()
    rng = lists["ranges"]
    for t in range(rng.shape[0]):
        assert np.all(lists["tile"][rng[t, 0]:rng[t, 1]] == t)
    assert rng[-1, 1] == lists["gid"].size
