"""Pins of the oracle's locality-preserving order (Sec. 3.3
"Locality-preserving densification": z-ordering of the Gaussians).

The z-order (Morton) code of a point interleaves the bits of its three
10-bit grid coordinates.  Pinned by: exact grid coordinates of points placed
at known fractions of the bounding box; codes built bit by bit from binary
strings; the textbook locality of the z-curve (on a 2^k grid each run of 8^j
consecutive codes fills one aligned cube of side 2^j); degenerate boxes; and
the stable order."""
import numpy as np
import pytest

import oracle


def _string_code(qx, qy, qz):
    """Interleave three 10-bit integers through their binary strings, most
    significant bit first: z, y, x for every bit position."""
    bx, by, bz = (format(int(v), "010b") for v in (qx, qy, qz))
    return int("".join(z + y + x for x, y, z in zip(bx, by, bz)), 2)


def test_grid_coordinates_of_known_fractions():
    """Box [-1, 1] x [0, 4] x [2, 2.5]: a point at fraction (q + 1/4) / 1024
    of each extent (exact in binary) has grid coordinate q; the box's far
    corner is clamped to 1023."""
    rng = np.random.default_rng(0)
    q = rng.integers(0, 1024, (50, 3))
    lo = np.array([-1.0, 0.0, 2.0])
    ext = np.array([2.0, 4.0, 0.5])
    pts = lo + ext * (q + 0.25) / 1024.0
    pts = np.vstack([pts, lo, lo + ext])            # the two corners fix the box
    got = oracle.morton_quantise(pts.astype(np.float32))
    np.testing.assert_array_equal(got[:50], q)
    np.testing.assert_array_equal(got[50], [0, 0, 0])
    np.testing.assert_array_equal(got[51], [1023, 1023, 1023])
    codes = oracle.morton_codes(pts.astype(np.float32))
    for i in range(50):
        assert int(codes[i]) == _string_code(*q[i])
    assert int(codes[50]) == 0 and int(codes[51]) == (1 << 30) - 1


def test_codes_match_bit_strings_on_random_points():
    rng = np.random.default_rng(1)
    pts = rng.normal(size=(300, 3)).astype(np.float32)
    q = oracle.morton_quantise(pts)
    codes = oracle.morton_codes(pts)
    assert q.min() >= 0 and q.max() <= 1023
    for i in range(300):
        assert int(codes[i]) == _string_code(*q[i])


@pytest.mark.parametrize("k", [2, 3])
def test_z_curve_fills_aligned_cubes(k):
    """Cell centres of a 2^k grid (box [0, 1]^3 fixed by its corners), in
    z-order: every run of 8^j consecutive points is one aligned cube of
    side 2^j, and consecutive runs of 8 tile the grid without overlap."""
    n = 1 << k
    idx = np.array([(x, y, z) for z in range(n) for y in range(n) for x in range(n)])
    pts = np.vstack([(idx + 0.5) / n, [[0, 0, 0], [1, 1, 1]]]).astype(np.float32)
    order = oracle.morton_order(pts)
    order = order[order < n ** 3]                   # drop the two corners
    cells = idx[order]
    for j in range(1, k + 1):
        run = 8 ** j
        side = 1 << j
        for s in range(0, n ** 3, run):
            c = cells[s:s + run]
            base = c.min(axis=0)
            assert np.all(base % side == 0)
            assert np.all(c.max(axis=0) - base == side - 1)
            assert len({tuple(v) for v in c}) == run


def test_flat_and_single_point_boxes():
    """A box flat along an axis maps that axis to 0; one point (or all
    equal) gives code 0 and the identity order."""
    rng = np.random.default_rng(2)
    pts = rng.uniform(-1, 1, (64, 3)).astype(np.float32)
    pts[:, 2] = 0.75
    q = oracle.morton_quantise(pts)
    assert not q[:, 2].any() and q[:, :2].any()
    same = np.tile(np.float32([0.1, -2.0, 3.0]), (17, 1))
    assert not oracle.morton_codes(same).any()
    np.testing.assert_array_equal(oracle.morton_order(same), np.arange(17))
    assert oracle.morton_codes(np.zeros((0, 3), np.float32)).size == 0


def test_order_is_stable_permutation_of_sorted_codes():
    rng = np.random.default_rng(3)
    base = rng.uniform(0, 1, (40, 3)).astype(np.float32)
    pts = np.vstack([base, base[::2], [[0, 0, 0], [1, 1, 1]]]).astype(np.float32)
    codes = oracle.morton_codes(pts)
    order = oracle.morton_order(pts)
    assert sorted(order.tolist()) == list(range(len(pts)))
    c = codes[order]
    assert np.all(c[1:] >= c[:-1])
    for i in range(len(order) - 1):                 # equal codes keep index order
        if c[i] == c[i + 1]:
            assert order[i] < order[i + 1]
