"""Pins of the oracle's spatial order (the Morton order of the means that the
library's row reordering uses): codes worked out by hand on exact lattices, the
textbook sort it reduces to on a line, stability, and invariance under exact
shifts and power-of-two scalings."""
import numpy as np

import oracle as orc

# the ten bits of 1023 spread to every third bit: sum of 8^b for b < 10
SPREAD_1023 = sum(8 ** b for b in range(10))


def test_spread_constant():
    assert SPREAD_1023 == (8 ** 10 - 1) // 7 == 153391689


def test_cube_corners():
    # the unit cube's corners: coordinate 1 lands on t = 1024, the last cell (all ten bits)
    corners = [(x, y, z) for z in (0, 1) for y in (0, 1) for x in (0, 1)]  # x fastest: the Z-order
    rng = np.random.default_rng(3)
    shuffle = rng.permutation(8)
    pts = np.array([corners[k] for k in shuffle], np.float32)
    perm, codes = orc.morton_order(pts)
    assert [tuple(pts[i].astype(int)) for i in perm] == corners
    want = {c: SPREAD_1023 * (c[0] + 2 * c[1] + 4 * c[2]) for c in corners}
    for i, p in enumerate(pts):
        assert codes[i] == want[tuple(p.astype(int))]
    assert max(codes) == 2 ** 30 - 1


def test_hand_computed_codes():
    # the x extent is 1024, so the scale is exactly 1 and the cells are the integer coordinates
    pts = {(0, 0, 0): 0, (1, 0, 0): 1, (0, 1, 0): 2, (0, 0, 1): 4, (2, 0, 0): 8,
           (3, 5, 0): 1 + 8 + 2 + 128,      # x = 11b -> bits 0, 3; y = 101b -> bits 1, 7
           (0, 0, 6): 32 + 256,             # z = 110b -> bits 5, 8
           (7, 7, 7): 511,                  # three bits of each axis -> bits 0..8
           (1024, 0, 0): SPREAD_1023}       # t = 1024 -> the last cell, 1023
    keys = list(pts)
    order = [keys[k] for k in (5, 2, 8, 0, 6, 3, 1, 7, 4)]
    perm, codes = orc.morton_order(np.array(order, np.float32))
    for i, p in enumerate(order):
        assert codes[i] == pts[p], p
    got = [order[i] for i in perm]
    assert got == sorted(keys, key=lambda p: pts[p])
    assert got[:5] == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0)]
    assert got[-1] == (1024, 0, 0)


def test_line_reduces_to_sort():
    # points on the z axis one unit apart: every point in its own cell, codes increasing with z
    rng = np.random.default_rng(5)
    z = rng.permutation(1000).astype(np.float32)
    pts = np.zeros((1000, 3), np.float32)
    pts[:, 2] = z
    perm, _ = orc.morton_order(pts)
    assert np.array_equal(perm, np.argsort(z, kind="stable"))


def test_ties_keep_row_order():
    rng = np.random.default_rng(7)
    base = rng.uniform(-5, 5, (40, 3)).astype(np.float32)
    pts = base[rng.integers(0, 6, 300)]  # 300 rows, six distinct points
    perm, codes = orc.morton_order(pts)
    assert sorted(perm.tolist()) == list(range(300))
    for a, b in zip(perm[:-1], perm[1:]):
        assert codes[a] < codes[b] or (codes[a] == codes[b] and a < b)


def test_degenerate_inputs():
    perm, codes = orc.morton_order(np.ones((17, 3), np.float32) * 2.5)  # zero extent: scale 0
    assert np.array_equal(perm, np.arange(17)) and not codes.any()
    perm, codes = orc.morton_order(np.array([[1.0, -2.0, 3.0]], np.float32))
    assert perm.tolist() == [0] and codes.tolist() == [0]
    perm, codes = orc.morton_order(np.zeros((0, 3), np.float32))
    assert perm.size == 0


def test_exact_shift_and_power_of_two_scale():
    # integer lattice points: shifts by integers and scalings by powers of two are exact in FP32,
    # so the cells, and the order, cannot change
    rng = np.random.default_rng(9)
    pts = rng.integers(0, 300, (500, 3)).astype(np.float32)
    perm, codes = orc.morton_order(pts)
    for shift in ((-512, -3, 100), (7, 0, -250)):
        p2, c2 = orc.morton_order(pts + np.array(shift, np.float32))
        assert np.array_equal(perm, p2) and np.array_equal(codes, c2)
    for s in (0.25, 4.0):
        p2, c2 = orc.morton_order(pts * np.float32(s))
        assert np.array_equal(perm, p2) and np.array_equal(codes, c2)
