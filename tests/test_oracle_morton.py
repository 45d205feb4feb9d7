"""Pins for the Morton-order oracle (oracle/morton.py). CPU only.

The code's bit layout is pinned on hand-worked values; the order it induces is
pinned against an independent definition of Z-order (compare the axis whose
coordinates differ in the most significant bit, the comparison of Chan 2002),
which shares nothing with bit interleaving; the quantisation on its end points,
its monotonicity and a degenerate axis."""
import functools

import numpy as np

from oracle import morton as M


def test_interleave_hand_values():
    cases = {(0, 0, 0): 0, (1, 0, 0): 1, (0, 1, 0): 2, (0, 0, 1): 4, (1, 1, 1): 7, (2, 0, 0): 8, (0, 2, 0): 16,
             (1023, 1023, 1023): (1 << 30) - 1, (512, 0, 0): 1 << 27,
             # x=011, y=101, z=110: level 0 takes (z,y,x) = (0,1,1) = 3, level 1 (1,0,1) = 5, level 2 (1,1,0) = 6
             (3, 5, 6): 3 | (5 << 3) | (6 << 6)}
    for (x, y, z), want in cases.items():
        assert int(M.interleave(np.array([x]), np.array([y]), np.array([z]))[0]) == want, (x, y, z)


def _less_msb(a, b):
    """The most significant set bit of a is below that of b."""
    return a < b and a < (a ^ b)


def _z_cmp(p, q):
    """Z-order comparison without interleaving: the axis whose coordinates
    differ in the highest bit decides; on equal highest bits z outranks y
    outranks x, so the axes are visited z first and a later axis must differ
    strictly higher to take over."""
    axis, best = 2, 0
    for k in (2, 1, 0):
        d = int(p[k]) ^ int(q[k])
        if _less_msb(best, d):
            axis, best = k, d
    return (int(p[axis]) > int(q[axis])) - (int(p[axis]) < int(q[axis]))


def test_code_order_equals_msb_comparison_order():
    rng = np.random.default_rng(0)
    pts = rng.integers(0, 1024, (400, 3))
    pts[50:60] = pts[0]  # duplicates
    codes = M.interleave(pts[:, 0], pts[:, 1], pts[:, 2])
    by_code = sorted(range(len(pts)), key=lambda i: (int(codes[i]), i))
    by_cmp = sorted(range(len(pts)), key=functools.cmp_to_key(lambda i, j: _z_cmp(pts[i], pts[j]) or (i - j)))
    assert by_code == by_cmp


def test_quantise_end_points_and_monotone():
    x = np.linspace(-3.0, 5.0, 10001, dtype=np.float32)
    q = M.quantise(x, np.float32(-3.0), np.float32(5.0))
    assert q[0] == 0 and q[-1] == 1023
    assert np.all(np.diff(q.astype(np.int64)) >= 0)
    assert len(np.unique(q)) == 1024
    # a cell is 8/1024 wide: x = -3 + 8 k / 1024 + small lands in cell k
    k = np.arange(0, 1023, 37)
    xs = (np.float32(-3.0) + np.float32(8.0 / 1024) * k.astype(np.float32) + np.float32(1e-3)).astype(np.float32)
    np.testing.assert_array_equal(M.quantise(xs, np.float32(-3.0), np.float32(5.0)), k)


def test_degenerate_axis_and_nan():
    m = np.zeros((5, 3), np.float32)
    m[:, 0] = np.arange(5)
    codes = M.morton_codes(m)
    np.testing.assert_array_equal(codes, M.interleave(M.quantise(m[:, 0], 0, 4), [0] * 5, [0] * 5))
    assert M.quantise(np.array([np.nan], np.float32), np.float32(0), np.float32(1))[0] == 0


def test_order_is_a_stable_permutation():
    rng = np.random.default_rng(1)
    m = rng.uniform(-10, 10, (5000, 3)).astype(np.float32)
    m[100:110] = m[7]
    perm, sc = M.morton_order(m)
    assert sorted(perm.tolist()) == list(range(5000))
    assert np.all(np.diff(sc.astype(np.int64)) >= 0)
    dup = [i for i in perm if i == 7 or 100 <= i < 110]
    assert dup == sorted(dup)


def test_order_groups_nearby_points():
    """Locality, the reason for the order: consecutive Gaussians along the
    curve are much closer in space than in the input order."""
    rng = np.random.default_rng(2)
    m = rng.uniform(0, 1, (20000, 3)).astype(np.float32)
    perm, _ = M.morton_order(m)
    d_in = np.linalg.norm(np.diff(m, axis=0), axis=1).mean()
    d_z = np.linalg.norm(np.diff(m[perm], axis=0), axis=1).mean()
    assert d_z < 0.1 * d_in
