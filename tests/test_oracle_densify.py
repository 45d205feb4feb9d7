"""Pins for the densification-statistics oracle (oracle/densify.py): a
hand-worked two-view example, invisible Gaussians left alone, and additivity
over passes. CPU only."""
import numpy as np

from oracle import densify as D


def _inputs():
    V, N = 2, 3
    proj = np.zeros((V, N, 12))
    proj[0, :, 7] = [3.0, 7.0, 100.0]
    proj[1, :, 7] = [5.0, 2.0, 100.0]
    counts = np.array([[1, 4, 0], [2, 0, 0]], np.uint32)
    dp = np.zeros((V, N, 9))
    dp[0, 0, :2] = [0.1, 0.0]     # view 0 is 200 x 100: (0.1 * 100, 0) -> 10
    dp[0, 1, :2] = [0.0, -0.2]    # (0, -0.2 * 50) -> 10
    dp[1, 0, :2] = [0.3, 0.4]     # view 1 is 100 x 50: (15, 10) -> sqrt(325)
    dp[1, 1, :2] = [9.0, 9.0]     # invisible in view 1: ignored
    dp[0, 2, :2] = [5.0, 5.0]     # invisible everywhere
    sizes = np.array([[200, 100], [100, 50]])
    return proj, counts, dp, sizes


def test_hand_worked_example():
    proj, counts, dp, sizes = _inputs()
    ga, dn, mr = D.densify_stats(proj, counts, dp, sizes, np.zeros(3), np.zeros(3), np.zeros(3))
    np.testing.assert_allclose(ga, [10.0 + np.sqrt(325.0), 10.0, 0.0], rtol=1e-15)
    np.testing.assert_array_equal(dn, [2.0, 1.0, 0.0])
    np.testing.assert_array_equal(mr, [5.0, 7.0, 0.0])


def test_accumulates_over_passes():
    proj, counts, dp, sizes = _inputs()
    a = D.densify_stats(proj, counts, dp, sizes, np.zeros(3), np.zeros(3), np.zeros(3))
    b = D.densify_stats(proj, counts, dp, sizes, *a)
    np.testing.assert_allclose(b[0], 2 * a[0], rtol=1e-15)
    np.testing.assert_array_equal(b[1], 2 * a[1])
    np.testing.assert_array_equal(b[2], a[2])
    c = D.densify_stats(proj, counts, dp, sizes, np.zeros(3), np.zeros(3), np.array([1.0, 9.0, 4.0]))
    np.testing.assert_array_equal(c[2], [5.0, 9.0, 4.0])
