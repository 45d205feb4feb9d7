"""Pins for the SSIM loss oracle (oracle/ssim.py). CPU only.

Each pin comes from outside the oracle's own formulas: scipy's Gaussian window
and 2D correlation, a per-pixel scalar loop written from the definition, the
identities SSIM(x, x) = 1 and SSIM(x, y) = SSIM(y, x), the closed form for
constant images, and central finite differences of the loss."""
import numpy as np
import pytest

from oracle import ssim as S

scipy_signal = pytest.importorskip("scipy.signal")


def test_window_matches_scipy_gaussian():
    ref = scipy_signal.windows.gaussian(11, std=1.5)
    ref = ref / ref.sum()
    np.testing.assert_allclose(S.gaussian_window(), ref, rtol=1e-14, atol=0)


def test_window_sum_matches_scipy_correlate2d():
    rng = np.random.default_rng(1)
    f = rng.standard_normal((13, 17))
    for w1 in (S.gaussian_window(), rng.uniform(0.1, 1.0, 5)):   # an asymmetric window pins the orientation
        ref = scipy_signal.correlate2d(f, np.outer(w1, w1), mode="same", boundary="fill", fillvalue=0.0)
        np.testing.assert_allclose(S.window_sum(f, w1), ref, rtol=1e-12, atol=1e-13)


def test_separable_path_equals_direct_sum():
    rng = np.random.default_rng(7)
    f = rng.uniform(0, 1, (23, 40))
    np.testing.assert_allclose(S.window_sum_separable(f, S.gaussian_window()), S.window_sum(f, S.gaussian_window()),
                               rtol=1e-12, atol=1e-14)
    img, tgt = rng.uniform(0, 1, (40 * 23 + 6 * 9, 3)), rng.uniform(0, 1, (40 * 23 + 6 * 9, 3))
    sizes = np.array([[40, 23], [6, 9]])
    a, b = S.ssim_loss(img, tgt, sizes), S.ssim_loss(img, tgt, sizes, fast=True)
    assert a[0] == pytest.approx(b[0], rel=1e-13)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-9, atol=1e-15)


def _ssim_scalar(x, y):
    """SSIM map by plain loops: every window sum over the in-image pixels."""
    H, W = x.shape
    w = S.gaussian_window()
    h = len(w) // 2
    out = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            mx = my = exx = eyy = exy = 0.0
            for a in range(-h, h + 1):
                for b in range(-h, h + 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < H and 0 <= jj < W:
                        g = w[a + h] * w[b + h]
                        mx += g * x[ii, jj]
                        my += g * y[ii, jj]
                        exx += g * x[ii, jj] ** 2
                        eyy += g * y[ii, jj] ** 2
                        exy += g * x[ii, jj] * y[ii, jj]
            vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
            out[i, j] = ((2 * mx * my + S.C1) * (2 * cxy + S.C2)) / ((mx * mx + my * my + S.C1) * (vx + vy + S.C2))
    return out


def test_ssim_map_matches_scalar_loops():
    rng = np.random.default_rng(2)
    x, y = rng.uniform(0, 1, (7, 9)), rng.uniform(0, 1, (7, 9))
    np.testing.assert_allclose(S.ssim_maps(x, y)[0], _ssim_scalar(x, y), rtol=1e-12, atol=1e-13)


def test_identical_images_give_ssim_one_and_zero_loss():
    rng = np.random.default_rng(3)
    img = rng.uniform(0, 1, (20 * 14 + 9 * 6, 3))
    sizes = np.array([[20, 14], [9, 6]])
    L, g, mean_ssim = S.ssim_loss(img, img, sizes)
    assert mean_ssim == pytest.approx(1.0, abs=1e-12)
    assert L == pytest.approx(0.0, abs=1e-12)
    assert np.abs(g).max() < 1e-12
    np.testing.assert_allclose(S.ssim_maps(img[:280, 0].reshape(14, 20), img[:280, 0].reshape(14, 20))[0], 1.0,
                               rtol=0, atol=1e-12)


def test_symmetric_in_its_arguments():
    rng = np.random.default_rng(4)
    x, y = rng.uniform(0, 1, (12, 10)), rng.uniform(0, 1, (12, 10))
    np.testing.assert_allclose(S.ssim_maps(x, y)[0], S.ssim_maps(y, x)[0], rtol=1e-13, atol=0)


def test_constant_images_closed_form_in_the_interior():
    a, b = 0.3, 0.7
    x, y = np.full((31, 33), a), np.full((31, 33), b)
    want = (2 * a * b + S.C1) / (a * a + b * b + S.C1)
    got = S.ssim_maps(x, y)[0]
    np.testing.assert_allclose(got[5:-5, 5:-5], want, rtol=1e-10)
    # at the border the zero padding lowers the means and makes the variances non-zero
    assert abs(got[0, 0] - want) > 1e-3


def test_loss_weights():
    rng = np.random.default_rng(5)
    img, tgt = rng.uniform(0, 1, (11 * 8, 3)), rng.uniform(0, 1, (11 * 8, 3))
    sizes = np.array([[11, 8]])
    L0, _, m = S.ssim_loss(img, tgt, sizes, lam=0.0)
    assert L0 == pytest.approx(np.abs(img - tgt).mean(), rel=1e-13)
    L1, _, m1 = S.ssim_loss(img, tgt, sizes, lam=1.0)
    assert L1 == pytest.approx(1.0 - m1, rel=1e-13)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    sizes = np.array([[12, 9], [5, 7]])
    P = 12 * 9 + 5 * 7
    img = rng.uniform(0.05, 0.95, (P, 3))
    tgt = rng.uniform(0.05, 0.95, (P, 3))
    tgt[:20] = img[:20] + 0.3   # keep |r| away from 0 where the L1 kink sits
    _, g, _ = S.ssim_loss(img, tgt, sizes)
    h = 1e-6
    fd = np.zeros_like(img)
    for idx in np.ndindex(*img.shape):
        p, m = img.copy(), img.copy()
        p[idx] += h
        m[idx] -= h
        fd[idx] = (S.ssim_loss(p, tgt, sizes)[0] - S.ssim_loss(m, tgt, sizes)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-9 * np.abs(fd).max())
