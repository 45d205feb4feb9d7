"""SSIM image loss and its gradient, written plainly in float64 numpy.

TEST INFRASTRUCTURE ONLY: tests/, the smoke check in __graft_entry__ and the
CPU-baseline leg of bench.py may use this module; the product package never
does. It shares no code with the CUDA library.

What it computes. The paper (arXiv 2606.11390, §4) runs a fused SSIM loss
operator per camera next to the rasteriser, citing SSIM (Wang et al. 2004)
and the fused SSIM of Taming 3DGS (Mallick et al. 2024); it states no
formula. The reading taken here is the usual Gaussian-splatting training loss

    L = (1 - lam) * mean|x - y| + lam * (1 - mean SSIM(x, y)),   lam = 0.2,

with the means over every pixel and colour channel of every view. SSIM is
evaluated per channel with an 11x11 Gaussian window of standard deviation 1.5
(normalised to sum 1) and the constants C1 = 0.01^2, C2 = 0.03^2 (dynamic
range 1), as in Wang et al. (2004). Window sums near the image border take the
pixels outside the image as zero and are not renormalised (the "same"
zero-padded filtering of the usual implementations). For pixel p:

    mu_x = G*x,  mu_y = G*y,  s_xx = G*(x x) - mu_x^2,  s_yy = G*(y y) - mu_y^2,
    s_xy = G*(x y) - mu_x mu_y,
    SSIM(p) = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)).

The gradient with respect to x is the chain rule through the three window
sums that depend on x (mu_x, G*(x x), G*(x y)): the per-pixel partials of SSIM
with respect to those sums are filtered back with the adjoint of the window
sum (the same symmetric window, restricted to in-image pixels).
"""
from __future__ import annotations

import numpy as np

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA = 0.2


def gaussian_window(size: int = WINDOW, sigma: float = SIGMA) -> np.ndarray:
    """1D Gaussian weights exp(-k^2 / (2 sigma^2)), k = -size//2 .. size//2,
    normalised to sum 1."""
    k = np.arange(size, dtype=np.float64) - (size // 2)
    w = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return w / w.sum()


def window_sum(f: np.ndarray, w1: np.ndarray) -> np.ndarray:
    """(G*f)(i, j) = sum_{a,b} w1[a] w1[b] f(i + a - h, j + b - h) over the
    in-image pixels (zero outside), h = len(w1)//2. f is [H, W]; the 2D window
    is the outer product of w1 with itself, summed directly (no separation)."""
    H, W = f.shape
    h = len(w1) // 2
    fp = np.zeros((H + 2 * h, W + 2 * h), np.float64)
    fp[h:h + H, h:h + W] = f
    out = np.zeros((H, W), np.float64)
    for a in range(len(w1)):
        for b in range(len(w1)):
            out += w1[a] * w1[b] * fp[a:a + H, b:b + W]
    return out


def window_sum_separable(f: np.ndarray, w1: np.ndarray) -> np.ndarray:
    """The same zero-padded window sum as window_sum, as two 1D correlations
    (scipy.ndimage.correlate1d along rows, then columns): equal up to rounding
    because the 2D window is an outer product. Used for full-size images,
    where the direct 121-term sum is too slow."""
    from scipy import ndimage

    f = np.asarray(f, np.float64)
    t = ndimage.correlate1d(f, w1, axis=1, mode="constant", cval=0.0)
    return ndimage.correlate1d(t, w1, axis=0, mode="constant", cval=0.0)


def ssim_maps(x: np.ndarray, y: np.ndarray, w1=None, fast: bool = False):
    """Per-pixel SSIM of one channel and its partials with respect to the
    window sums mu_x, G*(x x) and G*(x y). Returns (S, dS_dmux, dS_dexx, dS_dexy)."""
    w1 = gaussian_window() if w1 is None else w1
    ws = window_sum_separable if fast else window_sum
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mux, muy = ws(x, w1), ws(y, w1)
    exx, eyy, exy = ws(x * x, w1), ws(y * y, w1), ws(x * y, w1)
    sxx = exx - mux * mux
    syy = eyy - muy * muy
    sxy = exy - mux * muy
    a1 = 2.0 * mux * muy + C1
    a2 = 2.0 * sxy + C2
    b1 = mux * mux + muy * muy + C1
    b2 = sxx + syy + C2
    S = (a1 * a2) / (b1 * b2)
    # partials, holding the other window sums fixed
    d_exx = -S / b2                                   # via s_xx in b2
    d_exy = 2.0 * a1 / (b1 * b2)                      # via s_xy in a2
    d_mux = (2.0 * muy * a2 / (b1 * b2)               # via a1
             - 2.0 * muy * a1 / (b1 * b2)             # via s_xy in a2
             - 2.0 * mux * S / b1                     # via b1
             + 2.0 * mux * S / b2)                    # via s_xx in b2
    return S, d_mux, d_exx, d_exy


def _split_views(flat: np.ndarray, sizes) -> list:
    """Image [P][3] packed by view (view v: W_v x H_v pixels, row-major) ->
    list of [H_v, W_v, 3] arrays."""
    flat = np.asarray(flat, np.float64).reshape(-1, 3)
    out, base = [], 0
    for (W, H) in np.asarray(sizes).reshape(-1, 2):
        W, H = int(W), int(H)
        out.append(flat[base:base + W * H].reshape(H, W, 3))
        base += W * H
    if base != flat.shape[0]:
        raise ValueError("sizes do not match the image")
    return out


def ssim_loss(image, target, sizes, lam: float = LAMBDA, fast: bool = False):
    """L = (1 - lam) mean|x - y| + lam (1 - mean SSIM) over all views and
    channels; returns (L, dL/dimage shaped like image, mean SSIM). fast=True
    takes the separable window sums (full-size images)."""
    xs = _split_views(image, sizes)
    ys = _split_views(target, sizes)
    M = sum(x.size for x in xs)
    w1 = gaussian_window()
    ws = window_sum_separable if fast else window_sum
    l1 = 0.0
    s_sum = 0.0
    grads = []
    for x, y in zip(xs, ys):
        g = np.zeros_like(x)
        for c in range(3):
            xc, yc = x[:, :, c], y[:, :, c]
            S, d_mux, d_exx, d_exy = ssim_maps(xc, yc, w1, fast)
            s_sum += S.sum()
            # d(sum_p S(p)) / dx(q) = G^T d_mux + 2 x G^T d_exx + y G^T d_exy;
            # the window is symmetric, so G^T is the same zero-padded sum
            dssim = ws(d_mux, w1) + 2.0 * xc * ws(d_exx, w1) + yc * ws(d_exy, w1)
            r = xc - yc
            l1 += np.abs(r).sum()
            g[:, :, c] = (1.0 - lam) * np.sign(r) / M - lam * dssim / M
        grads.append(g.reshape(-1, 3))
    L = (1.0 - lam) * l1 / M + lam * (1.0 - s_sum / M)
    grad = np.concatenate(grads).reshape(np.shape(image))
    return L, grad, s_sum / M
