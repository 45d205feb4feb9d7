"""Pins for the oracle's analytic backward: central finite differences in
double through the whole forward (projection, SH colour, sort, compositing).
The paper (§4) accumulates these gradients with atomics; here we only fix
what they must equal. CPU only."""
import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _linear_loss(w):
    """L = sum(w * image); dL/dimage = w."""
    return lambda img: (float((img * w).sum()), w)


def _l1l2_loss(target, w1, w2):
    """The workloads' loss L = w1 mean|r| + w2 mean(r^2), r = image - target,
    in double, with its gradient written from the definition."""
    n = target.size

    def f(img):
        r = img - target
        return float(w1 * np.abs(r).sum() / n + w2 * (r * r).sum() / n), (w1 * np.sign(r) + 2 * w2 * r) / n
    return f


def _loss_and_state(oracle, s, loss_fn):
    proj, bins, ras = oracle.forward(s, "f64")
    return loss_fn(ras["image"])[0], proj, ras


def _fd_check(oracle, s, comps_per_param=None, seed=0, rel=1e-5, loss_fn=None):
    s = {k: (v.astype(np.float64) if k in PARAMS else v) for k, v in s.items()}
    rng = np.random.default_rng(seed)
    P = int((s["sizes"][:, 0].astype(np.int64) * s["sizes"][:, 1]).sum())
    if loss_fn is None:
        loss_fn = _linear_loss(rng.standard_normal((P, 3)))
    L0, proj0, ras0 = _loss_and_state(oracle, s, loss_fn)
    w = loss_fn(ras0["image"])[1]
    bins0 = oracle.bin_sort(s, proj0, "f64")
    _, grads = oracle.backward(s, proj0, bins0, w, "f64")
    n_checked = 0
    for name in PARAMS:
        flat = s[name].reshape(-1)
        gflat = grads[name].reshape(-1)
        scale = np.abs(gflat).max()
        idx = np.arange(flat.size)
        if comps_per_param is not None and flat.size > comps_per_param:
            idx = rng.choice(flat.size, comps_per_param, replace=False)
        for i in idx:
            if name == "sh" and (i // 3) % 16 >= (s["cfg"]["sh_degree"] + 1) ** 2:
                assert gflat[i] == 0
                continue
            x = flat[i]
            h = 1e-6 * max(1.0, abs(x))
            vals = []
            same = True
            for sgn in (1, -1):
                flat[i] = x + sgn * h
                L, proj, ras = _loss_and_state(oracle, s, loss_fn)
                same &= np.array_equal(proj["counts"], proj0["counts"]) and np.array_equal(proj["rects"], proj0["rects"])
                same &= np.array_equal(ras["hit_signature"], ras0["hit_signature"])
                vals.append(L)
            flat[i] = x
            if not same:
                continue  # a tile rectangle or the composited set moved: not differentiable here
            fd = (vals[0] - vals[1]) / (2 * h)
            tol = rel * max(abs(gflat[i]), 1e-3 * scale) + 1e-9
            assert abs(fd - gflat[i]) <= tol, (name, i, fd, gflat[i])
            n_checked += 1
    return n_checked


@pytest.mark.parametrize("seed,views,tile", [(31, 1, 16), (32, 2, 8), (36, 3, 16)])
def test_fd_small_scenes(oracle, seed, views, tile):
    s = scenes.random_small(seed, N=16, width=36, height=30, n_views=views, tile=tile, log_scale_mu=-1.8)
    n = _fd_check(oracle, s, seed=seed)
    assert n > 16 * 59 * 0.8


def test_fd_with_early_stop_and_alpha_cap(oracle):
    # high opacities: early stops and capped alphas occur, and gradients
    # through capped alphas are zero
    s = scenes.random_small(34, N=20, width=32, height=32, spread=0.5, log_scale_mu=-1.5)
    s["opacity_logits"] = s["opacity_logits"] + 4.0
    proj, bins, ras = oracle.forward(s, "f64")
    assert (ras["final_T"] < 1e-3).any()
    n = _fd_check(oracle, s, seed=34)
    assert n > 20 * 59 * 0.7


@pytest.fixture(scope="module")
def diff_4k_crop():
    """512 Gaussians nearest the ray through a 128x128 window at the centre of
    the 3840x2160 view of the 4M-Gaussian workload, rendered as a 128x128
    image with the principal point shifted."""
    full = scenes.diff_4k()
    assert full["means"].shape[0] == 4 << 20
    m = full["means"]
    d = np.hypot(m[:, 0] / m[:, 2], m[:, 1] / m[:, 2])
    d[m[:, 2] <= 0.5] = np.inf
    keep = np.sort(np.argsort(d)[:512])
    return scenes.crop_view(full, 1856, 1016, 128, 128, keep=keep)


def test_fd_diff_4k_crop(oracle, diff_4k_crop):
    n = _fd_check(oracle, diff_4k_crop, comps_per_param=40, seed=0)
    assert n > 150


def test_fd_diff_4k_crop_workload_loss(oracle, diff_4k_crop):
    """The same crop under the workloads' L1 + 0.2 L2 loss against a target
    whose residuals stay at least 0.05 away from zero (where |r| has no
    derivative): the scalar loss the autograd boundary is tested with."""
    s = diff_4k_crop
    s64 = {k: (v.astype(np.float64) if k in PARAMS else v) for k, v in s.items()}
    img0 = oracle.forward(s64, "f64")[2]["image"]
    rng = np.random.default_rng(3)
    off = rng.uniform(0.05, 0.1, img0.shape) * rng.choice([-1.0, 1.0], img0.shape)
    n = _fd_check(oracle, s, comps_per_param=40, seed=1, loss_fn=_l1l2_loss(img0 - off, 1.0, 0.2))
    assert n > 150
