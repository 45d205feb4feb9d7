"""Pins for the oracle's analytic backward: central finite differences in
double through the whole forward (projection, SH colour, sort, compositing).
The paper (§4) accumulates these gradients with atomics; here we only fix
what they must equal. CPU only."""
import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _loss_and_state(oracle, s, w):
    proj, bins, ras = oracle.forward(s, "f64")
    return float((ras["image"] * w).sum()), proj, ras


def _fd_check(oracle, s, comps_per_param=None, seed=0, rel=1e-5):
    s = {k: (v.astype(np.float64) if k in PARAMS else v) for k, v in s.items()}
    rng = np.random.default_rng(seed)
    P = int((s["sizes"][:, 0].astype(np.int64) * s["sizes"][:, 1]).sum())
    w = rng.standard_normal((P, 3))
    L0, proj0, ras0 = _loss_and_state(oracle, s, w)
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
                L, proj, ras = _loss_and_state(oracle, s, w)
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


def test_fd_diff_4k_crop(oracle):
    # 512 Gaussians nearest the ray through a 128x128 window at the centre of
    # the 3840x2160 view of the 4M-Gaussian scene, rendered as a 128x128 image
    # with the principal point shifted.
    full = scenes.diff_4k(N=1 << 20)
    m = full["means"]
    d = np.hypot(m[:, 0] / m[:, 2], m[:, 1] / m[:, 2])
    d[m[:, 2] <= 0.5] = np.inf
    keep = np.sort(np.argsort(d)[:512])
    s = scenes.crop_view(full, 1856, 1016, 128, 128, keep=keep)
    n = _fd_check(oracle, s, comps_per_param=40, seed=0)
    assert n > 150
