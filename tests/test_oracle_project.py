"""Pins for the oracle's projection (EWA splatting of 3D Gaussians, 3DGS as
cited in §4 of the paper): closed forms, an independent EWA construction, and
brute-force tile enumeration. CPU only."""
import math

import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes

# The configuration constants travel as float32 (0.3f).
EPS2D = float(np.float32(0.3))


def _one_gaussian_scene(mean, log_scale, quat, opac=2.0, W=64, H=48, fx=80.0, fy=80.0, cx=32.0, cy=24.0, tile=16,
                        viewmat=None):
    s = {
        "means": np.array([mean], np.float64),
        "log_scales": np.array([log_scale], np.float64),
        "quats": np.array([quat], np.float64),
        "opacity_logits": np.array([opac], np.float64),
        "sh": np.zeros((1, 16, 3)),
        "cams": scenes.camera_row(np.eye(4) if viewmat is None else viewmat, fx, fy, cx, cy)[None],
        "sizes": np.array([[W, H]], np.int32),
        "cfg": scenes.make_cfg(tile_w=tile, tile_h=tile),
    }
    return s


def _hamilton(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _rotate(q, v):
    q = np.asarray(q, np.float64) / np.linalg.norm(q)
    qc = q * np.array([1, -1, -1, -1])
    return _hamilton(_hamilton(q, np.concatenate([[0.0], v])), qc)[1:]


def test_isotropic_on_axis_closed_form(oracle):
    # An isotropic Gaussian on the optical axis projects to a circle of
    # variance (f s / d)^2 + eps2d centred on the principal point, whatever
    # its rotation.
    for ls, d, q in [(-2.0, 4.0, (1, 0, 0, 0)), (-1.5, 7.0, (0.3, -0.5, 0.2, 0.7)), (-3.0, 2.5, (0, 0, 1, 0))]:
        s = _one_gaussian_scene([0, 0, d], [ls] * 3, q)
        p = oracle.project(s, "f64")
        rec = p["projected"][0]
        sig2 = (80.0 * math.exp(ls) / d) ** 2 + EPS2D
        assert rec[0] == pytest.approx(32.0, abs=1e-12) and rec[1] == pytest.approx(24.0, abs=1e-12)
        assert rec[2] == pytest.approx(1 / sig2, rel=1e-10)
        assert rec[3] == pytest.approx(0.0, abs=1e-10 / sig2)
        assert rec[4] == pytest.approx(1 / sig2, rel=1e-10)
        assert rec[6] == pytest.approx(d, rel=1e-15)
        # radius: eigenvalues equal, so the 0.1 floor inside the square root applies
        assert rec[7] == math.ceil(3 * math.sqrt(sig2 + math.sqrt(0.1)))


def test_ewa_matches_numerical_jacobian(oracle):
    # Sigma2 - eps2d I must equal J_pi W Sigma W^T J_pi^T, with J_pi the
    # Jacobian of the pinhole map (by central differences) and Sigma built
    # from the quaternion by Hamilton-product rotation of the scaled axes.
    rng = np.random.default_rng(3)
    viewmat = scenes.look_at([0.3, -0.2, -0.5], [0.1, 0.0, 4.0], [0, -1, 0])
    fx, fy, cx, cy = 90.0, 85.0, 31.0, 25.5
    for _ in range(20):
        mean = rng.uniform(-0.6, 0.6, 3) + [0, 0, 4]
        ls = rng.normal(-2.0, 0.6, 3)
        q = rng.standard_normal(4)
        s = _one_gaussian_scene(mean, ls, q, fx=fx, fy=fy, cx=cx, cy=cy, viewmat=viewmat)
        p = oracle.project(s, "f64")
        if p["counts"][0] == 0:
            continue
        rec = p["projected"][0]
        conic = np.array([[rec[2], rec[3]], [rec[3], rec[4]]])
        S2 = np.linalg.inv(conic)
        vm = s["cams"][0, :16].astype(np.float64).reshape(4, 4)  # the float32 matrix the oracle sees
        W = vm[:3, :3]
        t = W @ mean + vm[:3, 3]

        def pi(X):
            return np.array([fx * X[0] / X[2] + cx, fy * X[1] / X[2] + cy])

        J = np.zeros((2, 3))
        for k in range(3):
            h = 1e-6 * max(1.0, abs(t[k]))
            e = np.zeros(3)
            e[k] = h
            J[:, k] = (pi(t + e) - pi(t - e)) / (2 * h)
        axes = np.stack([_rotate(q, np.eye(3)[k]) * math.exp(ls[k]) for k in range(3)], 1)
        Sigma = axes @ axes.T
        ref = J @ W @ Sigma @ W.T @ J.T + EPS2D * np.eye(2)
        np.testing.assert_allclose(S2, ref, rtol=1e-7, atol=1e-9)
        np.testing.assert_allclose(rec[:2], pi(t), rtol=1e-14)
        assert rec[6] == pytest.approx(t[2], rel=1e-14)
        lam = np.linalg.eigvalsh(ref)
        if (lam[1] - lam[0]) / 2 >= math.sqrt(0.1):
            assert rec[7] == math.ceil(3 * math.sqrt(lam[1]) - 1e-9) or rec[7] == math.ceil(3 * math.sqrt(lam[1]))


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16)])
def test_rect_equals_bruteforce_tile_enumeration(oracle, tile):
    # A tile belongs to the rectangle iff its pixel box [tx*tw, (tx+1)*tw) x ...
    # meets the open square (mean - r, mean + r)^2 and lies in the image.
    s = scenes.random_small(7, N=400, width=101, height=67, n_views=2, spread=1.4, log_scale_mu=-2.0)
    s["cfg"] = scenes.make_cfg(tile_w=tile[0], tile_h=tile[1])
    p = oracle.project(s, "f32")
    N = s["means"].shape[0]
    n_checked = 0
    for vg in range(2 * N):
        v = vg // N
        W, H = s["sizes"][v]
        ntx, nty = -(-W // tile[0]), -(-H // tile[1])
        rec = p["projected"][vg].astype(np.float64)
        if p["counts"][vg] == 0:
            continue
        mx, my, r = rec[0], rec[1], rec[7]
        want = set()
        for ty in range(nty):
            for tx in range(ntx):
                if (tx + 1) * tile[0] > mx - r and tx * tile[0] < mx + r and (ty + 1) * tile[1] > my - r and ty * tile[1] < my + r:
                    want.add((tx, ty))
        x0, y0, x1, y1 = p["rects"][vg]
        got = {(tx, ty) for ty in range(y0, y1) for tx in range(x0, x1)}
        assert got == want, (vg, rec[:8], (x0, y0, x1, y1))
        assert p["counts"][vg] == len(want)
        n_checked += 1
    assert n_checked > 300


def test_culling(oracle):
    # behind the camera, inside the near plane and beyond the far plane: no tiles
    for z in (-3.0, 0.005, 2e10):
        s = _one_gaussian_scene([0, 0, z], [-2, -2, -2], (1, 0, 0, 0))
        assert oracle.project(s, "f32")["counts"][0] == 0
    # far off to the side: rectangle clamps to nothing
    s = _one_gaussian_scene([40, 0, 4], [-2, -2, -2], (1, 0, 0, 0))
    assert oracle.project(s, "f32")["counts"][0] == 0


def test_sh_degree0_colour_is_view_independent(oracle):
    s = scenes.random_small(11, N=32, n_views=3, sh_degree=0)
    p = oracle.project(s, "f64")
    C0 = 1 / (2 * math.sqrt(math.pi))
    N = 32
    want = np.maximum(C0 * s["sh"][:, 0, :].astype(np.float64) + 0.5, 0)
    for v in range(3):
        vis = p["counts"][v * N:(v + 1) * N] > 0
        got = p["projected"][v * N:(v + 1) * N, 8:11]
        np.testing.assert_allclose(got[vis], want[vis], rtol=1e-14, atol=1e-15)
