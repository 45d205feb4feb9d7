"""Pins for the oracle's elementary pieces: the scale exponential, the real SH
basis, the loss gradient and Adam. CPU only."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ulp_dist(a: float, b: float) -> int:
    ia = np.array([a], np.float32).view(np.int32)[0]
    ib = np.array([b], np.float32).view(np.int32)[0]
    return abs(int(ia) - int(ib))


def test_exp_cody_waite_within_2ulp(oracle):
    rng = np.random.default_rng(0)
    xs = np.concatenate([np.linspace(-20, 10, 20001), rng.uniform(-87, 88, 20000), [0.0, -0.0, 1e-8, -1e-8]])
    worst = 0
    for x in xs.astype(np.float32):
        got = oracle.exp_cody_waite(float(x))
        ref = np.float32(math.exp(float(x)))
        worst = max(worst, _ulp_dist(got, float(ref)))
    assert worst <= 2, worst


def test_exp_cody_waite_clamps(oracle):
    assert oracle.exp_cody_waite(-1000.0) == pytest.approx(math.exp(-87.0), rel=1e-6)
    assert oracle.exp_cody_waite(1000.0) == pytest.approx(math.exp(88.0), rel=1e-6)
    assert oracle.exp_cody_waite(float("nan")) == pytest.approx(math.exp(-87.0), rel=1e-6)


def _fib_dirs(n):
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    r = np.sqrt(1 - z * z)
    phi = np.pi * (1 + 5 ** 0.5) * i
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)


def test_sh_orthonormal_by_quadrature(oracle):
    # Gauss-Legendre in cos(theta) x uniform phi integrates polynomials of
    # degree <= 6 on the sphere exactly.
    nz, nphi = 12, 24
    zs, wz = np.polynomial.legendre.leggauss(nz)
    phis = 2 * np.pi * np.arange(nphi) / nphi
    Z, PHI = np.meshgrid(zs, phis, indexing="ij")
    R = np.sqrt(1 - Z * Z)
    dirs = np.stack([R * np.cos(PHI), R * np.sin(PHI), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.sh_basis(dirs)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_matches_scipy_definition(oracle):
    sp = pytest.importorskip("scipy.special")
    dirs = _fib_dirs(257)
    Y = oracle.sh_basis(dirs)
    theta = np.arccos(np.clip(dirs[:, 2], -1, 1))
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            if hasattr(sp, "sph_harm_y"):
                c = sp.sph_harm_y(l, abs(m), theta, phi)
            else:  # older scipy: sph_harm(m, n, azimuth, polar)
                c = sp.sph_harm(abs(m), l, phi, theta)
            if m > 0:
                ref = math.sqrt(2) * c.real
            elif m < 0:
                ref = math.sqrt(2) * c.imag
            else:
                ref = c.real
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-12, err_msg=f"l={l} m={m}")


def test_sh_matches_golden_closed_forms(oracle):
    rows = []
    with open(os.path.join(GOLDEN, "sh_real_basis_l3.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                idx, l, m, norm, poly = line.split()
                rows.append((int(idx), norm, poly))
    assert [r[0] for r in rows] == list(range(16))
    dirs = _fib_dirs(101)
    Y = oracle.sh_basis(dirs)
    env = {"sqrt": math.sqrt, "pi": math.pi}
    for idx, norm, poly in rows:
        c = eval(norm, env)
        for d, y in zip(dirs, Y[:, idx]):
            x_, y_, z_ = d
            val = c * eval(poly, {"x": x_, "y": y_, "z": z_})
            assert y == pytest.approx(val, abs=1e-12)


def test_loss_gradient_matches_central_differences(oracle):
    rng = np.random.default_rng(1)
    img = rng.random((50, 3)).astype(np.float32)
    tgt = rng.random((50, 3)).astype(np.float32)
    L, g = oracle.loss(img, tgt, 1.0, 0.2)
    r = img.astype(np.float64) - tgt
    assert L == pytest.approx(np.mean(np.abs(r)) + 0.2 * np.mean(r * r), rel=1e-12)
    # mean|r| is piecewise linear, r^2 smooth: d/dimg = (sign r + 0.4 r)/n
    np.testing.assert_allclose(g, (np.sign(r) + 0.4 * r) / r.size, rtol=1e-12)


def test_adam_closed_forms(oracle):
    # Step 1: m_hat = g and v_hat = g^2, so the update is -lr g / (|g| + eps).
    rng = np.random.default_rng(2)
    p0 = rng.standard_normal(10)
    g = rng.standard_normal(10)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-15
    p, m, v = oracle.adam(p0, g, np.zeros(10), np.zeros(10), lr, b1, b2, eps, 1)
    np.testing.assert_allclose(p, p0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, (1 - b1) * g, rtol=1e-15)
    np.testing.assert_allclose(v, (1 - b2) * g * g, rtol=1e-15)
    # With a constant gradient the bias corrections make m_hat = g and
    # v_hat = g^2 at every step, so after t steps p = p0 - t lr g/(|g|+eps).
    p, m, v = p0.copy(), np.zeros(10), np.zeros(10)
    for t in range(1, 8):
        p, m, v = oracle.adam(p, g, m, v, lr, b1, b2, eps, t)
    np.testing.assert_allclose(p, p0 - 7 * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-13)
