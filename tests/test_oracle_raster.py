"""Pins for the oracle's key sort and compositing (front-to-back alpha
blending of depth-sorted splats per tile, §4 of the paper; 3DGS rules for the
alpha cap, the 1/255 cutoff and the transmittance stop). CPU only."""
import math

import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes


def _scene_variants():
    yield scenes.random_small(21, N=80, width=53, height=37, n_views=2)
    yield scenes.random_small(22, N=120, width=40, height=40, n_views=3, tile=8)
    s = scenes.random_small(23, N=60, width=70, height=29, n_views=1, log_scale_mu=-1.8)
    s["cfg"] = scenes.make_cfg(tile_w=32, tile_h=16)
    yield s


def test_sort_matches_python_sort_on_tile_depth_index(oracle):
    for s in _scene_variants():
        proj = oracle.project(s, "f32")
        bins = oracle.bin_sort(s, proj, "f32")
        N = s["means"].shape[0]
        sizes = s["sizes"]
        tw, th = s["cfg"]["tile_w"], s["cfg"]["tile_h"]
        base, bases, ntxs = 0, [], []
        for W, H in sizes:
            bases.append(base)
            ntxs.append(-(-W // tw))
            base += -(-W // tw) * -(-H // th)
        items = []
        for vg in range(len(proj["counts"])):
            if proj["counts"][vg] == 0:
                continue
            v = vg // N
            x0, y0, x1, y1 = proj["rects"][vg]
            d = float(np.float32(proj["projected"][vg, 6]))
            for ty in range(y0, y1):
                for tx in range(x0, x1):
                    items.append((bases[v] + ty * ntxs[v] + tx, d, vg))
        items.sort()
        assert bins["n_isect"] == len(items) == int(proj["counts"].sum())
        assert [it[2] for it in items] == bins["vals"].tolist()
        tiles = bins["keys"] >> np.uint64(32)
        depth = (bins["keys"] & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
        assert tiles.tolist() == [it[0] for it in items]
        assert depth.tolist() == [it[1] for it in items]
        # tile ranges partition the sorted list
        r = bins["ranges"]
        for t in range(r.shape[0]):
            seg = tiles[r[t, 0]:r[t, 1]]
            assert (seg == t).all()
            assert (r[t, 1] - r[t, 0]) == int((tiles == t).sum())


def test_sort_ties_broken_by_index(oracle):
    # duplicated Gaussians have identical keys; the stable sort keeps them in
    # index order
    s = scenes.random_small(24, N=20, width=48, height=48)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        s[k] = np.concatenate([s[k], s[k][:10]])
    proj = oracle.project(s, "f32")
    bins = oracle.bin_sort(s, proj, "f32")
    keys, vals = bins["keys"], bins["vals"]
    same = keys[1:] == keys[:-1]
    assert same.sum() > 0
    assert (vals[1:][same] > vals[:-1][same]).all()


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_tiled_equals_untiled_bruteforce(oracle, precision):
    for s in _scene_variants():
        proj, bins, ras = oracle.forward(s, precision)
        bf = oracle.render_bruteforce(s, proj, precision)
        np.testing.assert_array_equal(ras["image"], bf["image"])
        np.testing.assert_array_equal(ras["final_T"], bf["final_T"])


@pytest.mark.parametrize("precision,tol", [("f32", 2e-6), ("f64", 1e-12)])
def test_weights_plus_final_T_sum_to_one(oracle, precision, tol):
    # With every colour equal to 1 (SH degree 0, DC = 0.5 / C0) and a black
    # background, the image is sum_k alpha_k T_k, so image + T_final = 1.
    C0 = 1 / (2 * math.sqrt(math.pi))
    for s in _scene_variants():
        s["cfg"] = dict(s["cfg"], sh_degree=0)
        s["sh"][:, 0, :] = 0.5 / C0
        s["opacity_logits"] = s["opacity_logits"] + 2.0  # push some pixels to the early stop
        proj, bins, ras = oracle.forward(s, precision)
        total = ras["image"].astype(np.float64) + ras["final_T"][:, None]
        np.testing.assert_allclose(total, 1.0, atol=tol)
        assert (ras["final_T"] < 0.5).any()


def _splat_scene(layers, W=48, H=40, fx=60.0, tile=16):
    """Isotropic Gaussians on the optical axis; `layers` = [(depth, log_scale,
    opacity_logit, colour)]; colour via SH degree 0."""
    C0 = 1 / (2 * math.sqrt(math.pi))
    n = len(layers)
    s = {
        "means": np.array([[0, 0, d] for d, _, _, _ in layers], np.float64),
        "log_scales": np.array([[ls] * 3 for _, ls, _, _ in layers], np.float64),
        "quats": np.tile([1.0, 0, 0, 0], (n, 1)),
        "opacity_logits": np.array([o for _, _, o, _ in layers], np.float64),
        "sh": np.zeros((n, 16, 3)),
        "cams": scenes.camera_row(np.eye(4), fx, fx, W / 2, H / 2)[None],
        "sizes": np.array([[W, H]], np.int32),
        "cfg": scenes.make_cfg(tile_w=tile, tile_h=tile, sh_degree=0),
    }
    for i, (_, _, _, c) in enumerate(layers):
        s["sh"][i, 0, :] = (np.asarray(c, np.float64) - 0.5) / C0
    return s


def test_single_isotropic_splat_closed_form(oracle):
    d, ls, ol, col = 3.0, -2.2, 0.7, (0.9, 0.4, 0.2)
    s = _splat_scene([(d, ls, ol, col)])
    proj, bins, ras = oracle.forward(s, "f64")
    W, H = 48, 40
    sig2 = (60.0 * math.exp(ls) / d) ** 2 + float(np.float32(0.3))
    o = 1 / (1 + math.exp(-ol))
    amin = float(np.float32(1 / 255))
    ys, xs = np.mgrid[0:H, 0:W]
    r2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2
    alpha = np.minimum(float(np.float32(0.99)), o * np.exp(-r2 / (2 * sig2)))
    alpha = np.where(alpha >= amin, alpha, 0.0)
    # pixels outside the splat's 3-sigma tile rectangle see nothing
    x0, y0, x1, y1 = proj["rects"][0]
    inrect = (xs // 16 >= x0) & (xs // 16 < x1) & (ys // 16 >= y0) & (ys // 16 < y1)
    alpha = np.where(inrect, alpha, 0.0).reshape(-1)
    np.testing.assert_allclose(ras["final_T"], 1 - alpha, atol=1e-14)
    np.testing.assert_allclose(ras["image"], alpha[:, None] * np.array(col)[None], atol=1e-14)
    assert ((ras["last"] == 1) == (alpha > 0)).all()


def test_alpha_cap_and_early_stop(oracle):
    # Five nearly opaque splats (opacity 0.95) stacked along the axis: near
    # the centre T goes 1 -> ~0.05 -> ~0.0025 -> ~1.3e-4, and the fourth would
    # take it below 1e-4, so it is not composited and compositing stops.
    ol = math.log(0.95 / 0.05)
    layers = [(3.0 + 0.1 * k, -1.0, ol, (0.2 * (k + 1), 0.5, 1.0 - 0.2 * k)) for k in range(5)]
    s = _splat_scene(layers, W=16, H=16)
    proj, bins, ras = oracle.forward(s, "f64")
    c = 8 * 16 + 8  # pixel (8, 8), sampled at (8.5, 8.5); the splats project to (8, 8)
    sig2 = [(60.0 * math.exp(-1.0) / dd) ** 2 + float(np.float32(0.3)) for dd, _, _, _ in layers]
    r2 = 0.5 ** 2 + 0.5 ** 2
    a = [0.95 * math.exp(-r2 / (2 * v)) for v in sig2]
    T, img = 1.0, np.zeros(3)
    n = 0
    for k in range(5):
        Tn = T * (1 - a[k])
        if Tn < 1e-4:
            break
        img += np.array(layers[k][3]) * a[k] * T
        T = Tn
        n += 1
    assert n == 3
    assert ras["last"][c] == 3
    assert ras["final_T"][c] == pytest.approx(T, rel=1e-12)
    np.testing.assert_allclose(ras["image"][c], img, rtol=1e-12)
    # alpha cap: opacity 0.999 at the centre gives alpha = 0.99 exactly
    s = _splat_scene([(3.0, -0.5, math.log(0.999 / 0.001), (1, 1, 1))], W=16, H=16)
    proj, bins, ras = oracle.forward(s, "f64")
    assert ras["final_T"][c] == pytest.approx(1 - float(np.float32(0.99)), rel=1e-12)


def test_empty_tiles_and_empty_scene(oracle):
    s = scenes.random_small(25, N=4, width=64, height=64)
    s["means"][:, 2] = -5.0  # all behind the camera
    proj, bins, ras = oracle.forward(s, "f32")
    assert bins["n_isect"] == 0
    assert (ras["image"] == 0).all() and (ras["final_T"] == 1).all() and (ras["last"] == 0).all()
