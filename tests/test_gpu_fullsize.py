"""Parity at full size: the 4M-Gaussian 3840x2160 workload in the launch
configuration bench.py times (graph-captured batched step, the workload's
tile shape).

- every tile count, rectangle and projected record of the 4M Gaussians against
  the oracle's projection;
- the total intersection count;
- for sampled tiles, the sorted list (exact) against a brute-force list built
  from the oracle's rectangles and depths, and the rendered pixels;
- for sampled Gaussians whose tiles are all included, the complete parameter
  gradients under a seeded upstream gradient (zero on near-threshold pixels),
  with the oracle compositing those tiles from its own lists.
"""
import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes

from gpu_util import grad_close, to_np

pytestmark = pytest.mark.gpu


def _tile_list(proj, tile, ntx):
    """Oracle-side list of tile `tile` (view 0): visible records whose
    rectangle contains it, in (depth, index) order."""
    tx, ty = tile % ntx, tile // ntx
    r = proj["rects"]
    m = (proj["counts"] > 0) & (r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3])
    idx = np.nonzero(m)[0]
    depth = proj["projected"][idx, 6].astype(np.float32)
    return idx[np.lexsort((idx, depth))].astype(np.uint32)


def test_full_size_4k_sampled(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_11390_gb300 import _native
    from paper_2606_11390_gb300 import renderer as R

    _native.load()
    s = scenes.diff_4k()
    N = s["means"].shape[0]
    W, H = (int(x) for x in s["sizes"][0])
    st = R.TrainStep(s, mode="batched", graph=True).prepare()
    st.run()
    torch.cuda.synchronize()
    st.check()
    fr = st.frames[0]
    g_counts = to_np(fr.counts, np.uint32)
    g_rects = to_np(fr.rects).reshape(-1, 4)
    g_proj = to_np(fr.projected).reshape(-1, 12)
    g_ranges = to_np(fr.ranges, np.uint32).reshape(-1, 2)
    g_vals = to_np(fr.vals, np.uint32)
    g_img = to_np(st.image).reshape(-1, 3)

    # 1. projection of all Gaussians
    o_proj = oracle.project(s, "f32")
    np.testing.assert_array_equal(g_counts, o_proj["counts"])
    np.testing.assert_array_equal(g_rects, o_proj["rects"])
    vis = o_proj["counts"] > 0
    for k in (0, 1, 2, 3, 4, 6, 7):
        np.testing.assert_array_equal(g_proj[vis, k], o_proj["projected"][vis, k])
    np.testing.assert_allclose(g_proj[vis, 5], o_proj["projected"][vis, 5], rtol=2e-6)
    np.testing.assert_allclose(g_proj[vis, 8:11], o_proj["projected"][vis, 8:11], atol=2e-6)
    I = int(o_proj["counts"].astype(np.int64).sum())
    assert st.n_isect() == I

    # 2. sampled tiles: lists and pixels
    tw, th = s["cfg"]["tile_w"], s["cfg"]["tile_h"]
    ntx, nty = -(-W // tw), -(-H // th)
    rng = np.random.default_rng(11)
    lens = g_ranges[:, 1].astype(np.int64) - g_ranges[:, 0]
    heavy = np.argsort(lens)[-4:]
    tiles = np.unique(np.concatenate([rng.choice(ntx * nty, 20, replace=False), heavy, [0, ntx * nty - 1]]))
    lists = {}
    for t in tiles:
        lst = _tile_list(o_proj, int(t), ntx)
        lists[int(t)] = lst
        got = g_vals[g_ranges[t, 0]:g_ranges[t, 1]]
        np.testing.assert_array_equal(got, lst, err_msg=f"tile {t}")

    # 3. sampled Gaussians with small rectangles: complete gradients
    small = np.nonzero(vis & (o_proj["counts"] <= 4))[0]
    gsel = np.sort(rng.choice(small, 48, replace=False))
    gt = set()
    for g in gsel:
        x0, y0, x1, y1 = o_proj["rects"][g]
        gt.update(ty * ntx + tx for ty in range(y0, y1) for tx in range(x0, x1))
    for t in gt:
        if t not in lists:
            lists[t] = _tile_list(o_proj, t, ntx)
    all_tiles = np.array(sorted(lists), np.int64)
    vals_o = np.concatenate([lists[int(t)] for t in all_tiles]).astype(np.uint32)
    ranges_o = np.zeros((ntx * nty, 2), np.uint32)
    pos = 0
    for t in all_tiles:
        n = lists[int(t)].shape[0]
        ranges_o[t] = (pos, pos + n)
        pos += n
    bins_o = {"vals": vals_o, "ranges": ranges_o}
    ras = oracle.raster_fwd(s, o_proj, bins_o, "f32", tiles=all_tiles)
    pix = []
    for t in all_tiles:
        tx, ty = int(t) % ntx, int(t) // ntx
        ys, xs = np.mgrid[ty * th:min(ty * th + th, H), tx * tw:min(tx * tw + tw, W)]
        pix.append((ys * W + xs).reshape(-1))
    pix = np.concatenate(pix)
    marg = ras["marginal_pix"][pix].astype(bool)
    assert marg.mean() < 0.02
    np.testing.assert_allclose(g_img[pix][~marg], ras["image"][pix][~marg], atol=1e-5, rtol=0)
    np.testing.assert_allclose(to_np(fr.final_T)[pix][~marg], ras["final_T"][pix][~marg], atol=1e-5, rtol=0)

    P = W * H
    dl = (rng.standard_normal((P, 3)) / P).astype(np.float32)
    # near-threshold pixels of the sampled tiles get a zero upstream gradient
    # (each pixel composites on its own, so no other contribution changes)
    dl[pix[marg]] = 0
    grads = st.params.like()
    R.rasterize_bwd(st.params, st.cams, fr, torch.from_numpy(dl).cuda().view(-1), grads)
    torch.cuda.synchronize()
    assert fr.read_status() == 0
    d_o = oracle.raster_bwd(s, o_proj, bins_o, dl.astype(np.float64), "f32", tiles=all_tiles)
    print(f"near-threshold pixels {marg.mean():.4f}, sampled records touched by one "
          f"{(ras['marginal_vg'][gsel] != 0).mean():.4f}")
    grad_close(to_np(fr.d_projected).reshape(-1, 9)[gsel], d_o[gsel], name="d_projected")
    o_g = oracle.project_bwd(s, d_o, "f32", gaussians=gsel)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        grad_close(to_np(grads[k])[gsel], o_g[k], name=k)
