"""GPU vs oracle parity through the C ABI (libgs_gb300.so).

Bars: bit-exact tile counts, rectangles, depths, sorted keys/values and tile
ranges; images within 1e-5 absolute; gradients within 1e-3 relative (see
gpu_util.grad_close). Pixels whose compositing involved a decision within
1e-4 (relative) of a threshold (alpha cutoff, alpha cap, transmittance stop)
can legitimately go either way between two correct float implementations;
the oracle flags them, they are checked at 1e-2 and their share is bounded;
gradients are compared element-wise with their upstream gradient set to zero.
"""
import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes

from gpu_util import grad_close, norm_close, run_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_11390_gb300 import _native

    _native.load()


def _scenes():
    yield "tiny_cfg", scenes.tiny()
    yield "ragged_2view", scenes.random_small(101, N=1000, width=173, height=91, n_views=2, spread=1.5)
    s = scenes.random_small(102, N=777, width=97, height=131, n_views=3, tile=8, log_scale_mu=-2.2)
    yield "tile8_3view", s
    s = scenes.random_small(103, N=513, width=150, height=70, n_views=1, log_scale_mu=-1.5)
    s["cfg"] = scenes.make_cfg(tile_w=32, tile_h=16, bg=(0.2, 0.5, 0.9))
    yield "tile32x16_bg", s
    yield "sh_deg1", scenes.random_small(104, N=300, width=64, height=64, sh_degree=1)
    # 9 views take the projection backward whose SH slice is transposed in
    # shared memory; 1000 Gaussians leave a partial last slice
    yield "nine_views", scenes.random_small(105, N=1000, width=64, height=48, n_views=9, spread=1.5)
    # several views at SH degree 2: the tensor copies move all 48 coefficients
    # and the backward writes zeros past the degree (640: full slices only)
    yield "sh_deg2_3view", scenes.random_small(107, N=640, width=80, height=60, n_views=3, spread=1.5, sh_degree=2)
    s = scenes.random_small(110, N=900, width=150, height=100, n_views=2, spread=1.5)
    s["cfg"] = scenes.make_cfg(flags=2)  # two pixels per rasteriser thread
    yield "two_px_per_thread", s
    s = scenes.random_small(111, N=900, width=150, height=100, n_views=1, spread=1.5)
    s["cfg"] = scenes.make_cfg(tile_w=32, tile_h=16, flags=2)
    yield "tile32x16_two_px", s
    s = scenes.random_small(112, N=1500, width=200, height=150, n_views=2, spread=1.5)
    s["cfg"] = scenes.make_cfg(tile_w=32, tile_h=32)
    yield "tile32x32", s


SCENES = list(_scenes())
IDS = [n for n, _ in SCENES]


def _check_forward(s, g, o_proj, o_bins, o_ras):
    # integers and the strictly rounded projection path: bit-exact
    np.testing.assert_array_equal(g["counts"], o_proj["counts"])
    np.testing.assert_array_equal(g["rects"], o_proj["rects"])
    vis = o_proj["counts"] > 0
    for k, name in ((0, "mean2d.x"), (1, "mean2d.y"), (2, "A"), (3, "B"), (4, "C"), (6, "depth"), (7, "radius")):
        np.testing.assert_array_equal(g["projected"][vis, k], o_proj["projected"][vis, k], err_msg=name)
    np.testing.assert_allclose(g["projected"][vis, 5], o_proj["projected"][vis, 5], rtol=2e-6, err_msg="opacity")
    np.testing.assert_allclose(g["projected"][vis, 8:11], o_proj["projected"][vis, 8:11], atol=2e-6, err_msg="rgb")
    assert not g["projected"][~vis].any()
    # the depth keys gs_project writes for the sort: the depth's float bits where visible, 0 where culled
    np.testing.assert_array_equal(g["depth_keys"][vis], o_proj["projected"][vis, 6].astype(np.float32).view(np.uint32))
    assert not g["depth_keys"][~vis].any()
    # keys / values / ranges: bit-exact
    assert g["n_isect"] == o_bins["n_isect"]
    if g["keys"] is not None:
        np.testing.assert_array_equal(g["keys"], o_bins["keys"])
    np.testing.assert_array_equal(g["vals"], o_bins["vals"])
    np.testing.assert_array_equal(g["ranges"], o_bins["ranges"])
    # images
    marg = o_ras["marginal_pix"].astype(bool)
    assert marg.mean() < 0.01, marg.mean()
    np.testing.assert_allclose(g["image"][~marg], o_ras["image"][~marg], atol=1e-5, rtol=0)
    np.testing.assert_allclose(g["image"][marg], o_ras["image"][marg], atol=1e-2, rtol=0)
    np.testing.assert_allclose(g["final_T"][~marg], o_ras["final_T"][~marg], atol=1e-5, rtol=0)
    np.testing.assert_array_equal(g["last"][~marg], o_ras["last"][~marg])


@pytest.mark.parametrize("name,s", SCENES, ids=IDS)
def test_forward_parity(oracle, name, s):
    o_proj, o_bins, o_ras = oracle.forward(s, "f32")
    g = run_gpu(s)
    assert g["status"] == 0
    _check_forward(s, g, o_proj, o_bins, o_ras)


@pytest.mark.parametrize("name,s", SCENES, ids=IDS)
def test_forward_parity_without_keys(oracle, name, s):
    """Without the optional 64-bit keys the sort may take its packed path
    (per-tile counts, packed second pass): the same lists, ranges and image."""
    o_proj, o_bins, o_ras = oracle.forward(s, "f32")
    g = run_gpu(s, keep_keys=False)
    assert g["status"] == 0
    _check_forward(s, g, o_proj, o_bins, o_ras)


@pytest.mark.parametrize("name,s", SCENES, ids=IDS)
def test_backward_parity(oracle, name, s):
    """Element-wise on every record, with the upstream gradient of the
    near-threshold pixels set to zero: a pixel composites on its own, so this
    removes exactly the contributions that depend on a decision two correct
    float implementations may take differently. With the full upstream
    gradient, the relative-norm bound holds over all records."""
    rng = np.random.default_rng(7)
    P = s["target"].shape[0]
    dl = (rng.standard_normal((P, 3)) / P).astype(np.float32)
    o_proj, o_bins, o_ras = oracle.forward(s, "f32")
    marg = o_ras["marginal_pix"].astype(bool)
    print(f"{name}: near-threshold pixels {marg.mean():.4f}, records touched by one "
          f"{(o_ras['marginal_vg'] != 0).mean():.4f}")
    N = s["means"].shape[0]
    dl_m = dl.copy()
    dl_m[marg] = 0
    o_dproj, o_grads = oracle.backward(s, o_proj, o_bins, dl_m.astype(np.float64), "f32")
    g = run_gpu(s, dL_dimage=dl_m)
    assert g["status"] == 0
    grad_close(g["d_projected"], o_dproj, name="d_projected")
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        grad_close(g["grads"][k], o_grads[k], name=k)
    o_dproj, o_grads = oracle.backward(s, o_proj, o_bins, dl.astype(np.float64), "f32")
    g = run_gpu(s, dL_dimage=dl)
    assert g["status"] == 0
    norm_close(g["d_projected"], o_dproj, name="d_projected (full upstream)")
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        norm_close(g["grads"][k], o_grads[k], name=f"{k} (full upstream)")
    assert N > 0


def test_capacity_overflow_sets_status_and_recovers(oracle):
    s = scenes.random_small(105, N=400, width=96, height=80)
    o_proj, o_bins, _ = oracle.forward(s, "f32")
    g = run_gpu(s, capacity=17)  # render() grows the buffers and reruns
    assert g["capacity"] >= o_bins["n_isect"]
    np.testing.assert_array_equal(g["keys"], o_bins["keys"])


@pytest.mark.parametrize("order", [False, True])
def test_overflowed_sort_keeps_ranges_inside_the_capacity(oracle, order):
    """After an overflow the lists are unusable (GS_STATUS_CAPACITY), but a
    consumer that reads them before checking the status (a captured step's
    rasteriser) must stay inside `vals`: every range lies in [0, capacity]."""
    import torch

    from paper_2606_11390_gb300 import _native as gs
    from paper_2606_11390_gb300 import renderer as R

    s = scenes.random_small(201, N=3000, width=120, height=90, n_views=4, spread=1.5, tile=8)
    o_proj, o_bins, _ = oracle.forward(s, "f32")
    N = s["means"].shape[0]
    params = R.FlatParams(N).load_from(s)
    cams = R.Cameras(s["cams"], s["sizes"])
    for cap in (1, 1000, o_bins["n_isect"] // 2):
        fr = R.Frame(N, cams, s["cfg"], capacity=cap, keep_keys=True, tile_order=order)
        R.project(params, cams, fr)
        R.bin_sort(fr)
        torch.cuda.synchronize()
        assert fr.read_status() & gs.GS_STATUS_CAPACITY
        assert int(fr.n_isect.item()) == o_bins["n_isect"]  # the exact total, even when clipped
        rg = to_np(fr.ranges, np.uint32).reshape(-1, 2)
        assert (rg[:, 0] <= rg[:, 1]).all() and rg.max() <= cap


def test_empty_and_fully_culled(oracle):
    s = scenes.random_small(106, N=50, width=40, height=30)
    s["means"][:, 2] = -3.0
    g = run_gpu(s, dL_dimage=np.ones((1200, 3), np.float32))
    assert g["n_isect"] == 0 and g["status"] == 0
    assert (g["image"] == 0).all() and (g["final_T"] == 1).all() and (g["last"] == 0).all()
    for k, v in g["grads"].items():
        assert not v.any(), k


def test_single_pixel_image_and_one_gaussian(oracle):
    s = scenes.random_small(107, N=1, width=1, height=1, log_scale_mu=0.0, depth=3.0, spread=0.01)
    o_proj, o_bins, o_ras = oracle.forward(s, "f32")
    g = run_gpu(s)
    _check_forward(s, g, o_proj, o_bins, o_ras)


def test_ties_broken_by_index(oracle):
    s = scenes.random_small(108, N=200, width=80, height=64)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        s[k] = np.concatenate([s[k], s[k][:100], s[k][:50]])
    o_proj, o_bins, o_ras = oracle.forward(s, "f32")
    g = run_gpu(s)
    same = o_bins["keys"][1:] == o_bins["keys"][:-1]
    assert same.sum() > 100
    np.testing.assert_array_equal(g["keys"], o_bins["keys"])
    np.testing.assert_array_equal(g["vals"], o_bins["vals"])


def test_many_sort_tiles_and_passes(oracle):
    # > 4096 keys per sort tile and several hundred image tiles: exercises the
    # look-back across sort tiles and the tile-id digit passes
    s = scenes.random_small(109, N=20000, width=640, height=480, n_views=2, spread=2.0, log_scale_mu=-2.8)
    o_proj, o_bins, o_ras = oracle.forward(s, "f32")
    assert o_bins["n_isect"] > 50000
    g = run_gpu(s)
    _check_forward(s, g, o_proj, o_bins, o_ras)


@pytest.mark.parametrize("keep_keys", [True, False])
def test_three_tile_id_passes(oracle, keep_keys):
    """More than 65536 tiles (two 2048x2048 views in 8x8 tiles: 17 tile-id
    bits) takes three tile-id digit passes; lists, ranges and counts stay
    bit-exact."""
    s = scenes.random_small(112, N=3000, width=2048, height=2048, n_views=2, spread=2.5, tile=8, log_scale_mu=-3.5)
    o_proj = oracle.project(s, "f32")
    o_bins = oracle.bin_sort(s, o_proj, "f32")
    assert oracle.num_tiles(s) > 65536 and o_bins["n_isect"] > 1_000_000
    g = run_gpu(s, keep_keys=keep_keys)
    assert g["status"] == 0
    assert g["n_isect"] == o_bins["n_isect"]
    if keep_keys:
        np.testing.assert_array_equal(g["keys"], o_bins["keys"])
    np.testing.assert_array_equal(g["vals"], o_bins["vals"])
    np.testing.assert_array_equal(g["ranges"], o_bins["ranges"])


def test_image_loss(oracle):
    import torch

    from paper_2606_11390_gb300 import _native

    rng = np.random.default_rng(3)
    for n in (1, 7, 4096 * 3 + 5):
        img = rng.random(n).astype(np.float32)
        tgt = rng.random(n).astype(np.float32)
        L, g = oracle.loss(img, tgt, 1.0, 0.2)
        ti, tt = torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda()
        dl = torch.zeros(n, device="cuda")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        _native.gs_image_loss(ti, tt, 1.0, 0.2, dl, loss)
        torch.cuda.synchronize()
        assert loss.item() == pytest.approx(L, rel=1e-6)
        np.testing.assert_allclose(dl.cpu().numpy(), g, rtol=1e-5, atol=1e-9)


def test_adam(oracle):
    import torch

    from paper_2606_11390_gb300 import _native

    rng = np.random.default_rng(4)
    n = 1031
    p0 = rng.standard_normal(n)
    m = np.zeros(n)
    v = np.zeros(n)
    tp = torch.from_numpy(p0.astype(np.float32)).cuda()
    tm, tv = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = p0.astype(np.float32).astype(np.float64)
    for t in range(1, 6):
        gr = rng.standard_normal(n).astype(np.float32)
        p, m, v = oracle.adam(p, gr.astype(np.float64), m, v, 1e-3, 0.9, 0.999, 1e-15, t)
        step.fill_(t)
        _native.gs_adam_step(tp, torch.from_numpy(gr).cuda(), tm, tv, 1e-3, 0.9, 0.999, 1e-15, step)
    torch.cuda.synchronize()
    np.testing.assert_allclose(tp.cpu().numpy(), p, rtol=0, atol=2e-6)


def test_tile_order_is_longest_first_permutation(oracle):
    """With the tile-order flag gs_bin_sort appends a permutation of the tile
    ids whose list lengths never increase by more than a half-octave bucket,
    and the images equal those rendered in the natural tile order."""
    s = scenes.random_small(113, N=4000, width=300, height=200, n_views=2, spread=1.5)
    a = run_gpu(s)  # Frame default: tile order on
    from paper_2606_11390_gb300 import renderer as R
    import torch

    N = s["means"].shape[0]
    params = R.FlatParams(N).load_from(s)
    cams = R.Cameras(s["cams"], s["sizes"])
    fr = R.Frame(N, cams, s["cfg"], keep_keys=False, tile_order=False)
    R.render(params, cams, fr)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(to_np(fr.image).reshape(-1, 3), a["image"])
    np.testing.assert_array_equal(to_np(fr.ranges, np.uint32).reshape(-1, 2), a["ranges"])
    fo = R.Frame(N, cams, s["cfg"], keep_keys=False, tile_order=True)
    R.render(params, cams, fo)
    torch.cuda.synchronize()
    nt = fo.n_tiles
    order = to_np(fo.tile_ranges, np.uint32)[2 * nt:3 * nt]
    assert sorted(order.tolist()) == list(range(nt))
    lens = (a["ranges"][:, 1].astype(np.int64) - a["ranges"][:, 0])[order]
    nz = lens[lens > 0]
    # non-increasing up to the bucket width (a factor of 2 at most between neighbours out of order)
    assert np.all(nz[1:] <= 2 * nz[:-1])
    assert np.all(lens[len(nz):] == 0)


@pytest.mark.parametrize("idx", [1, 2, 7])
def test_forward_with_l1l2_loss(oracle, idx):
    """gs_rasterize_fwd_l1l2 equals gs_rasterize_fwd followed by gs_image_loss:
    image, final T, last and dL/dimage bit for bit, the loss up to the
    rounding of its float partial sums (grouped differently by the two
    kernels); one call for all views and one call per view (accumulated)."""
    import torch

    from paper_2606_11390_gb300 import _native
    from paper_2606_11390_gb300 import renderer as R

    name, s = SCENES[idx]
    N = int(s["means"].shape[0])
    params = R.FlatParams(N).load_from(s)
    cams = R.Cameras(s["cams"], s["sizes"])
    P = cams.n_pixels
    rng = np.random.default_rng(7 + idx)
    tgt = torch.from_numpy(rng.random(P * 3).astype(np.float32)).cuda()
    w1, w2 = 1.0, 0.2
    fa = R.Frame(N, cams, s["cfg"])
    R.render(params, cams, fa)
    dla = torch.zeros(P * 3, device="cuda")
    la = torch.zeros(1, dtype=torch.float64, device="cuda")
    _native.gs_image_loss(fa.image, tgt, w1, w2, dla, la)
    # one call for all views
    fb = R.Frame(N, cams, s["cfg"], capacity=fa.capacity)
    R.project(params, cams, fb)
    R.bin_sort(fb)
    dlb = torch.full((P * 3,), 7.0, device="cuda")
    lb = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
    R.rasterize_fwd_l1l2(fb, tgt, P * 3, w1, w2, False, dlb, lb)
    torch.cuda.synchronize()
    assert fb.read_status() == 0
    for a, b in ((fa.image, fb.image), (fa.final_T, fb.final_T), (fa.last, fb.last), (dla, dlb)):
        np.testing.assert_array_equal(to_np(a), to_np(b))
    assert lb.item() == pytest.approx(la.item(), rel=1e-6)
    L_ref, _ = oracle.loss(to_np(fa.image), to_np(tgt), w1, w2)
    assert lb.item() == pytest.approx(L_ref, rel=1e-6)
    # one call per view, the loss accumulated over the views
    dlc = torch.zeros(P * 3, device="cuda")
    lc = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
    img_c = torch.zeros(P * 3, device="cuda")
    for v in range(cams.V):
        cv = cams.view(v)
        a, b = int(cams.pix_base[v]) * 3, int(cams.pix_base[v + 1]) * 3
        fv = R.Frame(N, cv, s["cfg"], capacity=fa.capacity)
        R.project(params, cv, fv)
        R.bin_sort(fv)
        fv.image = img_c[a:b]
        R.rasterize_fwd_l1l2(fv, tgt[a:b], P * 3, w1, w2, v > 0, dlc[a:b], lc)
        torch.cuda.synchronize()
        assert fv.read_status() == 0
    np.testing.assert_array_equal(to_np(img_c), to_np(fa.image))
    np.testing.assert_array_equal(to_np(dlc), to_np(dla))
    assert lc.item() == pytest.approx(la.item(), rel=1e-6)
    # the mean must cover at least this call's values
    with pytest.raises(_native.GSError):
        R.rasterize_fwd_l1l2(fb, tgt, P * 3 - 1, w1, w2, False, dlb, lb)


@pytest.mark.parametrize("N", [1000, 777])
def test_accumulated_backward_adds(N):
    """A backward with GS_FLAG_ACCUMULATE_GRADS adds its gradients to those in
    the output arrays. With N = 1000 the SH gradient array is 16-byte aligned
    and leaves the projection backward by tensor reduce-adds; with N = 777 it
    is not and takes plain loads and stores."""
    import torch

    from paper_2606_11390_gb300 import renderer as R

    s = scenes.random_small(106, N=N, width=96, height=64, n_views=2, spread=1.5)
    params = R.FlatParams(N).load_from(s)
    cams = R.Cameras(s["cams"], s["sizes"])
    frame = R.Frame(N, cams, dict(s["cfg"]))
    R.render(params, cams, frame)
    rng = np.random.default_rng(3)
    dl = torch.from_numpy(rng.standard_normal(frame.image.numel()).astype(np.float32) / 1e3).cuda()
    fresh = params.like()
    R.rasterize_bwd(params, cams, frame, dl, fresh)
    summed = params.like()
    base = torch.from_numpy(rng.standard_normal(summed.flat.numel()).astype(np.float32)).cuda()
    summed.flat.copy_(base)
    R.rasterize_bwd(params, cams, frame, dl, summed, accumulate=True)
    torch.cuda.synchronize()
    assert frame.read_status() == 0
    want = base.cpu().numpy().astype(np.float64) + to_np(fresh.flat).astype(np.float64)
    got = to_np(summed.flat).astype(np.float64)
    # the two backward calls may sum their atomics in another order
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6)
    assert np.abs(to_np(fresh["sh"])).max() > 0
