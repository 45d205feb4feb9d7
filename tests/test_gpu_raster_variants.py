"""Rasteriser variants through the C ABI:

- the pair-counting entry points (gs_rasterize_fwd_counted,
  gs_rasterize_bwd_pixels_counted) give the outputs of the plain ones, and
  their counts are consistent: executed >= evaluated >= composited, the
  backward composites exactly the forward's pairs, the backward evaluates no
  more than sum(last) pairs, and the composited count equals the oracle's
  (up to the pairs of tiles holding a near-threshold pixel);
- every tile shape x pixels per thread x splats per shared-memory batch
  (the autotuner's search space) renders the default image bit for bit, and
  its backward matches the oracle within the gradient tolerance.
"""

import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes

from gpu_util import grad_close, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_11390_gb300 import _native

    _native.load()


def _render(s, cfg):
    from paper_2606_11390_gb300 import renderer as R
    import torch

    N = int(s["means"].shape[0])
    params = R.FlatParams(N).load_from(s)
    cams = R.Cameras(s["cams"], s["sizes"])
    frame = R.Frame(N, cams, cfg)
    R.render(params, cams, frame)
    torch.cuda.synchronize()
    assert frame.read_status() == 0
    return params, cams, frame


def _upstream(s, o_ras, seed=7):
    rng = np.random.default_rng(seed)
    P = s["target"].shape[0]
    dl = (rng.standard_normal((P, 3)) / P).astype(np.float32)
    dl[o_ras["marginal_pix"].astype(bool)] = 0
    return dl


def _marginal_pair_bound(s, cfg, bins, o_ras):
    """Pairs of the tiles that hold a near-threshold pixel: a bound on how far
    two correct float implementations' composited counts can differ."""
    tw, th = cfg["tile_w"], cfg["tile_h"]
    bound, base, pix = 0, 0, 0
    for W, H in s["sizes"]:
        W, H = int(W), int(H)
        ntx, nty = -(-W // tw), -(-H // th)
        m = o_ras["marginal_pix"][pix:pix + W * H].reshape(H, W).astype(bool)
        for ty, tx in zip(*np.nonzero(m)):
            t = base + (ty // th) * ntx + tx // tw
            a, b = bins["ranges"][t]
            bound += int(b - a)  # per marginal pixel: at most its whole list
        base += ntx * nty
        pix += W * H
    return bound


COUNT_SCENES = {
    "tiny": lambda: scenes.tiny(),
    "ragged_2view": lambda: scenes.random_small(101, N=1000, width=173, height=91, n_views=2, spread=1.5),
    "tile8_3view": lambda: scenes.random_small(102, N=777, width=97, height=131, n_views=3, tile=8,
                                               log_scale_mu=-2.2),
    "early_stop": lambda: _early_stop_scene(),
}


def _early_stop_scene():
    s = scenes.random_small(203, N=800, width=120, height=90, spread=1.0, log_scale_mu=-1.8)
    s["opacity_logits"] = s["opacity_logits"] + 2.5
    return s


@pytest.mark.parametrize("name", list(COUNT_SCENES))
def test_pair_counts(oracle, name):
    import torch

    from paper_2606_11390_gb300 import _native as gs

    s = COUNT_SCENES[name]()
    cfg = dict(s["cfg"])
    params, cams, fr = _render(s, cfg)
    o_proj, o_bins, o_ras = oracle.forward(s, "f32")
    img = torch.zeros_like(fr.image)
    fT = torch.zeros_like(fr.final_T)
    last = torch.zeros_like(fr.last)
    cf = torch.zeros(3, dtype=torch.int64, device="cuda")
    gs.gs_rasterize_fwd_counted(fr.projected, fr.vals, fr.tile_ranges, cams.sizes, fr.cfg, img, fT, last, cf)
    dl = torch.from_numpy(_upstream(s, o_ras).reshape(-1)).cuda()
    dp = torch.zeros_like(fr.d_projected)
    cb = torch.zeros(3, dtype=torch.int64, device="cuda")
    gs.gs_rasterize_bwd_pixels_counted(fr.projected, fr.vals, fr.tile_ranges, cams.sizes, fr.cfg, fr.N, fr.final_T,
                                       fr.last, dl, dp, cb)
    gs.gs_rasterize_bwd_pixels(fr.projected, fr.vals, fr.tile_ranges, cams.sizes, fr.cfg, fr.N, fr.final_T, fr.last,
                               dl, fr.d_projected)
    torch.cuda.synchronize()
    # same outputs as the plain kernels
    assert torch.equal(img, fr.image) and torch.equal(fT, fr.final_T) and torch.equal(last, fr.last)
    grad_close(to_np(dp).reshape(-1, 9), to_np(fr.d_projected).reshape(-1, 9).astype(np.float64), rel=1e-4,
               name="d_projected (counted vs plain)")
    ex_f, ev_f, co_f = (int(x) for x in cf.cpu())
    ex_b, ev_b, co_b = (int(x) for x in cb.cpu())
    sum_last = int(to_np(fr.last, np.uint32).astype(np.int64).sum())
    print(f"{name}: fwd executed {ex_f} evaluated {ev_f} composited {co_f}; bwd executed {ex_b} evaluated {ev_b} "
          f"composited {co_b}; sum(last) {sum_last}")
    assert ex_f >= ev_f >= co_f > 0
    assert ex_b >= ev_b >= co_b > 0
    assert co_b == co_f  # the backward takes exactly the forward's decisions
    assert ev_b <= sum_last
    o_co = int(o_ras["composited"].astype(np.int64).sum())
    bound = _marginal_pair_bound(s, cfg, o_bins, o_ras)
    assert abs(co_f - o_co) <= bound, (co_f, o_co, bound)
    if bound == 0:
        assert co_f == o_co


TUNE_SCENE = lambda: scenes.random_small(211, N=1500, width=211, height=133, n_views=2, spread=1.5)  # noqa: E731
TILES = [(8, 8, 0), (16, 16, 0), (16, 16, 2), (32, 16, 0), (32, 16, 2), (32, 32, 0), (32, 32, 2)]
BATCHES = [0, 64, 128, 256, 512]


@pytest.mark.parametrize("tw,th,flags", TILES, ids=[f"{a}x{b}{'_2px' if f else ''}" for a, b, f in TILES])
def test_every_batch_size_renders_the_same(oracle, tw, th, flags):
    import torch

    from paper_2606_11390_gb300 import renderer as R

    s = TUNE_SCENE()
    s["cfg"] = scenes.make_cfg(tile_w=tw, tile_h=th, flags=flags)
    o_proj, o_bins, o_ras = oracle.forward(s, "f32")
    dl_np = _upstream(s, o_ras)
    _, o_grads = oracle.backward(s, o_proj, o_bins, dl_np.astype(np.float64), "f32")
    dl = torch.from_numpy(dl_np.reshape(-1)).cuda()
    ref = None
    # each direction's batch sizes against the other's default
    # (512 backward splats take more than 48 KB of shared memory on tiles of
    # more than 4 warps, launched with the opt-in)
    combos = [(bf, 0) for bf in BATCHES] + [(0, bb) for bb in BATCHES[1:]]
    for bf, bb in combos:
        cfg = dict(s["cfg"], raster_batch_fwd=bf, raster_batch_bwd=bb)
        params, cams, fr = _render(s, cfg)
        grads = params.like()
        R.rasterize_bwd(params, cams, fr, dl, grads)
        torch.cuda.synchronize()
        assert fr.read_status() == 0
        img = to_np(fr.image)
        if ref is None:
            ref = (img, to_np(fr.final_T), to_np(fr.last))
            marg = o_ras["marginal_pix"].astype(bool)
            np.testing.assert_allclose(img.reshape(-1, 3)[~marg], o_ras["image"][~marg], atol=1e-5, rtol=0)
        else:
            np.testing.assert_array_equal(img, ref[0], err_msg=f"batch {bf}/{bb}")
            np.testing.assert_array_equal(to_np(fr.final_T), ref[1])
            np.testing.assert_array_equal(to_np(fr.last), ref[2])
        for k in ("means", "opacity_logits", "sh"):
            grad_close(to_np(grads[k]), o_grads[k], name=f"{k} batch {bf}/{bb}")


def test_bad_batch_size_is_rejected():
    import torch

    from paper_2606_11390_gb300 import _native as gs

    s = scenes.tiny()
    params, cams, fr = _render(s, dict(s["cfg"]))
    for val in (96, 1024, 32):
        with pytest.raises(gs.GSError):
            gs.gs_rasterize_fwd(fr.projected, fr.vals, fr.tile_ranges, cams.sizes, dict(fr.cfg, raster_batch_fwd=val),
                                fr.image, fr.final_T, fr.last)
        with pytest.raises(gs.GSError):
            gs.gs_rasterize_bwd_pixels(fr.projected, fr.vals, fr.tile_ranges, cams.sizes,
                                       dict(fr.cfg, raster_batch_bwd=val), fr.N, fr.final_T, fr.last,
                                       torch.zeros_like(fr.image), fr.d_projected)


@pytest.mark.parametrize("tw,th,flags", [(32, 16, 0), (16, 16, 2), (8, 8, 0), (32, 32, 2)],
                         ids=["32x16", "16x16_2px", "8x8", "32x32_2px_no_masks"])
def test_backward_with_the_forwards_cull_masks(oracle, tw, th, flags):
    """The backward reusing the forward's per-entry cull masks takes the same
    decisions as computing them itself: the same pair counts, and the same
    gradients up to the order of the FP32 atomics; a backward with another
    warp layout (pixels per thread) than the forward's ignores the masks."""
    import torch

    from paper_2606_11390_gb300 import _native as gs

    s = TUNE_SCENE()
    s["cfg"] = scenes.make_cfg(tile_w=tw, tile_h=th, flags=flags)
    params, cams, fr = _render(s, dict(s["cfg"]))  # the forward writes fr.cull
    o_proj, o_bins, o_ras = oracle.forward(s, "f32")
    dl_np = _upstream(s, o_ras)
    o_dproj, _ = oracle.backward(s, o_proj, o_bins, dl_np.astype(np.float64), "f32")
    dl = torch.from_numpy(dl_np.reshape(-1)).cuda()
    out = {}
    for name, cfg, masks in (("own", fr.cfg, None), ("handed", fr.cfg, fr.cull),
                             ("other_layout", dict(fr.cfg, flags=int(fr.cfg["flags"]) ^ gs.GS_FLAG_RASTER_2PX)
                              if tw != 8 else fr.cfg, fr.cull)):
        dp = torch.zeros_like(fr.d_projected)
        cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
        gs.gs_rasterize_bwd_pixels_counted(fr.projected, fr.vals, fr.tile_ranges, cams.sizes, cfg, fr.N, fr.final_T,
                                           fr.last, dl, dp, cnt, cull_masks=masks)
        torch.cuda.synchronize()
        out[name] = (to_np(dp).reshape(-1, 9), [int(x) for x in cnt.cpu()])
        grad_close(out[name][0], o_dproj, name=f"d_projected ({name})")
    assert out["handed"][1] == out["own"][1]
    if tw == 32 and th == 32 and flags:
        assert not fr.cull.any()  # layouts of more than 8 warps hand no masks over
    else:
        # entries the forward staged carry its layout's tag (the forward stops
        # staging a tile once all its pixels are done)
        n = int(fr.n_isect.item())
        tags = to_np(fr.cull[:n]).view(np.uint16) >> 8
        want = {(32, 16, 0): 0x85, (16, 16, 2): 0x82, (8, 8, 0): 0x81}[(tw, th, flags)]
        assert set(np.unique(tags).tolist()) <= {0, want}
        assert (tags == want).mean() > 0.5
