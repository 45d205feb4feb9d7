"""gs_bin_sort_static: the key sort for callers that cannot allocate device
memory (for example a plug-in whose host application owns all device
allocations, or a service that forbids allocation after start-up). It keeps
its scratch in a fixed device array inside the library instead of taking a
workspace. Its output must equal gs_bin_sort's, call after call, although the
shared array keeps whatever the previous call left in it.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_11390_gb300 import _native
    from paper_2606_11390_gb300 import renderer as R

    _native.load()
    return torch, _native, R


def _sorted_both_ways(rt, scene, tile_order=False):
    torch, gs, R = rt
    N = int(scene["means"].shape[0])
    params = R.FlatParams(N).load_from(scene)
    cams = R.Cameras(scene["cams"], scene["sizes"])
    frame = R.Frame(N, cams, scene["cfg"], keep_keys=True, tile_order=tile_order)
    R.render(params, cams, frame)  # gs_project + gs_bin_sort (workspace) with capacity sizing
    torch.cuda.synchronize()
    n = int(frame.n_isect.item())
    # with a tile order, tile_ranges also holds the order after the ranges
    ref = (frame.keys[:n].clone(), frame.vals[:n].clone(), frame.tile_ranges.clone(), n)
    # the allocation-free variant, into outputs pre-filled with junk
    keys = torch.full_like(frame.keys, -7)
    vals = torch.full_like(frame.vals, -7)
    ranges = torch.full_like(frame.tile_ranges, -7)
    n_isect = torch.full_like(frame.n_isect, -7)
    status = torch.zeros_like(frame.status)
    gs.gs_bin_sort_static(frame.projected, frame.rects, frame.counts, N, cams.sizes, frame.cfg, keys, vals,
                          frame.capacity, ranges, n_isect, status)
    torch.cuda.synchronize()
    got = (keys[:n], vals[:n], ranges, int(n_isect.item()))
    return ref, got, int(status.item())


def test_static_scratch_sort_matches_workspace_sort(rt):
    # two calls in a row on two different scenes, then the first one again:
    # the second and third calls start from the scratch the previous one left
    a = scenes.random_small(301, N=3000, width=203, height=117, n_views=2, spread=1.5)
    b = scenes.random_small(302, N=1200, width=96, height=64, n_views=1, tile=8)
    for s, order in ((a, False), (b, False), (a, False), (b, True), (a, True)):
        ref, got, status = _sorted_both_ways(rt, s, tile_order=order)
        assert status == 0
        assert got[3] == ref[3] > 0
        assert bool((got[0] == ref[0]).all()) and bool((got[1] == ref[1]).all())
        _check_ranges(got[2].cpu().numpy().view(np.uint32), ref[2].cpu().numpy().view(np.uint32), order)


def _bucket(n):
    """Half-octave length bucket of the longest-first tile order (empty last)."""
    n = n.astype(np.int64)
    lg = np.where(n > 0, np.floor(np.log2(np.maximum(n, 1))).astype(np.int64), 0)
    half = np.where(lg > 0, (n >> np.maximum(lg - 1, 0)) & 1, 0)
    return np.where(n == 0, 63, 62 - np.minimum(2 * lg + half, 62))


def _check_ranges(got, ref, order):
    """The [n_tiles][2] ranges bit for bit; with a tile order, the order is a
    permutation of the tiles that visits the same length buckets in the same
    sequence (the order within a bucket is left open)."""
    if not order:
        np.testing.assert_array_equal(got, ref)
        return
    nt = got.shape[0] // 3
    np.testing.assert_array_equal(got[:2 * nt], ref[:2 * nt])
    rg = ref[:2 * nt].reshape(-1, 2).astype(np.int64)
    length = rg[:, 1] - rg[:, 0]
    og, orf = got[2 * nt:].astype(np.int64), ref[2 * nt:].astype(np.int64)
    np.testing.assert_array_equal(np.sort(og), np.arange(nt))
    bg = _bucket(length[og])
    np.testing.assert_array_equal(bg, _bucket(length[orf]))
    assert (np.diff(bg) >= 0).all()


def test_static_scratch_rejects_oversized_problems(rt):
    torch, gs, R = rt
    cfg = scenes.make_cfg()
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    keys = torch.zeros(16, dtype=torch.int64, device="cuda")
    # 2^26 keys need about 1 GiB of scratch, far beyond the fixed array
    with pytest.raises(gs.GSError, match="too large"):
        gs.gs_bin_sort_static(dummy, dummy, dummy, 1, [[64, 64]], cfg, keys, dummy, 1 << 26, dummy, keys, dummy)


def test_static_scratch_argument_errors_match_gs_bin_sort(rt):
    """Sizes no workspace could serve are argument errors, as in gs_bin_sort,
    not GS_ERR_TOO_LARGE."""
    torch, gs, R = rt
    cfg = scenes.make_cfg()
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    keys = torch.zeros(16, dtype=torch.int64, device="cuda")
    for n, cap in ((1, (1 << 32) - 1), (1 << 32, 16), (-1, 16)):
        with pytest.raises(gs.GSError, match="invalid argument"):
            gs.gs_bin_sort_static(dummy, dummy, dummy, n, [[64, 64]], cfg, keys, dummy, cap, dummy, keys, dummy)
