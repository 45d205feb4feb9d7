"""The depth sort run as P merged partitions (gs_bin_sort_partitioned, the
paper's multi-device sort emulated on one GPU) gives exactly the keys, values,
ranges and counts of the oracle's stable sort, for any power-of-two P,
including P larger than the number of records, and at full size."""
import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes

from gpu_util import run_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    yield "ragged_2view", scenes.random_small(101, N=1000, width=173, height=91, n_views=2, spread=1.5)
    yield "tile8_3view", scenes.random_small(102, N=777, width=97, height=131, n_views=3, tile=8, log_scale_mu=-2.2)
    s = scenes.random_small(103, N=5000, width=150, height=70, n_views=1, log_scale_mu=-1.5)
    s["means"][100:400] = s["means"][7]  # equal depths across partitions
    yield "ties", s
    yield "fewer_records_than_partitions", scenes.random_small(104, N=20, width=40, height=30, n_views=1)


CASES = list(_cases())


@pytest.mark.parametrize("P", [2, 4, 8, 64])
@pytest.mark.parametrize("name,s", CASES, ids=[c[0] for c in CASES])
def test_partitioned_sort_matches_oracle(oracle, name, s, P):
    o_proj = oracle.project(s, "f32")
    o_bins = oracle.bin_sort(s, o_proj, "f32")
    g = run_gpu(s, partitions=P)
    assert g["status"] == 0
    I = int(o_proj["counts"].astype(np.int64).sum())
    assert g["n_isect"] == I
    np.testing.assert_array_equal(g["keys"], o_bins["keys"])
    np.testing.assert_array_equal(g["vals"], o_bins["vals"])
    np.testing.assert_array_equal(g["ranges"], o_bins["ranges"])


def _tile_list(proj, tile, ntx):
    """Oracle-side list of one tile of view 0: visible records whose rectangle
    contains it, in (depth, index) order."""
    tx, ty = tile % ntx, tile // ntx
    r = proj["rects"]
    m = (proj["counts"] > 0) & (r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3])
    idx = np.nonzero(m)[0]
    depth = proj["projected"][idx, 6].astype(np.float32)
    return idx[np.lexsort((idx, depth))].astype(np.uint32)


def test_partitioned_sort_full_size(oracle):
    """4M Gaussians at 3840x2160 in the bench's tile shape: with 8 partitions
    the intersection count equals the oracle's, sampled tile lists (random,
    the heaviest, the corners) equal the oracle's entry for entry, and the
    whole list equals the one-partition sort's."""
    import torch

    from paper_2606_11390_gb300 import renderer as R

    s = scenes.diff_4k()
    N = s["means"].shape[0]
    W, H = (int(x) for x in s["sizes"][0])
    tw, th = s["cfg"]["tile_w"], s["cfg"]["tile_h"]
    ntx, nty = -(-W // tw), -(-H // th)
    o_proj = oracle.project(s, "f32")
    I = int(o_proj["counts"].astype(np.int64).sum())
    params = R.FlatParams(N).load_from(s)
    cams = R.Cameras(s["cams"], s["sizes"])
    out = {}
    for P in (8, 1):
        fr = R.Frame(N, cams, s["cfg"], capacity=int(I * 1.05) + 4096, partitions=P)
        R.project(params, cams, fr)
        R.bin_sort(fr)
        torch.cuda.synchronize()
        assert fr.read_status() == 0
        assert int(fr.n_isect.item()) == I
        out[P] = (to_np(fr.vals, np.uint32)[:I].copy(), to_np(fr.ranges, np.uint32).reshape(-1, 2).copy())
        del fr
        torch.cuda.empty_cache()
    vals, ranges = out[8]
    lens = ranges[:, 1].astype(np.int64) - ranges[:, 0]
    rng = np.random.default_rng(12)
    tiles = np.unique(np.concatenate([rng.choice(ntx * nty, 16, replace=False), np.argsort(lens)[-3:],
                                      [0, ntx - 1, ntx * nty - 1]]))
    for t in tiles:
        np.testing.assert_array_equal(vals[ranges[t, 0]:ranges[t, 1]], _tile_list(o_proj, int(t), ntx),
                                      err_msg=f"tile {t}")
    np.testing.assert_array_equal(vals, out[1][0])
    np.testing.assert_array_equal(ranges, out[1][1])
