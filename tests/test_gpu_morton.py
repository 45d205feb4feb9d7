"""Morton ordering on the GPU (gs_morton_order, gs_gather_rows) against the
oracle: codes and permutation bit for bit, gathered rows exactly, and a
training step on the reordered Gaussians equal to the step on the original
order (same image bit for bit, the same gradients permuted)."""
import numpy as np
import pytest

from gpu_util import grad_close, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_11390_gb300 import _native

    _native.load()
    return _native


def _gpu_order(native, means):
    import torch

    N = means.shape[0]
    m = torch.from_numpy(np.ascontiguousarray(means, np.float32)).cuda()
    perm = torch.empty(max(N, 1), dtype=torch.int32, device="cuda")
    codes = torch.empty(max(N, 1), dtype=torch.int32, device="cuda")
    ws = torch.empty(native.gs_morton_workspace_bytes(N), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    native.gs_morton_order(m, N, perm, codes, ws, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    return to_np(perm, np.uint32)[:N], to_np(codes, np.uint32)[:N]


@pytest.mark.parametrize("N", [1, 7, 4096, 4097, 70001])
def test_morton_order_matches_oracle(native, N):
    from oracle import morton as M

    rng = np.random.default_rng(N)
    means = rng.normal(0, 3, (N, 3)).astype(np.float32)
    if N > 100:
        means[10:40] = means[3]          # equal codes keep index order
        means[50:60, 2] = means[5, 2]    # one flat axis among a few
    perm, codes = _gpu_order(native, means)
    operm, ocodes = M.morton_order(means)
    np.testing.assert_array_equal(codes, ocodes)
    np.testing.assert_array_equal(perm, operm)


def test_morton_order_of_a_workload(native):
    from oracle import morton as M
    from paper_2606_11390_gb300 import scenes

    s = scenes.diff_4k(N=300_000)
    perm, codes = _gpu_order(native, s["means"])
    operm, ocodes = M.morton_order(s["means"])
    np.testing.assert_array_equal(codes, ocodes)
    np.testing.assert_array_equal(perm, operm)


def test_flat_axis(native):
    from oracle import morton as M

    means = np.zeros((5000, 3), np.float32)
    means[:, 0] = np.random.default_rng(3).uniform(-1, 1, 5000)
    perm, codes = _gpu_order(native, means)
    np.testing.assert_array_equal(perm, M.morton_order(means)[0])


@pytest.mark.parametrize("width", [1, 3, 4, 48])
def test_gather_rows(native, width):
    import torch

    rng = np.random.default_rng(width)
    n = 10007
    src = rng.standard_normal((n, width)).astype(np.float32)
    perm = rng.permutation(n).astype(np.int32)
    s = torch.from_numpy(src).cuda()
    d = torch.full_like(s, float("nan"))
    p = torch.from_numpy(perm).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    native.gs_gather_rows(s, d, n, width, p, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    np.testing.assert_array_equal(to_np(d), src[perm])


def test_gather_rows_reports_bad_index(native):
    import torch

    src = torch.arange(40, dtype=torch.float32, device="cuda").view(10, 4)
    dst = torch.zeros_like(src)
    perm = torch.tensor([9, 8, 7, 6, 5, 4, 3, 2, 1, 1000], dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    native.gs_gather_rows(src, dst, 10, 4, perm, status)
    torch.cuda.synchronize()
    assert status.item() & native.GS_STATUS_BOUNDS
    np.testing.assert_array_equal(to_np(dst)[:9], to_np(src)[9:0:-1])
    assert np.all(to_np(dst)[9] == 0)


def test_step_on_morton_order_equals_original(native):
    import torch

    from paper_2606_11390_gb300 import renderer as R
    from paper_2606_11390_gb300 import scenes

    s = scenes.random_small(31, N=3000, width=120, height=90, n_views=2, spread=1.5, tile=16, loss=(1.0, 0.2))
    a = R.TrainStep(s, mode="batched").prepare()
    perm, status = R.morton_permutation(a.params)
    pm = R.permute_gaussians(a.params, perm, status=status)
    torch.cuda.synchronize()
    assert status.item() == 0
    b = R.TrainStep(s, mode="batched", params=pm).prepare()
    a.run()
    b.run()
    torch.cuda.synchronize()
    a.check()
    b.check()
    np.testing.assert_array_equal(to_np(a.image), to_np(b.image))
    p = to_np(perm, np.uint32)[:a.N].astype(np.int64)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        grad_close(to_np(b.grads[k]), to_np(a.grads[k])[p].astype(np.float64), rel=1e-3, name=k)
