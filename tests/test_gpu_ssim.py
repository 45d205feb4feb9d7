"""Parity of the fused SSIM loss kernel (gs_ssim_loss) with the float64 oracle.

Sizes span several 32x16 tiles with ragged edges, views smaller than one
tile, several views of different sizes in one call, and the full 3840x2160
view (checked against the oracle's separable path over the whole image).
Loss: relative 1e-5. Gradient: the per-tensor gradient tolerance (1e-3
relative per element, floored at 1e-3 of the largest, and on the norm)."""
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


def _images(seed, sizes, noise=0.1):
    rng = np.random.default_rng(seed)
    P = int(np.prod(np.asarray(sizes), axis=1).sum())
    img = rng.uniform(0.0, 1.0, (P, 3)).astype(np.float32)
    tgt = np.clip(img + noise * rng.standard_normal((P, 3)), 0.0, 1.0).astype(np.float32)
    return img, tgt


def _gpu(native, img, tgt, sizes, lam):
    import torch

    x = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    y = torch.from_numpy(np.ascontiguousarray(tgt)).cuda()
    g = torch.full_like(x, float("nan"))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    native.gs_ssim_loss(x, y, np.asarray(sizes, np.int32), lam, g, loss)
    torch.cuda.synchronize()
    return float(loss.item()), to_np(g)


CASES = {
    "one_view_ragged": [[100, 70]],
    "exact_tiles": [[64, 48]],
    "views_of_mixed_size": [[37, 23], [64, 32], [5, 3], [33, 17]],
    "single_pixel": [[1, 1]],
    "one_row": [[70, 1]],
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_ssim_loss_matches_oracle(native, name):
    from oracle import ssim as S

    sizes = CASES[name]
    img, tgt = _images(100 + sorted(CASES).index(name), sizes)
    L, g = _gpu(native, img, tgt, sizes, 0.2)
    Lo, go, _ = S.ssim_loss(img.astype(np.float64), tgt.astype(np.float64), np.asarray(sizes), 0.2)
    assert abs(L - Lo) <= 1e-5 * abs(Lo), (L, Lo)
    assert np.isfinite(g).all()
    grad_close(g, go, rel=1e-3, name="dL/dimage")


@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_ssim_loss_weight_ends(native, lam):
    from oracle import ssim as S

    sizes = [[45, 38], [16, 16]]
    img, tgt = _images(9, sizes)
    L, g = _gpu(native, img, tgt, sizes, lam)
    Lo, go, _ = S.ssim_loss(img.astype(np.float64), tgt.astype(np.float64), np.asarray(sizes), lam)
    assert abs(L - Lo) <= 1e-5 * abs(Lo)
    grad_close(g, go, rel=1e-3, name="dL/dimage")


def test_identical_images_give_zero_loss(native):
    sizes = [[77, 41]]
    img, _ = _images(3, sizes)
    L, g = _gpu(native, img, img, sizes, 0.2)
    assert abs(L) < 1e-6
    assert np.abs(g).max() * img.size < 1e-3   # gradients are O(1 / n) per element


def test_full_size_4k(native):
    from oracle import ssim as S

    sizes = [[3840, 2160]]
    img, tgt = _images(21, sizes, noise=0.05)
    L, g = _gpu(native, img, tgt, sizes, 0.2)
    Lo, go, _ = S.ssim_loss(img.astype(np.float64), tgt.astype(np.float64), np.asarray(sizes), 0.2, fast=True)
    assert abs(L - Lo) <= 1e-5 * abs(Lo), (L, Lo)
    grad_close(g, go, rel=1e-3, name="dL/dimage")


def test_rejects_bad_arguments(native):
    import torch

    x = torch.zeros(16 * 3, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(native.GSError):
        native.gs_ssim_loss(x, x, np.array([[4, 4]], np.int32), 1.5, x, loss)
    with pytest.raises(native.GSError):
        native.gs_ssim_loss(x, x, np.array([[0, 4]], np.int32), 0.2, x, loss)


def test_train_step_with_ssim_loss(native):
    """The fused SSIM loss inside the captured batched step: loss and image
    gradient against the oracle on the step's own rendered image; the graph
    replay and the per-view path agree."""
    import torch

    from oracle import ssim as S
    from paper_2606_11390_gb300 import renderer as R
    from paper_2606_11390_gb300 import scenes

    s = scenes.random_small(77, N=2000, width=96, height=72, n_views=3, spread=1.5, tile=16)
    st = R.TrainStep(s, mode="batched", loss="ssim").prepare()
    st.run()
    torch.cuda.synchronize()
    st.check()
    img = to_np(st.image).reshape(-1, 3).astype(np.float64)
    tgt = np.asarray(s["target"], np.float64).reshape(-1, 3)
    Lo, go, _ = S.ssim_loss(img, tgt, s["sizes"], 0.2)
    assert abs(st.loss.item() - Lo) <= 1e-5 * abs(Lo)
    grad_close(to_np(st.dL_dimage).reshape(-1, 3), go, rel=1e-3, name="dL/dimage")
    pv = R.TrainStep(s, mode="per_view", graph=False, loss="ssim").prepare()
    pv.run()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(to_np(pv.image), to_np(st.image))
    assert abs(pv.loss.item() - st.loss.item()) <= 1e-12 * abs(Lo)
    for k in ("means", "sh"):
        grad_close(to_np(st.grads[k]), to_np(pv.grads[k]).astype(np.float64), rel=1e-3, name=k)
