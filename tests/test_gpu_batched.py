"""Batched (one launch per stage for all views, replayed from a captured CUDA
graph) versus the plain per-view path, and graph replay versus eager launch.

Images and per-view sorted lists are identical bit for bit (same kernels on
the same records); gradients agree within the parity tolerance (FP32 atomics
sum in a different order)."""
import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes

from gpu_util import grad_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_11390_gb300 import _native
    from paper_2606_11390_gb300 import renderer

    _native.load()
    return renderer


def _scene(tile=16):
    s = scenes.random_small(201, N=3000, width=120, height=90, n_views=4, spread=1.5, tile=tile, loss=(1.0, 0.2))
    return s


def _run(R, s, mode, graph=True, steps=1):
    import torch

    st = R.TrainStep(s, mode=mode, graph=graph).prepare()
    for _ in range(steps):
        st.run()
    torch.cuda.synchronize()
    st.check()
    return st


@pytest.mark.parametrize("tile", [16, 8])
def test_batched_graph_equals_per_view(R, tile):
    s = _scene(tile)
    b = _run(R, s, "batched", graph=True)
    p = _run(R, s, "per_view", graph=False)
    np.testing.assert_array_equal(b.image.cpu().numpy(), p.image.cpu().numpy())
    assert abs(b.loss.item() - p.loss.item()) <= 1e-12 * max(1.0, abs(p.loss.item()))
    # per-view lists: batched tile ids are offset by the view's tile base and
    # record indices by v*N
    N = s["means"].shape[0]
    fb = b.frames[0]
    rb = fb.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
    vb = fb.vals.cpu().numpy().view(np.uint32)
    base = 0
    for v, fr in enumerate(p.frames):
        rp = fr.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
        vp = fr.vals.cpu().numpy().view(np.uint32)
        for t in range(rp.shape[0]):
            lb = vb[rb[base + t, 0]:rb[base + t, 1]]
            lp = vp[rp[t, 0]:rp[t, 1]]
            assert np.array_equal(lb, lp.astype(np.int64) + v * N), (v, t)
        base += rp.shape[0]
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        grad_close(b.grads[k].cpu().numpy(), p.grads[k].cpu().numpy().astype(np.float64), rel=1e-3, name=k)


def test_many_views_batched_equals_per_view(R):
    """17 small views (an odd count: the multi-view backward's per-thread
    pipeline alternates its two ring slots view by view, and many records
    are invisible in some views, whose copies it skips): the batched step's
    image and parameter gradients match the per-view loop's, which runs the
    single-view instance."""
    s = scenes.random_small(207, N=2500, width=64, height=48, n_views=17, spread=1.5, loss=(1.0, 0.2))
    b = _run(R, s, "batched", graph=True)
    p = _run(R, s, "per_view", graph=False)
    np.testing.assert_array_equal(b.image.cpu().numpy(), p.image.cpu().numpy())
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        grad_close(b.grads[k].cpu().numpy(), p.grads[k].cpu().numpy().astype(np.float64), rel=1e-3, name=k)


def test_graph_replay_equals_eager(R):
    s = _scene()
    g = _run(R, s, "batched", graph=True, steps=2)
    e = _run(R, s, "batched", graph=False, steps=2)
    np.testing.assert_array_equal(g.image.cpu().numpy(), e.image.cpu().numpy())
    for k in ("means", "sh"):
        grad_close(g.grads[k].cpu().numpy(), e.grads[k].cpu().numpy().astype(np.float64), rel=1e-3, name=k)


def test_per_view_captured_equals_per_view_eager(R):
    """The per-view loop (one launch per stage and view) captured in a graph:
    the same image and loss as launching it eagerly."""
    s = _scene()
    g = _run(R, s, "per_view", graph=True, steps=2)
    e = _run(R, s, "per_view", graph=False, steps=2)
    assert g.graph is not None and e.graph is None
    np.testing.assert_array_equal(g.image.cpu().numpy(), e.image.cpu().numpy())
    assert abs(g.loss.item() - e.loss.item()) <= 1e-12 * max(1.0, abs(e.loss.item()))
    for k in ("means", "sh"):
        grad_close(g.grads[k].cpu().numpy(), e.grads[k].cpu().numpy().astype(np.float64), rel=1e-3, name=k)


@pytest.mark.parametrize("px,batch", [(2, (64, 256)), (4, (256, 128)), (2, (0, 64))])
def test_tuned_step_equals_default(R, px, batch):
    """A step with another rasteriser configuration (pixels per thread,
    splats per batch) renders the default step's image bit for bit."""
    import torch

    s = _scene()
    d = _run(R, s, "batched")
    st = R.TrainStep(s, mode="batched", raster_px=px, raster_batch=batch).prepare()
    st.run()
    torch.cuda.synchronize()
    st.check()
    np.testing.assert_array_equal(st.image.cpu().numpy(), d.image.cpu().numpy())
    for k in ("means", "sh"):
        grad_close(st.grads[k].cpu().numpy(), d.grads[k].cpu().numpy().astype(np.float64), rel=1e-3, name=k)


def test_autotuner_on_the_gpu(R, tmp_path, monkeypatch):
    """best_config times its configurations (7 tile / pixel choices, 4
    forward batches, the backward batches the chosen tile has), returns one
    of them and caches it under the library digest; a second call reads the
    cache."""
    from paper_2606_11390_gb300 import autotune

    monkeypatch.setenv("GS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    s = _scene()
    best, times = autotune.best_config(s, steps=1)
    n_bwd = sum(autotune.batch_supported(best, "batch_bwd", b) for b in autotune.BATCHES)
    assert len(times) == 7 + len(autotune.BATCHES) + n_bwd and autotune.name(best) in times
    assert times[autotune.name(best)] == min(times.values())
    again, times2 = autotune.best_config(s, steps=1)
    assert again == best and times2 == times
    st = R.TrainStep(s, mode="batched", **autotune.step_kwargs(best)).prepare()
    st.run()


def test_adam_step_in_graph_moves_parameters(R, oracle):
    import torch

    s = _scene()
    st = R.TrainStep(s, mode="batched", adam=True, lr=1e-3).prepare()
    p0 = st.params.flat.clone()
    m0, v0 = st.exp_avg.clone(), st.exp_avg_sq.clone()
    t0 = int(st.step_count.item())
    st.run()
    torch.cuda.synchronize()
    st.check()
    g = st.grads.flat.cpu().numpy().astype(np.float64)
    want, _, _ = oracle.adam(p0.cpu().numpy(), g, m0.cpu().numpy(), v0.cpu().numpy(), 1e-3, 0.9, 0.999, 1e-15, t0 + 1)
    np.testing.assert_allclose(st.params.flat.cpu().numpy(), want, rtol=0, atol=5e-6)


def test_host_fed_steps_match_direct_steps(R):
    """HostFedStep (inputs copied in and gradients out every step, overlapped
    across neighbouring steps) returns, for alternating parameter sets, the
    gradients and loss of the same steps run directly on the device."""
    import torch

    s = _scene()
    st = R.TrainStep(s, mode="batched").prepare()
    pa = st.params.flat.clone()
    pb = pa.clone()
    pb[: st.N * 3] += 0.01  # shifted means
    want = []
    for p in (pa, pb):
        st.params.flat.copy_(p)
        st.run()
        torch.cuda.synchronize()
        want.append((st.grads.flat.cpu().numpy().astype(np.float64), float(st.loss.item())))
    host_p = [p.cpu().pin_memory() for p in (pa, pb)]
    host_t = st.target.cpu().pin_memory()
    host_c = torch.from_numpy(st.cams.host.copy()).pin_memory()
    host_g = [torch.empty_like(pa, device="cpu").pin_memory() for _ in range(4)]
    host_l = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(4)]
    fed = R.HostFedStep(st)
    for k in range(4):
        fed.run(host_p[k & 1], host_t, host_c, host_g[k], host_l[k])
    fed.sync()
    st.check()
    for k in range(4):
        g, L = want[k & 1]
        grad_close(host_g[k].numpy(), g, rel=1e-4, name=f"step {k} grads")
        assert abs(host_l[k].item() - L) <= 1e-9 * abs(L)


def test_host_fed_resident_params_match_direct_steps(R):
    """HostFedStep without stream_params (camera and target copied in, loss
    out, Gaussians resident): for alternating target images, each step's loss
    is that of the same step run directly, and the gradients left on the
    device are those of the last step."""
    import torch

    s = _scene()
    st = R.TrainStep(s, mode="batched").prepare()
    ta = st.target.clone()
    tb = ta.clone()
    tb.mul_(0.5).add_(0.25)
    want = []
    for t in (ta, tb):
        st.target.copy_(t)
        st.run()
        torch.cuda.synchronize()
        want.append((st.grads.flat.cpu().numpy().astype(np.float64), float(st.loss.item())))
    host_t = [t.cpu().pin_memory() for t in (ta, tb)]
    host_c = torch.from_numpy(st.cams.host.copy()).pin_memory()
    host_l = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(4)]
    fed = R.HostFedStep(st, stream_params=False)
    for k in range(4):
        fed.run(None, host_t[k & 1], host_c, None, host_l[k])
    fed.sync()
    st.check()
    for k in range(4):
        L = want[k & 1][1]
        assert abs(host_l[k].item() - L) <= 1e-9 * abs(L), (k, host_l[k].item(), L)
    grad_close(st.grads.flat.cpu().numpy(), want[1][0], rel=1e-4, name="resident grads")
