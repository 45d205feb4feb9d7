"""gs_densify_stats on the GPU against the oracle: statistics of the GPU's
backward (projection bit-exact, d_projected within the gradient tolerance)
versus those of the oracle's backward, over two accumulated passes."""
import numpy as np
import pytest

from gpu_util import grad_close, run_gpu

pytestmark = pytest.mark.gpu


def test_densify_stats_match_oracle(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import densify as D
    from paper_2606_11390_gb300 import _native as gs
    from paper_2606_11390_gb300 import scenes

    s = scenes.random_small(121, N=1500, width=140, height=100, n_views=3, spread=1.5)
    rng = np.random.default_rng(5)
    P = s["target"].shape[0]
    dl = (rng.standard_normal((P, 3)) / P).astype(np.float32)
    o_proj, o_bins, o_ras = oracle.forward(s, "f32")
    dl[o_ras["marginal_pix"].astype(bool)] = 0  # no near-threshold decision reaches a gradient
    o_dproj, _ = oracle.backward(s, o_proj, o_bins, dl.astype(np.float64), "f32")
    g = run_gpu(s, dL_dimage=dl)
    assert g["status"] == 0
    N, V = s["means"].shape[0], s["sizes"].shape[0]
    init = [np.zeros(N, np.float32), np.zeros(N, np.float32), np.full(N, 0.5, np.float32)]
    dev = [torch.from_numpy(a.copy()).cuda() for a in init]
    proj = torch.from_numpy(np.ascontiguousarray(g["projected"])).cuda()
    cnt = torch.from_numpy(g["counts"].view(np.int32)).cuda()
    dp = torch.from_numpy(np.ascontiguousarray(g["d_projected"], np.float32)).cuda()
    for _ in range(2):
        gs.gs_densify_stats(proj, cnt, dp, N, s["sizes"], *dev)
    torch.cuda.synchronize()
    want = D.densify_stats(o_proj["projected"], o_proj["counts"], o_dproj, s["sizes"], *init)
    want = D.densify_stats(o_proj["projected"], o_proj["counts"], o_dproj, s["sizes"], *want)
    ga, dn, mr = (d.cpu().numpy() for d in dev)
    np.testing.assert_array_equal(dn, want[1])
    np.testing.assert_array_equal(mr, want[2])
    grad_close(ga, want[0], name="grad_accum")
    assert V == 3


def test_train_step_gathers_densify_stats():
    """Inside the captured step: after two steps the statistics equal two
    direct calls on the step's own buffers (up to the rounding of the
    gradient atomics), and the per-view path agrees."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_11390_gb300 import _native as gs
    from paper_2606_11390_gb300 import renderer as R
    from paper_2606_11390_gb300 import scenes

    s = scenes.random_small(122, N=2000, width=120, height=90, n_views=3, spread=1.5, loss=(1.0, 0.2))
    st = R.TrainStep(s, mode="batched", densify_stats=True).prepare()
    assert float(st.denom.sum().item()) == 0.0
    st.run()
    st.run()
    torch.cuda.synchronize()
    st.check()
    fr = st.frames[0]
    ref = [torch.zeros(st.N, device="cuda") for _ in range(3)]
    for _ in range(2):
        gs.gs_densify_stats(fr.projected, fr.counts, fr.d_projected, st.N, st.cams.sizes, *ref)
    torch.cuda.synchronize()
    # the two steps' d_projected differ in the order of their FP32 atomics,
    # so the gradient norms agree to rounding; counts and radii exactly
    grad_close(st.grad_accum.cpu().numpy(), ref[0].cpu().numpy().astype(np.float64), rel=1e-5, name="grad_accum")
    np.testing.assert_array_equal(st.denom.cpu().numpy(), ref[1].cpu().numpy())
    np.testing.assert_array_equal(st.max_radii.cpu().numpy(), ref[2].cpu().numpy())
    vis = (fr.counts.view(torch.int32).cpu().numpy().reshape(3, -1) > 0).sum(axis=0)
    np.testing.assert_array_equal(st.denom.cpu().numpy(), 2 * vis)
    pv = R.TrainStep(s, mode="per_view", graph=False, densify_stats=True).prepare()
    pv.run()
    pv.run()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(pv.denom.cpu().numpy(), st.denom.cpu().numpy())
    np.testing.assert_array_equal(pv.max_radii.cpu().numpy(), st.max_radii.cpu().numpy())
    grad_close(pv.grad_accum.cpu().numpy(), st.grad_accum.cpu().numpy().astype(np.float64), name="grad_accum")
