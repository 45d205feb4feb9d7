"""Failure detection without a GPU fault: every device-side wait of the
library has an iteration bound. A test hook makes one look-back wait run out
on purpose (a tile that never publishes); the call must report
GS_STATUS_TIMEOUT through the status word, keep every access in bounds, and
leave the context usable for the next, correct call."""
import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_lookback_timeout_is_reported_and_recoverable(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_11390_gb300 import _native as gs
    from paper_2606_11390_gb300 import renderer as R

    gs.load()
    s = scenes.random_small(401, N=30000, width=320, height=240, spread=2.0, log_scale_mu=-3.0)
    N = s["means"].shape[0]
    params = R.FlatParams(N).load_from(s)
    cams = R.Cameras(s["cams"], s["sizes"])
    frame = R.Frame(N, cams, dict(s["cfg"], flags=gs.GS_FLAG_TEST_STALL_LOOKBACK), capacity=1 << 22,
                    keep_keys=True)
    R.project(params, cams, frame)
    frame.clear_status()
    R.bin_sort(frame)
    torch.cuda.synchronize()  # returns: the wait is bounded
    st = frame.read_status()
    assert st & gs.GS_STATUS_TIMEOUT
    # the context is still usable and a normal call is correct
    frame.cfg = dict(s["cfg"])
    frame.clear_status()
    R.bin_sort(frame)
    torch.cuda.synchronize()
    assert frame.read_status() == 0
    o_proj, o_bins, _ = oracle.forward(s, "f32")
    n = int(frame.n_isect.item())
    assert n == o_bins["n_isect"]
    np.testing.assert_array_equal(frame.keys.cpu().numpy().view(np.uint64)[:n], o_bins["keys"])
