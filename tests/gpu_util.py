"""Helpers for the GPU parity tests: run the CUDA library through its C ABI
(via the package's ctypes binding) on a scene and return numpy arrays."""
from __future__ import annotations

import numpy as np

FLAG_MARGINAL_TOL = 1e-2  # pixels with a near-threshold decision (see below)


def to_np(t, dtype=None):
    a = t.detach().cpu().numpy()
    return a.view(dtype) if dtype is not None else a


def run_gpu(scene, dL_dimage=None, capacity=None, tile=None, graph=False, partitions=1, keep_keys=True):
    """project -> bin_sort -> rasterize_fwd [-> rasterize_bwd with the given
    upstream gradient] on cuda:0. Returns numpy outputs."""
    import torch

    from paper_2606_11390_gb300 import renderer as R

    cfg = dict(scene["cfg"])
    if tile is not None:
        cfg["tile_w"], cfg["tile_h"] = tile
    N = int(scene["means"].shape[0])
    params = R.FlatParams(N).load_from(scene)
    cams = R.Cameras(scene["cams"], scene["sizes"])
    frame = R.Frame(N, cams, cfg, capacity=capacity, keep_keys=keep_keys, partitions=partitions)
    R.render(params, cams, frame)
    torch.cuda.synchronize()
    out = {
        "projected": to_np(frame.projected).reshape(-1, 12),
        "rects": to_np(frame.rects).reshape(-1, 4),
        "counts": to_np(frame.counts, np.uint32),
        "depth_keys": to_np(frame.depth_keys, np.uint32),
        "n_isect": int(frame.n_isect.item()),
        "status": frame.read_status(),
        "capacity": frame.capacity,
    }
    I = out["n_isect"]
    out["keys"] = to_np(frame.keys, np.uint64)[:I] if keep_keys else None
    out["vals"] = to_np(frame.vals, np.uint32)[:I]
    out["ranges"] = to_np(frame.ranges, np.uint32).reshape(-1, 2)
    out["image"] = to_np(frame.image).reshape(-1, 3)
    out["final_T"] = to_np(frame.final_T)
    out["last"] = to_np(frame.last, np.uint32)
    if dL_dimage is not None:
        grads = params.like()
        dl = torch.from_numpy(np.ascontiguousarray(dL_dimage, np.float32).reshape(-1)).cuda()
        R.rasterize_bwd(params, cams, frame, dl, grads)
        torch.cuda.synchronize()
        out["status"] |= frame.read_status()
        out["d_projected"] = to_np(frame.d_projected).reshape(-1, 9)
        out["grads"] = {k: to_np(grads[k]) for k in R.PARAM_NAMES}
    return out


def grad_close(got, ref, rel=1e-3, mask=None, name=""):
    """Per-tensor gradient check: elementwise |d| <= rel * max(|ref|, 1e-3 max|ref|)
    (on `mask` if given) and ||d|| / ||ref|| <= rel over all entries."""
    got = np.asarray(got, np.float64).reshape(ref.shape[0], -1)
    ref = np.asarray(ref, np.float64).reshape(ref.shape[0], -1)
    scale = np.abs(ref).max() if ref.size else 0.0
    d = np.abs(got - ref)
    tol = rel * np.maximum(np.abs(ref), 1e-3 * scale) + 1e-12
    bad = d > tol
    if mask is not None:
        bad &= mask.reshape(-1, 1)
    nrm = np.linalg.norm(ref)
    rel_norm = np.linalg.norm(got - ref) / nrm if nrm > 0 else np.linalg.norm(got - ref)
    assert not bad.any(), (f"{name}: {bad.sum()} of {bad.size} entries out of tolerance; worst "
                           f"{(d / tol).max():.3g}x tol at {np.unravel_index(np.argmax(d / tol), d.shape)}")
    assert rel_norm <= rel, f"{name}: relative norm error {rel_norm:.3g}"


def norm_close(got, ref, rel=1e-3, name=""):
    """||got - ref||_2 <= rel * ||ref||_2 over all entries."""
    got = np.asarray(got, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nrm = np.linalg.norm(ref)
    err = np.linalg.norm(got - ref)
    assert err <= rel * nrm + 1e-12, f"{name}: relative norm error {err / max(nrm, 1e-300):.3g}"
