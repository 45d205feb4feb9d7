"""ctypes binding of libgs_gb300.so: the C ABI of include/gs.h, one Python
function per entry point, with the same names.

Argument marshalling only: tensors become device pointers, the gs_config
struct is filled from a dict, the stream is the current torch stream. Every
step of the computation runs in the CUDA library; there is no fallback. If
the library has not been built (see paper_2606_11390_gb300.build) the first
call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

GS_OK, GS_ERR_ARG, GS_ERR_CUDA, GS_ERR_UNSUPPORTED, GS_ERR_TOO_LARGE = 0, 1, 2, 3, 4
GS_STATUS_CAPACITY, GS_STATUS_TIMEOUT, GS_STATUS_BOUNDS = 1, 2, 4
GS_FLAG_TILE_ORDER = 8
GS_MAX_VIEWS = 64
GS_FLAG_ACCUMULATE_GRADS = 1
GS_FLAG_RASTER_2PX = 2
GS_FLAG_TEST_STALL_LOOKBACK = 4
RECORD_FLOATS = 12
DRECORD_FLOATS = 9


class GSConfig(ctypes.Structure):
    _fields_ = [
        ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("near_plane", ctypes.c_float), ("far_plane", ctypes.c_float), ("eps2d", ctypes.c_float),
        ("alpha_cap", ctypes.c_float), ("alpha_min", ctypes.c_float), ("t_stop", ctypes.c_float),
        ("bg", ctypes.c_float * 3),
        ("raster_batch_fwd", ctypes.c_int32), ("raster_batch_bwd", ctypes.c_int32),
    ]


def make_config(cfg: dict) -> GSConfig:
    c = GSConfig()
    c.tile_w, c.tile_h, c.sh_degree = int(cfg["tile_w"]), int(cfg["tile_h"]), int(cfg["sh_degree"])
    c.flags = int(cfg.get("flags", 0))
    c.near_plane, c.far_plane, c.eps2d = cfg["near"], cfg["far"], cfg["eps2d"]
    c.alpha_cap, c.alpha_min, c.t_stop = cfg["alpha_cap"], cfg["alpha_min"], cfg["t_stop"]
    for i in range(3):
        c.bg[i] = cfg["bg"][i]
    c.raster_batch_fwd = int(cfg.get("raster_batch_fwd", 0))
    c.raster_batch_bwd = int(cfg.get("raster_batch_bwd", 0))
    return c


class GSError(RuntimeError):
    pass


_VP, _I64, _I32, _F32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
_SIGNATURES = {
    "gs_version": ([], ctypes.c_int),
    "gs_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "gs_layout_totals": ([_VP, _I32, _VP, _VP, _VP], ctypes.c_int),
    "gs_project": ([_VP] * 5 + [_I64, _VP, _VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "gs_bin_sort_workspace_bytes": ([_I64, _I32, _I64, _I64], ctypes.c_size_t),
    "gs_bin_sort": ([_VP, _VP, _VP, _VP, _I64, _VP, _I32, _VP, _VP, _VP, _I64, _VP, _VP, _VP, ctypes.c_size_t, _VP,
                     _VP], ctypes.c_int),
    "gs_bin_sort_static": ([_VP, _VP, _VP, _I64, _VP, _I32, _VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP], ctypes.c_int),
    "gs_rasterize_fwd": ([_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "gs_rasterize_fwd_counted": ([_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "gs_rasterize_fwd_l1l2": ([_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP, _VP, _VP, _I64, _F32, _F32, _I32, _VP, _VP,
                               _VP, _VP], ctypes.c_int),
    "gs_rasterize_bwd": ([_VP] * 5 + [_I64, _VP, _VP, _I32, _VP] + [_VP] * 7 + [_VP] * 6 + [_VP, _VP, _VP],
                         ctypes.c_int),
    "gs_rasterize_bwd_pixels": ([_VP, _VP, _VP, _VP, _I32, _VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "gs_rasterize_bwd_pixels_counted": ([_VP, _VP, _VP, _VP, _I32, _VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
                                        ctypes.c_int),
    "gs_project_bwd": ([_VP] * 5 + [_I64, _VP, _VP, _I32, _VP, _VP, _VP] + [_VP] * 5 + [_VP, _VP], ctypes.c_int),
    "gs_image_loss": ([_VP, _VP, _I64, _F32, _F32, _VP, _VP, _VP], ctypes.c_int),
    "gs_adam_step": ([_VP, _VP, _VP, _VP, _I64, _F32, _F32, _F32, _F32, _VP, _VP], ctypes.c_int),
    "gs_ssim_loss": ([_VP, _VP, _VP, _I32, _F32, _VP, _VP, _VP], ctypes.c_int),
    "gs_morton_workspace_bytes": ([_I64], ctypes.c_size_t),
    "gs_morton_order": ([_VP, _I64, _VP, _VP, _VP, ctypes.c_size_t, _VP, _VP], ctypes.c_int),
    "gs_gather_rows": ([_VP, _VP, _I64, _I32, _VP, _VP, _VP], ctypes.c_int),
    "gs_bin_sort_partitioned_workspace_bytes": ([_I64, _I32, _I64, _I64, _I32], ctypes.c_size_t),
    "gs_bin_sort_partitioned": ([_VP, _VP, _VP, _VP, _I64, _VP, _I32, _VP, _VP, _VP, _I64, _VP, _VP, _I32, _VP,
                                 ctypes.c_size_t, _VP, _VP], ctypes.c_int),
    "gs_densify_stats": ([_VP, _VP, _VP, _I64, _VP, _I32, _VP, _VP, _VP, _VP], ctypes.c_int),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Loads (and if needed builds) libgs_gb300.so. Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB_PATH
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise GSError(f"CUDA library not built: {path} is missing")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


def _check(rc: int, what: str):
    if rc != GS_OK:
        msg = load().gs_status_string(rc).decode()
        raise GSError(f"{what} failed: {msg} (code {rc})")


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _sizes(sizes) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(sizes, dtype=np.int32).reshape(-1, 2))


def _cfg_ref(cfg):
    c = cfg if isinstance(cfg, GSConfig) else make_config(cfg)
    return c, ctypes.byref(c)


def gs_version() -> int:
    return load().gs_version()


def gs_layout_totals(sizes, cfg):
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    nt, npix = ctypes.c_int64(), ctypes.c_int64()
    _check(load().gs_layout_totals(_ptr(sz), sz.shape[0], cref, ctypes.byref(nt), ctypes.byref(npix)),
           "gs_layout_totals")
    return nt.value, npix.value


def gs_project(means, log_scales, quats, opacity_logits, sh, cams, sizes, cfg, projected, rects, counts, status,
               stream=None, depth_keys=None):
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_project(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh),
                           means.shape[0], _ptr(cams), _ptr(sz), sz.shape[0], cref, _ptr(projected), _ptr(rects),
                           _ptr(counts), _ptr(depth_keys), _ptr(status), _stream(stream))
    _check(rc, "gs_project")


def gs_bin_sort_workspace_bytes(N, V, capacity, n_tiles) -> int:
    return int(load().gs_bin_sort_workspace_bytes(int(N), int(V), int(capacity), int(n_tiles)))


def gs_bin_sort(projected, rects, counts, N, sizes, cfg, keys, vals, capacity, tile_ranges, n_isect, workspace,
                status, stream=None, depth_keys=None):
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_bin_sort(_ptr(projected), _ptr(rects), _ptr(counts), _ptr(depth_keys), int(N), _ptr(sz),
                            sz.shape[0], cref,
                            _ptr(keys), _ptr(vals), int(capacity), _ptr(tile_ranges), _ptr(n_isect), _ptr(workspace),
                            workspace.numel() * workspace.element_size(), _ptr(status), _stream(stream))
    _check(rc, "gs_bin_sort")


def gs_bin_sort_partitioned_workspace_bytes(N, V, capacity, n_tiles, partitions) -> int:
    return int(load().gs_bin_sort_partitioned_workspace_bytes(int(N), int(V), int(capacity), int(n_tiles),
                                                              int(partitions)))


def gs_bin_sort_partitioned(projected, rects, counts, N, sizes, cfg, keys, vals, capacity, tile_ranges, n_isect,
                            partitions, workspace, status, stream=None, depth_keys=None):
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_bin_sort_partitioned(_ptr(projected), _ptr(rects), _ptr(counts), _ptr(depth_keys), int(N),
                                        _ptr(sz), sz.shape[0],
                                        cref, _ptr(keys), _ptr(vals), int(capacity), _ptr(tile_ranges),
                                        _ptr(n_isect), int(partitions), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), _ptr(status), _stream(stream))
    _check(rc, "gs_bin_sort_partitioned")


def gs_bin_sort_static(projected, rects, counts, N, sizes, cfg, keys, vals, capacity, tile_ranges, n_isect, status,
                       stream=None):
    """gs_bin_sort with the library's fixed device scratch instead of a
    caller workspace (for callers that cannot allocate device memory)."""
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_bin_sort_static(_ptr(projected), _ptr(rects), _ptr(counts), int(N), _ptr(sz), sz.shape[0], cref,
                                   _ptr(keys), _ptr(vals), int(capacity), _ptr(tile_ranges), _ptr(n_isect),
                                   _ptr(status), _stream(stream))
    _check(rc, "gs_bin_sort_static")


def gs_rasterize_fwd(projected, vals, tile_ranges, sizes, cfg, image, final_T, last, stream=None, cull_masks=None):
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_rasterize_fwd(_ptr(projected), _ptr(vals), _ptr(tile_ranges), _ptr(sz), sz.shape[0], cref,
                                 _ptr(image), _ptr(final_T), _ptr(last), _ptr(cull_masks), _stream(stream))
    _check(rc, "gs_rasterize_fwd")


def gs_rasterize_fwd_counted(projected, vals, tile_ranges, sizes, cfg, image, final_T, last, pair_counts,
                             stream=None, cull_masks=None):
    """gs_rasterize_fwd that also adds its (executed, evaluated, composited)
    pixel-splat pair counts into pair_counts (int64 [3] on the device)."""
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_rasterize_fwd_counted(_ptr(projected), _ptr(vals), _ptr(tile_ranges), _ptr(sz), sz.shape[0], cref,
                                         _ptr(image), _ptr(final_T), _ptr(last), _ptr(pair_counts), _ptr(cull_masks),
                                         _stream(stream))
    _check(rc, "gs_rasterize_fwd_counted")


def gs_rasterize_fwd_l1l2(projected, vals, tile_ranges, sizes, cfg, image, final_T, last, target, n_values, w_l1,
                          w_l2, accumulate, dL_dimage, loss, stream=None, cull_masks=None):
    """gs_rasterize_fwd with the L1 + L2 loss of gs_image_loss in the same kernel."""
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_rasterize_fwd_l1l2(_ptr(projected), _ptr(vals), _ptr(tile_ranges), _ptr(sz), sz.shape[0], cref,
                                      _ptr(image), _ptr(final_T), _ptr(last), _ptr(target), int(n_values),
                                      float(w_l1), float(w_l2), int(bool(accumulate)), _ptr(dL_dimage), _ptr(loss),
                                      _ptr(cull_masks), _stream(stream))
    _check(rc, "gs_rasterize_fwd_l1l2")


def gs_rasterize_bwd(means, log_scales, quats, opacity_logits, sh, cams, sizes, cfg, projected, counts, vals,
                     tile_ranges, final_T, last, dL_dimage, d_projected, d_means, d_log_scales, d_quats,
                     d_opacity_logits, d_sh, status, stream=None, cull_masks=None):
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_rasterize_bwd(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh),
                                 means.shape[0], _ptr(cams), _ptr(sz), sz.shape[0], cref, _ptr(projected),
                                 _ptr(counts), _ptr(vals), _ptr(tile_ranges), _ptr(final_T), _ptr(last),
                                 _ptr(dL_dimage), _ptr(d_projected), _ptr(d_means), _ptr(d_log_scales), _ptr(d_quats),
                                 _ptr(d_opacity_logits), _ptr(d_sh), _ptr(cull_masks), _ptr(status), _stream(stream))
    _check(rc, "gs_rasterize_bwd")


def gs_rasterize_bwd_pixels(projected, vals, tile_ranges, sizes, cfg, N, final_T, last, dL_dimage, d_projected,
                            stream=None, cull_masks=None):
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_rasterize_bwd_pixels(_ptr(projected), _ptr(vals), _ptr(tile_ranges), _ptr(sz), sz.shape[0], cref,
                                        int(N), _ptr(final_T), _ptr(last), _ptr(dL_dimage), _ptr(d_projected),
                                        _ptr(cull_masks), _stream(stream))
    _check(rc, "gs_rasterize_bwd_pixels")


def gs_rasterize_bwd_pixels_counted(projected, vals, tile_ranges, sizes, cfg, N, final_T, last, dL_dimage,
                                    d_projected, pair_counts, stream=None, cull_masks=None):
    """gs_rasterize_bwd_pixels that also adds its (executed, evaluated,
    composited) pixel-splat pair counts into pair_counts (int64 [3])."""
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_rasterize_bwd_pixels_counted(_ptr(projected), _ptr(vals), _ptr(tile_ranges), _ptr(sz),
                                                sz.shape[0], cref, int(N), _ptr(final_T), _ptr(last),
                                                _ptr(dL_dimage), _ptr(d_projected), _ptr(pair_counts),
                                                _ptr(cull_masks), _stream(stream))
    _check(rc, "gs_rasterize_bwd_pixels_counted")


def gs_project_bwd(means, log_scales, quats, opacity_logits, sh, cams, sizes, cfg, counts, d_projected, d_means,
                   d_log_scales, d_quats, d_opacity_logits, d_sh, status, stream=None):
    sz = _sizes(sizes)
    c, cref = _cfg_ref(cfg)
    rc = load().gs_project_bwd(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh),
                               means.shape[0], _ptr(cams), _ptr(sz), sz.shape[0], cref, _ptr(counts),
                               _ptr(d_projected), _ptr(d_means), _ptr(d_log_scales), _ptr(d_quats),
                               _ptr(d_opacity_logits), _ptr(d_sh), _ptr(status), _stream(stream))
    _check(rc, "gs_project_bwd")


def gs_image_loss(image, target, w_l1, w_l2, dL_dimage, loss, stream=None):
    rc = load().gs_image_loss(_ptr(image), _ptr(target), image.numel(), float(w_l1), float(w_l2), _ptr(dL_dimage),
                              _ptr(loss), _stream(stream))
    _check(rc, "gs_image_loss")


def gs_ssim_loss(image, target, sizes, lam, dL_dimage, loss, stream=None):
    sz = _sizes(sizes)
    rc = load().gs_ssim_loss(_ptr(image), _ptr(target), _ptr(sz), sz.shape[0], float(lam), _ptr(dL_dimage),
                             _ptr(loss), _stream(stream))
    _check(rc, "gs_ssim_loss")


def gs_morton_workspace_bytes(N):
    return int(load().gs_morton_workspace_bytes(int(N)))


def gs_morton_order(means, N, perm, codes, workspace, status, stream=None):
    rc = load().gs_morton_order(_ptr(means), int(N), _ptr(perm), _ptr(codes) if codes is not None else None,
                                _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(status),
                                _stream(stream))
    _check(rc, "gs_morton_order")


def gs_gather_rows(src, dst, n_rows, row_floats, perm, status, stream=None):
    rc = load().gs_gather_rows(_ptr(src), _ptr(dst), int(n_rows), int(row_floats), _ptr(perm), _ptr(status),
                               _stream(stream))
    _check(rc, "gs_gather_rows")


def gs_densify_stats(projected, counts, d_projected, N, sizes, grad_accum, denom, max_radii, stream=None):
    sz = _sizes(sizes)
    rc = load().gs_densify_stats(_ptr(projected), _ptr(counts), _ptr(d_projected), int(N), _ptr(sz), sz.shape[0],
                                 _ptr(grad_accum), _ptr(denom), _ptr(max_radii), _stream(stream))
    _check(rc, "gs_densify_stats")


def gs_adam_step(param, grad, exp_avg, exp_avg_sq, lr, beta1, beta2, eps, step, stream=None):
    rc = load().gs_adam_step(_ptr(param), _ptr(grad), _ptr(exp_avg), _ptr(exp_avg_sq), param.numel(), float(lr),
                             float(beta1), float(beta2), float(eps), _ptr(step), _stream(stream))
    _check(rc, "gs_adam_step")
