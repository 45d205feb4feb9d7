"""Runtime around the C ABI: device-resident scenes, per-call buffers, the
autograd Function, and the training-step runner (per-view or batched, the
latter captured in a CUDA graph).

PyTorch supplies device memory and streams only; every stage of the step runs
in libgs_gb300 kernels (see include/gs.h).
"""
from __future__ import annotations


import numpy as np
import torch

from . import _native as gs

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")
PARAM_WIDTH = {"means": 3, "log_scales": 3, "quats": 4, "opacity_logits": 1, "sh": 48}
FLOATS_PER_GAUSSIAN = sum(PARAM_WIDTH.values())  # 59


def _round_up(x, m):
    return (x + m - 1) // m * m


class FlatParams:
    """The five parameter arrays of N Gaussians as views into one flat float32
    device buffer. Each segment starts on a 16-byte boundary (N is padded to a
    multiple of 4), so kernels can stage them with TMA bulk copies and a single
    fused Adam launch covers all of them."""

    def __init__(self, N: int, device="cuda", buf: torch.Tensor | None = None):
        self.N = N
        self.Np = _round_up(max(N, 1), 4)
        self.numel = FLOATS_PER_GAUSSIAN * self.Np
        self.flat = buf if buf is not None else torch.zeros(self.numel, dtype=torch.float32, device=device)
        assert self.flat.numel() == self.numel
        self.views = {}
        off = 0
        for name in PARAM_NAMES:
            w = PARAM_WIDTH[name]
            seg = self.flat[off:off + w * N]
            shape = (N, 16, 3) if name == "sh" else ((N,) if w == 1 else (N, w))
            self.views[name] = seg.view(shape)
            off += w * self.Np

    def __getitem__(self, k):
        return self.views[k]

    def like(self):
        return FlatParams(self.N, self.flat.device)

    def load_from(self, scene: dict):
        for name in PARAM_NAMES:
            src = torch.from_numpy(np.ascontiguousarray(scene[name], np.float32))
            self.views[name].copy_(src.view(self.views[name].shape))
        return self


class Cameras:
    """Cameras of one batch: poses/intrinsics on the device (gs_camera records,
    20 floats each) and the (W, H) layout on the host."""

    def __init__(self, cams: np.ndarray, sizes: np.ndarray, device="cuda"):
        cams = np.ascontiguousarray(cams, np.float32).reshape(-1, 20)
        self.sizes = np.ascontiguousarray(sizes, np.int32).reshape(-1, 2)
        assert cams.shape[0] == self.sizes.shape[0]
        self.V = cams.shape[0]
        self.host = cams
        self.dev = torch.from_numpy(cams).to(device)
        self.n_pixels = int((self.sizes[:, 0].astype(np.int64) * self.sizes[:, 1]).sum())
        self.pix_base = np.concatenate([[0], np.cumsum(self.sizes[:, 0].astype(np.int64) * self.sizes[:, 1])])

    def view(self, v: int) -> "Cameras":
        c = Cameras.__new__(Cameras)
        c.sizes = self.sizes[v:v + 1]
        c.V = 1
        c.host = self.host[v:v + 1]
        c.dev = self.dev[v:v + 1]
        c.n_pixels = int(c.sizes[0, 0]) * int(c.sizes[0, 1])
        c.pix_base = np.array([0, c.n_pixels])
        return c


class Frame:
    """Device buffers of one rendering call for N Gaussians and a camera
    layout, with a key capacity that grows on demand."""

    def __init__(self, N: int, cams: Cameras, cfg: dict, capacity: int | None = None, device="cuda",
                 keep_keys: bool = False, partitions: int = 1, tile_order: bool = True):
        self.N, self.cams, self.cfg = N, cams, dict(cfg)
        if tile_order:  # rasterise the longest tile lists first (same results)
            self.cfg["flags"] = int(self.cfg.get("flags", 0)) | gs.GS_FLAG_TILE_ORDER
        self.partitions = int(partitions)  # > 1: the depth sort runs as merged partitions
        self.device = device
        self.keep_keys = keep_keys  # materialise the 64-bit sort keys (tests and inspection only)
        V = cams.V
        self.n_tiles, self.n_pixels = gs.gs_layout_totals(cams.sizes, cfg)
        i32 = dict(dtype=torch.int32, device=device)
        f32 = dict(dtype=torch.float32, device=device)
        self.projected = torch.zeros(V * N * gs.RECORD_FLOATS, **f32)
        self.rects = torch.zeros(V * N * 4, dtype=torch.int16, device=device)
        self.counts = torch.zeros(V * N, **i32)
        self.depth_keys = torch.zeros(V * N, **i32)  # depth bits of visible records, read by the sort
        order = bool(self.cfg.get("flags", 0) & gs.GS_FLAG_TILE_ORDER)
        self.tile_ranges = torch.zeros(self.n_tiles * (3 if order else 2), **i32)
        self.ranges = self.tile_ranges[:2 * self.n_tiles]  # [n_tiles][2] start, end
        self.n_isect = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, **i32)
        self.image = torch.zeros(self.n_pixels * 3, **f32)
        self.final_T = torch.zeros(self.n_pixels, **f32)
        self.last = torch.zeros(self.n_pixels, **i32)
        self.dL_dimage = torch.zeros(self.n_pixels * 3, **f32)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.d_projected = torch.zeros(V * N * gs.DRECORD_FLOATS, **f32)
        self.capacity = 0
        self.set_capacity(capacity if capacity is not None else max(1024, 8 * V * N))

    def set_capacity(self, capacity: int):
        capacity = int(capacity)
        if capacity == self.capacity:
            return
        self.capacity = capacity
        self.keys = (torch.zeros(max(capacity, 1), dtype=torch.int64, device=self.device) if self.keep_keys
                     else None)
        self.vals = torch.zeros(max(capacity, 1), dtype=torch.int32, device=self.device)
        # per list entry: the forward's cull mask for the backward (uint16 bits)
        self.cull = torch.zeros(max(capacity, 1), dtype=torch.int16, device=self.device)
        if self.partitions == 1:
            ws = gs.gs_bin_sort_workspace_bytes(self.N, self.cams.V, capacity, self.n_tiles)
        else:
            ws = gs.gs_bin_sort_partitioned_workspace_bytes(self.N, self.cams.V, capacity, self.n_tiles,
                                                            self.partitions)
            if ws == 0:
                raise ValueError("partitions must be a power of two in [1, 64]")
        self.workspace = torch.zeros(ws, dtype=torch.uint8, device=self.device)

    def read_status(self) -> int:
        return int(self.status.item())

    def clear_status(self):
        self.status.zero_()

    def hand_over(self) -> "FrameState":
        """Moves what a backward of the last render reads out of this frame
        into a FrameState (no copy) and gives the frame fresh buffers in their
        place, so that a later render on this frame cannot overwrite them:
        the projected records, tile counts, sorted list, its cull masks and
        tile ranges, and per pixel the image, final transmittance and
        last-contributor count.
        The camera records are copied (V x 80 bytes), since the caller may
        refill them."""
        st = FrameState(self)
        self.projected = torch.zeros_like(self.projected)
        self.counts = torch.zeros_like(self.counts)
        self.vals = torch.zeros_like(self.vals)
        self.cull = torch.zeros_like(self.cull)
        self.tile_ranges = torch.zeros_like(self.tile_ranges)
        self.ranges = self.tile_ranges[:2 * self.n_tiles]
        self.image = torch.zeros_like(self.image)
        self.final_T = torch.zeros_like(self.final_T)
        self.last = torch.zeros_like(self.last)
        return st


class FrameState:
    """The buffers of one rendered frame that its backward reads (see
    Frame.hand_over), with the attribute names rasterize_bwd uses; the
    backward's own scratch (d_projected, status) is allocated on demand."""

    def __init__(self, frame: Frame):
        c = frame.cams
        self.cams = Cameras.__new__(Cameras)
        self.cams.sizes, self.cams.V, self.cams.host = c.sizes.copy(), c.V, c.host.copy()
        self.cams.dev = c.dev.clone()
        self.cams.n_pixels, self.cams.pix_base = c.n_pixels, c.pix_base.copy()
        self.N, self.cfg, self.n_tiles = frame.N, dict(frame.cfg), frame.n_tiles
        self.projected, self.counts, self.vals, self.cull = frame.projected, frame.counts, frame.vals, frame.cull
        self.tile_ranges, self.image = frame.tile_ranges, frame.image
        self.final_T, self.last = frame.final_T, frame.last
        self.d_projected = None
        self.status = None

    def alloc_scratch(self):
        if self.d_projected is None:
            dev = self.projected.device
            self.d_projected = torch.empty(self.cams.V * self.N * gs.DRECORD_FLOATS, dtype=torch.float32, device=dev)
            self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        return self

    def read_status(self) -> int:
        return int(self.status.item()) if self.status is not None else 0


def project(params: FlatParams, cams: Cameras, frame: Frame, stream=None):
    gs.gs_project(params["means"], params["log_scales"], params["quats"], params["opacity_logits"], params["sh"],
                  cams.dev, cams.sizes, frame.cfg, frame.projected, frame.rects, frame.counts, frame.status, stream,
                  depth_keys=frame.depth_keys)


def bin_sort(frame: Frame, stream=None):
    if frame.partitions == 1:
        gs.gs_bin_sort(frame.projected, frame.rects, frame.counts, frame.N, frame.cams.sizes, frame.cfg, frame.keys,
                       frame.vals, frame.capacity, frame.tile_ranges, frame.n_isect, frame.workspace, frame.status,
                       stream, depth_keys=frame.depth_keys)
    else:
        gs.gs_bin_sort_partitioned(frame.projected, frame.rects, frame.counts, frame.N, frame.cams.sizes, frame.cfg,
                                   frame.keys, frame.vals, frame.capacity, frame.tile_ranges, frame.n_isect,
                                   frame.partitions, frame.workspace, frame.status, stream,
                                   depth_keys=frame.depth_keys)


def rasterize_fwd(frame: Frame, stream=None):
    gs.gs_rasterize_fwd(frame.projected, frame.vals, frame.tile_ranges, frame.cams.sizes, frame.cfg, frame.image,
                        frame.final_T, frame.last, stream, cull_masks=frame.cull)


def rasterize_fwd_l1l2(frame: Frame, target, n_values, w_l1, w_l2, accumulate, dL_dimage, loss, stream=None):
    """rasterize_fwd with the L1 + L2 image loss computed in the same kernel
    (target and dL_dimage laid out like frame.image)."""
    gs.gs_rasterize_fwd_l1l2(frame.projected, frame.vals, frame.tile_ranges, frame.cams.sizes, frame.cfg,
                             frame.image, frame.final_T, frame.last, target, n_values, w_l1, w_l2, accumulate,
                             dL_dimage, loss, stream, cull_masks=frame.cull)


def rasterize_bwd(params: FlatParams, cams: Cameras, frame: Frame, dL_dimage, grads: FlatParams, stream=None,
                  accumulate=False):
    flags = int(frame.cfg.get("flags", 0)) & ~gs.GS_FLAG_ACCUMULATE_GRADS
    cfg = dict(frame.cfg, flags=flags | (gs.GS_FLAG_ACCUMULATE_GRADS if accumulate else 0))
    gs.gs_rasterize_bwd(params["means"], params["log_scales"], params["quats"], params["opacity_logits"],
                        params["sh"], cams.dev, cams.sizes, cfg, frame.projected, frame.counts, frame.vals,
                        frame.tile_ranges, frame.final_T, frame.last, dL_dimage, frame.d_projected, grads["means"],
                        grads["log_scales"], grads["quats"], grads["opacity_logits"], grads["sh"], frame.status,
                        stream, cull_masks=frame.cull)


def render(params: FlatParams, cams: Cameras, frame: Frame, max_retries: int = 3):
    """project -> bin_sort -> rasterize_fwd, growing the key capacity (host
    check after the sort) until every intersection fits."""
    project(params, cams, frame)
    for _ in range(max_retries + 1):
        frame.clear_status()
        bin_sort(frame)
        st = frame.read_status()
        if st & gs.GS_STATUS_TIMEOUT:
            raise gs.GSError("gs_bin_sort: device wait timed out")
        if not (st & gs.GS_STATUS_CAPACITY):
            break
        need = int(frame.n_isect.item())
        frame.set_capacity(int(need * 1.25) + 1024)
    else:
        raise gs.GSError("gs_bin_sort: capacity retries exhausted")
    rasterize_fwd(frame)
    return frame


def morton_permutation(params: FlatParams, stream=None):
    """Permutation (int32 on the device) that lists the Gaussians along a 3D
    Morton curve of their means (gs_morton_order); returns (perm, status)."""
    N = params.N
    dev = params.flat.device
    perm = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
    ws = torch.empty(max(gs.gs_morton_workspace_bytes(N), 1), dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    if ws.data_ptr() % 256:
        raise gs.GSError("workspace allocation is not 256-byte aligned")
    gs.gs_morton_order(params["means"], N, perm, None, ws, status, stream)
    return perm, status


def permute_gaussians(params: FlatParams, perm, out: FlatParams | None = None, status=None, stream=None) -> FlatParams:
    """out[name][i] = params[name][perm[i]] for every parameter array (gs_gather_rows)."""
    out = out if out is not None else params.like()
    status = status if status is not None else torch.zeros(1, dtype=torch.int32, device=params.flat.device)
    for name in PARAM_NAMES:
        gs.gs_gather_rows(params[name], out[name], params.N, PARAM_WIDTH[name], perm, status, stream)
    return out


class GaussianRasterize(torch.autograd.Function):
    """image[P, 3] = render(means, log_scales, quats, opacity_logits, sh).

    The forward keeps only what the backward needs: the projected records, the
    sorted list and tile ranges, and per pixel the final transmittance and the
    last-contributor count (no per-pixel lists). It takes these buffers over
    from the frame (Frame.hand_over), so the frame can render again before
    this backward runs, in any order of forwards and backwards. The backward
    calls gs_rasterize_bwd, which recomputes transmittance in reverse from the
    final T and the last-contributor count."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, cams: Cameras, frame: Frame):
        N = means.shape[0]
        params = _PackedView(means, log_scales, quats, opacity_logits, sh, N)
        render(params, cams, frame)
        ctx.state = frame.hand_over()
        ctx.save_for_backward(means, log_scales, quats, opacity_logits, sh)
        return ctx.state.image.view(-1, 3)

    @staticmethod
    def backward(ctx, grad_image):
        means, log_scales, quats, opacity_logits, sh = ctx.saved_tensors
        st = ctx.state.alloc_scratch()
        N = means.shape[0]
        params = _PackedView(means, log_scales, quats, opacity_logits, sh, N)
        grads = FlatParams(N, means.device)
        rasterize_bwd(params, st.cams, st, grad_image.contiguous().view(-1), grads)
        ins = (means, log_scales, quats, opacity_logits, sh)
        out = tuple(grads[k].view(t.shape) if need else None
                    for k, t, need in zip(PARAM_NAMES, ins, ctx.needs_input_grad[:5]))
        return out + (None, None)


class _PackedView:
    """Parameter tensors in the form the binding functions index by name;
    each must be a contiguous float32 CUDA tensor with N rows of its width
    (sh as [N, 16, 3] or [N, 48], opacity_logits as [N] or [N, 1])."""

    def __init__(self, means, log_scales, quats, opacity_logits, sh, N):
        self.N = N
        self.views = {}
        for name, t in zip(PARAM_NAMES, (means, log_scales, quats, opacity_logits, sh)):
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor")
            if t.dim() == 0 or t.shape[0] != N or t.numel() != N * PARAM_WIDTH[name]:
                raise ValueError(f"{name}: expected {N} rows of {PARAM_WIDTH[name]} floats, got shape "
                                 f"{tuple(t.shape)}")
            self.views[name] = t.detach()

    def __getitem__(self, k):
        return self.views[k]


def rasterize(means, log_scales, quats, opacity_logits, sh, cams: Cameras, frame: Frame):
    """Differentiable render of all views of `cams`; returns image [P, 3]."""
    return GaussianRasterize.apply(means, log_scales, quats, opacity_logits, sh, cams, frame)


class TrainStep:
    """One training step (forward, image loss, backward, optionally Adam) over
    a batch of views, entirely in libgs_gb300 kernels.

    mode="batched": one launch per stage for all views; after `prepare()` the
    whole step is captured into a CUDA graph and `run()` is one graph replay.
    mode="per_view": every stage launched separately per view (the plain path
    a per-camera training loop would take), without graph capture.
    loss="l1l2": the scene's w_l1 mean|r| + w_l2 mean(r^2); loss="ssim": the
    fused SSIM loss (1 - ssim_lambda) mean|r| + ssim_lambda (1 - mean SSIM).
    Rasteriser launch configuration (see autotune.py): tile=(tw, th),
    raster_px (pixels per thread, 2 or 4; None keeps the scene's setting) and
    raster_batch=(forward, backward) splats per shared-memory batch (0: the
    default). graph: capture the step in a CUDA graph (default: batched mode
    only).
    """

    def __init__(self, scene: dict, mode="batched", adam=False, lr=1e-3, betas=(0.9, 0.999), eps=1e-15,
                 tile=None, device="cuda", graph=None, params: FlatParams | None = None, loss="l1l2",
                 ssim_lambda=0.2, densify_stats=False, raster_px=None, raster_batch=(0, 0)):
        if loss not in ("l1l2", "ssim"):
            raise ValueError(f"unknown loss {loss!r}")
        self.loss_kind, self.ssim_lambda = loss, float(ssim_lambda)
        # by default the batched step is captured and the per-view step (the
        # plain per-camera loop) is not; graph=True captures either
        self.mode, self.adam_on = mode, adam
        self.graph_on = (mode == "batched") if graph is None else bool(graph)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.cfg = dict(scene["cfg"])
        if tile is not None:
            self.cfg["tile_w"], self.cfg["tile_h"] = tile
        if raster_px is not None:
            if raster_px not in (2, 4):
                raise ValueError("raster_px must be 2 or 4")
            fl = int(self.cfg.get("flags", 0)) & ~gs.GS_FLAG_RASTER_2PX
            self.cfg["flags"] = fl | (gs.GS_FLAG_RASTER_2PX if raster_px == 2 else 0)
        self.cfg["raster_batch_fwd"], self.cfg["raster_batch_bwd"] = (int(b) for b in raster_batch)
        self.N = int(scene["means"].shape[0])
        self.params = params if params is not None else FlatParams(self.N, device).load_from(scene)
        self.grads = self.params.like()
        self.cams = Cameras(scene["cams"], scene["sizes"], device)
        self.target = torch.from_numpy(np.ascontiguousarray(scene["target"], np.float32).reshape(-1)).to(device)
        self.w_l1, self.w_l2 = scene["loss"]
        if mode == "batched":
            self.frame_cams = [self.cams]
        else:
            self.frame_cams = [self.cams.view(v) for v in range(self.cams.V)]
        self.frames = [Frame(self.N, c, self.cfg, device=device) for c in self.frame_cams]
        self.image = torch.zeros(self.cams.n_pixels * 3, dtype=torch.float32, device=device)
        self.dL_dimage = torch.zeros_like(self.image)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=device)
        self.densify_on = densify_stats
        if densify_stats:  # accumulated over steps until the caller resets them
            self.grad_accum = torch.zeros(self.N, dtype=torch.float32, device=device)
            self.denom = torch.zeros_like(self.grad_accum)
            self.max_radii = torch.zeros_like(self.grad_accum)
        if adam:
            self.exp_avg = torch.zeros_like(self.params.flat)
            self.exp_avg_sq = torch.zeros_like(self.params.flat)
        self.graph = None
        self.launches_per_step = None

    # -- stage launches ------------------------------------------------------
    def _enqueue(self, stream=None):
        """Enqueues one full step; returns the number of library kernels launched."""
        n = 0
        pv = self.mode == "per_view"
        # the L1 + L2 loss is computed by the forward kernel itself (its value
        # summed over the views); the SSIM loss needs whole windows and runs after
        fused_loss = self.loss_kind == "l1l2"
        for v, (fr, cams) in enumerate(zip(self.frames, self.frame_cams)):
            project(self.params, cams, fr, stream)
            bin_sort(fr, stream)
            # the frame's image is its slice of the packed image
            a, b = int(self.cams.pix_base[v]) * 3, int(self.cams.pix_base[v + 1 if pv else -1]) * 3
            fr.image = self.image[a:b]
            if fused_loss:
                rasterize_fwd_l1l2(fr, self.target[a:b], self.image.numel(), self.w_l1, self.w_l2, v > 0,
                                   self.dL_dimage[a:b], self.loss, stream)
            else:
                rasterize_fwd(fr, stream)
            n += 1 + self._sort_launches(fr) + 1  # project, sort, raster
        if not fused_loss:
            self.enqueue_loss(stream)
            n += 1
        for v, (fr, cams) in enumerate(zip(self.frames, self.frame_cams)):
            a, b = int(self.cams.pix_base[v]) * 3, int(self.cams.pix_base[v + 1 if pv else -1]) * 3
            rasterize_bwd(self.params, cams, fr, self.dL_dimage[a:b], self.grads, stream, accumulate=pv and v > 0)
            n += 2
            if self.densify_on:
                gs.gs_densify_stats(fr.projected, fr.counts, fr.d_projected, self.N, cams.sizes, self.grad_accum,
                                    self.denom, self.max_radii, stream)
                n += 1
        if self.adam_on:
            gs.gs_adam_step(self.params.flat, self.grads.flat, self.exp_avg, self.exp_avg_sq, self.lr, self.betas[0],
                            self.betas[1], self.eps, self.step_count, stream)
            n += 1
        return n

    def enqueue_loss(self, stream=None):
        """The image loss of the step: its value into self.loss, its gradient into self.dL_dimage."""
        if self.loss_kind == "ssim":
            gs.gs_ssim_loss(self.image, self.target, self.cams.sizes, self.ssim_lambda, self.dL_dimage, self.loss,
                            stream)
        else:
            gs.gs_image_loss(self.image, self.target, self.w_l1, self.w_l2, self.dL_dimage, self.loss, stream)

    @staticmethod
    def _sort_launches(fr: Frame) -> int:
        """Kernels gs_bin_sort launches: compaction, 4 depth passes, the
        super-tile emission, the super-tile passes (each scans its digit counts
        itself), the chunk offsets and the chunk table, the chunk counts, the
        per-super-tile scan, the tile scan and the scatter, then the optional
        64-bit keys and tile order."""
        tw, th = int(fr.cfg["tile_w"]), int(fr.cfg["tile_h"])
        n_super = 0
        for W, H in fr.cams.sizes:
            ntx, nty = -(-int(W) // tw), -(-int(H) // th)
            n_super += (-(-ntx // 8)) * (-(-nty // 8))
        bits = 0
        while (1 << bits) < n_super:
            bits += 1
        super_passes = (bits + 7) // 8
        order = 1 if fr.cfg.get("flags", 0) & gs.GS_FLAG_TILE_ORDER else 0
        return 1 + 4 + 1 + super_passes + 5 + 1 + (1 if fr.keep_keys else 0) + order

    def prepare(self, warmup_checks=2):
        """Sizes the key capacity from an eager run, then (batched mode)
        captures the step into a CUDA graph."""
        for fr in self.frames:
            fr.clear_status()
        for _ in range(warmup_checks + 3):
            if self.adam_on:
                self.step_count.fill_(1)
            self._enqueue()
            torch.cuda.synchronize()
            grew = False
            for fr in self.frames:
                st = fr.read_status()
                if st & gs.GS_STATUS_TIMEOUT:
                    raise gs.GSError("device wait timed out")
                if st & gs.GS_STATUS_CAPACITY:
                    fr.set_capacity(int(int(fr.n_isect.item()) * 1.15) + 4096)
                    grew = True
                fr.clear_status()
            if not grew:
                break
        else:
            raise gs.GSError("could not size the key capacity")
        self.launches_per_step = self._enqueue()  # counted on an eager step
        torch.cuda.synchronize()
        if self.graph_on:
            self.graph = self._capture()
        if self.densify_on:  # the sizing and capture steps do not count
            self.reset_densify_stats()
            torch.cuda.synchronize()
        return self

    def _capture(self):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self._enqueue(s)  # warm the capture stream
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self._enqueue(torch.cuda.current_stream())
        torch.cuda.synchronize()
        return graph

    def capture_fed(self, target, cams_dev):
        """One more graph of the (batched, captured) step that reads its target
        image and cameras from the given device buffers instead of self.target
        and self.cams.dev, so that a host-fed step needs no device copy of its
        inputs. The capture runs the step once on those buffers (an optimizer
        or densification statistics in the step advance with it)."""
        if self.graph is None or self.mode != "batched":
            raise ValueError("capture_fed needs a prepared batched step with a CUDA graph")
        old_t, old_c = self.target, self.cams.dev
        self.target, self.cams.dev = target, cams_dev
        try:
            return self._capture()
        finally:
            self.target, self.cams.dev = old_t, old_c

    def reset_densify_stats(self):
        """Starts a new densification-statistics window."""
        self.grad_accum.zero_()
        self.denom.zero_()
        self.max_radii.zero_()

    def run(self):
        """Enqueues one step (graph replay in batched mode)."""
        if self.adam_on:
            self._bump_step()
        if self.graph is not None:
            self.graph.replay()
        else:
            self._enqueue()

    def _bump_step(self):
        self.step_count.add_(1)

    def check(self):
        """Host check of the device status words (call after a sync)."""
        for fr in self.frames:
            st = fr.read_status()
            if st:
                raise gs.GSError(f"device status {st}: capacity/timeout/bounds")

    def n_isect(self) -> int:
        return int(sum(int(fr.n_isect.item()) for fr in self.frames))


class HostFedStep:
    """Training steps fed from host memory: every step copies its cameras and
    target image in from (pinned) host buffers and its loss back out; with
    stream_params=True it also copies the parameters in and the gradients
    out (a caller that keeps the Gaussians in host memory), otherwise the
    parameters stay resident in device memory as model state and the
    gradients stay there for an optimizer on the device. The copies run on
    two copy streams, double-buffered in device staging buffers, so the
    inputs of step k+1 and the outputs of step k move while step k computes;
    the link carries both directions at once. Stream order keeps every
    hazard: a staging buffer is refilled only after the step that used it has
    consumed it, and read out only after the step that fills it is done.

    run(...) enqueues one step and returns at once; the host buffers passed to
    a step must stay untouched until sync() (or until two later steps have
    been enqueued and synced). host_params and host_grads are ignored (and
    may be None) without stream_params."""

    def __init__(self, step: TrainStep, stream_params: bool = True):
        self.step = step
        self.stream_params = bool(stream_params)
        dev = step.params.flat.device
        sp = self.stream_params
        self.in_params = [torch.empty_like(step.params.flat) for _ in range(2)] if sp else None
        self.in_target = [torch.empty_like(step.target) for _ in range(2)]
        self.in_cams = [torch.empty_like(step.cams.dev) for _ in range(2)]
        self.out_grads = [torch.empty_like(step.grads.flat) for _ in range(2)] if sp else None
        self.out_loss = [torch.empty_like(step.loss) for _ in range(2)]
        self.h2d = torch.cuda.Stream(device=dev)
        self.d2h = torch.cuda.Stream(device=dev)
        ev = lambda: [torch.cuda.Event() for _ in range(2)]  # noqa: E731
        self.in_ready, self.in_free, self.out_ready, self.out_free = ev(), ev(), ev(), ev()
        self.k = 0
        # a captured step gets one graph per staging buffer, reading the
        # target image and cameras where they land (no device-to-device copy);
        # not with an optimizer or densification statistics in the step, whose
        # state the capture's own run would advance
        self.graphs = None
        if step.graph is not None and not step.adam_on and not step.densify_on:
            for b in range(2):  # valid contents for the capture's own run
                self.in_target[b].copy_(step.target)
                self.in_cams[b].copy_(step.cams.dev)
            self.graphs = [step.capture_fed(self.in_target[b], self.in_cams[b]) for b in range(2)]

    def run(self, host_params, host_target, host_cams, host_grads, host_loss):
        st, b = self.step, self.k & 1
        comp = torch.cuda.current_stream()
        if self.k >= 2:
            self.h2d.wait_event(self.in_free[b])
        sp = self.stream_params
        with torch.cuda.stream(self.h2d):
            if sp:
                self.in_params[b].copy_(host_params, non_blocking=True)
            self.in_target[b].copy_(host_target, non_blocking=True)
            self.in_cams[b].copy_(host_cams, non_blocking=True)
            self.in_ready[b].record(self.h2d)
        comp.wait_event(self.in_ready[b])
        if sp:
            st.params.flat.copy_(self.in_params[b])
        if self.graphs is not None:
            self.graphs[b].replay()
            self.in_free[b].record(comp)  # the step has read its inputs
        else:
            st.target.copy_(self.in_target[b])
            st.cams.dev.copy_(self.in_cams[b])
            self.in_free[b].record(comp)
            st.run()
        if self.k >= 2:
            comp.wait_event(self.out_free[b])
        if sp:
            self.out_grads[b].copy_(st.grads.flat)
        self.out_loss[b].copy_(st.loss)
        self.out_ready[b].record(comp)
        self.d2h.wait_event(self.out_ready[b])
        with torch.cuda.stream(self.d2h):
            if sp:
                host_grads.copy_(self.out_grads[b], non_blocking=True)
            host_loss.copy_(self.out_loss[b], non_blocking=True)
            self.out_free[b].record(self.d2h)
        self.k += 1

    def sync(self):
        """Waits for every enqueued step, its copies included."""
        torch.cuda.current_stream().synchronize()
        self.h2d.synchronize()
        self.d2h.synchronize()
