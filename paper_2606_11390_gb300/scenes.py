"""Seeded synthetic scenes: Gaussian parameters, cameras, target images.

This module only draws inputs. It holds none of the splatting arithmetic, so
the CUDA path and the CPU oracle can both be fed from it without sharing any
part of the method. Every generator uses numpy's PCG64 with an explicit seed.

A scene is a dict:
  means [N,3], log_scales [N,3], quats [N,4] (w,x,y,z), opacity_logits [N],
  sh [N,16,3] (coefficient-major, channel-minor), all float32;
  cams [V,20] float32 = row-major 4x4 world->camera matrix (OpenCV axes:
  +x right, +y down, +z forward) followed by fx, fy, cx, cy;
  sizes [V,2] int32 = (width, height) per view;
  target [P,3] float32 with P = sum of width*height, views packed in order;
  cfg: tile size, SH degree and the compositing constants;
  loss: (w_l1, w_l2) for L = w_l1 mean|r| + w_l2 mean(r^2).

The named workloads stand in for the paper's Mip-NeRF 360 and aerial scenes
(§5), which are not available here: same Gaussian counts and image sizes,
parameter distributions from the configuration each name describes.
"""
from __future__ import annotations

import numpy as np

BASE_CFG = dict(tile_w=16, tile_h=16, sh_degree=3, near=0.01, far=1e10, eps2d=0.3, alpha_cap=0.99,
                alpha_min=1.0 / 255.0, t_stop=1e-4, bg=(0.0, 0.0, 0.0))


# Tile shape of the single-camera workloads: the tile-size autotuner's sweep
# on GB300 for the 4M-Gaussian 3840x2160 step measured 16x16: 6.30 ms,
# 32x16: 5.82 ms, 32x32: 6.13 ms, 8x8: 14.0 ms per step. (The street scene,
# with its near-camera splats, is faster with 16x16: 104 vs 118 ms.)
WIDE_TILES = dict(tile_w=32, tile_h=16)


def make_cfg(**over):
    c = dict(BASE_CFG)
    c.update(over)
    return c


def look_at(eye, target, up):
    """World->camera 4x4 matrix for a camera at `eye` looking at `target`
    (OpenCV axes; `up` is the world up direction)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    down = -np.asarray(up, np.float64)
    right = np.cross(down, f)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    Rm = np.stack([right, down, f])
    M = np.eye(4)
    M[:3, :3] = Rm
    M[:3, 3] = -Rm @ eye
    return M


def camera_row(viewmat, fx, fy, cx, cy):
    return np.concatenate([np.asarray(viewmat, np.float64).reshape(16), [fx, fy, cx, cy]]).astype(np.float32)


def _params(rng, N, means, log_scale_mu=-3.0, log_scale_sigma=0.5):
    """Parameter distributions shared by the named configurations: log-scales
    N(mu, sigma), quaternions N(0,1)^4 normalised, opacity logits N(0,1), SH DC
    N(0.5, 0.2), higher bands N(0, 0.1)."""
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (N, 3)).astype(np.float32)
    q = rng.standard_normal((N, 4), dtype=np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = rng.standard_normal(N, dtype=np.float32)
    sh = np.empty((N, 16, 3), np.float32)
    sh[:, 0, :] = rng.normal(0.5, 0.2, (N, 3)).astype(np.float32)
    sh[:, 1:, :] = (0.1 * rng.standard_normal((N, 15, 3), dtype=np.float32))
    return dict(means=np.ascontiguousarray(means, np.float32), log_scales=log_scales, quats=q, opacity_logits=opac,
                sh=sh)


def _finish(rng, name, params, cams, sizes, cfg, loss):
    sizes = np.asarray(sizes, np.int32).reshape(-1, 2)
    P = int((sizes[:, 0].astype(np.int64) * sizes[:, 1]).sum())
    target = rng.random((P, 3), dtype=np.float32)
    s = dict(params)
    s.update(name=name, cams=np.stack(cams).astype(np.float32), sizes=sizes, cfg=cfg, loss=loss, target=target)
    return s


def clustered_means(rng, N, n_clusters, lo, hi, sigma):
    centres = rng.uniform(lo, hi, (n_clusters, 3))
    idx = rng.integers(0, n_clusters, N)
    return (centres[idx] + sigma * rng.standard_normal((N, 3))).astype(np.float32)


def tiny(seed=1000, N=4096, width=256, height=256, tile=16):
    """4096 Gaussians, one 256x256 pinhole camera (fx=fy=300, centred principal
    point) at the origin looking down +z; means uniform in [-1,1]^3 shifted 4
    units forward; L1 loss against a uniform [0,1] target."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-1, 1, (N, 3)).astype(np.float32) + np.float32([0, 0, 4])
    params = _params(rng, N, means)
    cam = camera_row(np.eye(4), 300.0, 300.0, width / 2, height / 2)
    return _finish(rng, "tiny", params, [cam], [(width, height)], make_cfg(tile_w=tile, tile_h=tile), (1.0, 0.0))


def train_1080p(seed=1001, N=1 << 20):
    """1M Gaussians in 64 isotropic clusters (sigma 0.5) with centres uniform in
    x in [-10,10], y in [-2.5,2.5], z in [3,23]; one 1920x1080 camera, fx=fy=1500;
    loss L1 + 0.2 L2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = clustered_means(rng, N, 64, [-10, -2.5, 3], [10, 2.5, 23], 0.5)
    params = _params(rng, N, means)
    cam = camera_row(np.eye(4), 1500.0, 1500.0, 960.0, 540.0)
    return _finish(rng, "train_1080p", params, [cam], [(1920, 1080)], make_cfg(**WIDE_TILES), (1.0, 0.2))


def diff_4k(seed=1002, N=4 << 20):
    """4M Gaussians, clustered layout scaled to a 40x10x40 box (x in [-20,20],
    y in [-5,5], z in [5,45], cluster sigma 1.0); one 3840x2160 view,
    fx=fy=3000; loss L1 + 0.2 L2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = clustered_means(rng, N, 64, [-20, -5, 5], [20, 5, 45], 1.0)
    params = _params(rng, N, means)
    cam = camera_row(np.eye(4), 3000.0, 3000.0, 1920.0, 1080.0)
    return _finish(rng, "diff_4k", params, [cam], [(3840, 2160)], make_cfg(**WIDE_TILES), (1.0, 0.2))


BATCH16_SIZES = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160)]


def batch16(seed=1003, N=8 << 20, sizes=None, tile=16):
    """8M Gaussians in the 40x10x40 clustered box; 16 views of mixed resolution
    (four each of 640x480, 1280x720, 1920x1080, 3840x2160, interleaved) on an
    orbit of radius 45 about the box centre, azimuth 2*pi*k/16 + U(-0.1, 0.1),
    elevation U(10, 30) degrees, looking at the centre, fx = fy = 0.78 W."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = clustered_means(rng, N, 64, [-20, -5, 5], [20, 5, 45], 1.0)
    params = _params(rng, N, means)
    centre = np.array([0.0, 0.0, 25.0])
    up = np.array([0.0, -1.0, 0.0])
    cams, szs = [], []
    sizes = sizes or BATCH16_SIZES
    for k in range(16):
        az = 2 * np.pi * k / 16 + rng.uniform(-0.1, 0.1)
        el = np.deg2rad(rng.uniform(10, 30))
        eye = centre + 45.0 * np.array([np.cos(el) * np.sin(az), -np.sin(el), -np.cos(el) * np.cos(az)])
        W, H = sizes[k % len(sizes)]
        f = 0.78 * W
        cams.append(camera_row(look_at(eye, centre, up), f, f, W / 2, H / 2))
        szs.append((W, H))
    return _finish(rng, "batch16", params, cams, szs, make_cfg(tile_w=tile, tile_h=tile), (1.0, 0.2))


def street(seed=1004, N=64 << 20, n_views=4, width=3840, height=2160, n_buildings=2000):
    """Street-like scene: 70% of means on a jittered ground plane (height
    N(0, 0.05)) over 1 km x 1 km, 30% on the faces of axis-aligned buildings
    (footprint U(10,40) m per side, height U(5,60) m) placed beside 20 m street
    lanes; log-scales N(-2.5, 0.7); views 1.5 m above the ground looking
    horizontally along a street, fx = fy = 3000. World up is +z."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_ground = int(0.7 * N)
    n_fac = N - n_ground
    ground = np.empty((n_ground, 3), np.float32)
    ground[:, 0] = rng.uniform(-500, 500, n_ground)
    ground[:, 1] = rng.uniform(-500, 500, n_ground)
    ground[:, 2] = rng.normal(0, 0.05, n_ground)
    # buildings on a 60 m block grid, leaving 20 m lanes along x and y
    bx = rng.integers(-8, 8, n_buildings) * 60.0 + 30.0
    by = rng.integers(-8, 8, n_buildings) * 60.0 + 30.0
    sx = rng.uniform(10, 40, n_buildings)
    sy = rng.uniform(10, 40, n_buildings)
    hz = rng.uniform(5, 60, n_buildings)
    area = 2 * (sx + sy) * hz
    b = rng.choice(n_buildings, n_fac, p=area / area.sum())
    face = rng.integers(0, 4, n_fac)
    t = rng.random(n_fac)
    h = rng.random(n_fac) * hz[b]
    x0, x1 = bx[b] - sx[b] / 2, bx[b] + sx[b] / 2
    y0, y1 = by[b] - sy[b] / 2, by[b] + sy[b] / 2
    fac = np.empty((n_fac, 3), np.float32)
    fac[:, 0] = np.where(face < 2, x0 + t * (x1 - x0), np.where(face == 2, x0, x1))
    fac[:, 1] = np.where(face < 2, np.where(face == 0, y0, y1), y0 + t * (y1 - y0))
    fac[:, 2] = h
    means = np.concatenate([ground, fac])
    params = _params(rng, N, means, log_scale_mu=-2.5, log_scale_sigma=0.7)
    cams = []
    for k in range(n_views):
        ex = float(rng.integers(-8, 8)) * 60.0
        ey = float(rng.uniform(-400, 400))
        eye = np.array([ex, ey, 1.5])
        heading = 1.0 if k % 2 == 0 else -1.0
        cams.append(camera_row(look_at(eye, eye + np.array([0.0, heading, 0.0]), [0.0, 0.0, 1.0]), 3000.0, 3000.0,
                               width / 2, height / 2))
    return _finish(rng, "street", params, cams, [(width, height)] * n_views, make_cfg(), (1.0, 0.2))


def random_small(seed, N=64, width=48, height=40, n_views=1, tile=16, sh_degree=3, spread=1.0, depth=4.0,
                 log_scale_mu=-2.5, loss=(1.0, 0.0)):
    """Small random scene for parity and pin tests: N Gaussians in a cube of
    half-size `spread` at distance `depth`, `n_views` cameras jittered around
    the origin, image sizes that are not multiples of the tile size."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = (rng.uniform(-spread, spread, (N, 3)) + np.array([0, 0, depth])).astype(np.float32)
    params = _params(rng, N, means, log_scale_mu=log_scale_mu)
    cams, szs = [], []
    for v in range(n_views):
        eye = rng.uniform(-0.3, 0.3, 3) if v > 0 else np.zeros(3)
        tgt = np.array([0, 0, depth]) + (rng.uniform(-0.2, 0.2, 3) if v > 0 else 0)
        W = width + 7 * v
        H = height + 5 * v
        f = 1.1 * max(W, H)
        cams.append(camera_row(look_at(eye, tgt, [0, -1, 0]), f, f * 1.05, W / 2 + 0.3, H / 2 - 0.2))
        szs.append((W, H))
    return _finish(rng, "random_small", params, cams, szs, make_cfg(tile_w=tile, tile_h=tile, sh_degree=sh_degree),
                   loss)


def crop_view(scene, x0, y0, w, h, keep=None):
    """A copy of a one-view scene restricted to the window [x0, x0+w) x [y0, y0+h):
    the principal point is shifted so that the window becomes the full image.
    `keep` optionally selects a subset of the Gaussians."""
    s = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    if keep is not None:
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            s[k] = np.ascontiguousarray(scene[k][keep])
    cam = s["cams"][0].copy()
    cam[18] -= x0
    cam[19] -= y0
    s["cams"] = cam[None, :]
    s["sizes"] = np.array([[w, h]], np.int32)
    W = int(scene["sizes"][0, 0])
    tgt = scene["target"].reshape(int(scene["sizes"][0, 1]), W, 3)[y0:y0 + h, x0:x0 + w]
    s["target"] = np.ascontiguousarray(tgt.reshape(-1, 3))
    return s


NAMED = {"tiny": tiny, "train_1080p": train_1080p, "diff_4k": diff_4k, "batch16": batch16, "street": street}


def make(name, **kw):
    return NAMED[name](**kw)


VIEW_SIZES = {"tiny": [(256, 256)], "train_1080p": [(1920, 1080)], "diff_4k": [(3840, 2160)],
              "batch16": [BATCH16_SIZES[k % 4] for k in range(16)], "street": [(3840, 2160)] * 4}


def make_sizes(name) -> np.ndarray:
    """The (W, H) of every view of a named workload, without building it."""
    return np.array(VIEW_SIZES[name], np.int32)
