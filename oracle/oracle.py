"""Python handle on the CPU oracle (oracle/gs_oracle.cpp).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check in __graft_entry__ and the
CPU-baseline leg of bench.py may import this module; the product package never
does. The oracle restates the Gaussian-splatting operators that the paper
(arXiv 2606.11390, §4 "Distributed Gaussian Splatting") distributes, following
the 3D Gaussian Splatting formulation it cites (Kerbl et al. 2023). It shares
no code with the CUDA library.

Precision: functions take ``precision="f32"`` (decisions and forward values in
float, the precision of the GPU kernels) or ``"f64"`` (everything in double,
used by the finite-difference pins). Gradients are always returned in double.

Threads: the oracle is built twice from the same source, serial (what the
tests use) and with OpenMP over Gaussians (projection and its backward) and
over tiles (compositing and its backward). Inside ``with parallel(n):`` the
functions run the OpenMP build on n host threads; it exists to time the
oracle on all cores of a host, and its gradient sums may differ from the
serial build's in the last bits (atomic adds in thread order).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgs_oracle.so")
_OMP_PATH = os.path.join(_BUILD, "libgs_oracle_omp.so")
_lock = threading.Lock()
_libs = {}
_use_omp = False

CXXFLAGS = ["-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def _build_one(path, extra, force):
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", *CXXFLAGS, *extra, "-o", tmp, _SRC])
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libgs_oracle.so (serial) and
    libgs_oracle_omp.so (OpenMP), host compiler only; returns the serial one."""
    os.makedirs(_BUILD, exist_ok=True)
    _build_one(_LIB_PATH, [], force)
    try:
        _build_one(_OMP_PATH, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass  # no OpenMP runtime: parallel() then raises
    return _LIB_PATH


@contextlib.contextmanager
def parallel(threads: int | None = None):
    """Runs the oracle's OpenMP build inside the block, on `threads` host
    threads (default: all the runtime offers). Yields the thread count."""
    global _use_omp
    build()
    if not os.path.exists(_OMP_PATH):
        raise RuntimeError("the OpenMP build of the oracle is not available (g++ -fopenmp failed)")
    L = _load(_OMP_PATH)
    if threads:
        L.oracle_set_threads(int(threads))
    old = _use_omp
    _use_omp = True
    try:
        yield int(L.oracle_max_threads())
    finally:
        _use_omp = old


class OConfig(ctypes.Structure):
    _fields_ = [
        ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("sh_degree", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("near_plane", ctypes.c_float), ("far_plane", ctypes.c_float), ("eps2d", ctypes.c_float),
        ("alpha_cap", ctypes.c_float), ("alpha_min", ctypes.c_float), ("t_stop", ctypes.c_float),
        ("bg", ctypes.c_float * 3),
    ]


def make_config(cfg: dict) -> OConfig:
    c = OConfig()
    c.tile_w, c.tile_h, c.sh_degree = int(cfg["tile_w"]), int(cfg["tile_h"]), int(cfg["sh_degree"])
    c.near_plane, c.far_plane, c.eps2d = cfg["near"], cfg["far"], cfg["eps2d"]
    c.alpha_cap, c.alpha_min, c.t_stop = cfg["alpha_cap"], cfg["alpha_min"], cfg["t_stop"]
    for i in range(3):
        c.bg[i] = cfg["bg"][i]
    return c


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32


def lib():
    """The serial build, or the OpenMP build inside parallel()."""
    if _use_omp:
        return _load(_OMP_PATH)
    return _load(build())


def _load(path):
    with _lock:
        if path not in _libs:
            L = ctypes.CDLL(path)
            _libs[path] = L
            L.oracle_exp_cody_waite.restype = ctypes.c_float
            L.oracle_exp_cody_waite.argtypes = [ctypes.c_float]
            L.oracle_sh_basis.argtypes = [_VP, _I64, _VP]
            L.oracle_num_tiles.restype = _I64
            L.oracle_num_tiles.argtypes = [_VP, _I32, _VP]
            for suf in ("f32", "f64"):
                getattr(L, f"oracle_project_{suf}").argtypes = [_VP] * 5 + [_I64, _VP, _VP, _I32, _VP, _VP, _VP, _VP]
                f = getattr(L, f"oracle_bin_sort_{suf}")
                f.restype = _I64
                f.argtypes = [_VP, _VP, _VP, _I64, _VP, _VP, _I32, _VP, _VP, _VP, _I64, _VP]
                getattr(L, f"oracle_raster_fwd_{suf}").argtypes = [_VP, _VP, _VP, _VP, _VP, _I32, _VP, _VP, _I64,
                                                                    _VP, _VP, _VP, _VP, _VP, _VP, _VP]
                getattr(L, f"oracle_raster_bwd_{suf}").argtypes = [_VP, _VP, _VP, _VP, _VP, _I32, _VP, _VP, _I64,
                                                                    _VP, _VP]
                getattr(L, f"oracle_project_bwd_{suf}").argtypes = [_VP] * 5 + [_I64, _VP, _VP, _I32, _VP, _VP, _VP,
                                                                                 _I64] + [_VP] * 5
                getattr(L, f"oracle_render_bruteforce_{suf}").argtypes = [_VP, _VP, _VP, _I64, _VP, _VP, _I32, _VP,
                                                                           _VP, _VP]
            L.oracle_loss.restype = ctypes.c_double
            L.oracle_loss.argtypes = [_VP, _VP, _I64, ctypes.c_double, ctypes.c_double, _VP]
            L.oracle_adam.argtypes = [_VP, _VP, _VP, _VP, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, _I32]
            L.oracle_max_threads.restype = ctypes.c_int
            L.oracle_max_threads.argtypes = []
            L.oracle_set_threads.argtypes = [ctypes.c_int]
    return _libs[path]


def _dt(precision):
    return np.float32 if precision == "f32" else np.float64


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _cams(scene):
    cams = _c(scene["cams"], np.float32).reshape(-1, 20)
    sizes = _c(scene["sizes"], np.int32).reshape(-1, 2)
    return cams, sizes


def exp_cody_waite(x: float) -> float:
    return lib().oracle_exp_cody_waite(float(x))


def sh_basis(dirs: np.ndarray) -> np.ndarray:
    d = _c(dirs, np.float64).reshape(-1, 3)
    out = np.zeros((d.shape[0], 16), np.float64)
    lib().oracle_sh_basis(_p(d), d.shape[0], _p(out))
    return out


def num_tiles(scene) -> int:
    _, sizes = _cams(scene)
    cfg = make_config(scene["cfg"])
    return int(lib().oracle_num_tiles(_p(sizes), sizes.shape[0], ctypes.byref(cfg)))


def _params(scene, precision):
    dt = _dt(precision)
    return [_c(scene[k], dt) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]


def project(scene, precision="f32"):
    """Per (view, Gaussian): 12-value record, int16 tile rectangle, tile count."""
    dt = _dt(precision)
    params = _params(scene, precision)
    N = params[0].shape[0]
    cams, sizes = _cams(scene)
    V = cams.shape[0]
    cfg = make_config(scene["cfg"])
    projected = np.zeros((V * N, 12), dt)
    rects = np.zeros((V * N, 4), np.int16)
    counts = np.zeros(V * N, np.uint32)
    getattr(lib(), f"oracle_project_{precision}")(*[_p(a) for a in params], N, _p(cams), _p(sizes), V,
                                                   ctypes.byref(cfg), _p(projected), _p(rects), _p(counts))
    return {"projected": projected, "rects": rects, "counts": counts}


def bin_sort(scene, proj, precision="f32"):
    """Stable sort of (tile | depth) keys; returns keys, vals, ranges, n_isect."""
    N = scene["means"].shape[0]
    cams, sizes = _cams(scene)
    V = cams.shape[0]
    cfg = make_config(scene["cfg"])
    nt = num_tiles(scene)
    I = int(proj["counts"].astype(np.int64).sum())
    keys = np.zeros(max(I, 1), np.uint64)
    vals = np.zeros(max(I, 1), np.uint32)
    ranges = np.zeros((nt, 2), np.uint32)
    got = getattr(lib(), f"oracle_bin_sort_{precision}")(
        _p(_c(proj["projected"], _dt(precision))), _p(_c(proj["rects"], np.int16)), _p(_c(proj["counts"], np.uint32)),
        N, _p(cams), _p(sizes), V, ctypes.byref(cfg), _p(keys), _p(vals), I, _p(ranges))
    assert got == I
    return {"keys": keys[:I], "vals": vals[:I], "ranges": ranges, "n_isect": I}


def raster_fwd(scene, proj, bins, precision="f32", tiles=None):
    """Image [P,3], final transmittance [P], last-contributor count [P],
    marginal-decision flags per (view, Gaussian) [V*N] and per pixel [P], a
    per-pixel signature of the set of composited list entries [P] and the
    number of entries composited per pixel [P]."""
    dt = _dt(precision)
    cams, sizes = _cams(scene)
    V = cams.shape[0]
    N = scene["means"].shape[0]
    cfg = make_config(scene["cfg"])
    P = int((sizes[:, 0].astype(np.int64) * sizes[:, 1]).sum())
    image = np.zeros((P, 3), dt)
    final_T = np.ones(P, dt)
    last = np.zeros(P, np.uint32)
    marg_vg = np.zeros(V * N, np.uint8)
    marg_pix = np.zeros(P, np.uint8)
    hitsig = np.zeros(P, np.uint64)
    ncomp = np.zeros(P, np.uint32)
    t = None if tiles is None else _c(tiles, np.int64)
    getattr(lib(), f"oracle_raster_fwd_{precision}")(
        _p(_c(proj["projected"], dt)), _p(_c(bins["vals"], np.uint32)), _p(_c(bins["ranges"], np.uint32)), _p(cams),
        _p(sizes), V, ctypes.byref(cfg), _p(t), 0 if t is None else t.shape[0], _p(image), _p(final_T), _p(last),
        _p(marg_vg), _p(marg_pix), _p(hitsig), _p(ncomp))
    return {"image": image, "final_T": final_T, "last": last, "marginal_vg": marg_vg, "marginal_pix": marg_pix,
            "hit_signature": hitsig, "composited": ncomp}


def raster_bwd(scene, proj, bins, dL_dimage, precision="f32", tiles=None):
    """Gradient w.r.t. the 9 rasterised values of each (view, Gaussian) record:
    mean2d x/y, conic A/B/C, r/g/b, opacity. Shape [V*N, 9], double."""
    dt = _dt(precision)
    cams, sizes = _cams(scene)
    V = cams.shape[0]
    N = scene["means"].shape[0]
    cfg = make_config(scene["cfg"])
    d_proj = np.zeros((V * N, 9), np.float64)
    t = None if tiles is None else _c(tiles, np.int64)
    getattr(lib(), f"oracle_raster_bwd_{precision}")(
        _p(_c(proj["projected"], dt)), _p(_c(bins["vals"], np.uint32)), _p(_c(bins["ranges"], np.uint32)), _p(cams),
        _p(sizes), V, ctypes.byref(cfg), _p(t), 0 if t is None else t.shape[0], _p(_c(dL_dimage, np.float64)),
        _p(d_proj))
    return d_proj


def project_bwd(scene, d_proj, precision="f32", gaussians=None):
    """Parameter gradients summed over views, in double. ``gaussians`` selects a subset."""
    params = _params(scene, precision)
    N = params[0].shape[0]
    cams, sizes = _cams(scene)
    V = cams.shape[0]
    cfg = make_config(scene["cfg"])
    sel = None if gaussians is None else _c(gaussians, np.int64)
    n = N if sel is None else sel.shape[0]
    out = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
           "opacity_logits": np.zeros(n), "sh": np.zeros((n, 16, 3))}
    getattr(lib(), f"oracle_project_bwd_{precision}")(
        *[_p(a) for a in params], N, _p(cams), _p(sizes), V, ctypes.byref(cfg), _p(_c(d_proj, np.float64)), _p(sel),
        n, _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]), _p(out["opacity_logits"]), _p(out["sh"]))
    return out


def render_bruteforce(scene, proj, precision="f32"):
    dt = _dt(precision)
    cams, sizes = _cams(scene)
    V = cams.shape[0]
    N = scene["means"].shape[0]
    cfg = make_config(scene["cfg"])
    P = int((sizes[:, 0].astype(np.int64) * sizes[:, 1]).sum())
    image = np.zeros((P, 3), dt)
    final_T = np.ones(P, dt)
    getattr(lib(), f"oracle_render_bruteforce_{precision}")(
        _p(_c(proj["projected"], dt)), _p(_c(proj["rects"], np.int16)), _p(_c(proj["counts"], np.uint32)), N,
        _p(cams), _p(sizes), V, ctypes.byref(cfg), _p(image), _p(final_T))
    return {"image": image, "final_T": final_T}


def loss(image, target, w_l1, w_l2):
    """L = w_l1 * mean|r| + w_l2 * mean(r^2), r = image - target; returns (L, dL/dimage)."""
    img = _c(image, np.float32).reshape(-1)
    tgt = _c(target, np.float32).reshape(-1)
    g = np.zeros(img.shape[0], np.float64)
    L = lib().oracle_loss(_p(img), _p(tgt), img.shape[0], float(w_l1), float(w_l2), _p(g))
    return L, g.reshape(np.shape(image))


def adam(param, grad, m, v, lr, beta1, beta2, eps, t):
    """One Adam step in place on double arrays; returns (param, m, v)."""
    p = _c(param, np.float64).copy()
    mm = _c(m, np.float64).copy()
    vv = _c(v, np.float64).copy()
    g = _c(grad, np.float64)
    lib().oracle_adam(_p(p), _p(g), _p(mm), _p(vv), p.size, lr, beta1, beta2, eps, int(t))
    return p, mm, vv


def forward(scene, precision="f32", tiles=None):
    """project -> bin_sort -> raster_fwd, all on the oracle."""
    proj = project(scene, precision)
    bins = bin_sort(scene, proj, precision)
    ras = raster_fwd(scene, proj, bins, precision, tiles)
    return proj, bins, ras


def backward(scene, proj, bins, dL_dimage, precision="f32", tiles=None, gaussians=None):
    d_proj = raster_bwd(scene, proj, bins, dL_dimage, precision, tiles)
    grads = project_bwd(scene, d_proj, precision, gaussians)
    return d_proj, grads
