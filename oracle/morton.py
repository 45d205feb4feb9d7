"""Morton (Z-order) ordering of Gaussians, written plainly in numpy.

TEST INFRASTRUCTURE ONLY: tests/, the smoke check in __graft_entry__ and the
CPU-baseline leg of bench.py may use this module; the product package never
does. It shares no code with the CUDA library.

What it computes. The paper (arXiv 2606.11390, §5.2) orders the Gaussians along
a three-dimensional Morton curve during densification, for memory locality in
rasterisation; it gives no quantisation. The reading taken here: per axis,
lo and hi are the minimum and maximum of the means; a coordinate becomes the
10-bit integer q = clamp(floor((x - lo) * (1024 / (hi - lo))), 0, 1023), with
the subtraction, the quotient 1024 / (hi - lo) and the product each rounded to
float32 (so the integer is decided in the precision of the GPU path; q = 0 on
an axis where hi == lo). The Morton code places bit b of qx, qy, qz at bits
3b, 3b + 1, 3b + 2. The permutation lists the Gaussians by code, equal codes in
index order (a stable sort).
"""
from __future__ import annotations

import numpy as np

BITS = 10


def quantise(x: np.ndarray, lo: np.float32, hi: np.float32) -> np.ndarray:
    """10-bit cell index of each coordinate, decided in float32."""
    x = np.asarray(x, np.float32)
    ext = np.float32(hi) - np.float32(lo)
    if not ext > 0:
        return np.zeros(x.shape, np.uint32)
    scale = np.float32(1024.0) / ext
    t = (x - np.float32(lo)) * scale
    f = np.floor(t)
    q = np.where(np.isnan(f) | (f <= 0), 0, np.where(f >= 1023, 1023, f))
    return q.astype(np.uint32)


def interleave(qx, qy, qz) -> np.ndarray:
    """Bit b of qx, qy, qz goes to bit 3b, 3b+1, 3b+2 of the code, one bit at a time."""
    qx, qy, qz = (np.asarray(q, np.uint64) for q in (qx, qy, qz))
    code = np.zeros(qx.shape, np.uint64)
    for b in range(BITS):
        code |= ((qx >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
        code |= ((qy >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + 1)
        code |= ((qz >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + 2)
    return code.astype(np.uint32)


def morton_codes(means: np.ndarray) -> np.ndarray:
    """30-bit Morton code of every mean [N][3] (float32), bounding box of all means."""
    m = np.asarray(means, np.float32).reshape(-1, 3)
    if m.shape[0] == 0:
        return np.zeros(0, np.uint32)
    lo, hi = m.min(axis=0), m.max(axis=0)
    q = [quantise(m[:, a], lo[a], hi[a]) for a in range(3)]
    return interleave(*q)


def morton_order(means: np.ndarray):
    """Returns (perm, sorted codes): perm[i] is the old index of the i-th
    Gaussian along the curve."""
    codes = morton_codes(means)
    perm = np.argsort(codes, kind="stable").astype(np.uint32)
    return perm, codes[perm]
