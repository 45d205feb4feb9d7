"""Densification statistics, written plainly in numpy.

TEST INFRASTRUCTURE ONLY: tests/, the smoke check in __graft_entry__ and the
CPU-baseline leg of bench.py may use this module; the product package never
does. It shares no code with the CUDA library.

What it computes. The paper (arXiv 2606.11390, §5.2) densifies (Kerbl et al.
2023) during training; the statistics densification reads are, per Gaussian,
the accumulated norm of the loss gradient with respect to its screen-space
position and its largest screen-space radius. The reading taken here follows
the 3DGS formulation: for every view where the Gaussian is visible (a
non-empty tile rectangle), add the Euclidean norm of dL/dmean2d expressed in
normalised device coordinates (the pixel-space gradient times W/2 and H/2),
count the view, and keep the largest radius in pixels.
"""
from __future__ import annotations

import numpy as np


def densify_stats(projected, counts, d_projected, sizes, grad_accum, denom, max_radii):
    """One backward pass's contribution, added to copies of the three running
    arrays; returns (grad_accum, denom, max_radii) as float64."""
    sizes = np.asarray(sizes).reshape(-1, 2)
    V = sizes.shape[0]
    N = np.asarray(grad_accum).shape[0]
    proj = np.asarray(projected, np.float64).reshape(V, N, 12)
    cnt = np.asarray(counts).reshape(V, N)
    dp = np.asarray(d_projected, np.float64).reshape(V, N, 9)
    ga = np.array(grad_accum, np.float64)
    dn = np.array(denom, np.float64)
    mr = np.array(max_radii, np.float64)
    for v in range(V):
        W, H = float(sizes[v, 0]), float(sizes[v, 1])
        for g in range(N):
            if cnt[v, g] == 0:
                continue
            ga[g] += np.hypot(dp[v, g, 0] * W / 2.0, dp[v, g, 1] * H / 2.0)
            dn[g] += 1.0
            mr[g] = max(mr[g], proj[v, g, 7])
    return ga, dn, mr
