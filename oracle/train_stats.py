"""Plain CPU reference of the densification and pruning statistics (Sec. 3.3).

TEST INFRASTRUCTURE: only ``tests/`` may import this module; the CUDA
renderer shares no code with it.

* :func:`densify_scores` -- per site, the norm of the position gradient
  times the approximate radius of its Voronoi cell, read here as half the mean
  distance to its Delaunay neighbours (the faces of the cell lie halfway to the
  neighbours).
* :func:`sample_multinomial` -- draws with probability proportional to the
  scores; the uniform numbers are inputs, and a draw u selects the first site
  whose inclusive cumulative weight exceeds u * total (FP64 sums).
* :func:`prune_mask` -- a site is pruned when its density and the density of
  every neighbour are below the threshold (low density and surrounded by
  low-density cells, so it neither renders nor bounds a surface).
"""
from __future__ import annotations

import numpy as np


def cell_radius(pos, adj_off, adj_idx) -> np.ndarray:
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    r = np.zeros(n)
    for i in range(n):
        nb = adj_idx[adj_off[i]:adj_off[i + 1]]
        if len(nb):
            r[i] = 0.5 * np.mean([np.linalg.norm(pos[j] - pos[i]) for j in nb])
    return r


def densify_scores(pos, adj_off, adj_idx, g_pos) -> np.ndarray:
    g = np.asarray(g_pos, np.float64)
    return np.sqrt(np.sum(g * g, axis=1)) * cell_radius(pos, adj_off, adj_idx)


def sample_multinomial(weights, u) -> np.ndarray:
    w = np.asarray(weights, np.float64)
    cdf = np.cumsum(w)
    target = np.asarray(u, np.float64) * cdf[-1]
    return np.searchsorted(cdf, target, side="right").astype(np.int64)


def prune_mask(density, adj_off, adj_idx, threshold) -> np.ndarray:
    d = np.asarray(density, np.float64)
    n = len(d)
    out = np.zeros(n, bool)
    for i in range(n):
        if d[i] < threshold:
            nb = adj_idx[adj_off[i]:adj_off[i + 1]]
            out[i] = all(d[j] < threshold for j in nb)
    return out
