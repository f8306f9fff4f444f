"""FP64 CPU oracle for the Voronoi adjacency N(i) the walk of Alg. 1 needs
(the Delaunay neighbours, rebuilt when sites move: Sec. 3.2 and the Voronoi
optimisation paragraph of Sec. 4).

TEST INFRASTRUCTURE: only ``tests/`` and the benchmark's CPU-baseline leg may
import this module; the CUDA adjacency builder shares no code with it.

* :func:`voronoi_neighbors` -- the definition, computed literally in C
  (``adjacency.c``): j is a neighbour of i iff the part of their bisector plane
  inside the domain box that is no farther from p_i than from any other site
  has a positive area.  The other sites are taken from a k-d tree, nearest
  first; the candidate set is grown until every site left out lies at least
  twice the cell's radius about p_i away, so that none of them can cut the
  cell (its bisector with p_i is then beyond the cell).
* :func:`delaunay_edges` -- the edges of Qhull's Delaunay tetrahedralisation
  (scipy), an independent cross-check of the definition.
* :func:`default_domain` -- the sites' bounding box grown by 5% of its extent
  on every side (at least 1e-3), the domain the adjacency is built in.
"""
from __future__ import annotations

import numpy as np

from . import _d, _i64, _p, lib


def default_domain(pos) -> np.ndarray:
    p = np.asarray(pos, np.float64).reshape(-1, 3)
    lo, hi = p.min(0), p.max(0)
    m = np.maximum(0.05 * (hi - lo), 1e-3)
    return np.concatenate([lo - m, hi + m])


def _faces(pos64, sites, cands, domain):
    """Face areas between each site and each of its candidates, and each
    site's cell radius, for candidate lists ``cands`` (list of int arrays)."""
    off = np.zeros(len(sites) + 1, np.int64)
    off[1:] = np.cumsum([len(c) for c in cands])
    cand = np.ascontiguousarray(np.concatenate(cands) if len(cands) else np.zeros(0), np.int64)
    qi = np.ascontiguousarray(sites, np.int64)
    area = np.zeros(len(cand))
    rmax = np.zeros(len(sites))
    dom = np.ascontiguousarray(domain, np.float64)
    lib().orc_voronoi_faces(len(pos64), _p(pos64, _d), len(qi), _p(qi, _i64), _p(off, _i64),
                            _p(cand, _i64), _p(dom, _d), _p(area, _d), _p(rmax, _d), 0)
    return [area[off[q]:off[q + 1]] for q in range(len(sites))], rmax


def voronoi_neighbors(pos, sites=None, domain=None, k0: int = 48, all_candidates: bool = False):
    """Neighbour ids (sorted) and face areas of ``sites`` (default: all).

    ``all_candidates``: cut every face by every other site (brute force, for
    small sets) instead of the k-d tree candidates."""
    pos64 = np.ascontiguousarray(np.asarray(pos, np.float64).reshape(-1, 3))
    n = len(pos64)
    sites = np.arange(n) if sites is None else np.asarray(sites, np.int64)
    domain = default_domain(pos64) if domain is None else np.asarray(domain, np.float64)
    nbrs = [None] * len(sites)
    areas = [None] * len(sites)
    if all_candidates or n <= k0 + 1:
        cands = [np.delete(np.arange(n), s) for s in sites]
        a, _ = _faces(pos64, sites, cands, domain)
        for q in range(len(sites)):
            keep = a[q] > 0
            order = np.argsort(cands[q][keep])
            nbrs[q], areas[q] = cands[q][keep][order], a[q][keep][order]
        return nbrs, areas
    from scipy.spatial import cKDTree

    tree = cKDTree(pos64)
    todo = np.arange(len(sites))
    k = k0
    while len(todo):
        kk = min(k + 1, n)
        dist, idx = tree.query(pos64[sites[todo]], k=kk)
        cands = []
        for q, s in enumerate(sites[todo]):
            c = idx[q][idx[q] != s]
            cands.append(c[: kk - 1])
        a, rmax = _faces(pos64, sites[todo], cands, domain)
        again = []
        for q, t in enumerate(todo):
            # every site outside the candidates is at least as far as the farthest candidate
            complete = kk >= n or dist[q][-1] >= 2.0 * rmax[q]
            if not complete:
                again.append(t)
                continue
            keep = a[q] > 0
            order = np.argsort(cands[q][keep])
            nbrs[t], areas[t] = cands[q][keep][order], a[q][keep][order]
        todo = np.asarray(again, np.int64)
        k *= 2
    return nbrs, areas


def adjacency(pos, domain=None, k0: int = 48):
    """CSR (int32 offsets [N+1], int32 ids) of the Voronoi adjacency of all
    sites in the domain, rows sorted, and the smallest face area of each row."""
    nbrs, areas = voronoi_neighbors(pos, None, domain, k0)
    off = np.zeros(len(nbrs) + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in nbrs])
    idx = np.concatenate(nbrs).astype(np.int32) if len(nbrs) else np.zeros(0, np.int32)
    amin = np.array([a.min() if len(a) else np.inf for a in areas])
    return off.astype(np.int32), idx, amin


def delaunay_edges(pos):
    """Qhull's Delaunay tetrahedralisation (scipy): symmetric CSR (int32) of
    its edges, and the simplices [T, 4]."""
    from scipy.spatial import Delaunay

    p = np.asarray(pos, np.float64).reshape(-1, 3)
    tri = Delaunay(p)
    s = tri.simplices.astype(np.int64)
    pairs = np.concatenate([s[:, [a, b]] for a in range(4) for b in range(a + 1, 4)])
    pairs = np.concatenate([pairs, pairs[:, ::-1]])
    key = np.unique(pairs[:, 0] * len(p) + pairs[:, 1])
    src, dst = key // len(p), key % len(p)
    off = np.zeros(len(p) + 1, np.int64)
    np.add.at(off, src + 1, 1)
    return np.cumsum(off).astype(np.int32), dst.astype(np.int32), s
