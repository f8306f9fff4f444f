"""Pins of the Voronoi-adjacency oracle (the neighbour lists N(i) of Alg. 1,
rebuilt by the GPU builder when sites move).

* the face-polygon definition against Qhull's Delaunay edges (scipy) in a
  domain large enough to hold every face, on uniform and clustered sets;
* the k-d tree candidate search against brute force over all sites;
* closed forms: two sites (the face is the box's cross-section), a regular
  tetrahedron with its centre (complete graph), an octahedron with its centre
  (opposite vertices are not neighbours), collinear sites (only consecutive
  ones), a face that lies outside the domain;
* Euler's relation V - E + F - T = 1 for the tetrahedralisation the edges
  come from, and the mean face count 2 + 48 pi^2 / 35 of a Poisson-Voronoi cell.
"""
import math

import numpy as np
import pytest

from oracle import adjacency as A
from paper_2502_01157_gb300 import scenes as S

BIG = np.array([-1e6, -1e6, -1e6, 1e6, 1e6, 1e6])   # holds the far faces of nearly coplanar hull sites


def _rows(off, idx):
    return [np.sort(idx[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


@pytest.mark.parametrize("kind,n,seed", [("uniform", 40, 0), ("uniform", 300, 1), ("mixture", 400, 2),
                                         ("uniform", 2000, 3)])
def test_definition_equals_qhull_in_a_large_domain(kind, n, seed):
    rng = np.random.default_rng(seed)
    p = S.uniform_sites(n, -1, 1, rng) if kind == "uniform" else S.mixture_sites(n, rng)
    p = p.astype(np.float64)
    nb, _ = A.voronoi_neighbors(p, domain=BIG, all_candidates=n <= 400)
    off, idx, _ = A.delaunay_edges(p)
    q = _rows(off, idx)
    bad = [i for i in range(n) if not np.array_equal(nb[i], q[i])]
    assert not bad, bad[:5]


@pytest.mark.parametrize("seed", [4, 5])
def test_kdtree_candidates_equal_brute_force(seed):
    rng = np.random.default_rng(seed)
    p = S.mixture_sites(600, rng).astype(np.float64)
    a, _ = A.voronoi_neighbors(p, all_candidates=True)
    b, _ = A.voronoi_neighbors(p, k0=8)            # forces the candidate set to grow
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_two_sites_face_is_the_box_cross_section():
    p = np.array([[-1.0, 0, 0], [1.0, 0, 0]])
    dom = np.array([-2.0, -2, -2, 2, 2, 2])
    nb, ar = A.voronoi_neighbors(p, domain=dom, all_candidates=True)
    assert [list(x) for x in nb] == [[1], [0]]
    assert ar[0][0] == pytest.approx(16.0, rel=1e-12)       # the square x = 0, |y|, |z| <= 2


def test_tetrahedron_with_centre_is_complete():
    t = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1], [0, 0, 0]], np.float64)
    nb, _ = A.voronoi_neighbors(t, domain=BIG, all_candidates=True)
    for i in range(5):
        assert list(nb[i]) == [j for j in range(5) if j != i]


def test_octahedron_with_centre():
    e = np.concatenate([np.eye(3), -np.eye(3), np.zeros((1, 3))])   # +x +y +z -x -y -z, centre 6
    nb, _ = A.voronoi_neighbors(e, domain=np.array([-3.0, -3, -3, 3, 3, 3]), all_candidates=True)
    assert list(nb[6]) == [0, 1, 2, 3, 4, 5]
    for v in range(6):
        opposite = (v + 3) % 6
        assert list(nb[v]) == sorted(set(range(7)) - {v, opposite})


def test_collinear_sites_only_neighbour_their_successors():
    x = np.array([0.0, 0.3, 1.1, 1.5, 2.6])
    p = np.stack([x, np.zeros(5), np.zeros(5)], 1)
    nb, _ = A.voronoi_neighbors(p, domain=np.array([-1.0, -1, -1, 4, 1, 1]), all_candidates=True)
    assert [list(a) for a in nb] == [[1], [0, 2], [1, 3], [2, 4], [3]]


def test_face_outside_the_domain_is_not_an_edge():
    # on the bisector x = 0 of sites 0 and 1, site 2 is farther only where
    # z <= -3/4: the face exists in a box reaching z = -1, not in one cut at -1/2
    p = np.array([[-1.0, 0, 0], [1.0, 0, 0], [0.0, 0, 0.5]])
    nb, ar = A.voronoi_neighbors(p, domain=np.array([-2.0, -1, -1, 2, 1, 1]), all_candidates=True)
    assert list(nb[0]) == [1, 2] and list(nb[1]) == [0, 2]
    assert ar[0][0] == pytest.approx(2 * 0.25, rel=1e-12)   # |y| <= 1, -1 <= z <= -3/4
    nb, _ = A.voronoi_neighbors(p, domain=np.array([-2.0, -1, -0.5, 2, 1, 1]), all_candidates=True)
    assert list(nb[0]) == [2] and list(nb[1]) == [2]


def test_euler_relation_of_the_tetrahedralisation():
    rng = np.random.default_rng(7)
    p = rng.uniform(-1, 1, (500, 3))
    off, idx, simp = A.delaunay_edges(p)
    V, E, T = len(p), len(idx) // 2, len(simp)
    tri = np.sort(np.concatenate([simp[:, [0, 1, 2]], simp[:, [0, 1, 3]], simp[:, [0, 2, 3]],
                                  simp[:, [1, 2, 3]]]), axis=1)
    F = len(np.unique(tri, axis=0))
    assert V - E + F - T == 1


def test_poisson_voronoi_mean_face_count():
    rng = np.random.default_rng(11)
    p = rng.uniform(0, 1, (40000, 3))
    inner = np.where(np.all((p > 0.2) & (p < 0.8), axis=1))[0][:4000]
    nb, _ = A.voronoi_neighbors(p, sites=inner)
    mean = np.mean([len(x) for x in nb])
    expect = 2 + 48 * math.pi ** 2 / 35       # 15.535...
    assert abs(mean - expect) < 0.2, mean      # standard error ~ 3.3 / sqrt(4000)
