"""Pins of the oracle's near-degenerate ray classes (the accuracy rule's
exception: visited cells may differ only on rays within 1e-6 of a Voronoi
edge or vertex).

Each case builds a geometry whose answer is known by hand: three sites in the
plane z = 0 have one Voronoi edge, the vertical line through their
circumcentre, so a ray's distance to that edge is plain line-to-line
geometry.  Each class is shown to fire on one side of its threshold and not
on the other, so a wrong sign, a dropped term or a wrong plane fails here.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2502_01157_gb300 import scenes as S
from tests.helpers import TinyScene

EDGE, CAMERA, STOP, GRAZE, BEND = (oracle.FLAG_EDGE, oracle.FLAG_CAMERA, oracle.FLAG_STOP,
                                   oracle.FLAG_GRAZE, oracle.FLAG_BEND)


def _three_sites(j=(1.0, 0.0, 0.0), k=(0.0, 1.0, 0.0), half=1.5, sigma=0.5):
    """Sites i = origin, j, k in the plane z = 0; every pair shares a face.
    Their Voronoi edge is the vertical line through the circumcentre."""
    pos = np.array([[0.0, 0.0, 0.0], j, k], np.float32)
    off = np.array([0, 2, 4, 6], np.int32)
    idx = np.array([1, 2, 0, 2, 0, 1], np.int32)
    return TinyScene(pos, off, idx, np.full(3, sigma, np.float32), np.zeros((3, 1, 3), np.float32), 0,
                     np.full(3, -half, np.float32), np.full(3, half, np.float32))


def _ray_cam(eye, direction):
    eye = np.asarray(eye, np.float64)
    return S.Camera(S.look_at(eye, eye + np.asarray(direction, np.float64)), 1.0, 1.0, 0.5, 0.5, 1, 1)


def _edge_point(sc):
    """Circumcentre of the three sites in the plane z = 0 (FP64 of the stored FP32)."""
    p = sc.pos.astype(np.float64)
    a, b, c = p[0, :2], p[1, :2], p[2, :2]
    A = 2 * np.array([b - a, c - a])
    rhs = np.array([b @ b - a @ a, c @ c - a @ a])
    return np.linalg.solve(A, rhs)


def _dist_to_vertical_line(o, d, q):
    """Distance between the line o + t d and the vertical line through (q, z)."""
    w = np.cross(d, [0.0, 0.0, 1.0])
    if np.linalg.norm(w) < 1e-15:
        return float(np.hypot(o[0] - q[0], o[1] - q[1]))
    return float(abs(np.dot(np.array([q[0], q[1], 0.0]) - o, w)) / np.linalg.norm(w))


def _one_ray(sc, cam, **kw):
    out = oracle.render(sc, cam, trace=16, **kw)
    o, d = oracle.camera_rays(cam)
    return out, o[0], d[0]


@pytest.mark.parametrize("h_over_tau", [0.3, -0.3, 10.0, -10.0])
def test_ray_through_a_voronoi_edge_is_flagged_and_one_ten_tau_away_is_not(h_over_tau):
    sc = _three_sites()
    cam0 = _ray_cam((0.1, 0.3, 0.0), (1.0, 0.0, 0.0))
    tau = oracle.render(sc, cam0)["tau"]
    # the ray from o passes the edge point (0.5, 0.5) at distance h, offset
    # perpendicular to its own direction in the plane (its z slope keeps the
    # closest approach at that offset)
    o = np.array([0.1, 0.3, 0.0])
    q0 = np.array([0.5, 0.5, 0.2])
    dxy = (q0 - o)[:2] / np.linalg.norm((q0 - o)[:2])
    perp = np.array([dxy[1], -dxy[0], 0.0])
    q = q0 + h_over_tau * tau * perp
    out, ro, rd = _one_ray(sc, _ray_cam(o, q - o))
    h = _dist_to_vertical_line(ro, rd, _edge_point(sc))
    assert abs(h / tau - abs(h_over_tau)) < 0.1 * abs(h_over_tau)   # the geometry is what we built
    f = int(out["flags"][0])
    assert bool(f & EDGE) == (abs(h_over_tau) < 1.0)
    assert not f & (CAMERA | STOP | GRAZE | BEND)
    # the side of the edge decides the cells: into j (x = 0.5 first) or into k
    cells = [c for c in out["trace_cells"][0] if c >= 0]
    assert cells[:2] == ([0, 1] if h_over_tau > 0 else [0, 2])
    assert out["tie"][0] == bool(f & EDGE) and out["degen"][0] == bool(f)


@pytest.mark.parametrize("delta,edge", [(1e-3, True), (0.1, False)])
def test_grazing_exit_near_an_edge_uses_the_distance_to_the_edge_line(delta, edge):
    # the ray runs nearly parallel to the face x = 0.5 (cosine 1e-4 to its
    # normal) and crosses it delta before it would reach the face y = 0.5: the
    # exit point is ~delta from the plane y = 0.5, but the ray passes within
    # ~1e-4 delta of the edge they share, so a 1e-3 gap is an FP32 tie
    sc = _three_sites()
    c = 1e-4
    a = c * (0.3 - delta)
    out, ro, rd = _one_ray(sc, _ray_cam((0.5 - a, 0.2, 0.0), (c, 1.0, 0.0)))
    tau = out["tau"]
    h = _dist_to_vertical_line(ro, rd, _edge_point(sc))
    f = int(out["flags"][0])
    cells = [x for x in out["trace_cells"][0] if x >= 0]
    assert cells[:2] == [0, 1]                        # it leaves by x = 0.5
    t_exit = out["trace_t"][0][0]
    p = ro + t_exit * rd
    assert 0.5 - p[1] > 100 * tau                     # the exit point is far from y = 0.5
    assert (h < tau) == edge
    assert bool(f & EDGE) == edge
    assert f & GRAZE                                  # cos 1e-4: gradient conditioning


def test_box_exit_next_to_a_grazing_face_is_an_edge_tie():
    # two cells split by x = 0; the ray runs up the box nearly parallel to the
    # face and leaves the box at y = 1 a little before it would cross x = 0:
    # the box face and the cell face meet in an edge the ray passes close by
    pos = np.array([[-1.0, 0, 0], [1.0, 0, 0]], np.float32)
    sc = TinyScene(pos, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32),
                   np.array([0.5, 0.5], np.float32), np.zeros((2, 1, 3), np.float32), 0,
                   np.full(3, -1.0, np.float32), np.full(3, 1.0, np.float32))
    c = 1e-4
    res = {}
    for gap in (1e-3, 0.2):   # t(x = 0) - t(box exit)
        a = c * (1.9 + gap)
        out, ro, rd = _one_ray(sc, _ray_cam((-a, -0.9, 0.0), (c, 1.0, 0.0)))
        assert list(out["trace_cells"][0][:2]) == [0, -1]   # it never reaches x = 0
        w = np.cross(rd, [0.0, 0.0, 1.0])
        h = abs(np.dot(np.array([0.0, 1.0, 0.0]) - ro, w)) / np.linalg.norm(w)  # to the line x = 0, y = 1
        res[gap] = (bool(out["flags"][0] & EDGE), h / out["tau"])
    assert res[1e-3][0] and res[1e-3][1] < 1
    assert not res[0.2][0] and res[0.2][1] > 10


@pytest.mark.parametrize("g_over_tau,flagged", [(0.3, True), (10.0, False)])
def test_camera_next_to_a_bisector_is_flagged(g_over_tau, flagged):
    # the camera sits g from the bisector x = 0.5 of its two nearest sites
    sc = _three_sites()
    tau = oracle.render(sc, _ray_cam((0.2, 0.3, 0.0), (0.0, 0.0, 1.0)))["tau"]
    out, ro, _ = _one_ray(sc, _ray_cam((0.5 + g_over_tau * tau, 0.3, 0.0), (0.0, 0.0, 1.0)))
    i, gap = oracle.nearest_site(sc.pos, ro)
    # the bisector of sites 0 and 1 is x = 0.5 (the FP32 camera moved a little)
    assert i == 1 and gap == pytest.approx(abs(ro[0] - 0.5), rel=1e-9)
    assert gap == pytest.approx(g_over_tau * tau, rel=0.2)
    assert bool(out["flags"][0] & CAMERA) == flagged
    assert out["tie"][0] == flagged


@pytest.mark.parametrize("rel,flagged", [(5e-4, True), (-5e-4, True), (1e-2, False), (-1e-2, False)])
def test_transmittance_next_to_eps_at_a_stop_test_is_flagged(rel, flagged):
    # two cells split by x = 0; the ray crosses the first over length 0.5 with
    # T = exp(-0.5 sigma) = eps (1 + rel) at the face: whether it walks on
    # into the second cell is decided by T > eps
    eps = 1e-4
    sigma = -math.log(eps * (1 + rel)) / 0.5
    sc = TinyScene(np.array([[-1.0, 0, 0], [1.0, 0, 0]], np.float32), np.array([0, 1, 2], np.int32),
                   np.array([1, 0], np.int32), np.array([sigma, 0.5], np.float32),
                   np.zeros((2, 1, 3), np.float32), 0, np.full(3, -1.0, np.float32),
                   np.full(3, 1.0, np.float32))
    out = oracle.render(sc, _ray_cam((-0.5, 0.0, 0.0), (1.0, 0.0, 0.0)), eps=eps)
    T1 = np.exp(-0.5 * np.float64(np.float32(sigma)))
    assert out["steps"][0] == (2 if T1 > eps else 1)
    assert bool(out["flags"][0] & STOP) == flagged
    assert out["stop_tie"][0] == flagged and not out["tie"][0]


def _bounce_then_edge(disc_rel, h_over_tau):
    """A ray along +x hits a mirror sphere with relative discriminant
    disc_rel; the sites are placed so that the reflected ray passes the
    Voronoi edge at h_over_tau * tau (geometry in FP64 from the stored FP32
    camera, sphere and sites)."""
    r = np.float32(0.1)
    centre = np.array([-0.3, 0.0, 0.0], np.float32).astype(np.float64)
    b = float(r) * math.sqrt(1 - disc_rel)
    cam = _ray_cam((-0.8, b, 0.0), (1.0, 0.0, 0.0))
    sph = S.Sphere(tuple(centre), float(r), ior=0.0, max_bounces=1)
    o, d = oracle.camera_rays(cam)
    o, d = o[0], d[0]
    fx = sph.as_f64()
    c64, r64 = np.asarray(fx[1:4], np.float64), float(fx[4])
    oc = o - c64
    bb = d @ oc
    ts = -bb - math.sqrt(bb * bb - (oc @ oc - r64 * r64))
    P = o + ts * d
    n = (P - c64) / r64
    d2 = d - 2 * (d @ n) * n
    d2 /= np.linalg.norm(d2)
    tau = 1e-6
    # edge point 0.6 past the hit along the reflected ray, moved h to the
    # ray's right, so the ray passes on its left: it reaches y = y_e first (k)
    e = P + 0.6 * d2 + h_over_tau * tau * np.array([d2[1], -d2[0], 0.0])
    sc = _three_sites(j=(2 * e[0], 0.0, 0.0), k=(0.0, 2 * e[1], 0.0), half=1.0)
    h = _dist_to_vertical_line(P, d2, _edge_point(sc))
    return sc, cam, sph, h / tau


@pytest.mark.parametrize("disc_rel,expect_edge", [(1e-3, True), (0.05, False)])
def test_edge_distance_after_a_bounce_grows_with_the_bent_rays_error(disc_rel, expect_edge):
    # the same edge pass at ~12 tau: after a near-tangent hit (the FP32
    # reflected direction is off by ~1e-5) it is a tie, after a well-
    # conditioned one it is not; a straight ray at that distance is not
    sc, cam, sph, h = _bounce_then_edge(disc_rel, 12.0)
    assert 11.0 < h < 13.0
    out = oracle.render(sc, cam, effects=sph, trace=16)
    assert out["tau"] == pytest.approx(1e-6)
    f = int(out["flags"][0])
    assert bool(f & BEND) == (disc_rel < 1e-2)
    assert bool(f & EDGE) == expect_edge
    cells = [x for x in out["trace_cells"][0] if x >= 0]
    assert cells[:3] == [0, 0, 2]        # the bounce stays in cell i, then k
