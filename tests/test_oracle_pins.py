"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself:

* the Voronoi definition, Eq. (5), by brute force over all sites;
* closed forms of Eq. (3)-(4) (homogeneous media, empty media, a two-cell
  scene and an early-stop chain derived by hand);
* the real spherical harmonics against scipy and against orthonormality;
* the analytic backward against central finite differences of the forward;
* ray generation against the pinhole projection it inverts.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2502_01157_gb300 import scenes as S
from tests.helpers import TinyScene, camera_at, csr_from_lists, random_scene


# ---------------------------------------------------------------------------
# Spherical harmonics (Sec. 3.4: view-dependent colour by SH of degree three)
# ---------------------------------------------------------------------------
def _sphere_quadrature(n_theta=24, n_phi=48):
    x, w = np.polynomial.legendre.leggauss(n_theta)  # x = cos(theta)
    phi = (np.arange(n_phi) + 0.5) * 2 * np.pi / n_phi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wts = (w[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).reshape(-1)
    return dirs, wts


def test_sh_orthonormal():
    dirs, wts = _sphere_quadrature()
    Y = oracle.sh_basis(3, dirs)
    G = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_matches_scipy_complex_harmonics():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(0)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = oracle.sh_basis(3, d)
    for l in range(4):
        for m in range(-l, l + 1):
            Ylm = sp.sph_harm_y(l, abs(m), theta, phi)  # Condon-Shortley phase included
            if m > 0:
                ref = math.sqrt(2) * (-1) ** m * Ylm.real
            elif m < 0:
                ref = math.sqrt(2) * (-1) ** m * Ylm.imag
            else:
                ref = Ylm.real
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-12,
                                       err_msg=f"l={l} m={m}")


def test_sh_degree0_constant():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(0, d)
    np.testing.assert_allclose(Y[:, 0], 1 / (2 * math.sqrt(math.pi)), rtol=1e-15)


# ---------------------------------------------------------------------------
# Rays and nn(o)
# ---------------------------------------------------------------------------
def test_camera_rays_reproject_to_pixel_centres():
    rng = np.random.default_rng(2)
    for _ in range(5):
        eye = rng.uniform(-3, 3, 3)
        cam = S.Camera(S.look_at(eye, rng.uniform(-1, 1, 3)), 40.0, 55.0, 13.3, 9.1, 27, 19)
        o, d = oracle.camera_rays(cam)
        np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
        R = cam.c2w[:, :3].astype(np.float64)
        t = cam.c2w[:, 3].astype(np.float64)
        np.testing.assert_allclose(o, np.broadcast_to(t, o.shape), atol=0)
        pc = np.linalg.solve(R, (o + 2.5 * d - t).T).T   # back into the camera frame
        u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
        v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
        uu, vv = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
        np.testing.assert_allclose(u, uu.reshape(-1) + 0.5, atol=1e-9)
        np.testing.assert_allclose(v, vv.reshape(-1) + 0.5, atol=1e-9)
        assert np.all(pc[:, 2] > 0)


def test_nearest_site_is_bruteforce_argmin():
    rng = np.random.default_rng(3)
    pos = rng.uniform(-1, 1, (500, 3)).astype(np.float32)
    for _ in range(20):
        q = rng.uniform(-1.5, 1.5, 3)
        i, gap = oracle.nearest_site(pos, q)
        dd = np.sum((pos.astype(np.float64) - q) ** 2, axis=1)
        assert i == int(np.argmin(dd))
        j = np.argsort(dd)[1]
        n = pos[j].astype(np.float64) - pos[i]
        assert gap == pytest.approx((dd[j] - dd[i]) / (2 * np.linalg.norm(n)), rel=1e-12)


# ---------------------------------------------------------------------------
# The walk against the Voronoi definition (Eq. 5) by brute force
# ---------------------------------------------------------------------------
def _nearest(pos, p):
    dd = np.sum((pos[None, :, :] - p[:, None, :]) ** 2, axis=2)
    return np.argmin(dd, axis=1), dd


@pytest.mark.parametrize("kind,n,seed,eye", [
    ("uniform", 400, 11, (0.05, -0.1, 0.2)),    # camera inside the foam
    ("uniform", 600, 12, (2.5, 1.5, -0.7)),     # camera outside the box
    ("mixture", 800, 13, (0.3, 0.2, -0.4)),     # strongly varying cell sizes
])
def test_walk_visits_the_voronoi_cells_in_order(kind, n, seed, eye):
    sc = random_scene(n, 0, seed, kind=kind)
    sc.density[:] = 1e-3  # no early stop: the whole ray is walked
    cam = camera_at(eye, (0.0, 0.0, 0.0), w=9, h=7, fov=70.0)
    out = oracle.render(sc, cam, trace=4096, eps=0.0)
    o, d = oracle.camera_rays(cam)
    pos = sc.pos.astype(np.float64)
    box = np.concatenate([sc.aabb_min, sc.aabb_max]).astype(np.float64)
    lo = (box[:3] - o) / d
    hi = (box[3:] - o) / d
    tmax_r = np.maximum(lo, hi).min(1)
    checked = 0
    for r in range(cam.n_rays):
        steps = out["steps"][r]
        if steps == 0:
            continue
        cells = out["trace_cells"][r, :steps]
        t1 = out["trace_t"][r, :steps]
        t0 = np.concatenate([[0.0], np.maximum.accumulate(t1[:-1])])
        # initial cell is nn(o)
        assert cells[0] == _nearest(pos, o[r][None])[0][0]
        # every finite exit point is on the bisector of the two cells and no
        # other site is closer (a point of the Voronoi face)
        for k in range(steps - 1):
            p = o[r] + t1[k] * d[r]
            dd = np.sum((pos - p) ** 2, axis=1)
            assert abs(dd[cells[k]] - dd[cells[k + 1]]) < 1e-9
            assert dd.min() > dd[cells[k]] - 1e-9
        # midpoints of segments lie in the visited cell
        tend = min(t1[-1], tmax_r[r])
        mids = []
        for k in range(steps):
            b = t1[k] if k < steps - 1 else tend
            if b - t0[k] > 1e-9:
                mids.append((k, 0.5 * (t0[k] + b)))
        P = o[r] + np.array([m for _, m in mids])[:, None] * d[r]
        nn = _nearest(pos, P)[0]
        assert np.array_equal(nn, cells[[k for k, _ in mids]])
        # dense sampling finds no cell the walk skipped
        ts = np.linspace(0.0, tend, 4000)
        seq = _nearest(pos, o[r] + ts[:, None] * d[r])[0]
        runs = seq[np.concatenate([[True], seq[1:] != seq[:-1]])]
        it = iter(cells.tolist())
        assert all(any(c == x for x in it) for c in runs.tolist())
        checked += 1
    assert checked >= 0.3 * cam.n_rays


def test_segment_widths_sum_to_the_clipped_ray_length():
    sc = random_scene(500, 0, 21)
    sig = float(np.float32(0.37))
    sc.density[:] = sig
    cam = camera_at((0.1, 0.0, 0.0), (1.0, 0.3, 0.2), w=8, h=8)
    out = oracle.render(sc, cam, eps=0.0)
    o, d = oracle.camera_rays(cam)
    # slab test by hand for the expected length
    lo = (sc.aabb_min.astype(np.float64) - o) / d
    hi = (sc.aabb_max.astype(np.float64) - o) / d
    tmax = np.minimum(lo, hi).max(1), np.maximum(lo, hi).min(1)
    L = tmax[1] - np.maximum(tmax[0], 0.0)
    np.testing.assert_allclose(-np.log(out["trans"]) / sig, L, rtol=1e-12)


# ---------------------------------------------------------------------------
# Closed forms of Eq. (3)-(4)
# ---------------------------------------------------------------------------
Y00 = 1 / (2 * math.sqrt(math.pi))


def test_homogeneous_medium():
    sc = random_scene(700, 0, 31)
    sig = float(np.float32(0.8))
    sc.density[:] = sig
    sc.sh[:, 0, :] = (np.array([0.2, 0.55, 0.9]) - 0.5) / Y00
    col = sc.sh[0, 0, :].astype(np.float64) * Y00 + 0.5   # the FP32-stored colour
    cam = camera_at((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), w=10, h=10)
    out = oracle.render(sc, cam, eps=0.0)
    o, d = oracle.camera_rays(cam)
    lo = (sc.aabb_min.astype(np.float64) - o) / d
    hi = (sc.aabb_max.astype(np.float64) - o) / d
    L = np.maximum(lo, hi).min(1)
    T = np.exp(-sig * L)
    np.testing.assert_allclose(out["trans"], T, rtol=1e-12)
    np.testing.assert_allclose(out["rgb"], (1 - T)[:, None] * col[None], rtol=1e-11, atol=1e-14)


def test_empty_medium():
    sc = random_scene(300, 3, 32)
    sc.density[:] = 0.0
    cam = camera_at((0.2, 0.1, 0.0), (0.0, 1.0, 0.0), w=6, h=6)
    out = oracle.render(sc, cam)
    assert np.all(out["rgb"] == 0) and np.all(out["trans"] == 1) and np.all(out["depth"] == 0)


def test_single_cell_depth_is_the_segment_midpoint():
    box = np.array([-1.0, -1.0, -1.0], np.float32), np.array([1.0, 1.0, 1.0], np.float32)
    sig = float(np.float32(0.6))
    sc = TinyScene(np.zeros((1, 3), np.float32), np.array([0, 0], np.int32),
                   np.zeros(0, np.int32), np.array([sig], np.float32),
                   np.array([[[0.0, 0.0, 0.0]]], np.float32), 0, box[0], box[1])
    cam = S.Camera(S.look_at((-3.0, 0.0, 0.0), (0.0, 0.0, 0.0)), 1.0, 1.0, 0.5, 0.5, 1, 1)
    out = oracle.render(sc, cam)
    # box entry at t=2, exit at t=4
    a = 1 - math.exp(-sig * 2.0)
    assert out["trans"][0] == pytest.approx(math.exp(-sig * 2.0), rel=1e-14)
    assert out["depth"][0] == pytest.approx(a * 3.0, rel=1e-14)
    np.testing.assert_allclose(out["rgb"][0], 0.5 * a, rtol=1e-14)


def test_two_cells_by_hand():
    # sites at x=-1 and x=+1: one bisector plane x=0; the ray starts at x=-2
    # (inside the box [-3,3]^3) and runs along +x: segments [0,2] and [2,5]
    pos = np.array([[-1, 0, 0], [1, 0, 0]], np.float32)
    off, idx = csr_from_lists([[1], [0]])
    sA, sB = 0.3, 0.7
    cA, cB = np.array([0.1, 0.4, 0.9]), np.array([0.8, 0.3, 0.2])
    sh = np.stack([(cA - 0.5) / Y00, (cB - 0.5) / Y00])[:, None, :].astype(np.float32)
    sc = TinyScene(pos, off, idx, np.array([sA, sB], np.float32), sh, 0,
                   np.full(3, -3, np.float32), np.full(3, 3, np.float32))
    cam = S.Camera(S.look_at((-2.0, 0.0, 0.0), (5.0, 0.0, 0.0)), 1.0, 1.0, 0.5, 0.5, 1, 1)
    out = oracle.render(sc, cam, trace=8)
    sA, sB = float(np.float32(sA)), float(np.float32(sB))
    cA = (sh[0, 0].astype(np.float64) * Y00 + 0.5)
    cB = (sh[1, 0].astype(np.float64) * Y00 + 0.5)
    eA, eB = math.exp(-2 * sA), math.exp(-3 * sB)
    np.testing.assert_allclose(out["rgb"][0], (1 - eA) * cA + eA * (1 - eB) * cB, rtol=1e-12)
    assert out["trans"][0] == pytest.approx(eA * eB, rel=1e-14)
    assert out["depth"][0] == pytest.approx((1 - eA) * 1.0 + eA * (1 - eB) * 3.5, rel=1e-13)
    assert out["steps"][0] == 2
    assert list(out["trace_cells"][0, :2]) == [0, 1]
    assert out["trace_t"][0, 0] == pytest.approx(2.0, rel=1e-15)


def test_early_stop_in_the_predicted_cell():
    # slab cells along x (sites at x = 0..9): the ray starts at x=-0.4 in cell 0;
    # segment widths 0.9, 1, 1, ...; with sigma=2.8, T before cell 4 is
    # exp(-2.8*2.9) = 3.0e-4 > 1e-4 and after it exp(-2.8*3.9) = 1.8e-5 <= 1e-4:
    # Alg. 1 composites exactly 4 cells.
    n = 10
    pos = np.stack([np.arange(n), np.zeros(n), np.zeros(n)], 1).astype(np.float32)
    off, idx = csr_from_lists([[j for j in (i - 1, i + 1) if 0 <= j < n] for i in range(n)])
    sc = TinyScene(pos, off, idx, np.full(n, 2.8, np.float32),
                   np.zeros((n, 1, 3), np.float32), 0,
                   np.array([-1, -1, -1], np.float32), np.array([n, 1, 1], np.float32))
    cam = S.Camera(S.look_at((-0.4, 0.0, 0.0), (5.0, 0.0, 0.0)), 1.0, 1.0, 0.5, 0.5, 1, 1)
    out = oracle.render(sc, cam, trace=16, eps=1e-4)
    assert out["steps"][0] == 4
    assert list(out["trace_cells"][0, :4]) == [0, 1, 2, 3]
    s = float(np.float32(2.8))
    assert out["trans"][0] == pytest.approx(math.exp(-s * 3.9), rel=1e-12)


def test_max_steps_sets_status():
    sc = random_scene(400, 0, 41)
    sc.density[:] = 1e-3
    cam = camera_at((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), w=4, h=4)
    out = oracle.render(sc, cam, max_steps=3)
    assert np.all(out["steps"] <= 3)
    assert np.any(out["status"] == oracle.RAY_MAX_STEPS)


def test_pixel_subset_equals_full_render():
    sc = random_scene(500, 2, 42)
    cam = camera_at((0.1, 0.2, 0.0), (0.0, 0.0, 1.0), w=11, h=7)
    full = oracle.render(sc, cam)
    px = np.array([0, 5, 76, 13, 40])
    sub = oracle.render(sc, cam, pixels=px)
    for k in ("rgb", "trans", "depth", "steps"):
        np.testing.assert_array_equal(sub[k], full[k][px])


# ---------------------------------------------------------------------------
# Backward against central finite differences of the forward
# ---------------------------------------------------------------------------
def _loss(sc, cam, g, eps):
    out = oracle.render(sc, cam, eps=eps, tau=0.0)
    return (np.sum(g[0] * out["rgb"]) + np.sum(g[1] * out["trans"])
            + np.sum(g[2] * out["depth"]))


@pytest.mark.parametrize("eye,fwd", [((0.05, 0.02, -0.03), (0.3, 0.1, 1.0)),
                                     ((2.2, -1.7, 0.4), (0.0, 0.0, 0.0))])
def test_backward_matches_finite_differences(eye, fwd):
    sc = random_scene(120, 3, 51)
    rng = np.random.default_rng(52)
    sc.sh[:, 1:, :] = rng.normal(0, 0.2, sc.sh[:, 1:, :].shape)
    sc.density[:] = rng.uniform(0.2, 1.5, sc.n_sites)
    # FD on FP64 copies (the oracle takes doubles)
    sc.pos = sc.pos.astype(np.float64)
    sc.sh = sc.sh.astype(np.float64)
    sc.density = sc.density.astype(np.float64)
    cam = camera_at(eye, fwd, w=5, h=4, fov=50.0)
    R = cam.n_rays
    g = (rng.normal(size=(R, 3)), rng.normal(size=R), rng.normal(size=R))
    ref = oracle.render(sc, cam, eps=0.0)
    assert not ref["degen"].any()
    G = oracle.render_bwd(sc, cam, g[0], g[1], g[2], eps=0.0)

    def fd(arr, idx, h):
        old = arr[idx]
        arr[idx] = old + h
        lp = _loss(sc, cam, g, 0.0)
        arr[idx] = old - h
        lm = _loss(sc, cam, g, 0.0)
        arr[idx] = old
        return (lp - lm) / (2 * h)

    # the cells the rays actually visit
    tr = oracle.render(sc, cam, eps=0.0, trace=512)
    visited = np.unique(tr["trace_cells"][tr["trace_cells"] >= 0])
    pick = visited[:: max(1, len(visited) // 12)]
    for i in pick:
        assert G["density"][i] == pytest.approx(fd(sc.density, i, 1e-6), rel=1e-5, abs=1e-8)
        for k in (0, 3, 8, 15):
            for ch in (0, 2):
                assert G["sh"][i, k, ch] == pytest.approx(fd(sc.sh, (i, k, ch), 1e-6),
                                                          rel=1e-5, abs=1e-8)
        for a in range(3):
            assert G["pos"][i, a] == pytest.approx(fd(sc.pos, (i, a), 1e-6),
                                                   rel=1e-4, abs=1e-7)
    # a bisector moves rigidly when both sites translate along their
    # difference: the total position gradient along the ray's cells is the
    # sum of the per-site terms (checked above); sites not visited get none
    untouched = np.setdiff1d(np.arange(sc.n_sites), visited)
    assert np.all(G["density"][untouched] == 0)
    assert np.all(G["sh"][untouched] == 0)


def test_prepared_scene_gives_the_same_results():
    # the FP64 copy and the start cell made once must not change any value
    sc = random_scene(700, 2, 77)
    cams = [camera_at((0.1, 0.2, -0.1), (1.0, 0.3, 0.2), w=11, h=9),
            camera_at((2.2, -1.5, 0.7), (0.0, 0.0, 0.0), w=7, h=5)]
    P = oracle.prepare(sc)
    assert oracle.prepare(P) is P
    for cam in cams:
        a = oracle.render(sc, cam, trace=64)
        b = oracle.render(P, cam, trace=64)
        for k in ("rgb", "trans", "depth", "steps", "flags", "trace_cells"):
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)
        g = np.random.default_rng(1).normal(size=(cam.n_rays, 3))
        ga = oracle.render_bwd(sc, cam, g)
        gb = oracle.render_bwd(P, cam, g)
        for k in ga:
            np.testing.assert_allclose(ga[k], gb[k], rtol=1e-12, atol=1e-15)
        assert P.start_info(cam)[0] == oracle.nearest_site(sc.pos, cam.c2w[:, 3])[0]
