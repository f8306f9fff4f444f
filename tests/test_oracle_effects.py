"""Pins of the oracle's ray-generation variants and sphere bounces (Fig. 2):
an equidistant fisheye, a rolling shutter and an analytic sphere -- a mirror,
or clear glass with Snell refraction and total internal reflection -- met in
the same walk through the foam.

* fisheye: every ray's angle to the optical axis equals the normalised image
  radius, its azimuth the pixel's;
* rolling shutter: each image row equals the same row of a global-shutter
  camera moved to that row's origin;
* single homogeneous cell: transmittance exp(-sigma L) with the bent path
  length L worked out from angles (Snell's law, the deviation through a sphere,
  the chords of total internal reflection), depth from the path segments;
* many cells: a bounced ray equals the composition of straight renders of its
  legs (each leg a straight walk of Alg. 1, pinned elsewhere);
* the backward pass against central finite differences with bounces.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2502_01157_gb300 import scenes as S
from tests.helpers import TinyScene, camera_at, random_scene

Y00 = 0.5 / math.sqrt(math.pi)


def _one_cell(sigma, colour, half=1.0):
    sh = np.zeros((1, 1, 3), np.float32)
    sh[0, 0, :] = (np.asarray(colour, np.float64) - 0.5) / Y00
    return TinyScene(np.zeros((1, 3), np.float32), np.array([0, 0], np.int32), np.zeros(0, np.int32),
                     np.array([sigma], np.float32), sh, 0, np.full(3, -half, np.float32),
                     np.full(3, half, np.float32))


def _ray_cam(eye, direction, t_far=0.0):
    """1x1 pinhole camera whose single ray leaves ``eye`` along ``direction``."""
    eye = np.asarray(eye, np.float64)
    return S.Camera(S.look_at(eye, eye + np.asarray(direction, np.float64)), 1.0, 1.0, 0.5, 0.5, 1, 1,
                    t_far=t_far)


def _slab_exit(p, d, half):
    """Distance from p (inside the box [-half, half]^3) along d to the box."""
    t = np.inf
    for a in range(3):
        if d[a] > 0:
            t = min(t, (half - p[a]) / d[a])
        elif d[a] < 0:
            t = min(t, (-half - p[a]) / d[a])
    return t


# ---------------------------------------------------------------------------
# camera models
# ---------------------------------------------------------------------------
def test_fisheye_rays_follow_the_equidistant_model():
    c2w = S.look_at((0.3, -0.2, 0.1), (1.0, 0.5, -0.4))
    cam = S.fisheye(40, 30, 220.0, c2w=c2w)
    o, d = oracle.camera_rays(cam)
    R = cam.c2w[:, :3].astype(np.float64)
    dc = np.linalg.solve(R, d.T).T
    dc /= np.linalg.norm(dc, axis=1, keepdims=True)
    v, u = np.divmod(np.arange(cam.n_rays), cam.width)
    x = (u + 0.5 - cam.cx) / cam.fx
    y = (v + 0.5 - cam.cy) / cam.fy
    r = np.hypot(x, y)
    theta = np.arccos(np.clip(dc[:, 2], -1, 1))
    np.testing.assert_allclose(theta, r, atol=2e-6)
    assert r.max() > math.pi / 2           # the corners look behind the camera
    az_ok = r > 1e-3
    dphi = np.angle(np.exp(1j * (np.arctan2(dc[az_ok, 1], dc[az_ok, 0]) - np.arctan2(y, x)[az_ok])))
    assert np.max(np.abs(dphi)) < 2e-5
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    np.testing.assert_array_equal(o, np.tile(cam.c2w[:, 3].astype(np.float64), (cam.n_rays, 1)))


def test_fisheye_renders_behind_the_camera():
    sc = random_scene(300, 1, 70)
    cam = S.fisheye(12, 10, 300.0, c2w=S.look_at((0.05, 0.02, -0.03), (1.0, 0.0, 0.0)))
    out = oracle.render(sc, cam)
    assert np.all(out["trans"] < 1.0) and np.all(out["steps"] > 0)


@pytest.mark.parametrize("model", [S.Camera.PINHOLE, S.Camera.FISHEYE])
def test_rolling_shutter_row_equals_a_global_camera_at_the_row_origin(model):
    sc = random_scene(400, 1, 7)
    vel = np.array([0.45, -0.3, 0.2])
    base = camera_at((0.05, -0.1, 0.02), (0.8, 0.5, 0.3), w=9, h=7, fov=70.0)
    cam = S.Camera(base.c2w, base.fx, base.fy, base.cx, base.cy, base.width, base.height,
                   model=model, shutter=vel)
    vel = np.asarray(cam.shutter)
    out = oracle.render(sc, cam)
    o, d = oracle.camera_rays(cam)
    t = cam.c2w[:, 3].astype(np.float64)
    starts = set()
    for v in range(cam.height):
        ov = t + ((v + 0.5) / cam.height - 0.5) * vel
        px = np.arange(v * cam.width, (v + 1) * cam.width)
        np.testing.assert_allclose(o[px], np.tile(ov, (cam.width, 1)), atol=1e-15)
        c2w = cam.c2w.astype(np.float64).copy()
        c2w[:, 3] = ov
        g = S.Camera(c2w, cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, model=model)
        ref = oracle.render(sc, g, pixels=px)
        starts.add(oracle.nearest_site(sc.pos, np.asarray(g.c2w[:, 3], np.float64))[0])
        ok = ~(ref["degen"] | out["degen"][px])
        for k in ("rgb", "trans", "depth"):
            np.testing.assert_allclose(out[k][px][ok], ref[k][ok], atol=2e-5)
    assert len(starts) > 1          # the rows really start in different cells


# ---------------------------------------------------------------------------
# sphere: one homogeneous cell, paths from angles
# ---------------------------------------------------------------------------
def test_mirror_on_axis_closed_form():
    sig, col = 0.7, (0.2, 0.6, 0.9)
    sc = _one_cell(sig, col)
    s = float(np.float32(sig))
    cam = _ray_cam((-3.0, 0.0, 0.0), (1.0, 0.0, 0.0))
    out = oracle.render(sc, cam, eps=0.0, effects=S.Sphere((0, 0, 0), 0.5))
    # in the box: [2, 2.5] towards the mirror, then 0.5 back to x = -1
    e = math.exp(-0.5 * s)
    T = e * e
    assert out["trans"][0] == pytest.approx(T, rel=1e-13)
    c = ((np.asarray(col) - 0.5) / Y00).astype(np.float32).astype(np.float64) * Y00 + 0.5
    np.testing.assert_allclose(out["rgb"][0], (1 - T) * c, rtol=1e-12)
    depth = (1 - e) * 2.25 + e * (1 - e) * (2.5 + 0.25)
    assert out["depth"][0] == pytest.approx(depth, rel=1e-13)
    assert out["steps"][0] == 2
    # no bounces allowed: the sphere is ignored
    straight = oracle.render(sc, cam, eps=0.0, effects=S.Sphere((0, 0, 0), 0.5, max_bounces=0))
    assert straight["trans"][0] == pytest.approx(math.exp(-2 * s), rel=1e-13)


def test_glass_through_the_centre_equals_no_sphere():
    sc = _one_cell(0.4, (0.3, 0.3, 0.7))
    glass = S.Sphere((0.0, 0.0, 0.0), 0.5, ior=1.5)
    cam = _ray_cam((-3.0, 0.0, 0.0), (1.0, 0.0, 0.0))
    a = oracle.render(sc, cam, eps=0.0, effects=glass)
    b = oracle.render(sc, cam, eps=0.0)
    for k in ("rgb", "trans"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-13)
    assert a["steps"][0] == 3
    # depth is composited per segment (midpoints of [2, 2.5], [2.5, 3.5], [3.5, 4])
    s = float(np.float32(0.4))
    T = [1.0, math.exp(-0.5 * s), math.exp(-1.5 * s), math.exp(-2.0 * s)]
    mids = [2.25, 3.0, 3.75]
    assert a["depth"][0] == pytest.approx(sum((T[k] - T[k + 1]) * mids[k] for k in range(3)),
                                          rel=1e-13)
    # from the centre every ray meets the surface head on
    inner = camera_at((0.0, 0.0, 0.0), (0.3, 1.0, -0.2), w=5, h=4, fov=90.0)
    a = oracle.render(sc, inner, eps=0.0, effects=glass)
    b = oracle.render(sc, inner, eps=0.0)
    for k in ("rgb", "trans"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-15)
    assert np.all(a["steps"] == 2)


@pytest.mark.parametrize("h,n", [(0.3, 1.5), (0.7, 1.5), (0.95, 1.33), (-0.6, 2.4)])
def test_glass_off_axis_path_from_snell_angles(h, n):
    sig, half, r = 0.05, 10.0, 1.0
    sc = _one_cell(sig, (0.5, 0.5, 0.5), half)
    s = float(np.float32(sig))
    n = float(np.float32(n))
    h = float(np.float32(h))
    cam = _ray_cam((-3.0, h, 0.0), (1.0, 0.0, 0.0))
    out = oracle.render(sc, cam, eps=0.0, effects=S.Sphere((0, 0, 0), r, ior=n))
    # 2-D geometry in the z = 0 plane, by angles
    sgn = math.copysign(1.0, h)
    ti = math.asin(abs(h) / r)
    tt = math.asin(math.sin(ti) / n)
    l1 = 3.0 - r * math.cos(ti)                  # to the entry point
    chord = 2.0 * r * math.cos(tt)
    phi_x = sgn * (2.0 * tt - ti)                # polar angle of the exit point
    px = np.array([r * math.cos(phi_x), r * math.sin(phi_x), 0.0])
    dev = 2.0 * (ti - tt)                        # total deviation, towards the axis
    dx = np.array([math.cos(dev), -sgn * math.sin(dev), 0.0])
    l3 = _slab_exit(px, dx, half)
    L = l1 + chord + l3
    assert -math.log(out["trans"][0]) / s == pytest.approx(L, rel=1e-10)
    T1, T2 = math.exp(-s * l1), math.exp(-s * (l1 + chord))
    depth = ((1 - T1) * l1 / 2 + (T1 - T2) * (l1 + chord / 2)
             + T2 * (1 - math.exp(-s * l3)) * (l1 + chord + l3 / 2))
    assert out["depth"][0] == pytest.approx(depth, rel=1e-10)


@pytest.mark.parametrize("m", [1, 2, 5])
def test_total_internal_reflection_chords(m):
    sig, half, r, n, b = 0.05, 10.0, 1.0, 1.5, 0.8
    sc = _one_cell(sig, (0.5, 0.5, 0.5), half)
    s = float(np.float32(sig))
    cam = _ray_cam((0.0, b, 0.0), (1.0, 0.0, 0.0))
    out = oracle.render(sc, cam, eps=0.0, effects=S.Sphere((0, 0, 0), r, ior=n, max_bounces=m))
    b = float(np.float32(b))
    th = math.asin(b / r)                       # beyond the critical angle asin(1/n)
    assert th > math.asin(1 / float(np.float32(n)))
    c = math.sqrt(r * r - b * b)
    phi = [math.atan2(b, c) - k * (math.pi - 2 * th) for k in range(m + 1)]
    p = [np.array([r * math.cos(f), r * math.sin(f), 0.0]) for f in phi]
    # p[k]: the (k+1)-th point on the surface; after the m-th (last allowed)
    # reflection at p[m-1] the ray runs along the next chord and out of the glass
    d_out = (p[m] - p[m - 1]) / np.linalg.norm(p[m] - p[m - 1])
    L = c + 2 * c * (m - 1) + _slab_exit(p[m - 1], d_out, half)
    assert -math.log(out["trans"][0]) / s == pytest.approx(L, rel=1e-10)
    assert out["steps"][0] == m + 1


# ---------------------------------------------------------------------------
# sphere in a foam: a bounced ray is the composition of its straight legs
# ---------------------------------------------------------------------------
def _sphere_entry(o, d, c, r, inside):
    """Next crossing by the closest-approach construction."""
    tc = np.dot(c - o, d)
    h2 = np.dot(c - o, c - o) - tc * tc
    if h2 > r * r:
        return None
    w = math.sqrt(r * r - h2)
    t = tc + w if inside else tc - w
    return t if t > 0 else None


def _legs(o, d, sph):
    """Straight legs (origin, direction, length or None) of a ray meeting
    ``sph``, with the textbook reflection (Householder) and Snell refraction."""
    c = np.asarray(sph.centre, np.float64)
    r, n = sph.radius, sph.ior
    inside = np.linalg.norm(o - c) < r
    legs = []
    for _ in range(sph.max_bounces):
        t = _sphere_entry(o, d, c, r, inside)
        if t is None:
            break
        legs.append((o, d, t))
        p = o + t * d
        nrm = (p - c) / r
        if n > 0:
            nn = -nrm if inside else nrm
            eta = n if inside else 1.0 / n
            ci = -np.dot(d, nn)
            k = 1 - eta * eta * (1 - ci * ci)
            if k >= 0:
                d = eta * d + (eta * ci - math.sqrt(k)) * nn
                inside = not inside
            else:
                d = (np.eye(3) - 2 * np.outer(nrm, nrm)) @ d
        else:
            d = (np.eye(3) - 2 * np.outer(nrm, nrm)) @ d
        d = d / np.linalg.norm(d)
        o = p
    legs.append((o, d, None))
    return legs


@pytest.mark.parametrize("ior,deg", [(0.0, 2), (1.5, 1), (1.9, 0)])
def test_bounced_ray_is_the_composition_of_straight_legs(ior, deg):
    sc = random_scene(500, deg, 31)
    sph = S.Sphere((0.1, 0.0, 0.05), 0.35, ior=ior, max_bounces=4)
    cam = camera_at((-0.85, 0.3, 0.2), (0.1, 0.0, 0.05), w=6, h=5, fov=40.0)
    out = oracle.render(sc, cam, eps=0.0, effects=sph)
    o_all, d_all = oracle.camera_rays(cam)
    n_checked = n_bounced = 0
    for px in range(cam.n_rays):
        if out["degen"][px]:
            continue
        legs = _legs(o_all[px], d_all[px], sph)
        C, T, D, s_off, bad = np.zeros(3), 1.0, 0.0, 0.0, False
        for k, (o, d, L) in enumerate(legs):
            if k == 0:
                g = S.Camera(cam.c2w, cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height,
                             t_far=L if L is not None else 0.0)
                part = oracle.render(sc, g, pixels=[px], eps=0.0)
            else:
                part = oracle.render(sc, _ray_cam(o, d, t_far=L if L is not None else 0.0),
                                     eps=0.0)
            bad |= bool(part["degen"][0])
            C += T * part["rgb"][0]
            D += T * (part["depth"][0] + s_off * (1 - part["trans"][0]))
            T *= part["trans"][0]
            s_off += L if L is not None else 0.0
        if bad:
            continue
        n_checked += 1
        n_bounced += len(legs) > 1
        np.testing.assert_allclose(out["rgb"][px], C, atol=2e-5)
        assert out["trans"][px] == pytest.approx(T, abs=2e-5)
        assert out["depth"][px] == pytest.approx(D, abs=1e-4)
    assert n_checked >= 20 and n_bounced >= 10


# ---------------------------------------------------------------------------
# backward with bounces
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ior", [0.0, 1.5])
def test_backward_with_bounces_matches_finite_differences(ior):
    sc = random_scene(150, 1, 81)
    rng = np.random.default_rng(82)
    sc.density[:] = rng.uniform(0.2, 1.5, sc.n_sites)
    sc.pos = sc.pos.astype(np.float64)
    sc.sh = sc.sh.astype(np.float64)
    sc.density = sc.density.astype(np.float64)
    sph = S.Sphere((0.05, 0.0, 0.0), 0.3, ior=ior, max_bounces=3)
    cam = camera_at((-0.8, 0.1, 0.05), (0.05, 0.0, 0.0), w=4, h=4, fov=35.0)
    R = cam.n_rays
    g = (rng.normal(size=(R, 3)), rng.normal(size=R), rng.normal(size=R), rng.normal(size=R))
    assert not oracle.render(sc, cam, eps=0.0, effects=sph)["degen"].any()
    G = oracle.render_bwd(sc, cam, g[0], g[1], g[2], eps=0.0, g_quantile=g[3], effects=sph)

    def loss():
        o = oracle.render(sc, cam, eps=0.0, tau=0.0, effects=sph)
        q = oracle.render_quantile(sc, cam, eps=0.0, effects=sph)
        return (np.sum(g[0] * o["rgb"]) + np.sum(g[1] * o["trans"]) + np.sum(g[2] * o["depth"])
                + np.sum(g[3] * q))

    def fd(arr, idx, h):
        old = arr[idx]
        arr[idx] = old + h
        lp = loss()
        arr[idx] = old - h
        lm = loss()
        arr[idx] = old
        return (lp - lm) / (2 * h)

    tr = oracle.render(sc, cam, eps=0.0, trace=512, effects=sph)
    visited = np.unique(tr["trace_cells"][tr["trace_cells"] >= 0])
    assert np.sum(tr["steps"]) > np.sum(oracle.render(sc, cam, eps=0.0)["steps"]) // 2
    for i in visited[:: max(1, len(visited) // 12)]:
        assert G["density"][i] == pytest.approx(fd(sc.density, i, 1e-6), rel=1e-5, abs=1e-8)
        for k in (0, 2):
            assert G["sh"][i, k, 1] == pytest.approx(fd(sc.sh, (i, k, 1), 1e-6), rel=1e-5, abs=1e-8)
        for a in range(3):
            assert G["pos"][i, a] == pytest.approx(fd(sc.pos, (i, a), 1e-6), rel=1e-4, abs=1e-7)


# ---------------------------------------------------------------------------
# near-degenerate flags (conditioning of the FP32 comparison)
# ---------------------------------------------------------------------------
def _two_cells():
    pos = np.array([[-1.0, 0, 0], [1.0, 0, 0]], np.float32)
    return TinyScene(pos, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32),
                     np.array([0.5, 0.5], np.float32), np.zeros((2, 1, 3), np.float32), 0,
                     np.full(3, -1.0, np.float32), np.full(3, 1.0, np.float32))


@pytest.mark.parametrize("theta,delta,flagged", [(1e-5, 1e-6, True), (1e-3, 1e-4, False), (0.5, 0.05, False)])
def test_grazing_face_crossing_is_flagged(theta, delta, flagged):
    # the ray crosses the face x = 0 at t = delta / sin(theta), at an angle
    # whose cosine to the face normal is sin(theta)
    sc = _two_cells()
    cam = _ray_cam((-delta, -0.9, 0.0), (math.sin(theta), math.cos(theta), 0.0))
    out = oracle.render(sc, cam, trace=8)
    assert list(out["trace_cells"][0][:2]) == [0, 1]      # it does cross
    assert bool(out["degen"][0]) == flagged


@pytest.mark.parametrize("h,flagged", [(0.5 * math.sqrt(1 - 1e-3), True), (0.3, False)])
def test_near_grazing_sphere_hit_is_flagged(h, flagged):
    sc = _one_cell(0.3, (0.5, 0.5, 0.5), 3.0)
    cam = _ray_cam((-2.0, h, 0.0), (1.0, 0.0, 0.0))
    out = oracle.render(sc, cam, effects=S.Sphere((0, 0, 0), 0.5, ior=0.0))
    assert bool(out["degen"][0]) == flagged


@pytest.mark.parametrize("b,flagged", [(1 / 1.5 * 1.0001, True), (0.3, False)])
def test_critical_angle_is_flagged(b, flagged):
    # from inside a glass sphere (n = 1.5) the ray meets the surface at
    # sin(theta_i) = b / r: total internal reflection starts at b = r / n
    sc = _one_cell(0.3, (0.5, 0.5, 0.5), 3.0)
    cam = _ray_cam((0.0, b, 0.0), (1.0, 0.0, 0.0))
    out = oracle.render(sc, cam, effects=S.Sphere((0, 0, 0), 1.0, ior=1.5, max_bounces=1))
    assert bool(out["degen"][0]) == flagged
