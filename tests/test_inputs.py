"""The seeded input generators hold the workload recipes (sites, attributes,
cameras, request arrivals): they must produce what the recipes state."""
import math

import numpy as np
import pytest

from paper_2502_01157_gb300 import scenes as S


def test_uniform_sites_are_in_the_box_and_seeded():
    a = S.uniform_sites(5000, -1.0, 1.0, np.random.default_rng(3))
    b = S.uniform_sites(5000, -1.0, 1.0, np.random.default_rng(3))
    assert a.dtype == np.float32 and a.shape == (5000, 3)
    assert np.array_equal(a, b)
    assert a.min() >= -1.0 and a.max() <= 1.0
    # each coordinate ~ U[-1, 1]: mean 0, variance 1/3
    assert np.all(np.abs(a.mean(0)) < 0.05) and np.all(np.abs(a.var(0) - 1 / 3) < 0.02)


def test_mixture_components_have_the_stated_shape():
    rng = np.random.default_rng(11)
    # one Gaussian, no background: the sample covariance is R diag(s^2) R^T
    # with each axis scale s in [0.1, 1]
    g = S.mixture_sites(40000, rng, n_gauss=1, frac_gauss=1.0).astype(np.float64)
    ev = np.linalg.eigvalsh(np.cov(g.T))
    assert np.all(ev > 0.01 * 0.9) and np.all(ev < 1.0 * 1.1)
    assert np.all(np.abs(g.mean(0)) <= 8.0 + 0.05)   # centre ~ U[-8, 8]^3
    # background only: U[-10, 10]^3
    u = S.mixture_sites(20000, rng, frac_gauss=0.0)
    assert u.min() >= -10.0 and u.max() <= 10.0
    assert np.all(np.abs(u.var(0) - 100 / 3) < 2.0)
    # the split: 90% from the Gaussians, 10% background.  With one Gaussian
    # (axis scales <= 1) nearly no Gaussian site lies 6 from its centre, so the
    # sites that far are the background ones that far
    m = S.mixture_sites(100000, np.random.default_rng(12), n_gauss=1).astype(np.float64)
    c = np.median(m, axis=0)
    far = np.mean(np.linalg.norm(m - c, axis=1) > 6.0)
    bg = np.random.default_rng(13).uniform(-10, 10, size=(200000, 3))
    expect = 0.1 * np.mean(np.linalg.norm(bg - c, axis=1) > 6.0)
    assert abs(far - expect) < 0.005


def test_dedupe_moves_only_duplicates():
    rng = np.random.default_rng(5)
    p = S.uniform_sites(1000, -1, 1, rng)
    p[10] = p[20]
    p[30] = p[20]
    before = p.copy()
    q = S.dedupe_sites(p, rng)
    assert len(np.unique(q, axis=0)) == 1000
    moved = np.any(q != before, axis=1)
    assert moved.sum() == 2 and not moved[[i for i in range(1000) if i not in (10, 20, 30)]].any()
    assert np.abs(q - before).max() < 1e-2


def test_lognormal_density():
    d = S.lognormal_density(200000, np.random.default_rng(8)).astype(np.float64)
    assert np.all(d > 0)
    ld = np.log(d)
    assert abs(ld.mean()) < 0.01 and abs(ld.std() - 1.0) < 0.01
    assert abs(np.median(d) - 1.0) < 0.01


def test_sh_coefficients():
    rng = np.random.default_rng(9)
    k = S.sh_coeffs(20000, 3, rng)
    assert k.shape == (20000, 16, 3) and k.dtype == np.float32
    assert abs(k.std() - 0.3) < 0.005
    c = S.sh_coeffs(20000, 3, rng, dc="uniform_colour")
    # base colour = k00 * Y00 + 0.5 with Y00 = 1 / (2 sqrt(pi)) is uniform on [0, 1]
    base = c[:, 0, :].astype(np.float64) / (2 * math.sqrt(math.pi)) + 0.5
    assert base.min() >= 0.0 and base.max() <= 1.0
    assert abs(base.mean() - 0.5) < 0.01 and abs(base.var() - 1 / 12) < 0.003
    assert abs(c[:, 1:, :].std() - 0.3) < 0.005


def test_pinhole_intrinsics():
    cam = S.pinhole(1920, 1080, 60.0)
    # the top edge of the image is 30 degrees above the axis
    assert math.isclose(math.degrees(math.atan((cam.height / 2) / cam.fy)), 30.0, rel_tol=1e-6)
    assert cam.fx == cam.fy and cam.cx == 960.0 and cam.cy == 540.0 and cam.n_rays == 2073600


def test_fisheye_image_circle_spans_the_field_of_view():
    cam = S.fisheye(400, 300, 200.0)
    # equidistant: angle = radius / f, so the inscribed circle (radius 150) is 100 degrees
    assert math.isclose(math.degrees(150.0 / cam.fx), 100.0, rel_tol=1e-6)
    assert cam.model == S.Camera.FISHEYE


@pytest.mark.parametrize("eye,target", [((3.0, -2.0, 1.0), (0.0, 0.0, 0.0)),
                                        ((0.0, 0.0, 5.0), (0.0, 0.0, 0.0)),   # along the up axis
                                        ((0.1, 0.2, -0.3), (1.0, 0.5, 0.2))])
def test_look_at_is_a_proper_rotation_towards_the_target(eye, target):
    c2w = S.look_at(eye, target)
    R, t = c2w[:, :3], c2w[:, 3]
    assert np.allclose(R.T @ R, np.eye(3), atol=1e-12) and math.isclose(np.linalg.det(R), 1.0, rel_tol=1e-12)
    fwd = np.asarray(target, float) - np.asarray(eye, float)
    assert np.allclose(R[:, 2], fwd / np.linalg.norm(fwd), atol=1e-12)
    assert np.allclose(t, eye)


def test_c4_cameras_and_poses():
    cams = S.config_cameras("c4")
    assert [(c.width, c.height) for c in cams] == S.C4_RESOLUTIONS
    assert sum(c.n_rays for c in cams) == 9484800
    for c in cams:
        eye = c.c2w[:, 3].astype(np.float64)
        assert math.isclose(np.linalg.norm(eye), 12.0, rel_tol=1e-6)
        # the optical axis passes through the origin
        axis = c.c2w[:, 2].astype(np.float64)
        assert np.allclose(axis, -eye / np.linalg.norm(eye), atol=1e-6)
    assert S.config_cameras("c3")[0].n_rays == 2073600 and S.config_cameras("c2")[0].n_rays == 921600


def test_sphere_poses_are_uniform_on_the_sphere():
    poses = S.sphere_poses(4000, 12.0, 77)
    eyes = np.array([p[:, 3] for p in poses])
    assert np.allclose(np.linalg.norm(eyes, axis=1), 12.0)
    # uniform directions: each coordinate of the unit vector has mean 0, variance 1/3
    u = eyes / 12.0
    assert np.all(np.abs(u.mean(0)) < 0.05) and np.all(np.abs(u.var(0) - 1 / 3) < 0.03)


def test_poisson_arrivals():
    t = S.poisson_arrivals(500.0, 40000, 3)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() * 500.0 - 1.0) < 0.02
    # exponential gaps: standard deviation equals the mean
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03


def test_random_target_is_uniform():
    y = S.random_target(50000, 2024)
    assert y.shape == (50000, 3) and y.min() >= 0 and y.max() <= 1
    assert abs(y.mean() - 0.5) < 0.01
