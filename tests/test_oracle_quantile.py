"""Pins of the oracle's quantile loss (Eq. 6): L = E|W^-1(u1) - W^-1(u2)| with
u1, u2 ~ U[0,1] and W^-1 the quantile function of a ray's (normalised)
volume-rendering weight distribution.

* against the paper's definition itself: the CDF of a hand-known slab chain,
  inverted on a fine grid, and the expectation over a uniform grid of quantile
  pairs (independent of the oracle's per-segment closed form);
* against the exponential distribution (E|X - X'| = 1/sigma) and a quadrature
  of 2 int F (1 - F) for a single homogeneous cell;
* its backward against central finite differences.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2502_01157_gb300 import scenes as S
from tests.helpers import TinyScene, camera_at, csr_from_lists, random_scene


def _slab_chain(sig):
    n = len(sig)
    pos = np.stack([np.arange(n), np.zeros(n), np.zeros(n)], 1).astype(np.float32)
    off, idx = csr_from_lists([[j for j in (i - 1, i + 1) if 0 <= j < n] for i in range(n)])
    return TinyScene(pos, off, idx, np.asarray(sig, np.float32), np.zeros((n, 1, 3), np.float32), 0,
                     np.array([-1, -1, -1], np.float32), np.array([n, 1, 1], np.float32))


def _ray_along_x(x0):
    return S.Camera(S.look_at((x0, 0.0, 0.0), (x0 + 5.0, 0.0, 0.0)), 1.0, 1.0, 0.5, 0.5, 1, 1)


def _mean_abs_diff_of_quantiles(t, F, n=4000):
    """E|F^-1(u1) - F^-1(u2)| on the midpoint grid u_k = (k + 1/2)/n."""
    u = (np.arange(n) + 0.5) / n
    q = np.interp(u, F, t)          # F increasing: quantile function by inversion
    q.sort()
    k = np.arange(n)
    return 2.0 * np.sum(q * (2 * k - (n - 1))) / n ** 2


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_quantile_loss_is_the_expected_quantile_distance(seed):
    rng = np.random.default_rng(seed)
    sig = rng.uniform(0.05, 2.0, 10).astype(np.float32)
    sc = _slab_chain(sig)
    x0 = -0.4
    cam = _ray_along_x(x0)
    Lq = oracle.render_quantile(sc, cam, eps=0.0)[0]
    # weight CDF from the slab geometry (boundaries at x = k + 1/2) and the
    # exponential transmittance, composited on [box entry, box exit] = [0, 10.4]
    t = np.linspace(0.0, 10.4, 400001)
    x = x0 + t
    cell = np.clip(np.floor(x + 0.5).astype(int), 0, len(sig) - 1)
    s = sig.astype(np.float64)[cell]
    tau = np.concatenate([[0.0], np.cumsum(0.5 * (s[1:] + s[:-1]) * np.diff(t))])
    W = 1.0 - np.exp(-tau)
    F = W / W[-1]
    ref = _mean_abs_diff_of_quantiles(t, F)
    assert Lq == pytest.approx(ref, rel=2e-4)


def test_quantile_loss_with_early_stop_uses_the_composited_segments():
    sig = np.full(10, 2.8, np.float32)
    sc = _slab_chain(sig)
    cam = _ray_along_x(-0.4)
    out = oracle.render(sc, cam, eps=1e-4)
    assert out["steps"][0] == 4          # stops after 4 cells (see the early-stop pin)
    Lq = oracle.render_quantile(sc, cam, eps=1e-4)[0]
    t = np.linspace(0.0, 3.9, 200001)     # the four composited segments end at t = 3.9
    W = 1.0 - np.exp(-float(np.float32(2.8)) * t)
    ref = _mean_abs_diff_of_quantiles(t, W / W[-1])
    assert Lq == pytest.approx(ref, rel=2e-4)


def test_single_cell_exponential_and_quadrature():
    quad = pytest.importorskip("scipy.integrate").quad
    box = (np.full(3, -1, np.float32), np.full(3, 1, np.float32))
    for sig in (0.3, 2.0, 50.0):
        sc = TinyScene(np.zeros((1, 3), np.float32), np.array([0, 0], np.int32), np.zeros(0, np.int32),
                       np.array([sig], np.float32), np.zeros((1, 1, 3), np.float32), 0, box[0], box[1])
        cam = S.Camera(S.look_at((-3.0, 0.0, 0.0), (0.0, 0.0, 0.0)), 1.0, 1.0, 0.5, 0.5, 1, 1)
        Lq = oracle.render_quantile(sc, cam, eps=0.0)[0]
        s = float(np.float32(sig))
        L = 2.0
        F = lambda t: (1 - math.exp(-s * t)) / (1 - math.exp(-s * L))
        ref = quad(lambda t: 2 * F(t) * (1 - F(t)), 0.0, L, epsabs=1e-13, epsrel=1e-12, limit=200)[0]
        assert Lq == pytest.approx(ref, rel=1e-9)
        if s * L > 50:
            assert Lq == pytest.approx(1.0 / s, rel=1e-9)   # exponential: E|X - X'| = 1/sigma


def test_no_density_gives_zero():
    sc = random_scene(300, 0, 4)
    sc.density[:] = 0
    cam = camera_at((0.1, 0.0, 0.0), (1.0, 0.0, 0.0), w=4, h=4)
    assert np.all(oracle.render_quantile(sc, cam) == 0)


@pytest.mark.parametrize("eye,fwd", [((0.05, 0.02, -0.03), (0.3, 0.1, 1.0)),
                                     ((2.2, -1.7, 0.4), (0.0, 0.0, 0.0))])
def test_quantile_backward_matches_finite_differences(eye, fwd):
    sc = random_scene(120, 1, 61)
    rng = np.random.default_rng(62)
    sc.density[:] = rng.uniform(0.2, 1.5, sc.n_sites)
    sc.pos = sc.pos.astype(np.float64)
    sc.sh = sc.sh.astype(np.float64)
    sc.density = sc.density.astype(np.float64)
    cam = camera_at(eye, fwd, w=5, h=4, fov=50.0)
    R = cam.n_rays
    gq = rng.normal(size=R)
    assert not oracle.render(sc, cam, eps=0.0)["degen"].any()
    G = oracle.render_bwd(sc, cam, np.zeros((R, 3)), eps=0.0, g_quantile=gq)
    loss = lambda: float(np.sum(gq * oracle.render_quantile(sc, cam, eps=0.0)))

    def fd(arr, idx, h):
        old = arr[idx]
        arr[idx] = old + h
        lp = loss()
        arr[idx] = old - h
        lm = loss()
        arr[idx] = old
        return (lp - lm) / (2 * h)

    tr = oracle.render(sc, cam, eps=0.0, trace=512)
    visited = np.unique(tr["trace_cells"][tr["trace_cells"] >= 0])
    for i in visited[:: max(1, len(visited) // 10)]:
        assert G["density"][i] == pytest.approx(fd(sc.density, i, 1e-6), rel=1e-5, abs=1e-9)
        for a in range(3):
            assert G["pos"][i, a] == pytest.approx(fd(sc.pos, (i, a), 1e-6), rel=1e-4, abs=1e-8)
    assert np.all(G["sh"] == 0)   # the weights do not depend on colour
