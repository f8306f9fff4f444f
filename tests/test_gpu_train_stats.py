"""Densification / pruning statistics on the GPU against the plain CPU
reference (Sec. 3.3): scores to FP32 rounding, masks and draws bit-exact."""
import numpy as np
import pytest
import torch

from oracle import train_stats as TS
from paper_2502_01157_gb300 import rf
from tests.helpers import random_scene
from tests.parity import foam_of

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_scores_and_prune_mask(dt):
    sc = random_scene(3000, 1, 71)
    rng = np.random.default_rng(72)
    sc.density[:] = np.where(rng.uniform(size=sc.n_sites) < 0.7, 0.01, 2.0).astype(np.float32)
    foam = foam_of(sc, dt)
    g = rng.normal(size=(sc.n_sites, 3)).astype(np.float32)
    s = foam.densify_scores(torch.from_numpy(g).cuda()).cpu().numpy()
    ref = TS.densify_scores(sc.pos, sc.adj_off, sc.adj_idx, g)
    np.testing.assert_allclose(s, ref, rtol=2e-6, atol=1e-9)
    dens = torch.from_numpy(sc.density).to(torch.bfloat16 if dt == "bf16" else torch.float32).float().numpy()
    m = foam.prune_mask(0.1).cpu().numpy()
    np.testing.assert_array_equal(m, TS.prune_mask(dens, sc.adj_off, sc.adj_idx, 0.1))
    assert 0 < m.sum() < sc.n_sites


@pytest.mark.parametrize("n", [1, 7, 4096, 4097, 100_000, 3_000_000])
def test_multinomial_draws(n):
    rng = np.random.default_rng(n)
    w = rng.lognormal(size=n).astype(np.float32)
    w[rng.uniform(size=n) < 0.2] = 0.0
    if w.sum() == 0:
        w[0] = 1.0
    u = rng.uniform(size=5000).astype(np.float32)
    got = rf.sample_multinomial(torch.from_numpy(w).cuda(), torch.from_numpy(u).cuda()).cpu().numpy()
    ref = TS.sample_multinomial(w, u)
    # a draw may differ only where u * total falls within rounding of a boundary
    cdf = np.cumsum(w.astype(np.float64))
    bad = got != ref
    if bad.any():
        t = u[bad].astype(np.float64) * cdf[-1]
        gap = np.abs(cdf[np.minimum(ref[bad], n - 1)] - t)
        assert np.all(gap <= 1e-9 * cdf[-1]), (got[bad], ref[bad])
    assert np.all(w[got] > 0)
