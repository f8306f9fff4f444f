"""Pins of the densification / pruning statistics oracle (Sec. 3.3)."""
import math

import numpy as np
import pytest

from oracle import train_stats as TS
from tests.helpers import csr_from_lists


def test_radius_and_score_on_a_hand_built_chain():
    # sites on a line at x = 0, 1, 3: neighbours 0-1, 1-2
    pos = np.array([[0, 0, 0], [1, 0, 0], [3, 0, 0]], np.float32)
    off, idx = csr_from_lists([[1], [0, 2], [1]])
    r = TS.cell_radius(pos, off, idx)
    np.testing.assert_allclose(r, [0.5, 0.5 * (1 + 2) / 2, 1.0])
    g = np.array([[3, 4, 0], [0, 0, 0], [1, 0, 0]], np.float32)
    np.testing.assert_allclose(TS.densify_scores(pos, off, idx, g), [2.5, 0.0, 1.0])


def test_prune_needs_low_density_around():
    #  0 - 1 - 2 - 3, densities 0, 0, 5, 0
    off, idx = csr_from_lists([[1], [0, 2], [1, 3], [2]])
    dens = np.array([0.0, 0.0, 5.0, 0.0])
    m = TS.prune_mask(dens, off, idx, 0.1)
    assert list(m) == [True, False, False, False]   # 1 and 3 border the dense cell 2
    iso_off, iso_idx = csr_from_lists([[]])
    assert TS.prune_mask(np.array([0.0]), iso_off, iso_idx, 0.1)[0]


def test_multinomial_frequencies_follow_the_weights():
    rng = np.random.default_rng(0)
    w = np.array([0.0, 1.0, 3.0, 0.0, 6.0])
    u = rng.uniform(size=200_000)
    idx = TS.sample_multinomial(w, u)
    assert not np.isin(idx, [0, 3]).any()           # zero weight is never drawn
    freq = np.bincount(idx, minlength=5) / len(u)
    p = w / w.sum()
    # chi-square with 2 dof, far below the 1e-6 tail
    chi2 = np.sum((freq[p > 0] - p[p > 0]) ** 2 / p[p > 0]) * len(u)
    assert chi2 < 27.6
    # boundaries: u exactly at a cumulative fraction selects the next site
    assert list(TS.sample_multinomial(w, [0.0, 0.1, 0.4, 0.9999])) == [1, 2, 4, 4]
