"""Host-side helpers of the binding (no GPU): g(r) normalisation and the
free-energy profile of a well-tempered bias."""
import math

import numpy as np

from paper_2503_23728_gb300 import pimd as P


def test_rdf_normalize_ideal_counts_give_one():
    """Counts equal to the ideal-gas expectation give g = 1 for every pair."""
    n_per, V, r_max, n_bins, n_conf = [10, 6], 1000.0, 5.0, 20, 3
    edges = np.linspace(0, r_max, n_bins + 1)
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    pairs = [10 * 9 / 2, 10 * 6, 6 * 5 / 2]
    counts = np.stack([n_conf * p * shell / V for p in pairs])
    g = P.rdf_normalize(counts, n_per, V, r_max, n_conf)
    assert np.allclose(g, 1.0, rtol=1e-12)


def test_metad_fes_of_one_hill():
    """One hill of height h: F(s) = -(gamma/(gamma-1)) h exp(-(s-c)^2/(2 sigma^2)),
    shifted so that min F = 0 (the minimum sits at the hill's centre)."""
    s = np.linspace(-1, 1, 201)
    F = P.metad_fes(s, [0.2], [0.03], 0.1, 10.0)
    want = -10.0 / 9.0 * 0.03 * np.exp(-0.5 * (s - 0.2) ** 2 / 0.01)
    assert np.allclose(F, want - want.min(), atol=1e-15)
    assert abs(s[np.argmin(F)] - 0.2) < 1e-12
