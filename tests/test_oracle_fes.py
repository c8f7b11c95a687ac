"""Pins for the oracle's free-energy and g(r) routines (Sec. 2.5: the
well-tempered bias and the path-integral reweighting of the bead CVs; Figs.
8, 9: radial distribution functions). Closed forms, exact lattice
coordination numbers and sampling from known densities; none of these
retypes the oracle's formulas."""
import math

import numpy as np
from scipy.special import ndtr

import oracle as O

KB = 8.617333262e-5


def _gauss_bin_F(edges, sigma, T):
    """-k_B T ln of the exact bin-averaged density of N(0, sigma^2)"""
    p = (ndtr(edges[1:] / sigma) - ndtr(edges[:-1] / sigma)) / np.diff(edges)
    return -KB * T * np.log(p)


def test_pi_fes_of_gaussian_bead_samples():
    """Independent N(0, sigma^2) CV samples on P = 4 beads without a bias:
    every F_k and the path-integral F equal -k_B T ln of the Gaussian's
    bin-averaged density within sampling error, and F is the log-mean-exp
    of the F_k (the second form of the equation in Sec. 2.5)."""
    P, T, sigma, n_bins, lo, hi = 4, 300.0, 0.3, 36, -0.9, 0.9
    h = O.CvHistogram(P, lo, hi, n_bins, T)
    rng = np.random.default_rng(7)
    S = rng.normal(scale=sigma, size=(200000, P))
    for s in S:
        h.add(s)
    F, Fk = h.fes()
    edges = np.linspace(lo, hi, n_bins + 1)
    want = _gauss_bin_F(edges, sigma, T)
    cnt = h.hist.sum(axis=0)
    err = KB * T / np.sqrt(cnt)                     # sampling error of -kT ln(count)
    assert np.all(np.abs(F - want) < 5 * err + 1e-4)
    for k in range(P):
        errk = KB * T / np.sqrt(h.hist[k])
        assert np.all(np.abs(Fk[k] - want) < 5 * errk + 1e-4)
    kT = KB * T
    lme = -kT * np.log(np.mean(np.exp(-Fk / kT), axis=0))
    assert np.allclose(F, lme, rtol=1e-12, atol=1e-14)
    assert abs(h.wsum[0] - len(S)) == 0.0            # every sample counted once, weight 1


def test_pi_fes_reweighting_removes_the_bias():
    """A harmonic bias V_b(s) = kappa s^2 / 2 on each of P = 2 beads, sampled
    at the ring polymer's temperature T_P = P T: each bead's CV follows
    N(0, sigma_b^2) with 1/sigma_b^2 = 1/sigma_0^2 + kappa / (k_B T P). The
    weights exp(sum_k V_b(s_k) / (k_B T P)) restore the unbiased
    N(0, sigma_0^2) profile. (With k_B T instead of k_B T P in the weight the
    profile would come out flat; without weights it keeps the biased
    curvature.)"""
    P, T, s0 = 2, 300.0, 0.3
    kTP = KB * T * P
    kappa = kTP / s0 ** 2
    sb = 1.0 / math.sqrt(1.0 / s0 ** 2 + kappa / kTP)
    n_bins, lo, hi = 30, -0.6, 0.6
    h = O.CvHistogram(P, lo, hi, n_bins, T)
    rng = np.random.default_rng(11)
    S = rng.normal(scale=sb, size=(400000, P))
    for s in S:
        h.add(s, 0.5 * kappa * s * s)
    F, _ = h.fes()
    want = _gauss_bin_F(np.linspace(lo, hi, n_bins + 1), s0, T)
    centre = np.abs(0.5 * (np.linspace(lo, hi, n_bins + 1)[1:] + np.linspace(lo, hi, n_bins + 1)[:-1])) < 0.4
    assert np.all(np.abs(F[centre] - want[centre]) < 0.08 * KB * T)
    # the profile's curvature is the unbiased one: a quadratic fit of F
    x = 0.5 * (np.linspace(lo, hi, n_bins + 1)[1:] + np.linspace(lo, hi, n_bins + 1)[:-1])[centre]
    a = np.polyfit(x, F[centre], 2)[0]
    assert abs(a / (KB * T / (2 * s0 ** 2)) - 1.0) < 0.05


def test_pi_fes_empty_bins_and_shift():
    """Empty bins give +inf; a constant log-weight shift changes nothing."""
    h1 = O.CvHistogram(3, 0.0, 1.0, 10, 250.0)
    h2 = O.CvHistogram(3, 0.0, 1.0, 10, 250.0, log_w_shift=7.5)
    rng = np.random.default_rng(3)
    for _ in range(500):
        s = rng.uniform(0.0, 0.5, size=3)
        v = rng.uniform(0.0, 0.05, size=3)
        h1.add(s, v)
        h2.add(s, v)
    F1, _ = h1.fes()
    F2, _ = h2.fes()
    assert np.all(np.isinf(F1[5:])) and np.all(np.isfinite(F1[:5]))
    assert np.allclose(F1[:5], F2[:5], rtol=1e-12)


def test_metad_fes_of_known_hills():
    """Two hills (Sec. 2.5: V = sum_k h_k exp(-(s - s_k)^2 / (2 sigma^2))):
    F = -(gamma / (gamma - 1)) V, so at a lone hill's centre F = -gamma h /
    (gamma - 1), and far from all hills F = 0."""
    md = O.Metad(("distances", [(0, 1, 1.0)]), 2, 1, 0.1, 0.2, 15.0, 10)
    md.set_hills([0.0, 5.0], [0.3, 0.1])
    F = md.fes([0.0, 5.0, 50.0, 0.2])
    g = 15.0 / 14.0
    assert abs(F[0] - (-g * (0.3 + 0.1 * math.exp(-0.5 * 25.0 / 0.04)))) < 1e-15
    assert abs(F[1] - (-g * 0.1)) < 1e-15
    assert F[2] == 0.0
    assert abs(F[3] - (-g * 0.3 * math.exp(-0.5))) < 1e-15


def test_rdf_gr_lattice_coordination_numbers():
    """Simple cubic lattice (spacing a) in a periodic box: the coordination
    number n(R) = rho sum_k g_k shell_k over the shells below R, rho =
    (N - 1) / V, counts 6, 18 and 26 neighbours for R between the first,
    second, third and fourth neighbour distances a, sqrt2 a, sqrt3 a, 2a."""
    n, a = 6, 2.0
    L = n * a
    g3 = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    x = (g3 * a + 0.013).astype(np.float64)
    N = len(x)
    r_max, n_bins = 5.0, 100
    counts = O.rdf_counts(x, (L, L, L), np.zeros(N, dtype=np.int32), 1, r_max, n_bins)
    g = O.rdf_gr(counts, [N], L ** 3, r_max, 1)
    dr = r_max / n_bins
    k = np.arange(n_bins)
    shell = 4.0 / 3.0 * np.pi * (((k + 1) * dr) ** 3 - (k * dr) ** 3)
    cum = np.cumsum((N - 1) / L ** 3 * g[0] * shell)
    for R, want in ((1.2 * a, 6), (1.5 * a, 18), (1.9 * a, 26)):
        assert abs(cum[int(R / dr) - 1] - want) < 1e-9, (R, cum[int(R / dr) - 1])


def test_rdf_gr_of_uniform_points_is_one():
    """Uniform random points of two types in a periodic box: g = 1 for every
    pair type and shell within sampling error."""
    rng = np.random.default_rng(5)
    L, na, nb = 10.0, 40, 25
    r_max, n_bins = 4.0, 8
    types = np.array([0] * na + [1] * nb, dtype=np.int32)
    counts = np.zeros((3, n_bins), dtype=np.uint64)
    n_conf = 400
    for _ in range(n_conf):
        x = rng.uniform(0.0, L, size=(na + nb, 3))
        counts += O.rdf_counts(x, (L, L, L), types, 2, r_max, n_bins)
    g = O.rdf_gr(counts, [na, nb], L ** 3, r_max, n_conf)
    rel = 1.0 / np.sqrt(np.maximum(counts.astype(float), 1.0))
    assert np.all(np.abs(g[:, 1:] - 1.0) < 5 * rel[:, 1:])
