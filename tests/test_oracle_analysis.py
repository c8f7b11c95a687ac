"""Pins of the oracle's structural analysis (RDF pair counts, Sec. 3.2
Figs. 8-9; proton-transfer coordinate, Sec. 3.2 Fig. 11) against closed forms
on lattices and hand-built geometries."""
import math

import numpy as np
import pytest

import oracle as O


def _cubic(nside, a, two_types=False):
    g = np.arange(nside)
    pts = np.array([(i, j, k) for i in g for j in g for k in g], dtype=np.float64) * a
    types = ((pts / a).round().astype(int).sum(axis=1) % 2) if two_types else np.zeros(len(pts), int)
    return pts, types


def test_rdf_simple_cubic_shells():
    """Simple cubic lattice, 4^3 sites, spacing a: coordination shells at a,
    sqrt2 a, sqrt3 a, 2a hold 6, 12, 8, 6 neighbours per site; pair counts
    are N z / 2 in the bins of those radii and zero elsewhere."""
    a = 1.5
    x, t = _cubic(4, a)
    L = 4 * a
    n_bins, r_max = 60, 2.95       # bin width 0.0492 A; shells well inside bins
    c = O.rdf_counts(x, (L, L, L), t, 1, r_max, n_bins)[0]
    dr = r_max / n_bins
    want = np.zeros(n_bins, dtype=np.uint64)
    for r, z in ((a, 6), (math.sqrt(2) * a, 12), (math.sqrt(3) * a, 8)):
        want[int(r / dr)] += len(x) * z // 2
    assert np.array_equal(c, want)
    # the 2a shell sits at L / 2: include it with r_max just above
    c2 = O.rdf_counts(x, (L, L, L), t, 1, 3.05, 61)[0]
    # at 2a = L/2 the +2a and -2a images are the same atom: 3 partners per site
    assert int(c2.sum()) == len(x) * (6 + 12 + 8) // 2 + len(x) * 3 // 2


def test_rdf_rock_salt_type_pairs():
    """Rock-salt colouring of the cubic lattice: nearest neighbours are all
    unlike (pair type (0,1)), the sqrt2 a shell all like (0,0) and (1,1)."""
    a = 1.225                     # shells at 24.5 and 34.6 bin widths: away from edges
    x, t = _cubic(4, a, two_types=True)
    L = 4 * a
    c = O.rdf_counts(x, (L, L, L), t, 2, 2.0, 40)
    n = len(x)
    k1, k2 = int(a / 0.05), int(math.sqrt(2) * a / 0.05)
    assert c[1, k1] == n * 6 // 2 and c[0, k1] == 0 and c[2, k1] == 0
    assert c[0, k2] == (n // 2) * 12 // 2 and c[2, k2] == (n // 2) * 12 // 2 and c[1, k2] == 0
    assert int(c.sum()) == n * 6 // 2 + n * 12 // 2


def test_rdf_ideal_gas_is_flat():
    """Uniform random points in a periodic box: g(r) = counts / (pairs
    density x shell volume) is 1 within sampling error in every bin."""
    rng = np.random.default_rng(4)
    L, n, r_max, n_bins = 20.0, 2000, 6.0, 12
    tot = np.zeros(n_bins)
    n_conf = 4
    for _ in range(n_conf):
        x = rng.uniform(0, L, size=(n, 3))
        tot += O.rdf_counts(x, (L, L, L), np.zeros(n, int), 1, r_max, n_bins)[0]
    edges = np.linspace(0, r_max, n_bins + 1)
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    expect = n_conf * n * (n - 1) / 2 / L ** 3 * shell
    g = tot / expect
    sig = 1.0 / np.sqrt(expect)
    assert np.all(np.abs(g[2:] - 1) < 5 * sig[2:]), g


def test_pt_coordinate_linear_geometry():
    """O1 - H ... O2 on a line, O1 at 0 and O2 at 2.5 A: v = d(O1,H) - d(O2,H)
    = 2 x_H - 2.5, with values exact in FP32; the bonding oxygen is O1 even
    when H sits nearer O2 (v > 0)."""
    for xh, want in ((1.0, -0.5), (1.25, 0.0), (1.5, 0.5)):
        x = np.array([[0.0, 0, 0], [xh, 0, 0], [2.5, 0, 0]])
        v, h = O.pt_coordinate(x, None, [-1, 0, -1], [1, 0, 1], -1.0, 1.0, 8)
        assert v[1] == np.float32(want) and np.isnan(v[0]) and np.isnan(v[2])
        k = int((want + 1.0) / 0.25)
        assert h[k] == 1 and h.sum() == 1


def test_pt_coordinate_periodic_image_and_nearest_acceptor():
    """The non-bonding acceptor is the nearest other oxygen, through the
    periodic boundary when that image is closest."""
    L = 10.0
    x = np.array([[1.0, 5, 5], [2.0, 5, 5], [9.5, 5, 5], [5.0, 5, 5]])   # O, H, O (wraps to -0.5), O
    v, _ = O.pt_coordinate(x, (L, L, L), [-1, 0, -1, -1], [1, 0, 1, 1], -3.0, 3.0, 6)
    # d(O_bond, H) = 1; other O: |9.5 - 2 - 10| = 2.5 and 3 -> v = 1 - 2.5
    assert abs(float(v[1]) + 1.5) < 1e-6
