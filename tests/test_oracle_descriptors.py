"""Pins for the oracle's neighbour rule, symmetry functions and network
(descriptor-based energy model of ref. [17], Sec. 1; graph edges within the
0.6 nm cutoff of Tables S1-S2)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_23728_gb300 import synth as s


def _model(widths=(16, 16), seed=3):
    return s.xavier_model((1, 6, 8), widths, seed)


def _fc(r, rc=6.0):
    return 0.5 * (math.cos(math.pi * r / rc) + 1.0) if r < rc else 0.0


# ---------------------------------------------------------------- neighbours
def test_neighbours_match_kdtree_periodic():
    """Set equality with scipy's periodic k-d tree (an independent library
    search), excluding pairs within 1e-4 A of the cutoff where FP32 and FP64
    may round differently."""
    from scipy.spatial import cKDTree
    r = s.water_box(4, seed=99)
    L = np.array(r.box)
    nb, _, _ = O.neighbours(r.x0, r.box, 6.0)
    tree = cKDTree(np.mod(r.x0, L), boxsize=L)
    pairs = tree.query_pairs(6.0 + 1e-4)
    near = set()
    for (i, j) in pairs:
        d = r.x0[j] - r.x0[i]
        d -= L * np.round(d / L)
        dist = np.linalg.norm(d)
        if abs(dist - 6.0) < 1e-4:
            near.add((i, j))
    for i in range(r.n_atoms):
        got = set(int(j) for j in nb[i])
        want = {j for (a, j) in pairs if a == i} | {a for (a, j) in pairs if j == i}
        fuzzy = {j for (a, j) in near if a == i} | {a for (a, j) in near if j == i}
        assert got - fuzzy == want - fuzzy
        assert list(nb[i]) == sorted(nb[i])
        assert i not in got


def test_neighbours_are_symmetric_and_gas_phase_matches_brute_force():
    reps = s.batch(n_rep=4, seed=5)
    for r in reps:
        nb, _, _ = O.neighbours(r.x0, None, 6.0)
        D = np.linalg.norm(r.x0[:, None] - r.x0[None], axis=2)
        for i in range(r.n_atoms):
            for j in nb[i]:
                assert i in nb[j]
            want = [j for j in range(r.n_atoms) if j != i and D[i, j] < 6.0 - 1e-4]
            assert set(want) <= set(int(j) for j in nb[i])


def test_neighbour_overflow_is_reported():
    r = s.water_box(4, seed=99)
    with pytest.raises(ValueError):
        O.neighbours(r.x0, r.box, 6.0, maxnb=16)


# ---------------------------------------------------------------- descriptors
def test_isolated_atom_has_zero_descriptor():
    m = _model()
    x = np.array([[0.0, 0.0, 0.0], [10.0, 0.0, 0.0]])
    G = O.descriptors(m, x, None)
    assert np.all(G == 0.0)


def test_isolated_pair_closed_form():
    """Two atoms at distance r: G2_mu = exp(-eta (r - r_mu)^2) fc(r) and no
    angular term (no pair of neighbours)."""
    m = _model()
    d = m.desc
    r = 2.345
    x = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3 + r]])
    G = O.descriptors(m, x, None)
    want = np.array([math.exp(-d["eta_R"] * (r - rm) ** 2) * _fc(r) for rm in d["r_mu"]])
    np.testing.assert_allclose(G[0, :32], want, rtol=1e-13, atol=1e-300)
    np.testing.assert_allclose(G[1, :32], want, rtol=1e-13, atol=1e-300)
    assert np.all(G[:, 32:] == 0.0)


@pytest.mark.parametrize("theta", [90.0, 180.0, 60.0])
def test_symmetric_triangle_angular_values(theta):
    """Centre atom with exactly two neighbours at equal distance r and angle
    theta (one neighbour pair): G5_(zeta,lambda,eta) = A(zeta,lambda)
    e^(-2 eta r^2) fc(r)^2 with the angular factor A worked by hand:
    90 deg: 2^(1-zeta); 180 deg: 0 for lambda = +1 and 2 for lambda = -1;
    60 deg: 2^(1-zeta) 1.5^zeta and 2^(1-zeta) 0.5^zeta."""
    m = _model()
    d = m.desc
    r = 3.0
    t = math.radians(theta)
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0], [r * math.cos(t), r * math.sin(t), 0.0]])
    G = O.descriptors(m, x, None)
    fc2 = _fc(r) ** 2
    for zi, zeta in enumerate(d["zeta"]):
        for li, lam in enumerate(d["lam"]):
            if theta == 90.0:
                A = 2.0 ** (1 - zeta)
            elif theta == 180.0:
                A = 0.0 if lam > 0 else 2.0
            else:
                A = 2.0 ** (1 - zeta) * (1.5 ** zeta if lam > 0 else 0.5 ** zeta)
            for ei, eta in enumerate(d["eta_A"]):
                nu = (zi * 2 + li) * 4 + ei
                want = A * math.exp(-2 * eta * r * r) * fc2
                np.testing.assert_allclose(G[0, 32 + nu], want, rtol=1e-12, atol=1e-15)


def test_descriptor_invariances(fad_model):
    """Translation, rotation and same-element permutation invariance."""
    _, r, m = fad_model
    G0 = O.descriptors(m, r.x0, None)
    rng = np.random.default_rng(0)
    G1 = O.descriptors(m, r.x0 + rng.normal(size=3) * 5.0, None)
    np.testing.assert_allclose(G1, G0, rtol=1e-12, atol=1e-12)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    R = s._rotation(np.random.default_rng(4))
    G2 = O.descriptors(m, r.x0 @ R.T, None)
    np.testing.assert_allclose(G2, G0, rtol=1e-12, atol=1e-12)
    # swap the two carbons and two oxygens
    perm = np.arange(r.n_atoms)
    perm[[0, 5]] = perm[[5, 0]]
    perm[[1, 6]] = perm[[6, 1]]
    G3 = O.descriptors(m, r.x0[perm], None)
    np.testing.assert_allclose(G3, G0[perm], rtol=1e-12, atol=1e-12)


def test_periodic_translation_invariance():
    m = _model()
    r = s.water_box(4, seed=21)
    G0 = O.descriptors(m, r.x0, r.box)
    L = np.array(r.box)
    x1 = np.mod(r.x0 + np.array([3.3, -7.1, 11.9]), L)
    G1 = O.descriptors(m, x1, r.box)
    np.testing.assert_allclose(G1, G0, rtol=1e-10, atol=1e-10)


# ---------------------------------------------------------------- network
def _numpy_energy(m, z, G):
    blob = m.params[z]
    h = (G - s.view(blob, m.widths, "mu")) / s.view(blob, m.widths, "sigma")
    for l in range(len(m.widths)):
        h = np.tanh(s.view(blob, m.widths, "W%d" % l) @ h + s.view(blob, m.widths, "b%d" % l))
    y = s.view(blob, m.widths, "w_out") @ h + s.view(blob, m.widths, "b_out")[0]
    return s.view(blob, m.widths, "s_E")[0] * y + s.view(blob, m.widths, "e_Z")[0]


def test_mlp_matches_numpy_and_finite_differences():
    m = _model((24, 20, 12), seed=9)
    rng = np.random.default_rng(1)
    for z in m.elements:
        blob = m.params[z]
        s.view(blob, m.widths, "b0")[:] = rng.normal(size=24) * 0.1
        s.view(blob, m.widths, "mu")[:] = rng.normal(size=64)
        s.view(blob, m.widths, "sigma")[:] = rng.uniform(0.5, 2.0, size=64)
        s.view(blob, m.widths, "s_E")[:] = 0.7
        s.view(blob, m.widths, "e_Z")[:] = -1.5
        G = rng.normal(size=64) * 2.0
        E, g = O.mlp(m, z, G)
        assert abs(E - _numpy_energy(m, z, G)) < 1e-13
        h = 1e-6
        fd = np.array([(_numpy_energy(m, z, G + h * e) - _numpy_energy(m, z, G - h * e)) / (2 * h)
                       for e in np.eye(64)])
        np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)
