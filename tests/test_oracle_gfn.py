"""Pins of the FP64 graph-field-network oracle (direct-force head, Sec. 2.2).

The paper prints no values for the head, so the oracle is pinned by what its
definition forces: Newton's third law and zero torque for free clusters, the
rotation / translation / permutation behaviour, the virial of central pair
forces, pairwise additivity with no message passing, locality, the cutoff,
and which parameters may or may not reach the forces after L iterations (a
wrong iteration order or the post-update node state in the edge update
fails those)."""
import math

import numpy as np
import pytest

import oracle.gfn as G
from paper_2503_23728_gb300 import synth as s


def _cluster(n=12, seed=3):
    rng = np.random.default_rng(seed)
    return s.cluster(rng, n)


def _model(els, F=16, L=3, seed=5):
    return s.gfn_model(els, F, L, seed)


def _rot(seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def test_newton_third_law_and_torque_cluster():
    Z, x = _cluster()
    m = _model(set(Z.tolist()))
    F, W = G.forces(m, Z, x)
    scale = np.abs(F).max()
    assert scale > 1e-3
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * scale * len(x)
    torque = np.cross(x, F).sum(axis=0)
    assert np.abs(torque).max() < 1e-11 * scale * np.abs(x).max() * len(x)
    # central pair forces: the virial is sum_i x_i (x) F_i for a free cluster, and symmetric
    assert np.allclose(W, np.einsum("ia,ib->ab", x, F), rtol=0, atol=1e-11 * np.abs(W).max())
    assert np.allclose(W, W.T, atol=1e-11 * np.abs(W).max())


def test_newton_third_law_periodic():
    rep = s.water_box(4, seed=71, n_beads=1)   # 64 H2O in a 12.42 A box
    m = _model((1, 8), F=16, L=2)
    F, _ = G.forces(m, rep.Z, rep.x0, rep.box)
    assert np.abs(F.sum(axis=0)).max() < 1e-11 * np.abs(F).max() * rep.n_atoms


def test_rotation_translation_permutation():
    Z, x = _cluster(10, seed=8)
    m = _model(set(Z.tolist()), F=12, L=3, seed=9)
    F, W = G.forces(m, Z, x)
    R = _rot(4)
    F2, W2 = G.forces(m, Z, x @ R.T)
    assert np.abs(F2 - F @ R.T).max() < 1e-11 * np.abs(F).max()
    assert np.abs(W2 - R @ W @ R.T).max() < 1e-10 * np.abs(W).max()
    F3, _ = G.forces(m, Z, x + np.array([3.7, -1.25, 12.0]))
    assert np.abs(F3 - F).max() < 1e-10 * np.abs(F).max()
    p = np.random.default_rng(1).permutation(len(x))
    F4, _ = G.forces(m, Z[p], x[p])
    assert np.abs(F4 - F[p]).max() < 1e-12 * np.abs(F).max()


def test_no_iterations_is_pairwise_additive():
    """L = 0: F_ij depends on r_ij only, so every force is the sum of the
    forces the atom feels from each neighbour alone."""
    Z, x = _cluster(8, seed=12)
    m = _model(set(Z.tolist()), F=10, L=0, seed=13)
    F, _ = G.forces(m, Z, x)
    F_pairs = np.zeros_like(F)
    for i in range(len(x)):
        for j in range(len(x)):
            if i != j:
                f2, _ = G.forces(m, Z[[i, j]], x[[i, j]])
                F_pairs[i] += f2[0]
    assert np.abs(F - F_pairs).max() < 1e-12 * np.abs(F).max()


def test_message_passing_is_not_pairwise():
    Z, x = _cluster(8, seed=12)
    m = _model(set(Z.tolist()), F=10, L=2, seed=13)
    F, _ = G.forces(m, Z, x)
    F_pairs = np.zeros_like(F)
    for i in range(len(x)):
        for j in range(len(x)):
            if i != j:
                F_pairs[i] += G.forces(m, Z[[i, j]], x[[i, j]])[0][0]
    assert np.abs(F - F_pairs).max() > 1e-3 * np.abs(F).max()


def _perturbed(m, keys, seed=0):
    m2 = s.GfnModel(m.elements, m.F, m.L, m.blob.copy(), m.desc)
    rng = np.random.default_rng(seed)
    for k in keys:
        v = m2.view(k)
        v[...] = v + rng.normal(scale=0.3, size=v.shape)
    return m2


def test_parameters_that_reach_the_forces():
    """e^(L) uses n^(0..L-1): the node update of the last iteration and, at
    L = 1, the messages never reach the forces; earlier ones do."""
    Z, x = _cluster(9, seed=21)
    els = set(Z.tolist())
    m1 = _model(els, F=8, L=1, seed=22)
    F1, _ = G.forces(m1, Z, x)
    F1b, _ = G.forces(_perturbed(m1, ["W_m0", "b_m0", "W_v10", "b_v10", "W_v20", "b_v20"]), Z, x)
    assert np.array_equal(F1, F1b)
    F1c, _ = G.forces(_perturbed(m1, ["W_a10"]), Z, x)
    assert np.abs(F1c - F1).max() > 1e-4 * np.abs(F1).max()
    m2 = _model(els, F=8, L=2, seed=23)
    F2, _ = G.forces(m2, Z, x)
    F2b, _ = G.forces(_perturbed(m2, ["W_m1", "b_m1", "W_v11", "W_v21", "b_v21"]), Z, x)
    assert np.array_equal(F2, F2b)
    for key in ("W_m0", "W_v10", "W_v20", "W_a11"):
        F2c, _ = G.forces(_perturbed(m2, [key]), Z, x)
        assert np.abs(F2c - F2).max() > 1e-4 * np.abs(F2).max(), key


def test_locality_and_isolated_atoms():
    Z1, x1 = _cluster(7, seed=31)
    Z2, x2 = _cluster(6, seed=32)
    els = set(Z1.tolist()) | set(Z2.tolist()) | {8}
    m = _model(els, F=8, L=3, seed=33)
    xa = np.concatenate([x1, x2 + np.array([40.0, 0, 0]), np.array([[0.0, 40.0, 0.0]])])
    Za = np.concatenate([Z1, Z2, np.array([8], dtype=Z1.dtype)])
    F, _ = G.forces(m, Za, xa)
    F1, _ = G.forces(m, Z1, x1)
    F2, _ = G.forces(m, Z2, x2)
    assert np.abs(F[:7] - F1).max() < 1e-12 * np.abs(F1).max()
    assert np.abs(F[7:13] - F2).max() < 1e-12 * np.abs(F2).max()
    assert np.abs(F[13]).max() == 0.0


def test_cutoff_behaviour():
    """The pair force carries fc(r): it vanishes quadratically at r_c and is
    exactly zero beyond."""
    m = _model((1, 8), F=8, L=2, seed=41)
    Z = np.array([8, 1])
    rc = m.desc["cutoff"]

    def f(r):
        return G.forces(m, Z, np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]]))[0][0, 0]

    d = 1e-3
    ratio = f(rc - 2 * d) / f(rc - d)
    assert abs(ratio - 4.0) < 1e-2
    assert f(rc + 1e-6) == 0.0
    # the force lies along the bond and is equal and opposite
    F, _ = G.forces(m, Z, np.array([[0.0, 0.0, 0.0], [1.1, 0.7, -0.3]]))
    u = np.array([1.1, 0.7, -0.3]) / math.sqrt(1.1 ** 2 + 0.7 ** 2 + 0.3 ** 2)
    assert np.abs(np.cross(F[0], u)).max() < 1e-12 * np.abs(F).max()
    assert np.abs(F[0] + F[1]).max() < 1e-14 * np.abs(F).max() + 1e-300


def test_messages_are_summed_over_neighbours():
    """Collinear A-B-A' with |AA'| = 2r beyond the cutoff: A sees only B, and
    B's message at iteration 0 holds two identical terms instead of the
    dimer's one. Summed messages change B's node state and so, from L = 2 on,
    the force on A; averaged ones would not. At L = 1 (node states unused)
    the forces on A agree."""
    Z = np.array([1, 8, 1])
    r = 3.4
    tri = np.array([[-r, 0.0, 0.0], [0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    for L, same in ((1, True), (2, False)):
        m = _model((1, 8), F=8, L=L, seed=51)
        Ft, _ = G.forces(m, Z, tri)
        Fd, _ = G.forces(m, Z[:2], tri[:2])
        assert np.abs(Ft[0] - Ft[2] * np.array([-1, 1, 1])).max() < 1e-14 * np.abs(Ft).max()   # mirror image
        diff = np.abs(Ft[0] - Fd[0]).max()
        if same:
            assert diff < 1e-14 * np.abs(Fd).max()
        else:
            assert diff > 1e-3 * np.abs(Fd).max()
