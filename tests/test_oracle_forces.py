"""Pins for the oracle's analytic forces and virial (forces as the gradient of
the energy model, Sec. 2.2): central finite differences, translation and
rotation invariance, and the strain derivative of the energy."""
import numpy as np

import oracle as O


def _V(m, r, x, box=None):
    E, _, _ = O.energy_forces(m, r.Z, x, r.box if box is None else box)
    return E.sum()


def test_forces_match_central_differences_water(water64_model):
    """Directional derivative along a random unit vector for 8 random atoms
    of the periodic water box, h = 1e-5 A (truncation error ~h^2 is then
    ~1e-9 eV/A), relative error <= 1e-6."""
    _, r, m = water64_model
    E, F, _ = O.energy_forces(m, r.Z, r.x0, r.box)
    rng = np.random.default_rng(2)
    h = 1e-5
    for i in rng.choice(r.n_atoms, size=8, replace=False):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        xp, xm = r.x0.copy(), r.x0.copy()
        xp[i] += h * u
        xm[i] -= h * u
        fd = -(_V(m, r, xp) - _V(m, r, xm)) / (2 * h)
        an = F[i] @ u
        assert abs(fd - an) <= 1e-6 * max(abs(an), np.abs(F).max() * 1e-2), (i, fd, an)


def test_forces_match_central_differences_gas(fad_model):
    _, r, m = fad_model
    _, F, _ = O.energy_forces(m, r.Z, r.x0, None)
    h = 1e-5
    for i in range(r.n_atoms):
        for a in range(3):
            xp, xm = r.x0.copy(), r.x0.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -(_V(m, r, xp) - _V(m, r, xm)) / (2 * h)
            assert abs(fd - F[i, a]) <= 1e-6 * np.abs(F).max()


def test_total_force_and_torque_vanish(fad_model, water64_model):
    _, r, m = fad_model
    _, F, _ = O.energy_forces(m, r.Z, r.x0, None)
    scale = np.abs(F).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * scale * r.n_atoms
    torque = np.cross(r.x0, F).sum(axis=0)
    assert np.abs(torque).max() < 1e-11 * scale * np.abs(r.x0).max() * r.n_atoms
    _, rw, mw = water64_model
    _, Fw, _ = O.energy_forces(mw, rw.Z, rw.x0, rw.box)
    assert np.abs(Fw.sum(axis=0)).max() < 1e-11 * np.abs(Fw).max() * rw.n_atoms


def test_virial_is_strain_derivative_gas(fad_model):
    """W_ba = -dV/d eps_ab under x_a -> x_a + eps_ab x_b (all 9 components)."""
    _, r, m = fad_model
    _, _, W = O.energy_forces(m, r.Z, r.x0, None)
    eps = 1e-6
    for a in range(3):
        for b in range(3):
            S = np.eye(3)
            S[a, b] += eps
            Vp = _V(m, r, r.x0 @ S.T)
            S[a, b] -= 2 * eps
            Vm = _V(m, r, r.x0 @ S.T)
            dV = (Vp - Vm) / (2 * eps)
            assert abs(W[b, a] + dV) <= 1e-6 * np.abs(W).max() + 1e-9


def test_virial_is_strain_derivative_periodic(water64_model):
    """Diagonal strain of the periodic box (box deformed with the atoms)."""
    _, r, m = water64_model
    _, _, W = O.energy_forces(m, r.Z, r.x0, r.box)
    eps = 1e-6
    for a in range(3):
        sc = np.ones(3)
        sc[a] += eps
        Vp = _V(m, r, r.x0 * sc, tuple(np.array(r.box) * sc))
        sc[a] -= 2 * eps
        Vm = _V(m, r, r.x0 * sc, tuple(np.array(r.box) * sc))
        dV = (Vp - Vm) / (2 * eps)
        assert abs(W[a, a] + dV) <= 1e-6 * np.abs(W).max()
