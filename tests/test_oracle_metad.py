"""Pins of the oracle's collective variables and well-tempered metadynamics
(Sec. 2.5; CVs of Secs. S2-S3) against closed forms, finite differences and
energy conservation."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_23728_gb300 import synth as s

KB = 8.617333262e-5
Q_XRD = 4 * math.pi * math.sin(math.radians(11.95)) / 1.54


def test_xrd_two_atoms_closed_form():
    """Two atoms at distance R: s = (f1^2 + f2^2 + 2 f1 f2 sin(QR)/(QR)) / 2
    and ds/dR = f1 f2 Q (QR cos QR - sin QR) / (QR)^2."""
    f1, f2, R = 7.3, 0.8, 1.37
    md = O.Metad(("xrd", Q_XRD, [f1, f2]), 2, 1, 0.01, 0.1, 10, 8)
    x = np.array([[0.2, -0.1, 0.4], [0.2 + R, -0.1, 0.4]])
    val, g, vir = md.cv(x, None, grad=True)
    y = Q_XRD * R
    assert abs(val - 0.5 * (f1 * f1 + f2 * f2 + 2 * f1 * f2 * math.sin(y) / y)) < 1e-13
    dsdR = f1 * f2 * Q_XRD * (y * math.cos(y) - math.sin(y)) / (y * y)
    assert abs(g[1, 0] - dsdR) < 1e-12 and abs(g[0, 0] + dsdR) < 1e-12
    assert abs(vir[0, 0] - R * dsdR) < 1e-12


@pytest.mark.parametrize("kind", ["xrd", "distances"])
def test_cv_gradient_and_virial_by_finite_differences(kind):
    rng = np.random.default_rng(9)
    n, L = 12, 7.0
    x = rng.uniform(0, L, size=(n, 3))
    box = (L, L, L)
    if kind == "xrd":
        md = O.Metad(("xrd", Q_XRD, rng.uniform(0.5, 8, n)), n, 1, 0.01, 0.1, 10, 8)
    else:
        md = O.Metad(("distances", [(0, 1, 1.0), (2, 1, -1.0), (3, 4, 0.5), (5, 6, -2.0)]), n, 1, 0.01, 0.1, 10, 8)
    val, g, vir = md.cv(x, box, grad=True)
    h = 1e-6
    for i in (0, 1, 4, 7):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = (md.cv(xp, box)[0] - md.cv(xm, box)[0]) / (2 * h)
            assert abs(fd - g[i, a]) < 1e-7 * max(1.0, abs(g).max()), (i, a)
    # uniform strain: ds/d eps = trace of the pair virial
    eps = 1e-6
    sp = md.cv(x * (1 + eps), tuple(np.array(box) * (1 + eps)))[0]
    sm = md.cv(x * (1 - eps), tuple(np.array(box) * (1 - eps)))[0]
    assert abs((sp - sm) / (2 * eps) - np.trace(vir)) < 1e-6 * max(1.0, abs(np.trace(vir)))
    # translation invariance
    assert np.abs(g.sum(axis=0)).max() < 1e-10 * max(1.0, abs(g).max())


def test_fad_dimer_cv_of_the_template():
    """The undistorted template has O-H 0.97 A with H on the O...O line and
    O...O 2.70 A, so s = 2 (0.97 - 1.73) = -1.52."""
    Z, x = s.fad_template()
    md = O.Metad(("distances", s.fad_dimer_cv_terms()), len(Z), 1, 0.01, 0.1, 10, 8)
    assert abs(md.cv(x, None)[0] + 1.52) < 1e-12


def test_bias_and_deposition_closed_forms():
    md = O.Metad(("distances", [(0, 1, 1.0)]), 2, 4, 0.02, 0.15, 10.0, 1, max_hills=16)
    T = 300.0
    md.deposit([0.3, 0.3, 0.5, 0.7], [0.0] * 4, T)
    s_h, h_h = md.hills
    assert np.array_equal(s_h, [0.3, 0.3, 0.5, 0.7]) and np.allclose(h_h, 0.005, rtol=0, atol=1e-16)
    sv = 0.41
    v, dv = md.bias(sv)
    want = sum(0.005 * math.exp(-0.5 * (sv - c) ** 2 / 0.15 ** 2) for c in (0.3, 0.3, 0.5, 0.7))
    dwant = sum(-0.005 * (sv - c) / 0.15 ** 2 * math.exp(-0.5 * (sv - c) ** 2 / 0.15 ** 2) for c in (0.3, 0.3, 0.5, 0.7))
    assert abs(v - want) < 1e-16 and abs(dv - dwant) < 1e-15
    # well-tempered height: (h0 / P) exp(-V / (k_B T (gamma - 1)))
    md.deposit([0.41] * 4, [v] * 4, T)
    assert abs(md.hills[1][-1] - 0.005 * math.exp(-v / (KB * T * 9.0))) < 1e-16
    # no room: a deposition that does not fit is dropped whole
    for _ in range(5):
        md.deposit([0.0] * 4, [0.0] * 4, T)
    assert len(md.hills[0]) == 16


def test_biased_forces_are_gradients_of_biased_energy(fad_model):
    """Forces of a biased bead = -grad (network energy + bias), checked by
    finite differences of the bead energy."""
    w, r, m = fad_model
    rep = s.Replica(r.Z, r.x0, r.box, 2, r.T, r.seed)
    md = O.Metad(("distances", s.fad_dimer_cv_terms()), r.n_atoms, 2, 0.05, 0.2, 10.0, 1000)
    md.deposit([-1.4, -1.6], [0.0, 0.0], r.T)
    sysm = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m, metad=md)
    sysm.q[1] += np.random.default_rng(2).normal(scale=0.05, size=sysm.q[1].shape)
    sysm.compute_forces()
    f0 = sysm.f.copy()
    C = O.nm_matrix(2)
    h = 1e-5
    for (i, a) in ((3, 0), (8, 1), (1, 2)):
        dq = np.zeros_like(sysm.q)
        dq[:, i, a] = C[0, :] * h          # moves bead 0's atom i along a by h
        sysm.q += dq
        sysm.compute_forces()
        vp = sysm.V[0]
        sysm.q -= 2 * dq
        sysm.compute_forces()
        vm = sysm.V[0]
        sysm.q += dq
        assert abs(-(vp - vm) / (2 * h) - f0[0, i, a]) < 1e-6 * max(1.0, abs(f0).max()), (i, a)


def test_nve_with_fixed_bias_conserves_energy(fad_model):
    """No thermostat, hills fixed: the ring-polymer Hamiltonian including the
    bias is conserved to O(dt^2) fluctuations, without drift."""
    w, r, m = fad_model
    amp = []
    for dt in (0.1, 0.05):
        rep = s.Replica(r.Z, r.x0, r.box, 4, 300.0, r.seed)
        md = O.Metad(("distances", s.fad_dimer_cv_terms()), r.n_atoms, 4, 0.05, 0.1, 10.0, 10 ** 9, max_hills=64)
        md.deposit([-1.5, -1.45, -1.55, -1.5], [0.0] * 4, 300.0)
        sysm = O.System(rep, s.MASS, dt, 0.0, model=m, thermostat=False, metad=md)
        H = []
        for _ in range(int(round(10.0 / dt))):
            sysm.step(1)
            H.append(sysm.estimators()["H_cons"])
        H = np.array(H)
        slope = np.polyfit(np.arange(len(H)), H, 1)[0]
        amp.append(H.std())
        assert abs(slope * len(H)) < 3 * H.std() + 1e-12
        assert np.abs(md.bias(md.cv_last[0])[0]) > 0     # the bias acts
    assert 2.5 < amp[0] / amp[1] < 6.0, amp
