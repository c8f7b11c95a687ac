"""Pins for the oracle's ring-polymer part (Sec. 2.1: effective Hamiltonian,
normal-mode transformation, H_eff = H_p + U splitting, finite-P estimator;
Sec. S1: harmonic-oscillator validation)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_23728_gb300 import synth as s

KB = 8.617333262e-5
HBAR = 0.6582119569
MVV2E = 103.64269652680505


@pytest.mark.parametrize("P", [1, 2, 3, 8, 16, 31, 32])
def test_normal_modes_orthogonal_and_diagonalise_springs(P):
    C = O.nm_matrix(P)
    np.testing.assert_allclose(C.T @ C, np.eye(P), atol=1e-14)
    wP = 0.37
    K = np.zeros((P, P))
    for j in range(P):
        K[j, j] += 2.0
        K[j, (j + 1) % P] -= 1.0
        K[j, (j - 1) % P] -= 1.0
    K *= wP * wP
    if P == 1:
        K[:] = 0.0
    if P == 2:
        K = wP * wP * np.array([[2.0, -2.0], [-2.0, 2.0]])
    ev = np.sort(np.linalg.eigvalsh(K))
    wk = O.nm_freqs(P, wP)
    np.testing.assert_allclose(np.sort(wk ** 2), ev, atol=1e-12)
    # and the columns of C are the matching eigenvectors, mode 0 = centroid
    D = C.T @ K @ C
    np.testing.assert_allclose(D, np.diag(wk ** 2), atol=1e-12)
    np.testing.assert_allclose(C[:, 0], 1.0 / math.sqrt(P))


def _harmonic_system(P, N=1, T=300.0, omega=0.0, dt=0.5, gamma0=0.01, thermostat=True, seed=5,
                     splitting="obabo", free_rp="exact"):
    x0 = np.random.default_rng(seed).normal(size=(N, 3)) * 0.1
    rep = s.Replica(np.full(N, s.H, dtype=np.int32), x0, (0.0, 0.0, 0.0), P, T, seed)
    return O.System(rep, s.MASS, dt, gamma0, thermostat=thermostat, potential="harmonic", omega=omega,
                    splitting=splitting, free_rp=free_rp)


def test_free_ring_polymer_matches_ode_solver():
    """With V = 0 and no thermostat the exact normal-mode propagation must
    reproduce the bead-space spring dynamics m q_j'' = -m w_P^2 (2 q_j -
    q_{j-1} - q_{j+1}) integrated by scipy's DOP853."""
    from scipy.integrate import solve_ivp
    P, N = 8, 2
    sysm = _harmonic_system(P, N, omega=0.0, dt=2.0, thermostat=False)
    rng = np.random.default_rng(3)
    sysm.q[:] = rng.normal(size=sysm.q.shape) * 0.2
    sysm.p[:] = rng.normal(size=sysm.p.shape) * 0.05
    C = O.nm_matrix(P)
    qb0 = np.einsum("jk,kia->jia", C, sysm.q)
    pb0 = np.einsum("jk,kia->jia", C, sysm.p)
    m = s.MASS[s.H]
    wP = P * KB * 300.0 / HBAR
    nsteps = 40
    sysm.step(nsteps)
    qb = np.einsum("jk,kia->jia", C, sysm.q)

    def rhs(t, y):
        q = y[: P * N * 3].reshape(P, N, 3)
        p = y[P * N * 3:].reshape(P, N, 3)
        f = -m * wP * wP * (2 * q - np.roll(q, 1, axis=0) - np.roll(q, -1, axis=0))
        return np.concatenate([(p / m).ravel(), f.ravel()])

    sol = solve_ivp(rhs, (0.0, nsteps * 2.0), np.concatenate([qb0.ravel(), pb0.ravel()]),
                    method="DOP853", rtol=1e-12, atol=1e-12)
    qode = sol.y[: P * N * 3, -1].reshape(P, N, 3)
    np.testing.assert_allclose(qb, qode, atol=1e-8)


def test_step_is_time_reversible():
    sysm = _harmonic_system(8, 3, omega=0.02, dt=0.5, thermostat=False)
    q0, p0 = sysm.q.copy(), sysm.p.copy()
    sysm.step(25)
    sysm.s.dt = -0.5
    sysm.step(25)
    np.testing.assert_allclose(sysm.q, q0, atol=1e-11)
    np.testing.assert_allclose(sysm.p, p0, atol=1e-11)


def test_initial_state_and_equipartition():
    """All beads start at x0; momenta are drawn at T_P = P T. Under PILE-L on a
    free ring polymer <p^2/m> -> k_B T_P per degree of freedom."""
    P, N, T = 8, 16, 200.0
    sysm = _harmonic_system(P, N, T=T, omega=0.0, dt=1.0, gamma0=0.02)
    xb = sysm.beads()
    for j in range(P):
        np.testing.assert_allclose(xb[j], xb[0], atol=1e-13)
    tk = []
    for _ in range(400):
        sysm.step(5)
        tk.append(sysm.estimators()["T_kin"])
    tk = np.array(tk[40:])
    assert abs(tk.mean() / (P * T) - 1.0) < 0.02


def _qho_exact_EP(P, T, omega):
    """<E_P> of a 3D oscillator with P beads (Sec. S1, with the square of the
    bracket restored): 3 k_B T sum_l 1 / (1 + [(2 P k_B T / hbar w) sin(l pi / P)]^2)."""
    kT = KB * T
    return 3 * kT * sum(1.0 / (1.0 + ((2 * P * kT / (HBAR * omega)) * math.sin(l * math.pi / P)) ** 2)
                        for l in range(1, P + 1))


def _block_mean(x, nblock=20):
    x = np.asarray(x)
    n = len(x) // nblock
    b = x[: n * nblock].reshape(nblock, n).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nblock)


def test_qho_closed_form_limits():
    w, T = 0.0786, 300.0
    kT = KB * T
    assert abs(_qho_exact_EP(1, T, w) - 3 * kT) < 1e-15
    big = _qho_exact_EP(4096, T, w)
    exact = 3 * 0.5 * HBAR * w / math.tanh(HBAR * w / (2 * kT))
    assert abs(big / exact - 1) < 1e-5


@pytest.mark.parametrize("P", [1, 4, 16])
def test_qho_thermostatted_averages_match_closed_form(P):
    """Harmonic oscillator (hbar w / k_B T ~ 2): PILE-L averages of the
    virial and primitive estimators against the P-bead closed form."""
    T, w, N = 300.0, 0.0786, 8
    sysm = _harmonic_system(P, N, T=T, omega=w, dt=0.25, gamma0=0.08)
    sysm.step(2000)
    Ev, Kp, Kc, x2 = [], [], [], []
    m = s.MASS[s.H]
    for _ in range(6000):
        sysm.step(10)
        e = sysm.estimators()
        Ev.append(e["E_tot"] / N)
        Kp.append(e["K_prim"] / N)
        Kc.append(e["K_cv"] / N)
        x2.append((sysm.beads() ** 2).sum(axis=2).mean())
    exact = _qho_exact_EP(P, T, w)
    mean, err = _block_mean(Ev)
    assert abs(mean - exact) < 4 * err + 0.004 * exact, (mean, err, exact)
    mk, ek = _block_mean(Kc)
    assert abs(mk - exact / 2) < 4 * ek + 0.004 * exact
    mp, ep = _block_mean(Kp)
    assert abs(mp - exact / 2) < 4 * ep + 0.004 * exact
    # <|x|^2> per atom = 3 / (beta m) sum_k 1 / (w^2 + w_k^2)
    wP = P * KB * T / HBAR
    wk = 2 * wP * np.sin(np.arange(P) * np.pi / P)
    x2_exact = 3 * (KB * T / MVV2E) / m * np.sum(1.0 / (w * w + wk ** 2))
    mx, ex = _block_mean(x2)
    assert abs(mx - x2_exact) < 4 * ex + 0.004 * x2_exact


def test_nve_energy_conservation(fad_model):
    """No thermostat: the ring-polymer Hamiltonian H_P shows no drift and its
    fluctuation scales as dt^2 (symplectic splitting)."""
    w, r, m = fad_model
    amp = []
    for dt in (0.1, 0.05):
        rep = s.Replica(r.Z, r.x0, r.box, 4, 300.0, r.seed)
        sysm = O.System(rep, s.MASS, dt, 0.0, model=m, thermostat=False)
        H = []
        nst = int(round(10.0 / dt))
        for _ in range(nst):
            sysm.step(1)
            H.append(sysm.estimators()["H_cons"])
        H = np.array(H)
        t = np.arange(len(H))
        slope = np.polyfit(t, H, 1)[0]
        amp.append(H.std())
        assert abs(slope * len(H)) < 3 * H.std() + 1e-12
    ratio = amp[0] / amp[1]
    assert 2.5 < ratio < 6.0, amp


# ---------------------------------------------------------------- integrator variants
@pytest.mark.parametrize("m,w,h", [(1.008, 0.3, 0.25), (15.999, 2.0, 0.5), (1.008, 400.0, 0.5)])
def test_cayley_free_rp_step_is_a_rotation(m, w, h):
    """The Cayley transform of h L (L = [[0, -m w^2], [1/m, 0]]) has the
    eigenvalues (1 + i w h / 2) / (1 - i w h / 2) = exp(+-i theta) with
    tan(theta / 2) = w h / 2: from (p, q) = (0, 1) one step gives
    q = cos theta, p = -m w sin theta; the mode energy p^2/2m + m w^2 q^2/2 is
    conserved for any w h, and a step of -h undoes a step of h."""
    th = 2.0 * math.atan(0.5 * w * h)
    p, q = O.free_rp_step("cayley", m, w, h, 0.0, 1.0)
    assert abs(q - math.cos(th)) < 1e-13
    assert abs(p + m * w * math.sin(th)) < 1e-13 * m * w
    p0, q0 = 0.7, -0.3

    def energy(p, q):
        return p * p / (2 * m) + 0.5 * m * w * w * q * q

    p1, q1 = O.free_rp_step("cayley", m, w, h, p0, q0)
    assert abs(energy(p1, q1) - energy(p0, q0)) < 1e-13 * energy(p0, q0)
    p2, q2 = O.free_rp_step("cayley", m, w, -h, p1, q1)
    assert abs(p2 - p0) < 1e-12 * max(1.0, m * w) and abs(q2 - q0) < 1e-12


def test_cayley_free_rp_step_is_second_order_accurate():
    """Local error against the exact rotation is O(h^3): halving h divides it
    by ~8 (theta - w h = -(w h)^3 / 12 + ...)."""
    m, w = 1.008, 0.8
    errs = []
    for h in (0.2, 0.1, 0.05):
        pe, qe = O.free_rp_step("exact", m, w, h, 0.4, 0.9)
        pc, qc = O.free_rp_step("cayley", m, w, h, 0.4, 0.9)
        errs.append(abs(qc - qe) + abs(pc - pe) / (m * w))
    assert 7.5 < errs[0] / errs[1] < 8.5 and 7.5 < errs[1] / errs[2] < 8.5
    # free drift of the centroid is the same for both
    assert O.free_rp_step("cayley", m, 0.0, 0.3, 0.5, 1.0) == O.free_rp_step("exact", m, 0.0, 0.3, 0.5, 1.0)


def test_baoab_without_thermostat_is_obabo(fad_model):
    """With the thermostat off both splittings are velocity Verlet: B A(dt/2)
    A(dt/2) B equals B A(dt) B because the exact free ring-polymer flow
    composes."""
    w, r, m = fad_model
    rep = s.Replica(r.Z, r.x0, r.box, 4, r.T, r.seed, r.name)
    a = O.System(rep, s.MASS, 0.25, 0.0, model=m, thermostat=False, splitting="obabo")
    b = O.System(rep, s.MASS, 0.25, 0.0, model=m, thermostat=False, splitting="baoab")
    a.step(20)
    b.step(20)
    assert np.abs(a.q - b.q).max() < 1e-10 * np.abs(a.q).max()
    assert np.abs(a.p - b.p).max() < 1e-10 * np.abs(a.p).max()


@pytest.mark.parametrize("splitting,free_rp", [("baoab", "exact"), ("obabo", "cayley"), ("baoab", "cayley")])
def test_qho_averages_with_other_integrators(splitting, free_rp):
    """The P = 4 oscillator averages of the closed form hold for BAOAB and
    for the Cayley propagator too (within sampling error + O(dt^2))."""
    P, T, w, N = 4, 300.0, 0.0786, 8
    sysm = _harmonic_system(P, N, T=T, omega=w, dt=0.25, gamma0=0.08, splitting=splitting, free_rp=free_rp)
    sysm.step(2000)
    Ev, x2 = [], []
    for _ in range(6000):
        sysm.step(10)
        Ev.append(sysm.estimators()["E_tot"] / N)
        x2.append((sysm.beads() ** 2).sum(axis=2).mean())
    exact = _qho_exact_EP(P, T, w)
    mean, err = _block_mean(Ev)
    assert abs(mean - exact) < 4 * err + 0.004 * exact, (mean, err, exact)
    m = s.MASS[s.H]
    wP = P * KB * T / HBAR
    wk = 2 * wP * np.sin(np.arange(P) * np.pi / P)
    x2_exact = 3 * (KB * T / MVV2E) / m * np.sum(1.0 / (w * w + wk ** 2))
    mx, ex = _block_mean(x2)
    assert abs(mx - x2_exact) < 4 * ex + 0.004 * x2_exact


# ---------------------------------------------------------------- staging transform
def test_staging_round_trip_and_spring_identity():
    """u -> x -> u is the identity, and the ring's spring energy
    sum_k (x_k - x_(k+1))^2 equals sum_(k>=2) k/(k-1) u_k^2 (the staging
    masses m_k' = k/(k-1) m)."""
    rng = np.random.default_rng(12)
    for P in (1, 2, 5, 32):
        x = rng.normal(size=(P, 3, 3))
        u = O.beads_to_staging(x)
        assert np.abs(O.staging_to_beads(u) - x).max() < 1e-13
        spring = ((x - np.roll(x, -1, axis=0)) ** 2).sum()
        k = np.arange(1, P + 1, dtype=float)
        fac = np.where(k >= 2, k / np.maximum(k - 1, 1), 0.0)
        assert abs(spring - (fac[:, None, None] * u ** 2).sum()) < 1e-12 * max(1.0, spring)
        assert np.abs(u[0] - x[0]).max() == 0.0


def test_staging_forces_are_minus_gradients():
    """-dPhi/du from the force recursion equals a finite difference of
    Phi(x(u)) for a random quadratic bead potential."""
    rng = np.random.default_rng(3)
    P = 7
    A = rng.normal(size=(P, P))
    A = A @ A.T
    c = rng.normal(size=P)

    def beads(u):
        u3 = np.zeros((P, 1, 3))
        u3[:, 0, 0] = u
        return O.staging_to_beads(u3)[:, 0, 0]

    def phi_of_u(u):
        x = beads(u)
        return 0.5 * x @ A @ x + c @ x

    u = rng.normal(size=P)
    x = beads(u)
    f = -(A @ x + c)
    Fu = O.staging_forces(f)
    h = 1e-6
    for k in range(P):
        up, um = u.copy(), u.copy()
        up[k] += h
        um[k] -= h
        fd = -(phi_of_u(up) - phi_of_u(um)) / (2 * h)
        assert abs(fd - Fu[k]) < 1e-6 * max(1.0, abs(Fu).max()), k


@pytest.mark.parametrize("P", [4, 16])
def test_qho_averages_with_staging(P):
    """Staging coordinates (masses k/(k-1) m, exact propagation at w_P)
    sample the same P-bead oscillator: closed-form <E_P> and <|x|^2>."""
    T, w, N = 300.0, 0.0786, 8
    x0 = np.random.default_rng(5).normal(size=(N, 3)) * 0.1
    rep = s.Replica(np.full(N, s.H, dtype=np.int32), x0, (0.0, 0.0, 0.0), P, T, 5)
    sysm = O.System(rep, s.MASS, 0.25, 0.08, potential="harmonic", omega=w, transform="staging")
    sysm.step(2000)
    Ev, x2 = [], []
    for _ in range(6000):
        sysm.step(10)
        Ev.append(sysm.estimators()["E_tot"] / N)
        x2.append((sysm.beads() ** 2).sum(axis=2).mean())
    exact = _qho_exact_EP(P, T, w)
    mean, err = _block_mean(Ev)
    assert abs(mean - exact) < 4 * err + 0.004 * exact, (mean, err, exact)
    m = s.MASS[s.H]
    wP = P * KB * T / HBAR
    wk = 2 * wP * np.sin(np.arange(P) * np.pi / P)
    x2_exact = 3 * (KB * T / MVV2E) / m * np.sum(1.0 / (w * w + wk ** 2))
    mx, ex = _block_mean(x2)
    assert abs(mx - x2_exact) < 4 * ex + 0.004 * x2_exact


def test_staging_nve_energy_conservation():
    """Staging NVE on oscillators (P = 4, 200 fs): no drift of H_P and
    fluctuations that scale as dt^2. (In staging coordinates u_1 carries the
    whole ring's force on one bead's mass, so its motion is sqrt(P) faster
    than a bead's; the random-init network's steep regions make FAD runs a
    poor conservation probe at these steps.)"""
    amp = []
    x0 = np.random.default_rng(5).normal(size=(3, 3)) * 0.1
    for dt in (0.1, 0.05):
        rep = s.Replica(np.full(3, s.H, dtype=np.int32), x0, (0.0, 0.0, 0.0), 4, 300.0, 5)
        sysm = O.System(rep, s.MASS, dt, 0.0, potential="harmonic", omega=0.0786, thermostat=False,
                        transform="staging")
        H = []
        for _ in range(int(round(200.0 / dt))):
            sysm.step(1)
            H.append(sysm.estimators()["H_cons"])
        H = np.array(H)
        slope = np.polyfit(np.arange(len(H)), H, 1)[0]
        amp.append(H.std())
        assert abs(slope * len(H)) < 3 * H.std() + 1e-12
    assert 2.5 < amp[0] / amp[1] < 6.0, amp


# ---------------------------------------------------------------- thermostat heat
def _free_ring_energy(sysm, transform):
    """H_P of a ring polymer with V = 0, from the state arrays alone: the
    kinetic energy of every coordinate plus the spring energy. Normal modes:
    masses m, spring sum_k m w_k^2 q_k^2 / 2 (w_k = 2 w_P sin(k pi / P));
    staging: masses m'_1 = m, m'_k = k / (k - 1) m, spring
    sum_(k>=2) m'_k w_P^2 u_k^2 / 2 (the spring identity pinned above)."""
    P, N = sysm.P, sysm.N
    m = sysm.mass[None, :, None]
    wP = P * KB * sysm.s.T / HBAR
    if transform == "staging":
        k = np.arange(1, P + 1, dtype=float)
        fac = np.where(k >= 2, k / np.maximum(k - 1, 1), 1.0)[:, None, None]
        mk = fac * m
        w2 = np.where(k >= 2, wP * wP, 0.0)[:, None, None]
    else:
        mk = np.broadcast_to(m, (P, N, 1))
        w2 = (2 * wP * np.sin(np.arange(P) * np.pi / P))[:, None, None] ** 2
    kin = (sysm.p ** 2 / (2 * mk)).sum()
    spring = (0.5 * mk * w2 * sysm.q ** 2).sum()
    return (kin + spring) * MVV2E


@pytest.mark.parametrize("P,splitting,free_rp,transform", [
    (1, "obabo", "exact", "normal_modes"), (8, "obabo", "exact", "normal_modes"),
    (5, "baoab", "exact", "normal_modes"), (8, "obabo", "cayley", "normal_modes"),
    (6, "obabo", "exact", "staging")])
def test_thermostat_heat_is_the_kinetic_energy_change_of_the_O_steps(P, splitting, free_rp, transform):
    """Sec. 2.1 (H_eff) with PILE-L on (Tables S2-S3): with V = 0 the B steps
    do nothing and the free ring-polymer A step conserves each mode's energy
    exactly (the exact rotation and the Cayley rotation alike), so the
    ring-polymer energy H_P changes only in the O steps. The accumulated heat
    Q_thermo must therefore equal H_P(now) - H_P(start), with H_P computed
    here from q and p, and H_cons = H_P - Q_thermo must stay at its initial
    value. A sign or factor error in the heat, a dropped O step or the wrong
    mode mass each break it."""
    N, T = 5, 300.0
    x0 = np.random.default_rng(9).normal(size=(N, 3)) * 0.1
    Z = np.array([s.H, s.O, s.C, s.H, s.O], dtype=np.int32)
    rep = s.Replica(Z, x0, (0.0, 0.0, 0.0), P, T, 17)
    sysm = O.System(rep, s.MASS, 0.5, 0.05, potential="harmonic", omega=0.0, splitting=splitting,
                    free_rp=free_rp, transform=transform)
    H0 = _free_ring_energy(sysm, transform)
    Hc0 = sysm.estimators()["H_cons"]
    assert abs(Hc0 - H0) < 1e-12 * max(1.0, abs(H0))
    for _ in range(6):
        sysm.step(7)
        e = sysm.estimators()
        dH = _free_ring_energy(sysm, transform) - H0
        assert abs(e["Q_thermo"]) > 1e-3          # the thermostat did move energy
        assert abs(e["Q_thermo"] - dH) < 1e-10 * max(1.0, abs(dH))
        assert abs(e["H_cons"] - H0) < 1e-10 * max(1.0, abs(H0))


def test_conserved_energy_with_pile_l_on(fad_model):
    """FAD, P = 4, PILE-L on: H_P itself fluctuates with the heat the
    thermostat exchanges, but H_cons = H_P - Q_thermo shows no drift and its
    fluctuation is the integrator's O(dt^2) error (pooled over three noise
    seeds, halving dt divides it by ~4). H_P + Q_thermo (a sign error in the
    heat) fluctuates a thousand times more."""
    w, r, m = fad_model
    amp = {0.1: [], 0.05: []}
    for seed in (1, 2, 3):
        for dt in (0.1, 0.05):
            rep = s.Replica(r.Z, r.x0, r.box, 4, 300.0, seed)
            sysm = O.System(rep, s.MASS, dt, 0.01, model=m, thermostat=True)
            H, Hw = [], []
            for _ in range(int(round(10.0 / dt))):
                sysm.step(1)
                e = sysm.estimators()
                H.append(e["H_cons"])
                Hw.append(e["H_cons"] + 2.0 * e["Q_thermo"])
            H, Hw = np.array(H), np.array(Hw)
            slope = np.polyfit(np.arange(len(H)), H, 1)[0]
            assert abs(slope * len(H)) < 4 * H.std() + 1e-12
            assert H.std() < 0.01 * Hw.std()
            amp[dt].append(H.std())
    ratio = np.mean(amp[0.1]) / np.mean(amp[0.05])
    assert 2.5 < ratio < 8.0, amp
