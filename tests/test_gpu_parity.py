"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Bars: neighbour lists bit-exact; FP32 path forces within 1e-5 relative
max-norm; FP64 path within 1e-10; trajectories over <= 10 steps with the same
Philox noise."""
import numpy as np
import pytest

import oracle as O
from paper_2503_23728_gb300 import synth as s

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _P():
    import __graft_entry__ as ge
    ge.build()
    from paper_2503_23728_gb300 import pimd as P
    return P


def _relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _bead_positions(rep, P, seed, sigma=0.08, f32=True):
    rng = np.random.default_rng(seed)
    x = np.repeat(rep.x0[None], P, axis=0) + rng.normal(scale=sigma, size=(P, rep.n_atoms, 3))
    if f32:
        x = x.astype(np.float32).astype(np.float64)
    return x


def _with_beads(rep, P):
    return s.Replica(rep.Z, rep.x0, rep.box, P, rep.T, rep.seed, rep.name)


# ---------------------------------------------------------------- water-64, FP32
@pytest.fixture(scope="module")
def water_fp32(water64_model):
    P = _P()
    w, r, m = water64_model
    rep = _with_beads(r, 7)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    ctx.set_weights(m)
    xb = _bead_positions(rep, 7, seed=17)
    return P, w, rep, m, ctx, xb


def test_neighbours_bit_exact(water_fp32):
    P, w, rep, m, ctx, xb = water_fp32
    ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    nnb, nbr = ctx.neighbours()
    for k in range(rep.n_beads):
        want, _, _ = O.neighbours(xb[k], rep.box, 6.0)
        for i in range(rep.n_atoms):
            b = k * rep.n_atoms + i
            got = nbr[b, :nnb[b]]
            assert np.array_equal(np.sort(got), want[i]), (k, i)


def test_descriptors_fp32(water_fp32):
    P, w, rep, m, ctx, xb = water_fp32
    G = ctx.descriptors(torch.tensor(xb.reshape(-1, 3), device="cuda")).cpu().numpy()
    for k in range(rep.n_beads):
        Go = O.descriptors(m, xb[k], rep.box)
        Gg = G[k * rep.n_atoms:(k + 1) * rep.n_atoms]
        scale = np.abs(Go).max(axis=0) + 1e-30
        assert np.all(np.abs(Gg - Go) <= 1e-5 * scale), k


def test_energy_forces_virial_fp32(water_fp32):
    P, w, rep, m, ctx, xb = water_fp32
    e, f, v = ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    e, f, v = e.cpu().numpy(), f.cpu().numpy().reshape(rep.n_beads, rep.n_atoms, 3), v.cpu().numpy()
    Eo, Fo, Wo = O.energy_forces_batch(m, rep.Z, xb, rep.box)
    assert _relmax(f, Fo) < 1e-5
    assert np.abs(e - Eo.sum(axis=1)).max() / rep.n_atoms < 1e-5
    assert _relmax(v, Wo) < 1e-5
    # translation invariance of the GPU forces
    assert np.abs(f.sum(axis=1)).max() < 1e-4 * np.abs(f).max()


# ---------------------------------------------------------------- FAD, FP64
@pytest.fixture(scope="module")
def fad_fp64(fad_model):
    P = _P()
    w, r, m = fad_model
    ctx = P.Context([r], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths)
    ctx.set_weights(m)
    return P, w, r, m, ctx


def test_energy_forces_fp64(fad_fp64):
    P, w, rep, m, ctx = fad_fp64
    xb = _bead_positions(rep, rep.n_beads, seed=3, sigma=0.1, f32=False)
    e, f, v = ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    e, f, v = e.cpu().numpy(), f.cpu().numpy().reshape(rep.n_beads, rep.n_atoms, 3), v.cpu().numpy()
    Eo, Fo, Wo = O.energy_forces_batch(m, rep.Z, xb, None)
    assert _relmax(f, Fo) < 1e-10
    assert np.abs(e - Eo.sum(axis=1)).max() < 1e-10 * np.abs(Eo.sum(axis=1)).max()
    assert _relmax(v, Wo) < 1e-10


def test_trajectory_fp64_matches_oracle(fad_model):
    """Config-1 shape (FAD, P = 16, 0.25 fs, PILE-L): 10 GPU steps against 10
    oracle steps with the same Philox noise."""
    P = _P()
    w, rep, m = fad_model
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths)
    ctx.set_weights(m)
    q0, p0, st0, _ = ctx.get_state()
    so = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m)
    np.testing.assert_allclose(q0.reshape(so.q.shape), so.q, rtol=0, atol=1e-12)
    np.testing.assert_allclose(p0.reshape(so.p.shape), so.p, rtol=1e-12, atol=1e-14)
    ctx.step(10)
    so.step(10)
    q, p, st, Q = ctx.get_state()
    assert st == 10
    np.testing.assert_allclose(q.reshape(so.q.shape), so.q, rtol=0, atol=1e-9)
    np.testing.assert_allclose(p.reshape(so.p.shape), so.p, rtol=0, atol=1e-9 * np.abs(so.p).max())
    eg = ctx.estimators()[0]
    eo = so.estimators()
    for k in ("V_mean", "K_prim", "K_cv", "E_tot", "H_cons", "Q_thermo", "T_kin"):
        assert abs(eg[k] - eo[k]) <= 1e-8 * max(1.0, abs(eo[k])), k
    np.testing.assert_allclose(eg["W"], eo["W"], atol=1e-8 * np.abs(eo["W"]).max())


def test_trajectory_fp32_matches_oracle(water64_model):
    """Water-64 (P = 4): 5 steps on the FP32 path against the FP64 oracle."""
    P = _P()
    w, r, m = water64_model
    rep = _with_beads(r, 4)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    ctx.set_weights(m)
    so = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m)
    ctx.step(5)
    so.step(5)
    q, p, _, _ = ctx.get_state()
    np.testing.assert_allclose(q.reshape(so.q.shape), so.q, rtol=0, atol=2e-5)
    assert _relmax(p.reshape(so.p.shape), so.p) < 1e-4
    eg, eo = ctx.estimators()[0], so.estimators()
    for k in ("V_mean", "K_cv", "E_tot"):
        assert abs(eg[k] - eo[k]) <= 1e-4 * max(1.0, abs(eo[k])), k


# ---------------------------------------------------------------- harmonic oscillator
def test_qho_gpu_matches_closed_form():
    """Sec. S1 check on the GPU integrator: 3D oscillators with P = 8 beads,
    PILE-L, FP64; <E> of the virial estimator vs the P-bead closed form."""
    P = _P()
    KB, HBAR = 8.617333262e-5, 0.6582119569
    T, wq, N, Pb = 300.0, 0.0786, 256, 8
    x0 = np.random.default_rng(1).normal(size=(N, 3)) * 0.1
    rep = s.Replica(np.full(N, s.H, dtype=np.int32), x0, (0.0, 0.0, 0.0), Pb, T, 99)
    ctx = P.Context([rep], 0.25, 0.08, precision="fp64", potential=P.POT_HARMONIC, omega=wq)
    ctx.step(2000)
    E = []
    for _ in range(1500):
        ctx.step(10)
        E.append(ctx.estimators()[0]["E_tot"] / N)
    E = np.array(E)
    kT = KB * T
    exact = 3 * kT * sum(1.0 / (1.0 + ((2 * Pb * kT / (HBAR * wq)) * np.sin(l * np.pi / Pb)) ** 2)
                         for l in range(1, Pb + 1))
    blocks = E[: len(E) // 15 * 15].reshape(15, -1).mean(axis=1)
    err = blocks.std(ddof=1) / np.sqrt(len(blocks))
    assert abs(E.mean() - exact) < 4 * err + 0.004 * exact, (E.mean(), err, exact)


# ---------------------------------------------------------------- state, errors
def test_checkpoint_resume(water64_model):
    """A run resumed from get_state/set_state follows the uninterrupted run.
    Force accumulation uses atomics, so the two agree to round-off (FP32
    path: 1e-5 relative) rather than bit for bit."""
    P = _P()
    w, r, m = water64_model
    rep = _with_beads(r, 4)
    a = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    a.set_weights(m)
    a.step(3)
    q, p, st, Q = a.get_state()
    a.step(4)
    qa, pa, sa, Qa = a.get_state()
    b = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    b.set_weights(m)
    b.set_state(q, p, st, Q)
    b.step(4)
    qb, pb, sb, Qb = b.get_state()
    assert sa == sb == 7
    np.testing.assert_allclose(qb, qa, rtol=0, atol=1e-5)
    assert _relmax(pb, pa) < 1e-5
    np.testing.assert_allclose(Qb, Qa, rtol=1e-6, atol=1e-9)


def test_neighbour_overflow_is_reported(water64_model):
    P = _P()
    w, r, m = water64_model
    ctx = P.Context([_with_beads(r, 2)], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths,
                    max_neighbours=32)
    with pytest.raises(P.PimdError) as ei:
        ctx.set_weights(m)
    assert ei.value.code == -7


def test_autograd_energy(water_fp32):
    """The torch.autograd.Function's backward (the adjoint kernel) against the
    oracle's analytic gradient: x.grad of sum_k c_k e_k equals -c_k F_k with
    F the FP64 oracle's forces on the same FP32 bead positions (1e-5
    relative max-norm), and the forward's energies equal the oracle's."""
    P, w, rep, m, ctx, xb = water_fp32
    x = torch.tensor(xb.reshape(-1, 3), device="cuda", requires_grad=True)
    e = P.pimd_energy(x, ctx)
    coef = torch.linspace(0.5, 1.5, e.shape[0], device="cuda", dtype=torch.float64)
    (e * coef).sum().backward()
    Eo, Fo, _ = O.energy_forces_batch(m, rep.Z, xb, rep.box)
    c = coef.cpu().numpy()
    want = -(c[:, None, None] * Fo)
    got = x.grad.cpu().numpy().reshape(want.shape)
    assert _relmax(got, want) < 1e-5
    assert np.abs(e.detach().cpu().numpy() - Eo.sum(axis=1)).max() / rep.n_atoms < 1e-5


def test_energy_central_differences_fp32(water64_model):
    """Config 2's finite-difference check on the GPU: central differences of
    the FP32 path's energy (through pimd_energy) for 8 random atoms of
    water-64 against the oracle's analytic forces. The step is the FP32
    rounding of x +- h, h = 2e-3 A; the FP32 energy's rounding (~1e-6 eV)
    over 2h bounds the error at ~1e-3 of the force scale."""
    P = _P()
    w, r, m = water64_model
    rep = _with_beads(r, 1)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    ctx.set_weights(m)
    x0 = _bead_positions(rep, 1, seed=29)[0]
    _, Fo, _ = O.energy_forces(m, rep.Z, x0, rep.box)
    atoms = np.random.default_rng(31).choice(rep.n_atoms, size=8, replace=False)
    h = 2e-3
    fd = np.zeros((8, 3))
    for a, i in enumerate(atoms):
        for d in range(3):
            xp, xm = x0.copy(), x0.copy()
            xp[i, d] = np.float32(x0[i, d] + h)
            xm[i, d] = np.float32(x0[i, d] - h)
            with torch.no_grad():
                ep = P.pimd_energy(torch.tensor(xp, device="cuda"), ctx).item()
                em = P.pimd_energy(torch.tensor(xm, device="cuda"), ctx).item()
            fd[a, d] = -(ep - em) / (xp[i, d] - xm[i, d])
    assert np.abs(fd - Fo[atoms]).max() < 3e-3 * np.abs(Fo).max()


# ---------------------------------------------------------------- uneven replicas
def test_uneven_replicas_fp32():
    P = _P()
    reps = s.batch(n_rep=6, seed=77, beads=(3, 5, 8))
    m = s.xavier_model(s.elements_of(reps), (64, 64), seed=4)
    G = np.concatenate([O.descriptors(m, r.x0, None) for r in reps])
    Z = np.concatenate([r.Z for r in reps])
    s.set_normalisation(m, G, Z)
    ctx = P.Context(reps, 0.25, 0.01, precision="fp32", widths=(64, 64))
    ctx.set_weights(m)
    xs = [_bead_positions(r, r.n_beads, seed=10 + k, sigma=0.05) for k, r in enumerate(reps)]
    e, f, _ = ctx.energy_forces(torch.tensor(np.concatenate([x.reshape(-1, 3) for x in xs]), device="cuda"))
    e, f = e.cpu().numpy(), f.cpu().numpy()
    b0 = s0 = 0
    for r, x in zip(reps, xs):
        Eo, Fo, _ = O.energy_forces_batch(m, r.Z, x, None)
        n = r.n_atoms * r.n_beads
        assert _relmax(f[b0:b0 + n].reshape(Fo.shape), Fo) < 1e-5
        assert np.abs(e[s0:s0 + r.n_beads] - Eo.sum(axis=1)).max() < 1e-5 * r.n_atoms
        b0 += n
        s0 += r.n_beads
    ctx.step(5)
    est = ctx.estimators()
    assert len(est) == len(reps) and all(np.isfinite(x["E_tot"]) for x in est)


def test_cell_lists_equal_all_pairs():
    """Ice (4 x 3 x 3 cells per bead, cells forced): cell-list neighbour lists
    are the same arrays as the all-pairs scan, and the forces agree."""
    P = _P()
    w = s.workload("ice")
    r = w.replicas[0]
    rep = _with_beads(r, 3)
    m = s.xavier_model(s.elements_of([rep]), w.widths, seed=2)
    G = O.descriptors(m, rep.x0, rep.box)
    s.set_normalisation(m, G, rep.Z)
    xb = _bead_positions(rep, 3, seed=9, sigma=0.3)
    out = []
    for algo in (2, 1):
        ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths, nbr_algo=algo)
        ctx.set_weights(m)
        _, f, _ = ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
        nnb, nbr = ctx.neighbours()
        out.append((nnb, nbr, f.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0])
    for b in range(len(out[0][0])):
        n = out[0][0][b]
        assert np.array_equal(out[0][1][b, :n], out[1][1][b, :n])
    assert _relmax(out[0][2], out[1][2]) < 1e-6
    want, _, _ = O.neighbours(xb[1], rep.box, 6.0)
    for i in range(0, rep.n_atoms, 5):
        b = rep.n_atoms + i
        assert np.array_equal(out[0][1][b, :out[0][0][b]], want[i])


@pytest.mark.parametrize("band", [0, 1, 4, 7, 12, 16])
def test_every_pair_schedule_matches_oracle(water_fp32, band):
    """The descriptor / adjoint pair schedules (flat walk, bands of 1..16
    with shuffle carries) all give the oracle's forces."""
    P, w, rep, m, ctx, xb = water_fp32
    ctx.set_angular("pairs")
    ctx.set_schedule(band)
    try:
        e, f, _ = ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
        Eo, Fo, _ = O.energy_forces_batch(m, rep.Z, xb, rep.box)
        assert _relmax(f.cpu().numpy().reshape(Fo.shape), Fo) < 1e-5
        assert np.abs(e.cpu().numpy() - Eo.sum(axis=1)).max() / rep.n_atoms < 1e-5
    finally:
        ctx.set_schedule(8)
        ctx.set_angular("moments")


def test_tuner_keeps_forces_correct(water64_model):
    P = _P()
    w, r, m = water64_model
    rep = _with_beads(r, 4)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    ctx.set_weights(m)
    res = ctx.tune(reps=2)
    assert res["best_ms"] > 0 and res["best_ms"] <= res["default_ms"] + 1e-9
    assert res["band_length"] in (0, 4, 6, 8, 10, 12, 16)
    assert res["angular"] in ("pairs", "moments") and ctx.angular == res["angular"]
    xb = _bead_positions(rep, 4, seed=31)
    _, f, _ = ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    _, Fo, _ = O.energy_forces_batch(m, rep.Z, xb, rep.box)
    assert _relmax(f.cpu().numpy().reshape(Fo.shape), Fo) < 1e-5
    ctx.step(3)
    assert np.isfinite(ctx.estimators()[0]["E_tot"])


def test_nonfinite_forces_are_reported(water64_model):
    """Two atoms on top of each other give non-finite forces; the library
    reports NONFINITE at the next synchronising call instead of faulting, and
    a fresh context on valid input works afterwards."""
    P = _P()
    w, r, m = water64_model
    x0 = r.x0.copy()
    x0[5] = x0[4]
    bad = s.Replica(r.Z, x0, r.box, 2, r.T, r.seed)
    ctx = P.Context([bad], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    with pytest.raises(P.PimdError) as ei:
        ctx.set_weights(m)
    assert ei.value.code == -5
    ctx.close()
    ok = P.Context([_with_beads(r, 2)], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    ok.set_weights(m)
    ok.step(2)
    assert np.isfinite(ok.estimators()[0]["E_tot"])


@pytest.mark.parametrize("which", ["water", "water-pairs", "fad"])
def test_deterministic_mode_resume_is_bit_identical(water64_model, fad_model, which):
    """deterministic = 1: forces summed in a fixed order (pair vectors
    gathered per atom; ordered pairs for small neighbour counts), virial and
    thermostat heat reduced in fixed order, so a resumed run reproduces the
    uninterrupted one bit for bit, and matches the oracle."""
    P = _P()
    w, r, m = fad_model if which == "fad" else water64_model
    rep = _with_beads(r, 4)

    def ctx():
        c = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths, deterministic=True)
        if which == "water-pairs":
            c.set_angular("pairs")
        c.set_weights(m)
        return c

    a = ctx()
    a.step(3)
    q, p, st, Q = a.get_state()
    a.step(4)
    qa, pa, sa, Qa = a.get_state()
    b = ctx()
    b.set_state(q, p, st, Q)
    b.step(4)
    qb, pb, sb, Qb = b.get_state()
    assert sa == sb == 7
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb) and np.array_equal(Qa, Qb)
    xb = _bead_positions(rep, 4, seed=5)
    _, f, _ = b.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    _, Fo, _ = O.energy_forces_batch(m, rep.Z, xb, rep.box)
    assert _relmax(f.cpu().numpy().reshape(Fo.shape), Fo) < 1e-5
    assert b.kernels_per_step() == 9


# ---------------------------------------------------------------- Verlet candidates
@pytest.mark.parametrize("which,skin,precision", [("ice", 0.5, "fp32"), ("ice", 0.08, "fp32"), ("water", -1.0, "fp32"),
                                                  ("ice", 1.5, "bf16_tc"), ("water", -1.0, "bf16_tc")])
def test_verlet_candidates_give_the_same_lists_and_trajectory(water64_model, ice_model, which, skin, precision):
    """Neighbour lists filtered from Verlet candidates (rebuilt when an atom
    has moved by half the skin) equal a full rebuild every step: deterministic
    trajectories with and without the skin are bit-identical, and the lists
    match the oracle's at the end. On the BF16 moment path the descriptor
    forward filters the candidates itself."""
    P = _P()
    w, r, m = ice_model if which == "ice" else water64_model
    rep = _with_beads(r, 4)
    out = []
    for sk in (skin, 0.0):
        ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision=precision, widths=w.widths, deterministic=True,
                        nbr_skin=sk)
        ctx.set_weights(m)
        ctx.step(40)
        q, p_, st, Q = ctx.get_state()
        nnb, nbr = ctx.neighbours()
        out.append((q, p_, nnb, nbr))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
    for b in range(len(out[0][2])):
        n = out[0][2][b]
        assert np.array_equal(out[0][3][b, :n], out[1][3][b, :n])


@pytest.mark.parametrize("precision", ["fp32", "bf16_tc"])
def test_verlet_candidate_overflow_falls_back(ice_model, precision):
    """Candidate slots too few for r_c + skin (ice, 96 neighbour slots, 144
    candidate slots, skin 1.2 A: ~149 candidates): the affected atoms scan
    directly, lists still exact (on the BF16 moment path the forward filters
    the candidates of the other atoms)."""
    P = _P()
    w, r, m = ice_model
    rep = _with_beads(r, 2)
    xb = _bead_positions(rep, 2, seed=41)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision=precision, widths=w.widths, max_neighbours=96,
                    nbr_skin=1.2)
    ctx.set_weights(m)
    ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    nnb, nbr = ctx.neighbours()
    for k in range(2):
        want, _, _ = O.neighbours(xb[k], rep.box, 6.0)
        for i in range(rep.n_atoms):
            b = k * rep.n_atoms + i
            assert np.array_equal(nbr[b, :nnb[b]], want[i]), (k, i)


def test_bounded_wait_times_out_and_gpu_stays_usable(water64_model):
    """A spin wait on a barrier that nothing completes gives up at its bound
    and reports TIMEOUT; the device keeps working afterwards."""
    P = _P()
    assert P.pimd_selftest_bounded_wait(0.2) == -6
    assert "bounded wait expired" in P.pimd_last_error()
    w, r, m = water64_model
    ctx = P.Context([_with_beads(r, 2)], w.dt_fs, w.gamma0_per_fs, precision="bf16_tc", widths=w.widths)
    ctx.set_weights(m)
    ctx.step(2)
    assert np.isfinite(ctx.estimators()[0]["E_tot"])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16_tc"])
def test_small_bead_neighbours_bit_exact(fad_model, precision):
    """Contexts whose beads all have at most 32 atoms (no cells, no Verlet
    candidates) build their lists with one warp per bead: the lists equal
    the oracle's exact FP32 rule for a gas-phase replica (FAD, 10 atoms) and
    a periodic one (24 atoms in a 12.5 A box, minimum images)."""
    P = _P()
    w, r, m = fad_model
    gas = _with_beads(r, 3)
    rng = np.random.default_rng(5)
    grid = np.stack(np.meshgrid(np.arange(3), np.arange(2), np.arange(4), indexing="ij"), -1).reshape(-1, 3)
    box = np.array([12.5, 12.5, 12.5])
    x0 = (grid * np.array([4.1, 6.2, 3.1]) + rng.normal(scale=0.3, size=grid.shape)) % box
    Z = np.resize(r.Z, len(x0)).astype(np.int32)
    per = s.Replica(Z, x0, box, 2, r.T, 9, "periodic24")
    ctx = P.Context([gas, per], w.dt_fs, w.gamma0_per_fs, precision=precision, widths=w.widths)
    ctx.set_weights(m)
    xs = [_bead_positions(gas, 3, seed=1, sigma=0.3), _bead_positions(per, 2, seed=2, sigma=0.3)]
    ctx.energy_forces(torch.tensor(np.concatenate([x.reshape(-1, 3) for x in xs]), device="cuda"))
    nnb, nbr = ctx.neighbours()
    b = 0
    for rep, xb in zip((gas, per), xs):
        for k in range(rep.n_beads):
            want, _, _ = O.neighbours(xb[k], rep.box, 6.0)
            for i in range(rep.n_atoms):
                assert np.array_equal(nbr[b, :nnb[b]], want[i]), (rep.name, k, i)
                b += 1
    ctx.close()


@pytest.mark.parametrize("precision,splitting", [("fp32", "obabo"), ("fp32", "baoab"), ("fp64", "obabo"),
                                                 ("bf16_tc", "obabo")])
def test_multistep_launch_fuses_ring_kernels_bit_identically(water64_model, precision, splitting):
    """pimd_step(8) runs one graph whose inner step boundaries fuse the ring
    finish with the next ring start; eight pimd_step(1) calls run the two
    kernels separately. Deterministic mode: positions, momenta, step counter
    and thermostat heat are bit-identical."""
    P = _P()
    w, r, m = water64_model
    rep = _with_beads(r, 4)

    def ctx():
        c = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision=precision, widths=w.widths, deterministic=True,
                      splitting=splitting)
        c.set_weights(m)
        return c

    a, b = ctx(), ctx()
    a.step(8)
    for _ in range(8):
        b.step(1)
    qa, pa, sa, Qa = a.get_state()
    qb, pb, sb, Qb = b.get_state()
    assert sa == sb == 8
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb) and np.array_equal(Qa, Qb)
    # and both continue identically (the fused graph leaves the state of a ring finish)
    a.step(1)
    b.step(1)
    qa, pa, _, _ = a.get_state()
    qb, pb, _, _ = b.get_state()
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)
    a.close()
    b.close()
