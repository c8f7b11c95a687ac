"""GPU parity of the graph-field-network force head (Sec. 2.2, direct
forces, FP32 on CUDA cores) against the FP64 numpy oracle on the same seeded
inputs and neighbour rule: forces and pair-force virials element by element
(bar 1e-4 relative max-norm, 1e-5 relative RMS: FP32 products over K <= 256
terms through L iterations), several feature widths and iteration counts,
isolated atoms and one-atom replicas, neighbour lists over two 128-slot
ranges, and dynamics driven by the head. The tensor-core variant (BF16
operands, FP32 accumulation, F = 64 / 128) is held to 3e-2 relative RMS
against the oracle on the same cases."""
import numpy as np
import pytest

import oracle.gfn as OG
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


def _relrms(a, b):
    return float(np.sqrt(((a - b) ** 2).mean() / (b ** 2).mean()))


def _beads(rep, P, seed, sigma=0.05):
    rng = np.random.default_rng(seed)
    x = np.repeat(rep.x0[None], P, axis=0) + rng.normal(scale=sigma, size=(P, rep.n_atoms, 3))
    return x.astype(np.float32).astype(np.float64)


def _with_beads(rep, P):
    return s.Replica(rep.Z, rep.x0, rep.box, P, rep.T, rep.seed, rep.name)


def _run(P, reps, model, xs, maxnb=128, dt=0.5, precision="fp32"):
    ctx = P.Context(reps, dt, 0.001, precision=precision, potential=P.POT_GFN, gfn=(model.F, model.L),
                    max_neighbours=maxnb)
    ctx.set_gfn(model)
    x = torch.tensor(np.concatenate([q.reshape(-1, 3) for q in xs]), device="cuda")
    e, f, v = ctx.energy_forces(x)
    out = (e.cpu().numpy(), f.cpu().numpy(), v.cpu().numpy().reshape(-1, 3, 3))
    ctx.close()
    return out


@pytest.mark.parametrize("F, L", [(32, 0), (64, 1), (128, 3)])
def test_fad_against_oracle(F, L):
    P = _P()
    rep = _with_beads(s.fad(), 4)
    m = s.gfn_model(s.elements_of([rep]), F, L, seed=100 + F + L)
    xb = _beads(rep, 4, seed=3, sigma=0.08)
    e, f, v = _run(P, [rep], m, [xb], dt=0.25)
    assert np.all(e == 0.0)
    f = f.reshape(4, rep.n_atoms, 3)
    for k in range(4):
        Fo, Wo = OG.forces(m, rep.Z, xb[k], None)
        assert _relmax(f[k], Fo) < 1e-4, (k, _relmax(f[k], Fo))
        assert _relrms(f[k], Fo) < 1e-5
        assert _relmax(v[k], Wo) < 1e-4
        assert np.abs(f[k].sum(axis=0)).max() < 1e-5 * np.abs(Fo).max()


def test_water64_sampled_beads():
    """Periodic 64-molecule box, F = 128, L = 3 (Table S1 sizes), 4 beads."""
    P = _P()
    w = s.workload("water64")
    rep = _with_beads(w.replicas[0], 4)
    m = s.gfn_model(s.elements_of([rep]), 128, 3, seed=7)
    xb = _beads(rep, 4, seed=11)
    e, f, v = _run(P, [rep], m, [xb])
    f = f.reshape(4, rep.n_atoms, 3)
    for k in (0, 3):
        Fo, Wo = OG.forces(m, rep.Z, xb[k], rep.box)
        assert _relmax(f[k], Fo) < 1e-4, (k, _relmax(f[k], Fo))
        assert _relrms(f[k], Fo) < 1e-5
        assert _relmax(v[k], Wo) < 1e-4


def test_two_neighbour_ranges_and_isolated_atoms():
    """Compressed water (~170 neighbours, 256 slots: lists longer than 128),
    plus gas-phase replicas with an isolated atom and a one-atom replica."""
    P = _P()
    dense = s.water_box(5, spacing=2.5, seed=515, n_beads=2)
    reps = [dense]
    cl = s.batch(n_rep=3, seed=93, beads=(2, 3))
    r0 = cl[0]
    x0 = r0.x0.copy()
    x0[0] += np.array([40.0, 0.0, 0.0])
    cl[0] = s.Replica(r0.Z, x0, r0.box, r0.n_beads, r0.T, r0.seed)
    reps += cl
    reps.append(s.Replica(np.array([8], dtype=np.int32), np.zeros((1, 3)), (0.0, 0.0, 0.0), 2, 300.0, 5))
    m = s.gfn_model(s.elements_of(reps), 64, 2, seed=17)
    xs = [_beads(r, r.n_beads, seed=40 + k) for k, r in enumerate(reps)]
    e, f, v = _run(P, reps, m, xs, maxnb=256)
    b0 = s0 = 0
    for k, (r, x) in enumerate(zip(reps, xs)):
        n = r.n_atoms * r.n_beads
        fg = f[b0:b0 + n].reshape(r.n_beads, r.n_atoms, 3)
        for q in range(r.n_beads):
            Fo, Wo = OG.forces(m, r.Z, x[q], r.box if r.box[0] > 0 else None, maxnb=256)
            if np.abs(Fo).max() > 0:
                assert _relmax(fg[q], Fo) < 1e-4, (k, q)
                assert _relmax(v[s0 + q], Wo) < 1e-4
            else:
                assert np.abs(fg[q]).max() == 0.0
        b0 += n
        s0 += r.n_beads
    n0 = reps[0].n_atoms * reps[0].n_beads
    assert np.abs(f[n0:n0 + cl[0].n_atoms * cl[0].n_beads].reshape(cl[0].n_beads, -1, 3)[:, 0]).max() == 0.0
    assert np.abs(f[-2:]).max() == 0.0


def test_dynamics_conserve_momentum_and_errors():
    """NVE ring-polymer steps on the head's forces: sum_i F_i = 0 on every
    bead, so the total momentum stays at its initial value; the head's
    context rejects the network's weights and vice versa."""
    P = _P()
    rep = _with_beads(s.fad(), 8)
    m = s.gfn_model(s.elements_of([rep]), 64, 3, seed=21)
    s.set_force_scale(m, 0.05)
    ctx = P.Context([rep], 0.25, 0.0, precision="fp32", thermostat=False, potential=P.POT_GFN, gfn=(64, 3))
    ctx.set_gfn(m)
    q0, p0, _, _ = ctx.get_state()
    ctx.step(200)
    q1, p1, _, _ = ctx.get_state()
    est = ctx.estimators()[0]
    assert np.all(np.isfinite(q1)) and np.all(np.isfinite(p1))
    assert est["V_mean"] == 0.0
    # centroid-mode momenta (mode 0 holds sqrt(P) x the centroid momentum)
    P_tot0 = p0.reshape(-1, 3)[:rep.n_atoms].sum(axis=0)
    P_tot1 = p1.reshape(-1, 3)[:rep.n_atoms].sum(axis=0)
    assert np.abs(P_tot1 - P_tot0).max() < 1e-4 * np.abs(p1).max()
    with pytest.raises(P.PimdError) as ei:
        ctx.set_weights(s.xavier_model(s.elements_of([rep]), (64, 64), seed=1))
    assert ei.value.code == -2
    ctx.close()
    c2 = P.Context([rep], 0.25, 0.01, precision="fp32", widths=(64, 64))
    with pytest.raises(P.PimdError) as ei:
        c2.set_gfn(m)
    assert ei.value.code == -2
    c2.close()


@pytest.mark.parametrize("wl, F, L", [("fad", 64, 2), ("water64", 128, 3)])
def test_tensor_core_head(wl, F, L):
    P = _P()
    w = s.workload(wl)
    rep = _with_beads(w.replicas[0], 3)
    m = s.gfn_model(s.elements_of([rep]), F, L, seed=31)
    xb = _beads(rep, 3, seed=12)
    box = rep.box if rep.box[0] > 0 else None
    e, f, v = _run(P, [rep], m, [xb], precision="bf16_tc")
    e32, f32, v32 = _run(P, [rep], m, [xb], precision="fp32")
    assert np.all(e == 0.0)
    f = f.reshape(3, rep.n_atoms, 3)
    f32 = f32.reshape(3, rep.n_atoms, 3)
    for k in range(3):
        Fo, Wo = OG.forces(m, rep.Z, xb[k], box)
        assert _relrms(f[k], Fo) < 3e-2, (k, _relrms(f[k], Fo))
        assert _relrms(f32[k], Fo) < 1e-5
        assert _relmax(v[k], Wo) < 5e-2
        # pair forces stay equal and opposite in BF16
        assert np.abs(f[k].sum(axis=0)).max() < 1e-4 * np.abs(Fo).max() * rep.n_atoms


def test_tensor_core_head_ragged_lists():
    """BF16 head on lists longer than 128 slots (two tiles per atom), gas-phase
    clusters with an isolated atom (no tile) and a one-atom replica."""
    P = _P()
    dense = s.water_box(5, spacing=2.5, seed=516, n_beads=2)
    cl = s.batch(n_rep=3, seed=94, beads=(2, 3))
    r0 = cl[0]
    x0 = r0.x0.copy()
    x0[0] += np.array([40.0, 0.0, 0.0])
    cl[0] = s.Replica(r0.Z, x0, r0.box, r0.n_beads, r0.T, r0.seed)
    reps = [dense] + cl + [s.Replica(np.array([8], dtype=np.int32), np.zeros((1, 3)), (0.0, 0.0, 0.0), 2, 300.0, 5)]
    m = s.gfn_model(s.elements_of(reps), 64, 2, seed=18)
    xs = [_beads(r, r.n_beads, seed=60 + k) for k, r in enumerate(reps)]
    e, f, v = _run(P, reps, m, xs, maxnb=256, precision="bf16_tc")
    b0 = 0
    for k, (r, x) in enumerate(zip(reps, xs)):
        n = r.n_atoms * r.n_beads
        fg = f[b0:b0 + n].reshape(r.n_beads, r.n_atoms, 3)
        for q in range(r.n_beads):
            Fo, _ = OG.forces(m, r.Z, x[q], r.box if r.box[0] > 0 else None, maxnb=256)
            if np.abs(Fo).max() > 0:
                assert _relrms(fg[q], Fo) < 3e-2, (k, q, _relrms(fg[q], Fo))
            else:
                assert np.abs(fg[q]).max() == 0.0
        b0 += n
    n0 = dense.n_atoms * dense.n_beads
    assert np.abs(f[n0:n0 + cl[0].n_atoms * cl[0].n_beads].reshape(cl[0].n_beads, -1, 3)[:, 0]).max() == 0.0
    assert np.abs(f[-2:]).max() == 0.0
