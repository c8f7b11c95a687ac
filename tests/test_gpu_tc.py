"""GPU parity of the BF16 tensor-core network path (tcgen05) and full-size
sampled checks on the ice workload in the benchmark's launch configuration.

Bars for BF16: forces within 1e-2 relative RMS and energies within 1 meV per
atom of the FP64 oracle; FP32 path: 1e-5 relative max-norm."""
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


def _relrms(a, b):
    return float(np.sqrt(((a - b) ** 2).mean() / (b ** 2).mean()))


def _relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _beads(rep, P, seed, sigma=0.08):
    rng = np.random.default_rng(seed)
    x = np.repeat(rep.x0[None], P, axis=0) + rng.normal(scale=sigma, size=(P, rep.n_atoms, 3))
    return x.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("P_beads", [7])
def test_bf16_water_against_oracle_and_fp32(water64_model, P_beads):
    P = _P()
    w, r, m = water64_model
    rep = s.Replica(r.Z, r.x0, r.box, P_beads, r.T, r.seed)
    xb = _beads(rep, P_beads, seed=23)
    xt = torch.tensor(xb.reshape(-1, 3), device="cuda")
    tc = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="bf16_tc", widths=w.widths)
    tc.set_weights(m)
    e, f, v = tc.energy_forces(xt)
    e, f = e.cpu().numpy(), f.cpu().numpy().reshape(P_beads, rep.n_atoms, 3)
    Eo, Fo, _ = O.energy_forces_batch(m, rep.Z, xb, rep.box)
    assert _relrms(f, Fo) < 1e-2
    assert np.abs(e - Eo.sum(axis=1)).max() / rep.n_atoms < 1e-3
    # and close to the FP32 path on the same inputs
    f32 = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    f32.set_weights(m)
    e2, f2, _ = f32.energy_forces(xt)
    assert _relrms(f, f2.cpu().numpy().reshape(f.shape)) < 1e-2


def test_bf16_small_network_and_ragged_tiles():
    """2 x 64 network on uneven gas-phase replicas (element groups that do
    not fill whole 128-row tiles)."""
    P = _P()
    reps = s.batch(n_rep=5, seed=81, beads=(3, 7))
    m = s.xavier_model(s.elements_of(reps), (64, 64), seed=12)
    G = np.concatenate([O.descriptors(m, r.x0, None) for r in reps])
    s.set_normalisation(m, G, np.concatenate([r.Z for r in reps]))
    F = np.concatenate([O.energy_forces(m, r.Z, r.x0, None)[1] for r in reps])
    s.set_energy_scale(m, 1.0 / float(np.sqrt((F ** 2).mean())))
    ctx = P.Context(reps, 0.25, 0.01, precision="bf16_tc", widths=(64, 64))
    ctx.set_weights(m)
    xs = [_beads(r, r.n_beads, seed=40 + k, sigma=0.05) for k, r in enumerate(reps)]
    e, f, _ = ctx.energy_forces(torch.tensor(np.concatenate([x.reshape(-1, 3) for x in xs]), device="cuda"))
    e, f = e.cpu().numpy(), f.cpu().numpy()
    b0 = s0 = 0
    for r, x in zip(reps, xs):
        Eo, Fo, _ = O.energy_forces_batch(m, r.Z, x, None)
        n = r.n_atoms * r.n_beads
        assert _relrms(f[b0:b0 + n].reshape(Fo.shape), Fo) < 1e-2
        assert np.abs(e[s0:s0 + r.n_beads] - Eo.sum(axis=1)).max() / r.n_atoms < 1e-3
        b0 += n
        s0 += r.n_beads


@pytest.mark.parametrize("widths", [(128,), (128, 128), (64, 64, 64, 64), (256,), (256, 256, 256),
                                    (256, 256, 256, 256)])
def test_bf16_network_depths(widths):
    P = _P()
    w = s.workload("water64")
    r = w.replicas[0]
    rep = s.Replica(r.Z, r.x0, r.box, 2, r.T, r.seed)
    m = s.xavier_model(s.elements_of([rep]), widths, seed=31)
    G = O.descriptors(m, rep.x0, rep.box)
    s.set_normalisation(m, G, rep.Z)
    _, F, _ = O.energy_forces(m, rep.Z, rep.x0, rep.box)
    s.set_energy_scale(m, 1.0 / float(np.sqrt((F ** 2).mean())))
    xb = _beads(rep, 2, seed=8)
    ctx = P.Context([rep], 0.5, 0.001, precision="bf16_tc", widths=widths)
    ctx.set_weights(m)
    e, f, _ = ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    Eo, Fo, _ = O.energy_forces_batch(m, rep.Z, xb, rep.box)
    assert _relrms(f.cpu().numpy().reshape(Fo.shape), Fo) < 1e-2
    assert np.abs(e.cpu().numpy() - Eo.sum(axis=1)).max() / rep.n_atoms < 1e-3


# ---------------------------------------------------------------- ice, full size
@pytest.mark.parametrize("precision", ["bf16_tc", "fp32"])
def test_ice_full_size_sampled_beads(ice_model, precision):
    """Ice Ih, 1296 atoms x 32 beads (41,472 bead-atoms) in the benchmark's
    launch configuration: after 3 steps, the forces and energies of two
    sampled beads match the oracle evaluated on the same FP32 bead positions."""
    P = _P()
    w, r, m = ice_model
    ctx = P.Context(w.replicas, w.dt_fs, w.gamma0_per_fs, precision=precision, widths=w.widths, timing=True)
    ctx.set_weights(m)
    ctx.step(3)
    x, f, V = ctx.get_forces()
    x = x.reshape(r.n_beads, r.n_atoms, 3)
    f = f.reshape(r.n_beads, r.n_atoms, 3)
    for k in (0, 19):
        Eo, Fo, _ = O.energy_forces(m, r.Z, x[k], r.box)
        if precision == "fp32":
            assert _relmax(f[k], Fo) < 1e-5
            assert abs(V[k] - Eo.sum()) / r.n_atoms < 1e-5
        else:
            assert _relrms(f[k], Fo) < 1e-2
            assert abs(V[k] - Eo.sum()) / r.n_atoms < 1e-3
    nnb, nbr = ctx.neighbours()
    want, _, _ = O.neighbours(x[5], r.box, 6.0)
    for i in range(0, r.n_atoms, 7):
        b = 5 * r.n_atoms + i
        assert np.array_equal(np.sort(nbr[b, :nnb[b]]), want[i])
    st = ctx.stage_times()
    assert all(v >= 0 for v in st.values()) and st["adjoint"] > 0
    # ring start, skin check, lists, descriptors, network, adjoint, ring
    # finish (which ends the step); the FP32 path adds the energy reduction
    # (the BF16 adjoint sums the per-bead energies and virials itself). The
    # BF16 step runs the descriptors, network and adjoint once per half of
    # the bead-atoms (overlapped halves, on by default here).
    if precision == "bf16_tc":
        assert ctx.kernels_per_step() == 10
        ctx.set_overlap(False)
        assert ctx.kernels_per_step() == 7
    else:
        assert ctx.kernels_per_step() == 8
