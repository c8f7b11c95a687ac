"""GPU parity of the moment-tensor evaluation of the angular symmetry
functions (O(n) per atom) against the FP64 oracle's pair sums and against the
pair-sum kernels on the same inputs.

Bars as for the FP32 path: descriptors within 1e-5 of each channel's scale,
forces and virial within 1e-5 relative max-norm."""
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


def _beads(rep, P, seed, sigma=0.08):
    rng = np.random.default_rng(seed)
    x = np.repeat(rep.x0[None], P, axis=0) + rng.normal(scale=sigma, size=(P, rep.n_atoms, 3))
    return x.astype(np.float32).astype(np.float64)


def _with_beads(rep, P):
    return s.Replica(rep.Z, rep.x0, rep.box, P, rep.T, rep.seed, rep.name)


def test_default_selection_and_errors(water64_model, fad_model):
    P = _P()
    w, r, m = water64_model
    c = P.Context([_with_beads(r, 2)], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    assert c.angular == "moments"          # ~90 neighbours per atom
    wf, rf, mf = fad_model
    c2 = P.Context([_with_beads(rf, 2)], wf.dt_fs, wf.gamma0_per_fs, precision="fp32", widths=wf.widths)
    assert c2.angular == "pairs"           # 9 neighbours
    c3 = P.Context([_with_beads(r, 2)], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths)
    assert c3.angular == "pairs"
    with pytest.raises(P.PimdError) as ei:
        c3.set_angular("moments")
    assert ei.value.code == -8
    with pytest.raises(P.PimdError) as ei:
        c.set_angular(5)
    assert ei.value.code == -1


@pytest.mark.parametrize("precision", ["fp32", "bf16_tc"])
def test_water_descriptors_forces_virial(water64_model, precision):
    P = _P()
    w, r, m = water64_model
    rep = _with_beads(r, 5)
    xb = _beads(rep, 5, seed=23)
    x = torch.tensor(xb.reshape(-1, 3), device="cuda")
    out = {}
    for algo in ("moments", "pairs"):
        ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision=precision, widths=w.widths)
        ctx.set_weights(m)
        ctx.set_angular(algo)
        G = ctx.descriptors(x).cpu().numpy()
        e, f, v = ctx.energy_forces(x)
        out[algo] = (G, e.cpu().numpy(), f.cpu().numpy().reshape(5, rep.n_atoms, 3), v.cpu().numpy())
    G, e, f, v = out["moments"]
    for k in range(5):
        Go = O.descriptors(m, xb[k], rep.box)
        Gg = G[k * rep.n_atoms:(k + 1) * rep.n_atoms]
        scale = np.abs(Go).max(axis=0) + 1e-30
        assert np.all(np.abs(Gg - Go) <= 1e-5 * scale), k
    if precision == "fp32":
        Eo, Fo, Wo = O.energy_forces_batch(m, rep.Z, xb, rep.box)
        assert _relmax(f, Fo) < 1e-5
        assert _relmax(v, Wo) < 1e-5
        assert np.abs(e - Eo.sum(axis=1)).max() / rep.n_atoms < 1e-5
    else:
        # same BF16 network on both sides: the angular evaluation changes only
        # FP32 rounding of the descriptors and of the adjoint
        _, ep, fp, vp = out["pairs"]
        assert np.sqrt(((f - fp) ** 2).mean() / (fp ** 2).mean()) < 1e-2
        assert np.abs(e - ep).max() / rep.n_atoms < 1e-3
    assert np.abs(f.sum(axis=1)).max() < 1e-4 * np.abs(f).max()


def test_fad_forced_moments(fad_model):
    """Small neighbour counts (9): the moment path is still exact."""
    P = _P()
    w, r, m = fad_model
    rep = _with_beads(r, 6)
    xb = _beads(rep, 6, seed=4, sigma=0.1)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    ctx.set_weights(m)
    ctx.set_angular("moments")
    e, f, v = ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    Eo, Fo, Wo = O.energy_forces_batch(m, rep.Z, xb, None)
    assert _relmax(f.cpu().numpy().reshape(Fo.shape), Fo) < 1e-5
    assert _relmax(v.cpu().numpy(), Wo) < 1e-5


def test_clusters_with_isolated_atom_and_empty_lists():
    """Replicas of 1..24 atoms, one atom far from the others (no neighbours):
    moment path forced, forces match the oracle, isolated atom gets zero."""
    P = _P()
    reps = s.batch(n_rep=5, seed=91, beads=(2, 3))
    r0 = reps[0]
    x0 = r0.x0.copy()
    x0[0] += np.array([40.0, 0.0, 0.0])
    reps[0] = s.Replica(r0.Z, x0, r0.box, r0.n_beads, r0.T, r0.seed)
    lone = s.Replica(np.array([8], dtype=np.int32), np.zeros((1, 3)), (0.0, 0.0, 0.0), 2, 300.0, 5)
    reps.append(lone)
    m = s.xavier_model(s.elements_of(reps), (64, 64), seed=6)
    G = np.concatenate([O.descriptors(m, r.x0, None) for r in reps])
    Z = np.concatenate([r.Z for r in reps])
    s.set_normalisation(m, G, Z)
    ctx = P.Context(reps, 0.25, 0.01, precision="fp32", widths=(64, 64))
    ctx.set_weights(m)
    ctx.set_angular("moments")
    xs = [_beads(r, r.n_beads, seed=50 + k, sigma=0.05) for k, r in enumerate(reps)]
    e, f, _ = ctx.energy_forces(torch.tensor(np.concatenate([x.reshape(-1, 3) for x in xs]), device="cuda"))
    e, f = e.cpu().numpy(), f.cpu().numpy()
    b0 = s0 = 0
    for r, x in zip(reps, xs):
        Eo, Fo, _ = O.energy_forces_batch(m, r.Z, x, None)
        n = r.n_atoms * r.n_beads
        fg = f[b0:b0 + n].reshape(Fo.shape)
        if np.abs(Fo).max() > 0:
            assert _relmax(fg, Fo) < 1e-5
        else:
            assert np.abs(fg).max() == 0.0
        assert np.abs(e[s0:s0 + r.n_beads] - Eo.sum(axis=1)).max() < 1e-5 * max(1, r.n_atoms)
        b0 += n
        s0 += r.n_beads
    assert np.abs(f[:reps[0].n_atoms * reps[0].n_beads].reshape(reps[0].n_beads, -1, 3)[:, 0]).max() == 0.0


def test_ice_full_size_moments_vs_pairs(ice_model):
    """Ice Ih, 1296 atoms x 32 beads, moment path as launched by the bench:
    forces of sampled beads against the oracle, and the whole batch against
    the pair-sum kernels."""
    P = _P()
    w, r, m = ice_model
    rep = r
    xb = _beads(rep, rep.n_beads, seed=77, sigma=0.05)
    x = torch.tensor(xb.reshape(-1, 3), device="cuda")
    res = {}
    for algo in ("moments", "pairs"):
        ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
        ctx.set_weights(m)
        ctx.set_angular(algo)
        e, f, v = ctx.energy_forces(x)
        res[algo] = (e.cpu().numpy(), f.cpu().numpy().reshape(rep.n_beads, rep.n_atoms, 3), v.cpu().numpy())
        ctx.close()
    e, f, v = res["moments"]
    ep, fp, vp = res["pairs"]
    for k in (0, 13, 31):
        Eo, Fo, Wo = O.energy_forces_batch(m, rep.Z, xb[k:k + 1], rep.box)
        assert _relmax(f[k:k + 1], Fo) < 1e-5, ("moments", k, _relmax(f[k:k + 1], Fo))
        assert _relmax(fp[k:k + 1], Fo) < 1e-5, ("pairs", k, _relmax(fp[k:k + 1], Fo))
        assert abs(e[k] - Eo.sum()) / rep.n_atoms < 1e-5
    # two FP32 evaluations, each within 1e-5 of the oracle
    assert _relmax(f, fp) < 2e-5
    assert _relmax(v, vp) < 2e-5


def test_deterministic_moments_bit_identical(water64_model):
    P = _P()
    w, r, m = water64_model
    rep = _with_beads(r, 3)
    xb = _beads(rep, 3, seed=8)
    x = torch.tensor(xb.reshape(-1, 3), device="cuda")
    outs = []
    for _ in range(2):
        ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths, deterministic=True)
        ctx.set_weights(m)
        assert ctx.angular == "moments"
        _, f, v = ctx.energy_forces(x)
        outs.append((f.cpu().numpy(), v.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_bf16_adjoint_deterministic_mode_and_summed_virial(water64_model):
    """BF16 moment adjoint (two neighbours per lane, one-level fold). In
    deterministic mode (pair vectors gathered per atom, energies and virials
    reduced in a fixed order) two runs are bit-identical. They agree with the
    default mode, whose adjoint adds the per-bead energies and virials itself
    (FP64 atomics) and scatters forces with FP32 atomics: only the summation
    order differs. The virial equals the BF16 pair-sum path's (same network).
    It is 3.7e-2 (relative RMS) from the FP64 oracle, the diagonal ~3.5 %
    low, on both BF16 paths: they share only the BF16 network, and the FP32
    path is within 1e-5. Forces keep the 1e-2 bar, but the virial diagonal
    adds the network's errors up without cancellation."""
    P = _P()
    w, r, m = water64_model
    rep = _with_beads(r, 4)
    xb = _beads(rep, 4, seed=31)
    x = torch.tensor(xb.reshape(-1, 3), device="cuda")
    runs = []
    for det in (False, True, True):
        c = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="bf16_tc", widths=w.widths, deterministic=det)
        c.set_weights(m)
        assert c.angular == "moments"
        e, f, v = c.energy_forces(x)
        runs.append((e.cpu().numpy(), f.cpu().numpy(), v.cpu().numpy()))
        c.close()
    (e0, f0, v0), (e1, f1, v1), (e2, f2, v2) = runs
    assert np.array_equal(e1, e2) and np.array_equal(f1, f2) and np.array_equal(v1, v2)
    assert _relmax(f0, f1) < 1e-5
    assert np.abs(e0 - e1).max() < 1e-9 * max(1.0, float(np.abs(e1).max()))
    assert _relmax(v0, v1) < 1e-6
    c = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="bf16_tc", widths=w.widths)
    c.set_weights(m)
    c.set_angular("pairs")
    _, _, vp = c.energy_forces(x)
    vp = vp.cpu().numpy()
    c.close()
    assert np.sqrt(((v0 - vp) ** 2).mean() / (vp ** 2).mean()) < 2e-3
    _, _, Wo = O.energy_forces_batch(m, rep.Z, xb, rep.box)
    Wo = np.asarray(Wo).reshape(v0.shape)
    assert np.sqrt(((v0 - Wo) ** 2).mean() / (Wo ** 2).mean()) < 5e-2


def test_bf16_reduced_forward_ragged_counts_and_empty_lists():
    """BF16 path, moment evaluation forced, on replicas of 1..24 atoms with an
    isolated atom: neighbour counts from 0 to 23 cover an empty list, a chunk
    of at most 16 neighbours (one half-warp's rows) and one of 17..31 (the
    second half-warp's rows padded with zero weights). Descriptors match the
    oracle within 1e-5 of each channel's scale (1e-30 absolute floor: far
    radial centres of a tiny cluster underflow in FP32); forces and energies
    match the pair-sum kernels with the same BF16 network; the isolated atom
    and the one-atom replica get exactly zero force."""
    P = _P()
    reps = s.batch(n_rep=5, seed=91, beads=(2, 3))
    r0 = reps[0]
    x0 = r0.x0.copy()
    x0[0] += np.array([40.0, 0.0, 0.0])
    reps[0] = s.Replica(r0.Z, x0, r0.box, r0.n_beads, r0.T, r0.seed)
    lone = s.Replica(np.array([8], dtype=np.int32), np.zeros((1, 3)), (0.0, 0.0, 0.0), 2, 300.0, 5)
    reps.append(lone)
    m = s.xavier_model(s.elements_of(reps), (64, 64), seed=6)
    G0 = np.concatenate([O.descriptors(m, r.x0, None) for r in reps])
    Z = np.concatenate([r.Z for r in reps])
    s.set_normalisation(m, G0, Z)
    xs = [_beads(r, r.n_beads, seed=50 + k, sigma=0.05) for k, r in enumerate(reps)]
    x = torch.tensor(np.concatenate([xx.reshape(-1, 3) for xx in xs]), device="cuda")
    out = {}
    for algo in ("moments", "pairs"):
        ctx = P.Context(reps, 0.25, 0.01, precision="bf16_tc", widths=(64, 64))
        ctx.set_weights(m)
        ctx.set_angular(algo)
        G = ctx.descriptors(x).cpu().numpy()
        e, f, _ = ctx.energy_forces(x)
        out[algo] = (G, e.cpu().numpy(), f.cpu().numpy())
    G, e, f = out["moments"]
    _, ep, fp = out["pairs"]
    b0 = 0
    for r, xx in zip(reps, xs):
        for k in range(r.n_beads):
            Go = O.descriptors(m, xx[k], None)
            Gg = G[b0:b0 + r.n_atoms]
            scale = np.abs(Go).max(axis=0)
            assert np.all(np.abs(Gg - Go) <= 1e-5 * scale + 1e-30), (r.n_atoms, k)
            b0 += r.n_atoms
    assert b0 == G.shape[0]
    assert np.sqrt(((f - fp) ** 2).mean() / (fp ** 2).mean()) < 1e-2
    assert np.abs(e - ep).max() < 1e-3 * max(r.n_atoms for r in reps)
    assert np.abs(f[:reps[0].n_atoms * reps[0].n_beads].reshape(reps[0].n_beads, -1, 3)[:, 0]).max() == 0.0
    assert np.abs(f[-lone.n_beads:]).max() == 0.0
