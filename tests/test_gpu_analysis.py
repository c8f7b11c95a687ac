"""GPU structural analysis (RDF pair counts, proton-transfer coordinate)
against the oracle: bit-exact integer counts and identical FP32 coordinates
on the same bead positions."""
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


def _beads(rep, P, seed, sigma=0.1):
    rng = np.random.default_rng(seed)
    x = np.repeat(rep.x0[None], P, axis=0) + rng.normal(scale=sigma, size=(P, rep.n_atoms, 3))
    return x


def _types(Z, elements):
    return np.searchsorted(np.asarray(sorted(elements)), Z)


def _bonds(rep, donor=1, acceptor=8):
    """bonding atom of each proton: its nearest acceptor in the initial structure"""
    x, L = rep.x0, np.asarray(rep.box)
    bond = np.full(rep.n_atoms, -1, dtype=np.int32)
    acc = np.where(rep.Z == acceptor)[0]
    for h in np.where(rep.Z == donor)[0]:
        d = x[acc] - x[h]
        if L[0] > 0:
            d -= L * np.round(d / L)
        bond[h] = acc[np.argmin((d ** 2).sum(axis=1))]
    return bond


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_rdf_counts_water_bit_exact(water64_model, precision):
    P = _P()
    w, r, m = water64_model
    rep = s.Replica(r.Z, r.x0, r.box, 3, r.T, r.seed, r.name)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision=precision, widths=w.widths)
    ctx.set_weights(m)
    xb = _beads(rep, 3, seed=12)
    ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    c = ctx.rdf_counts(6.0, 120).cpu().numpy().astype(np.uint64)
    t = _types(rep.Z, ctx.element_types() and [1, 8])
    want = sum(O.rdf_counts(xb[k], rep.box, t, 2, 6.0, 120) for k in range(3))
    assert np.array_equal(c, want)
    # accumulation into a caller's array
    c2 = ctx.rdf_counts(6.0, 120, counts=torch.tensor(c.astype(np.int64), device="cuda")).cpu().numpy()
    assert np.array_equal(c2, 2 * c.astype(np.int64))
    # g(r) on the device from the oracle's counts against the oracle's g(r)
    n_per = [int((rep.Z == 1).sum()), int((rep.Z == 8).sum())]
    g = ctx.rdf_gr(torch.tensor(want.astype(np.int64), device="cuda"), 6.0, 3).cpu().numpy()
    go = O.rdf_gr(want, n_per, float(np.prod(rep.box)), 6.0, 3)
    np.testing.assert_allclose(g, go, rtol=1e-13, atol=0)
    assert g[2, :15].max() == 0.0                         # no O-O pairs below 0.75 A


def test_rdf_counts_ice_full_size(ice_model):
    P = _P()
    w, r, m = ice_model
    ctx = P.Context([r], w.dt_fs, w.gamma0_per_fs, precision="bf16_tc", widths=w.widths)
    ctx.set_weights(m)
    xb = _beads(r, r.n_beads, seed=3, sigma=0.06)
    ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    c = ctx.rdf_counts(8.0, 400).cpu().numpy().astype(np.uint64)
    t = _types(r.Z, [1, 8])
    want = np.zeros_like(c)
    for k in range(r.n_beads):
        want += O.rdf_counts(xb[k], r.box, t, 2, 8.0, 400)
    assert np.array_equal(c, want)
    assert int(c.sum()) > 0


def test_rdf_counts_cluster_replica_and_errors(water64_model):
    P = _P()
    w, r, m = water64_model
    reps = s.batch(n_rep=3, seed=5, beads=(2, 4))
    m2 = s.xavier_model(s.elements_of(reps), (64, 64), seed=1)
    ctx = P.Context(reps, 0.25, 0.01, precision="fp32", widths=(64, 64))
    ctx.set_weights(m2)
    Zs = ctx.element_types()
    for q, rep in enumerate(reps):
        x = np.repeat(rep.x0[None], rep.n_beads, axis=0)
        c = ctx.rdf_counts(5.0, 50, replica=q).cpu().numpy().astype(np.uint64)
        t = _types(rep.Z, Zs)
        want = sum(O.rdf_counts(x[k], None, t, len(Zs), 5.0, 50) for k in range(rep.n_beads))
        assert np.array_equal(c, want), q
    with pytest.raises(P.PimdError):
        ctx.rdf_counts(5.0, 0)
    with pytest.raises(P.PimdError):
        ctx.rdf_counts(5.0, 50, replica=7)
    wp = s.Replica(r.Z, r.x0, r.box, 2, r.T, r.seed)
    ctx2 = P.Context([wp], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    with pytest.raises(P.PimdError):
        ctx2.rdf_counts(7.0, 10)                       # beyond half of the 12.42 A box


def test_pt_coordinate_water(water64_model):
    P = _P()
    w, r, m = water64_model
    rep = s.Replica(r.Z, r.x0, r.box, 4, r.T, r.seed, r.name)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    ctx.set_weights(m)
    xb = _beads(rep, 4, seed=21, sigma=0.12)
    ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    bond = _bonds(rep)
    v, h = ctx.pt_coordinate(bond, 8, (-2.5, 0.5), 60)
    v, h = v.cpu().numpy(), h.cpu().numpy().astype(np.uint64)
    acc = (rep.Z == 8).astype(np.int32)
    want_h = np.zeros(60, dtype=np.uint64)
    for k in range(4):
        vo, ho = O.pt_coordinate(xb[k], rep.box, bond, acc, -2.5, 0.5, 60)
        assert np.array_equal(np.isnan(v[k]), np.isnan(vo))
        ok = ~np.isnan(vo)
        assert np.array_equal(v[k][ok], vo[ok])
        want_h += ho
    assert np.array_equal(h, want_h)
    assert int(h.sum()) == 4 * int((rep.Z == 1).sum())
    with pytest.raises(P.PimdError):
        ctx.pt_coordinate(bond, 6, (-2.5, 0.5), 60)     # no carbon in water
