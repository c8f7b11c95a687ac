"""GPU well-tempered metadynamics (Sec. 2.5) against the oracle: biased
trajectories with hill deposition (dimer proton-transfer CV, FP64), XRD CV
values, bias energies and forces (FP32), hill checkpointing and errors."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_23728_gb300 import synth as s

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q_XRD = 4 * math.pi * math.sin(math.radians(11.95)) / 1.54
F_Z = {1: 1.0, 6: 6.0, 8: 8.0}        # forward-scattering factors f = Z


def _P():
    import __graft_entry__ as ge
    ge.build()
    from paper_2503_23728_gb300 import pimd as P
    return P


def test_dimer_cv_biased_trajectory_matches_oracle(fad_model):
    """FAD, P = 4, FP64: 40 steps with a hill every 5 steps; positions,
    momenta, hills and bead CVs against the oracle."""
    P = _P()
    w, r, m = fad_model
    rep = s.Replica(r.Z, r.x0, r.box, 4, r.T, r.seed, r.name)
    terms = s.fad_dimer_cv_terms()
    md = P.make_metad(("distances", terms), 0.02, 0.1, 10.0, 5, 64)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths, metad=md)
    ctx.set_weights(m)
    mo = O.Metad(("distances", terms), r.n_atoms, 4, 0.02, 0.1, 10.0, 5, max_hills=64)
    so = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m, metad=mo)
    ctx.step(40)
    so.step(40)
    q, p, st, _ = ctx.get_state()
    assert st == 40
    sh, hh = ctx.metad_hills()
    so_s, so_h = mo.hills
    assert len(sh) == len(so_s) == 32
    np.testing.assert_allclose(sh, so_s, rtol=0, atol=1e-9)
    np.testing.assert_allclose(hh, so_h, rtol=1e-9, atol=0)
    np.testing.assert_allclose(q.reshape(so.q.shape), so.q, rtol=0, atol=1e-8)
    np.testing.assert_allclose(p.reshape(so.p.shape), so.p, rtol=0, atol=1e-8 * np.abs(so.p).max())
    cv, vb = ctx.metad_cv()
    np.testing.assert_allclose(cv, mo.cv_last, rtol=0, atol=1e-9)
    np.testing.assert_allclose(vb, mo.vb_last, rtol=1e-8, atol=1e-14)
    eg, eo = ctx.estimators()[0], so.estimators()
    for k in ("V_mean", "E_tot", "H_cons"):
        assert abs(eg[k] - eo[k]) <= 1e-8 * max(1.0, abs(eo[k])), k


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_xrd_cv_bias_forces_match_oracle(water64_model, precision):
    """Water-64, P = 3, with preset hills: bead CVs, bias energies, forces and
    virials of the biased potential against the oracle."""
    P = _P()
    w, r, m = water64_model
    rep = s.Replica(r.Z, r.x0, r.box, 3, r.T, r.seed, r.name)
    md = P.make_metad(("xrd", Q_XRD, F_Z), 0.05, 0.5, 60.0, 100, 64, elements=[1, 8])
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision=precision, widths=w.widths, metad=md)
    ctx.set_weights(m)
    mo = O.Metad(("xrd", Q_XRD, [F_Z[int(z)] for z in rep.Z]), rep.n_atoms, 3, 0.05, 0.5, 60.0, 100)
    rng = np.random.default_rng(4)
    xb = (np.repeat(rep.x0[None], 3, axis=0) + rng.normal(scale=0.1, size=(3, rep.n_atoms, 3)))
    xb = xb.astype(np.float32).astype(np.float64)
    s0 = np.array([mo.cv(xb[k], rep.box)[0] for k in range(3)])
    hs, hh = s0 + np.array([0.3, -0.2, 0.1]), np.array([0.05, 0.03, 0.04])
    ctx.metad_set_hills(hs, hh)
    mo.deposit(hs, [0.0, 0.0, 0.0], rep.T)
    mo.hs[:3], mo.hh[:3] = hs, hh
    e, f, v = ctx.energy_forces(torch.tensor(xb.reshape(-1, 3), device="cuda"))
    cv, vb = ctx.metad_cv()
    tol = 1e-5 if precision == "fp32" else 1e-10
    for k in range(3):
        sk, g, vir = mo.cv(xb[k], rep.box, grad=True)
        bk, dv = mo.bias(sk)
        assert abs(cv[k] - sk) <= tol * abs(sk), (k, cv[k], sk)
        assert abs(vb[k] - bk) <= tol * 10 * max(abs(bk), 1e-3)
        Eo, Fo, Wo = O.energy_forces_batch(m, rep.Z, xb[k:k + 1], rep.box)
        Fb = Fo[0] - dv * g
        fk = f.cpu().numpy().reshape(3, rep.n_atoms, 3)[k]
        assert np.abs(fk - Fb).max() <= tol * np.abs(Fb).max(), k
        assert abs(e.cpu().numpy()[k] - (Eo.sum() + bk)) <= tol * rep.n_atoms
        Wb = np.asarray(Wo[0]).reshape(9) - dv * vir.reshape(9)
        assert np.abs(v.cpu().numpy()[k].reshape(9) - Wb).max() <= tol * np.abs(Wb).max()


def test_hill_capacity_and_checkpoint(fad_model):
    P = _P()
    w, r, m = fad_model
    rep = s.Replica(r.Z, r.x0, r.box, 4, r.T, r.seed, r.name)
    md = P.make_metad(("distances", s.fad_dimer_cv_terms()), 0.02, 0.1, 10.0, 1, 8)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths, metad=md)
    ctx.set_weights(m)
    ctx.step(2)                                   # 2 depositions of 4 hills: full
    sh, hh = ctx.metad_hills()
    assert len(sh) == 8 and np.all(hh > 0)
    with pytest.raises(P.PimdError) as ei:
        ctx.step(1)
        ctx.estimators()
    assert ei.value.code == -9
    assert len(ctx.metad_hills()[0]) == 8         # nothing written past the capacity
    ctx.metad_set_hills(sh[:4], hh[:4])
    s2, h2 = ctx.metad_hills()
    assert np.array_equal(s2, sh[:4]) and np.array_equal(h2, hh[:4])
    ctx.step(1)
    assert len(ctx.metad_hills()[0]) == 8
    bad = P.make_metad(("distances", [(0, 99, 1.0)]), 0.02, 0.1, 10.0, 1, 8)
    with pytest.raises(P.PimdError):
        P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths, metad=bad)
    bad2 = P.make_metad(("distances", s.fad_dimer_cv_terms()), 0.02, 0.1, 1.0, 1, 8)   # gamma must be > 1
    with pytest.raises(P.PimdError):
        P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths, metad=bad2)
