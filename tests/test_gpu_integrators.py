"""GPU parity of the integrator variants (BAOAB splitting, Cayley free
ring-polymer step) against the FP64 oracle with the same Philox noise."""
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


VARIANTS = [("baoab", "exact"), ("obabo", "cayley"), ("baoab", "cayley")]


@pytest.mark.parametrize("splitting,free_rp", VARIANTS)
def test_fp64_trajectory_matches_oracle(fad_model, splitting, free_rp):
    """FAD, P = 16, FP64, PILE-L: 10 steps on both sides."""
    P = _P()
    w, rep, m = fad_model
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths, splitting=splitting,
                    free_rp=free_rp)
    ctx.set_weights(m)
    so = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m, splitting=splitting, free_rp=free_rp)
    ctx.step(10)
    so.step(10)
    q, p, st, Q = ctx.get_state()
    assert st == 10
    np.testing.assert_allclose(q.reshape(so.q.shape), so.q, rtol=0, atol=1e-9)
    np.testing.assert_allclose(p.reshape(so.p.shape), so.p, rtol=0, atol=1e-9 * np.abs(so.p).max())
    eg, eo = ctx.estimators()[0], so.estimators()
    for k in ("V_mean", "K_prim", "K_cv", "E_tot", "H_cons", "Q_thermo", "T_kin"):
        assert abs(eg[k] - eo[k]) <= 1e-8 * max(1.0, abs(eo[k])), k


@pytest.mark.parametrize("splitting,free_rp", VARIANTS)
def test_fp32_water_trajectory_matches_oracle(water64_model, splitting, free_rp):
    P = _P()
    w, r, m = water64_model
    rep = s.Replica(r.Z, r.x0, r.box, 4, r.T, r.seed, r.name)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths, splitting=splitting,
                    free_rp=free_rp)
    ctx.set_weights(m)
    so = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m, splitting=splitting, free_rp=free_rp)
    ctx.step(5)
    so.step(5)
    q, p, _, _ = ctx.get_state()
    np.testing.assert_allclose(q.reshape(so.q.shape), so.q, rtol=0, atol=2e-5)
    assert float(np.abs(p.reshape(so.p.shape) - so.p).max() / np.abs(so.p).max()) < 1e-4


def test_large_omega_dt_cayley_stays_bounded():
    """P = 64 at 10 K with dt = 4 fs (omega_k dt up to ~5): with the Cayley
    step the free ring polymer's energy stays finite and the estimators are
    finite after many steps; it matches the oracle for the first steps."""
    P = _P()
    x0 = np.random.default_rng(2).normal(size=(4, 3)) * 0.1
    rep = s.Replica(np.full(4, s.H, dtype=np.int32), x0, (0.0, 0.0, 0.0), 64, 10.0, 7)
    ctx = P.Context([rep], 4.0, 0.01, precision="fp64", potential=P.POT_HARMONIC, omega=0.0786,
                    splitting="baoab", free_rp="cayley")
    so = O.System(rep, s.MASS, 4.0, 0.01, potential="harmonic", omega=0.0786, splitting="baoab",
                  free_rp="cayley")
    ctx.step(20)
    so.step(20)
    q, p, _, _ = ctx.get_state()
    np.testing.assert_allclose(q.reshape(so.q.shape), so.q, rtol=0, atol=1e-10)
    ctx.step(500)
    e = ctx.estimators()[0]
    assert all(np.isfinite(e[k]) for k in ("E_tot", "K_prim", "K_cv", "H_cons"))


@pytest.mark.parametrize("splitting", ["obabo", "baoab"])
def test_staging_fp64_trajectory_and_estimators_match_oracle(fad_model, splitting):
    """Staging coordinates (masses k/(k-1) m, all at omega_P), FAD P = 16,
    FP64: state after 10 steps and every estimator against the oracle."""
    P = _P()
    w, rep, m = fad_model
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths, splitting=splitting,
                    transform="staging")
    ctx.set_weights(m)
    so = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m, splitting=splitting, transform="staging")
    q0, p0, _, _ = ctx.get_state()
    np.testing.assert_allclose(q0.reshape(so.q.shape), so.q, rtol=0, atol=1e-12)
    np.testing.assert_allclose(p0.reshape(so.p.shape), so.p, rtol=1e-12, atol=1e-14)
    ctx.step(10)
    so.step(10)
    q, p, st, _ = ctx.get_state()
    np.testing.assert_allclose(q.reshape(so.q.shape), so.q, rtol=0, atol=1e-9)
    np.testing.assert_allclose(p.reshape(so.p.shape), so.p, rtol=0, atol=1e-9 * np.abs(so.p).max())
    eg, eo = ctx.estimators()[0], so.estimators()
    for k in ("V_mean", "K_prim", "K_cv", "E_tot", "H_cons", "Q_thermo", "T_kin"):
        assert abs(eg[k] - eo[k]) <= 1e-8 * max(1.0, abs(eo[k])), k


def test_staging_fp32_water_matches_oracle(water64_model):
    P = _P()
    w, r, m = water64_model
    rep = s.Replica(r.Z, r.x0, r.box, 4, r.T, r.seed, r.name)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths, transform="staging")
    ctx.set_weights(m)
    so = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m, transform="staging")
    ctx.step(5)
    so.step(5)
    q, p, _, _ = ctx.get_state()
    np.testing.assert_allclose(q.reshape(so.q.shape), so.q, rtol=0, atol=2e-5)
    assert float(np.abs(p.reshape(so.p.shape) - so.p).max() / np.abs(so.p).max()) < 1e-4
    eg, eo = ctx.estimators()[0], so.estimators()
    for k in ("V_mean", "K_cv", "E_tot"):
        assert abs(eg[k] - eo[k]) <= 1e-4 * max(1.0, abs(eo[k])), k
