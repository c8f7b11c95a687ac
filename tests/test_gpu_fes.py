"""GPU free-energy rows of Sec. 2.5 through the C ABI against the oracle:
the bead-resolved CV histogram (bins bit-exact; weights of a biased run to
FP64 rounding), the path-integral FES from a histogram, and the
well-tempered FES of a set of hills. Every input is seeded and synthetic
(bead positions from the test's generator, hills chosen here); histograms
fed to the GPU's FES call are the oracle's."""
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


def _configs(rep, P, n, seed):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        x = np.repeat(rep.x0[None], P, axis=0) + rng.normal(scale=0.12, size=(P, rep.n_atoms, 3))
        yield x


@pytest.mark.parametrize("biased", [False, True])
def test_cv_histogram_matches_oracle(fad_model, biased):
    """FAD, P = 8, FP64 path, dimer CV on every bead: 30 seeded bead
    configurations evaluated through pimd_energy_forces, each added to the
    histogram. Without hills every weight is 1 and the counts are bit-exact;
    with hills the weights exp(sum_k V_b / (k_B T P)) agree to 1e-12."""
    P = _P()
    w, r, m = fad_model
    nb = 8
    rep = s.Replica(r.Z, r.x0, r.box, nb, r.T, r.seed, r.name)
    terms = s.fad_dimer_cv_terms()
    md = P.make_metad(("distances", terms), 0.0, 0.1, 10.0, 1 << 30, 64)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths, metad=md)
    ctx.set_weights(m)
    mo = O.Metad(("distances", terms), rep.n_atoms, nb, 0.0, 0.1, 10.0, 1 << 30, max_hills=64)
    if biased:
        hs, hh = np.array([-1.6, -1.4, -1.5]), np.array([0.02, 0.015, 0.01])
        ctx.metad_set_hills(hs, hh)
        mo.set_hills(hs, hh)
    lo, hi, n_bins = -2.2, -0.8, 28
    shift = 0.5 if biased else 0.0
    hist, wsum = None, None
    ho = O.CvHistogram(nb, lo, hi, n_bins, rep.T, log_w_shift=shift)
    for x in _configs(rep, nb, 30, seed=41):
        ctx.energy_forces(torch.tensor(x.reshape(-1, 3), device="cuda"))
        hist, wsum = ctx.cv_histogram((lo, hi), n_bins, hist, wsum, log_w_shift=shift)
        sk = np.array([mo.cv(x[k], rep.box)[0] for k in range(nb)])
        vk = np.array([mo.bias(v)[0] for v in sk])
        ho.add(sk, vk)
    hg, wg = hist.cpu().numpy(), wsum.cpu().numpy()
    assert np.array_equal(hg > 0, ho.hist > 0)           # the same bins
    if biased:
        np.testing.assert_allclose(hg, ho.hist, rtol=1e-12, atol=0)
        np.testing.assert_allclose(wg, ho.wsum, rtol=1e-12)
    else:
        assert np.array_equal(hg, ho.hist)                # integer counts, weight 1
        assert wg[0] == ho.wsum[0] == 30.0
    assert ho.hist.sum() > 0


def test_pi_fes_matches_oracle(fad_model):
    """The oracle's bead-resolved histogram of 4 beads (Gaussian CV samples,
    some bins empty) uploaded to the device: pimd_pi_fes gives the oracle's
    F_k and path-integral F to 1e-12, +inf in the same empty bins."""
    P = _P()
    w, r, m = fad_model
    nb = 4
    rep = s.Replica(r.Z, r.x0, r.box, nb, r.T, r.seed, r.name)
    md = P.make_metad(("distances", s.fad_dimer_cv_terms()), 0.0, 0.1, 10.0, 1 << 30, 8)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths, metad=md)
    ctx.set_weights(m)
    lo, hi, n_bins = -1.0, 1.5, 40
    ho = O.CvHistogram(nb, lo, hi, n_bins, rep.T)
    rng = np.random.default_rng(2)
    for _ in range(3000):
        ho.add(rng.normal(scale=0.3, size=nb), rng.uniform(0, 0.01, size=nb))
    Fo, Fko = ho.fes()
    F, Fk = ctx.pi_fes(torch.tensor(ho.hist, device="cuda"), torch.tensor(ho.wsum, device="cuda"), (lo, hi))
    F, Fk = F.cpu().numpy(), Fk.cpu().numpy()
    assert np.array_equal(np.isinf(F), np.isinf(Fo)) and np.isinf(Fo).any()
    fin = np.isfinite(Fo)
    np.testing.assert_allclose(F[fin], Fo[fin], rtol=1e-12, atol=1e-15)
    finK = np.isfinite(Fko)
    assert np.array_equal(np.isfinite(Fk), finK)
    np.testing.assert_allclose(Fk[finK], Fko[finK], rtol=1e-12, atol=1e-15)


def test_metad_fes_matches_oracle(fad_model):
    """-(gamma / (gamma - 1)) V(s) of the same hills on both sides."""
    P = _P()
    w, r, m = fad_model
    rep = s.Replica(r.Z, r.x0, r.box, 4, r.T, r.seed, r.name)
    md = P.make_metad(("distances", s.fad_dimer_cv_terms()), 0.02, 0.1, 12.0, 5, 64)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths, metad=md)
    ctx.set_weights(m)
    mo = O.Metad(("distances", s.fad_dimer_cv_terms()), rep.n_atoms, 4, 0.02, 0.1, 12.0, 5, max_hills=64)
    rng = np.random.default_rng(8)
    hs, hh = rng.uniform(-2.0, 0.0, size=24), rng.uniform(0.001, 0.02, size=24)
    ctx.metad_set_hills(hs, hh)
    mo.set_hills(hs, hh)
    grid = np.linspace(-2.5, 0.5, 301)
    F = ctx.metad_fes(torch.tensor(grid)).cpu().numpy()
    np.testing.assert_allclose(F, mo.fes(grid), rtol=1e-13, atol=1e-16)
    assert ctx.metad_fes(torch.tensor(np.zeros(0))).numel() == 0


def test_fes_calls_reject_bad_arguments(fad_model):
    P = _P()
    w, r, m = fad_model
    rep = s.Replica(r.Z, r.x0, r.box, 4, r.T, r.seed, r.name)
    plain = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths)
    plain.set_weights(m)
    with pytest.raises(P.PimdError) as e:
        plain.cv_histogram((0.0, 1.0), 10)
    assert e.value.code == -2                             # STATE: no CV configured
    md = P.make_metad(("distances", s.fad_dimer_cv_terms()), 0.0, 0.1, 10.0, 1 << 30, 8)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp64", widths=w.widths, metad=md)
    ctx.set_weights(m)
    for bad in (((1.0, 1.0), 10), ((0.0, 1.0), 0)):
        with pytest.raises(P.PimdError) as e:
            ctx.cv_histogram(*bad)
        assert e.value.code == -1
    h = torch.zeros((4, 10), dtype=torch.float64, device="cuda")
    ws = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PimdError) as e:
        ctx.cv_histogram((0.0, 1.0), 10, h, ws, replica=3)
    assert e.value.code == -1
