"""The allocation-free descriptor entry point (pimd_descriptors_noalloc).

Some callers cannot allocate device memory at all -- for example a host MD
engine that reserves the whole GPU for its own memory pool -- so they cannot
hand pimd_create a workspace. pimd_descriptors_noalloc serves them with
scratch held in a fixed static device array inside the library. This test
calls it through the C ABI and checks it against the workspace-based
pimd_descriptors on the same positions, twice in a row (the static array keeps
the previous call's contents), plus its size limit."""
import ctypes as ct

import numpy as np
import pytest

from paper_2503_23728_gb300 import synth as s

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _max_atoms() -> int:
    """PIMD_NOALLOC_MAX_ATOMS as the library's header declares it."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "pimd.h")).read()
    return int(re.search(r"#define\s+PIMD_NOALLOC_MAX_ATOMS\s+(\d+)", text).group(1))


def test_noalloc_descriptors_match_workspace_path():
    import __graft_entry__ as ge
    ge.build()
    from paper_2503_23728_gb300 import pimd as P
    w = s.workload("water64")
    r = w.replicas[0]
    rep = s.Replica(r.Z, r.x0, r.box, 1, r.T, r.seed)
    m = s.xavier_model(s.elements_of([rep]), w.widths, seed=3)
    ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths)
    ctx.set_weights(m)
    d = m.desc
    rng = np.random.default_rng(12)
    for call in range(2):
        x = (r.x0 + rng.normal(scale=0.1, size=r.x0.shape)).astype(np.float32).astype(np.float64)
        xt = torch.tensor(x, device="cuda")
        want = ctx.descriptors(xt).cpu().numpy()
        G = torch.full((rep.n_atoms, 64), float("nan"), dtype=torch.float64, device="cuda")
        P.pimd_descriptors_noalloc(ct.c_void_p(xt.data_ptr()), rep.n_atoms, rep.box, d["cutoff"], d["eta_R"],
                                   d["r_mu"], d["eta_A"], ct.c_void_p(G.data_ptr()),
                                   ct.c_void_p(torch.cuda.current_stream().cuda_stream))
        got = G.cpu().numpy()
        scale = np.abs(want).max(axis=0) + 1e-30
        assert np.all(np.abs(got - want) <= 1e-5 * scale), call
    # beyond the static array's size: a clear error, nothing launched
    p_max = _max_atoms()
    big = torch.zeros(p_max + 1, 3, dtype=torch.float64, device="cuda")
    Gb = torch.zeros(1, 64, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PimdError) as ei:
        P.pimd_descriptors_noalloc(ct.c_void_p(big.data_ptr()), p_max + 1, None, 6.0, 1.0, d["r_mu"], d["eta_A"],
                                   ct.c_void_p(Gb.data_ptr()))
    assert ei.value.code == -1 and "scratch" in P.pimd_last_error(None)
    ctx.close()


def test_noalloc_gas_phase_cluster_and_neighbour_overflow():
    """A free 18-atom cluster (no box, the small-replica kernels) against the
    workspace path, then a dense cluster whose atoms have more neighbours
    than the static array's slots: NBR_OVERFLOW from the host, after the
    list writes stopped at the slot cap."""
    import __graft_entry__ as ge
    ge.build()
    from paper_2503_23728_gb300 import pimd as P
    rep = [r for r in s.batch(n_rep=12, seed=5) if 14 <= r.n_atoms <= 24][0]
    rep = s.Replica(rep.Z, rep.x0, rep.box, 1, rep.T, rep.seed)
    m = s.xavier_model(s.elements_of([rep]), (64, 64), seed=3)
    ctx = P.Context([rep], 0.25, 0.01, precision="fp32", widths=(64, 64))
    ctx.set_weights(m)
    d = m.desc
    x = rep.x0.astype(np.float32).astype(np.float64)
    xt = torch.tensor(x, device="cuda")
    want = ctx.descriptors(xt).cpu().numpy()
    G = torch.full((rep.n_atoms, 64), float("nan"), dtype=torch.float64, device="cuda")
    P.pimd_descriptors_noalloc(ct.c_void_p(xt.data_ptr()), rep.n_atoms, None, d["cutoff"], d["eta_R"], d["r_mu"],
                               d["eta_A"], ct.c_void_p(G.data_ptr()))
    scale = np.abs(want).max(axis=0) + 1e-30
    assert np.all(np.abs(G.cpu().numpy() - want) <= 1e-5 * scale)
    ctx.close()
    dense = np.random.default_rng(1).uniform(0.0, 5.0, size=(200, 3))
    xd = torch.tensor(dense, device="cuda")
    Gd = torch.zeros(200, 64, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PimdError) as ei:
        P.pimd_descriptors_noalloc(ct.c_void_p(xd.data_ptr()), 200, None, 6.0, d["eta_R"], d["r_mu"], d["eta_A"],
                                   ct.c_void_p(Gd.data_ptr()))
    assert ei.value.code == -7 and "neighbours" in P.pimd_last_error(None)
    with pytest.raises(ValueError):
        P.pimd_descriptors_noalloc(ct.c_void_p(xd.data_ptr()), 200, None, 6.0, d["eta_R"], d["r_mu"][:30],
                                   d["eta_A"], ct.c_void_p(Gd.data_ptr()))
