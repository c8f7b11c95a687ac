"""The autotuner on the GPU: it measures the ice workload's angular method,
pair schedule and overlapped halves, leaves the trajectory's state as it
found it, stores the choice, and a second context of the same shape takes
the choice from the cache."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tuner_measures_applies_and_caches(ice_model, tmp_path):
    import __graft_entry__ as ge
    ge.build()
    from paper_2503_23728_gb300 import pimd as P
    from paper_2503_23728_gb300 import tuner
    w, r, m = ice_model
    cache = str(tmp_path / "tune.json")
    ctx = P.Context(w.replicas, w.dt_fs, w.gamma0_per_fs, precision="bf16_tc", widths=w.widths, timing=True)
    ctx.set_weights(m)
    ctx.step(2)
    q0, p0, s0, Q0 = ctx.get_state()
    got = tuner.tune(ctx, cache=cache, reps=1, steps=3)
    assert got["source"] == "measured"
    assert got["angular"] in ("moments", "pairs") and isinstance(got["overlap"], bool)
    q1, p1, s1, Q1 = ctx.get_state()
    assert s1 == s0 and np.array_equal(q1, q0) and np.array_equal(p1, p0) and np.array_equal(Q1, Q0)
    assert ctx.angular == got["angular"]
    table = json.load(open(cache))
    assert got["key"] in table
    ctx.step(2)                                   # the tuned context steps
    ctx.close()
    ctx2 = P.Context(w.replicas, w.dt_fs, w.gamma0_per_fs, precision="bf16_tc", widths=w.widths)
    ctx2.set_weights(m)
    again = tuner.tune(ctx2, cache=cache)
    assert again["source"] == "cache" and again["angular"] == got["angular"]
    assert again["overlap"] == got["overlap"]


def test_adjoint_residency_changes_no_force(water64_model):
    """The BF16 moment adjoint at 12 and at 16 warps per SM: the same
    arithmetic per bead-atom, so deterministic-mode forces, energies and
    virials are bit-identical; other values are refused."""
    import __graft_entry__ as ge
    ge.build()
    from paper_2503_23728_gb300 import pimd as P
    w, r, m = water64_model
    ctx = P.Context(w.replicas, w.dt_fs, w.gamma0_per_fs, precision="bf16_tc", widths=w.widths,
                    deterministic=True)
    ctx.set_weights(m)
    ctx.set_angular("moments")
    assert ctx.adjoint_warps == 12
    e12, f12, v12 = (t.cpu().numpy() for t in ctx.energy_forces())
    ctx.set_adjoint_warps(16)
    assert ctx.adjoint_warps == 16
    e16, f16, v16 = (t.cpu().numpy() for t in ctx.energy_forces())
    assert np.array_equal(f12, f16) and np.array_equal(e12, e16) and np.array_equal(v12, v16)
    ctx.step(2)   # the step graph runs with the wide adjoint
    with pytest.raises(P.PimdError):
        ctx.set_adjoint_warps(14)
    ctx.close()
