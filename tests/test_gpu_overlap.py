"""Overlapped halves of the bead-atoms (two branches of the step's graph)
change the schedule only: in deterministic mode a trajectory with them is
bit-identical to one without."""
import numpy as np
import pytest

from paper_2503_23728_gb300 import synth as s

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_overlapped_halves_leave_the_trajectory_unchanged(ice_model):
    import __graft_entry__ as ge
    ge.build()
    from paper_2503_23728_gb300 import pimd as P
    w, r, m = ice_model
    runs = []
    for ov in (False, True):
        ctx = P.Context(w.replicas, w.dt_fs, w.gamma0_per_fs, precision="bf16_tc", widths=w.widths,
                        deterministic=True)
        ctx.set_weights(m)
        assert ctx.set_overlap(ov)                  # 41,472 bead-atoms: two halves of 16 beads
        ctx.step(4)
        q, p, st, _ = ctx.get_state()
        _, f, V = ctx.get_forces()
        runs.append((q, p, f, V))
        ctx.close()
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)
