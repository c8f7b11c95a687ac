"""Host logic of the autotuner (no GPU): the workload key, the cache round
trip, and that a cached choice is applied without timing anything."""
import json

import numpy as np

from paper_2503_23728_gb300 import tuner


class _Rep:
    def __init__(self, n, p):
        self.n_atoms, self.n_beads = n, p


class _FakeCtx:
    """Records the calls the tuner makes; timings are made up."""

    def __init__(self, reps, mean_nbrs=86.3):
        self.replicas = reps
        self.widths = (128, 128, 128)
        self.precision = "bf16_tc"
        self._nnb = np.full(sum(r.n_atoms * r.n_beads for r in reps), mean_nbrs)
        self.calls = []
        self.state = (np.zeros(3), np.zeros(3), 7, np.zeros(1))
        self.overlap = True

    def neighbours(self):
        return self._nnb, None

    def tune(self, reps=3):
        self.calls.append("tune")
        return {"angular": "moments", "band_length": 0, "best_ms": 0.3, "default_ms": 0.3, "adjoint_warps": 16}

    def set_angular(self, a):
        self.calls.append(("angular", a))

    def set_schedule(self, b):
        self.calls.append(("schedule", b))

    def set_adjoint_warps(self, n):
        self.calls.append(("adjoint_warps", n))

    def set_overlap(self, on):
        self.calls.append(("overlap", on))
        self.overlap = on
        return True

    def get_state(self):
        return self.state

    def set_state(self, q, p, step, Q):
        self.calls.append(("set_state", step))


def test_key_names_the_workload_shape():
    k1 = tuner.workload_key(_FakeCtx([_Rep(1296, 32)]))
    assert k1 == "1296x32x1|w128-128-128|bf16_tc"
    k2 = tuner.workload_key(_FakeCtx([_Rep(10, 8), _Rep(12, 16), _Rep(10, 8)], mean_nbrs=9.0))
    assert k2 == "10x8x2,12x16x1|w128-128-128|bf16_tc"


def test_cached_choice_is_applied_without_timing(tmp_path, monkeypatch):
    path = str(tmp_path / "cache.json")
    ctx = _FakeCtx([_Rep(1296, 32)])
    key = tuner.workload_key(ctx)
    json.dump({key: [{"angular": "pairs", "band_length": 10, "overlap": False, "mean_neighbours": 85.0,
                      "adjoint_warps": 16}]}, open(path, "w"))
    monkeypatch.setattr(tuner, "_step_ms", lambda *a, **k: (_ for _ in ()).throw(AssertionError("timed")))
    got = tuner.tune(ctx, cache=path)
    assert got["source"] == "cache" and got["band_length"] == 10
    assert "tune" not in ctx.calls
    assert ("angular", "pairs") in ctx.calls and ("schedule", 10) in ctx.calls and ("overlap", False) in ctx.calls
    assert ("adjoint_warps", 16) in ctx.calls


def test_measured_choice_is_stored_and_state_restored(tmp_path, monkeypatch):
    path = str(tmp_path / "cache.json")
    ctx = _FakeCtx([_Rep(1296, 32)])
    times = iter([0.42, 0.44])   # overlapped, then sequential
    monkeypatch.setattr(tuner, "_step_ms", lambda *a, **k: next(times))
    got = tuner.tune(ctx, cache=path)
    assert got["source"] == "measured" and got["overlap"] is True
    assert ctx.calls.count("tune") == 1 and ("set_state", 7) in ctx.calls
    assert ctx.overlap is True
    table = json.load(open(path))
    (entry,) = table[tuner.workload_key(ctx)]
    assert entry["overlap"] is True and entry["mean_neighbours"] == 86.3 and entry["adjoint_warps"] == 16
    # a second context of the same shape, its neighbour count drifted by a
    # fraction (beads spread from their initial positions), reads it back
    ctx2 = _FakeCtx([_Rep(1296, 32)], mean_nbrs=85.4)
    assert tuner.tune(ctx2, cache=path)["source"] == "cache"


def test_a_different_density_is_measured_and_stored_beside(tmp_path, monkeypatch):
    path = str(tmp_path / "cache.json")
    times = iter([0.42, 0.44, 0.50, 0.40])
    monkeypatch.setattr(tuner, "_step_ms", lambda *a, **k: next(times))
    assert tuner.tune(_FakeCtx([_Rep(1296, 32)], mean_nbrs=86.3), cache=path)["overlap"] is True
    got = tuner.tune(_FakeCtx([_Rep(1296, 32)], mean_nbrs=60.0), cache=path)
    assert got["source"] == "measured" and got["overlap"] is False
    table = json.load(open(path))
    assert sorted(e["mean_neighbours"] for e in table[got["key"]]) == [60.0, 86.3]
    # each density finds its own entry
    assert tuner.tune(_FakeCtx([_Rep(1296, 32)], mean_nbrs=61.0), cache=path)["overlap"] is False
    assert tuner.tune(_FakeCtx([_Rep(1296, 32)], mean_nbrs=88.0), cache=path)["overlap"] is True
