"""Autotuner with a persistent cache of its choices.

For a context it chooses, by timing them on the live workload:
  * how the angular terms are evaluated (moment tensors or pair sums) and,
    for pair sums, the band length of the pair schedule (`pimd_tune`, which
    times the descriptor forward and the adjoint of every candidate with
    CUDA events);
  * whether the step runs the two halves of its bead-atoms as overlapping
    branches of its graph (`pimd_set_overlap`), from whole-step timings.
The choices are stored in a JSON file under a key of the workload's shape:
atoms and beads of every replica (sorted multiset), the mean neighbour count
rounded to an integer, the network widths and the precision. A later context
with the same key applies them without timing anything.

The step timings advance the trajectory; the tuner puts the state back
(q, p, step counter and thermostat heat) before it returns.
"""
from __future__ import annotations

import json
import os

import numpy as np

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")


def workload_key(ctx) -> str:
    nnb, _ = ctx.neighbours()
    shapes = sorted((int(r.n_atoms), int(r.n_beads)) for r in ctx.replicas)
    # run-length form of the sorted (N, P) multiset keeps batch keys short
    runs = []
    for s in shapes:
        if runs and runs[-1][0] == s:
            runs[-1][1] += 1
        else:
            runs.append([s, 1])
    shp = ",".join("%dx%dx%d" % (n, p, c) for (n, p), c in runs)
    widths = "-".join(str(int(w)) for w in ctx.widths)
    return "%s|nb%d|w%s|%s" % (shp, int(round(float(nnb.mean()))), widths, ctx.precision)


def _load(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path: str, table: dict) -> None:
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _step_ms(ctx, steps: int) -> float:
    """Mean device time of single-step graph launches (CUDA events)."""
    torch = ctx.torch
    st = torch.cuda.current_stream() if ctx.stream is None else ctx.stream
    ctx.step(1)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for _ in range(steps):
        ctx.step(1)
    t1.record(st)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / steps


def apply(ctx, choice: dict) -> None:
    ctx.set_angular(choice["angular"])
    if choice["angular"] == "pairs":
        ctx.set_schedule(int(choice["band_length"]))
    ctx.set_overlap(bool(choice.get("overlap", True)))


def tune(ctx, cache: str | None = DEFAULT_CACHE, reps: int = 3, steps: int = 10, retune: bool = False) -> dict:
    """The tuned launch configuration of ctx (applied to it), from the cache
    when the workload's key is there, else measured and added to the cache.
    cache=None measures without reading or writing a file."""
    key = workload_key(ctx)
    table = _load(cache) if cache else {}
    if not retune and key in table:
        choice = dict(table[key])
        apply(ctx, choice)
        choice["source"] = "cache"
        choice["key"] = key
        return choice
    kern = ctx.tune(reps=reps)   # angular method and pair schedule, applied by the library
    choice = {"angular": kern["angular"], "band_length": int(kern["band_length"]),
              "kernels_ms": float(kern["best_ms"])}
    # overlapped halves, from whole-step timings (state restored afterwards)
    q, p, step, Q = ctx.get_state()
    has = ctx.set_overlap(True)
    choice["overlap"] = has
    if has:
        ms_on = _step_ms(ctx, steps)
        ctx.set_overlap(False)
        ms_off = _step_ms(ctx, steps)
        choice["overlap"] = bool(ms_on < ms_off)
        choice["step_ms"] = {"overlap": ms_on, "sequential": ms_off}
        ctx.set_overlap(choice["overlap"])
    ctx.set_state(q, p, step, Q)
    if cache:
        table = _load(cache)
        table[key] = {k: v for k, v in choice.items() if k not in ("source", "key")}
        _store(cache, table)
    choice["source"] = "measured"
    choice["key"] = key
    return choice
