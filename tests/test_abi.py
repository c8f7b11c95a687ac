"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/pimd.h declares, and validates arguments."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

import __graft_entry__ as ge
from paper_2503_23728_gb300 import pimd as P
from paper_2503_23728_gb300 import synth as s

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ge.build()
    return P.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|void|const char\*|size_t)\s+(pimd_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pimd_create" in names and "pimd_step" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(P.EXPORTS) <= names


def test_abi_version(lib):
    assert P.pimd_abi_version() == 3


def _cfg(**kw):
    base = dict(dt_fs=0.5, gamma0_per_fs=0.001, precision="fp32", widths=(128, 128, 128))
    base.update(kw)
    return P.make_config(**base)


def test_workspace_size_scales_with_system(lib):
    keep = P._Keep()
    w = s.workload("water64")
    small = P.make_replicas(w.replicas, keep)
    n1 = P.pimd_workspace_size(_cfg(), small)
    big = P.make_replicas([s.water_box(5, seed=3)], keep)
    n2 = P.pimd_workspace_size(_cfg(), big)
    assert 0 < n1 < n2
    # FP32 / BF16 hold the angular moments (6 x 32 float4 per bead-atom); FP64
    # records are larger than FP32 ones otherwise
    B = sum(r.n_atoms * r.n_beads for r in w.replicas)
    mom = 6 * 32 * 16 * B
    assert n1 > mom
    assert P.pimd_workspace_size(_cfg(precision="fp64"), small) > n1 - mom


@pytest.mark.parametrize("bad", [
    dict(dt_fs=0.0), dict(precision=7), dict(max_neighbours=40), dict(max_neighbours=512),
    dict(widths=(128, 64)), dict(widths=(96,)), dict(widths=()), dict(cutoff=-1.0),
])
def test_config_errors(lib, bad):
    keep = P._Keep()
    reps = P.make_replicas(s.workload("water64").replicas, keep)
    with pytest.raises(P.PimdError) as ei:
        P.pimd_workspace_size(_cfg(**bad), reps)
    assert ei.value.code in (-1, -8)
    assert P.pimd_last_error()


@pytest.mark.parametrize("bad, code", [
    (dict(precision="bf16_tc", gfn=(32, 3)), -8), (dict(precision="fp64"), -8), (dict(gfn=(48, 3)), -8),
    (dict(gfn=(64, 9)), -1), (dict(gfn=(64, -1)), -1), (dict(cutoff=0.0), -1),
])
def test_gfn_config_errors(lib, bad, code):
    keep = P._Keep()
    reps = P.make_replicas(s.workload("water64").replicas, keep)
    kw = dict(potential=P.POT_GFN, gfn=(64, 3))
    kw.update(bad)
    with pytest.raises(P.PimdError) as ei:
        P.pimd_workspace_size(_cfg(**kw), reps)
    assert ei.value.code == code


def test_gfn_workspace_holds_edge_states(lib):
    """The head keeps e_ij (maxnb slots x F floats per bead-atom) between
    iterations; no descriptors, network buffers or moments."""
    keep = P._Keep()
    w = s.workload("water64")
    reps = P.make_replicas(w.replicas, keep)
    B = sum(r.n_atoms * r.n_beads for r in w.replicas)
    n64 = P.pimd_workspace_size(_cfg(potential=P.POT_GFN, gfn=(64, 3)), reps)
    n128 = P.pimd_workspace_size(_cfg(potential=P.POT_GFN, gfn=(128, 3)), reps)
    assert n128 - n64 >= 4 * 64 * B * 128
    assert n64 > 4 * 64 * B * 128


def test_replica_errors(lib):
    keep = P._Keep()
    r = s.workload("water64").replicas[0]
    # box shorter than twice the cutoff
    small = s.Replica(r.Z, r.x0, (10.0, 10.0, 10.0), 4, 300.0, 1)
    with pytest.raises(P.PimdError):
        P.pimd_workspace_size(_cfg(), P.make_replicas([small], keep))
    # too many beads
    many = s.Replica(r.Z, r.x0, r.box, 300, 300.0, 1)
    with pytest.raises(P.PimdError):
        P.pimd_workspace_size(_cfg(), P.make_replicas([many], keep))
    # unknown element without a mass
    odd = s.Replica(np.array([1, 17], dtype=np.int32), np.zeros((2, 3)), (0, 0, 0), 4, 300.0, 1)
    with pytest.raises(P.PimdError):
        P.pimd_workspace_size(_cfg(), P.make_replicas([odd], keep))
    # ... which an explicit mass fixes
    assert P.pimd_workspace_size(_cfg(), P.make_replicas([odd], keep, masses={1: 1.008, 17: 35.45})) > 0
    with pytest.raises(P.PimdError):
        P.pimd_workspace_size(_cfg(), (P.pimd_replica_desc * 0)())


def test_create_rejects_small_or_misaligned_workspace(lib):
    keep = P._Keep()
    reps = P.make_replicas(s.workload("fad").replicas, keep)
    cfg = _cfg(widths=(64, 64))
    n = P.pimd_workspace_size(cfg, reps)
    with pytest.raises(P.PimdError) as ei:
        P.pimd_create(cfg, reps, 0x100000, n - 4096)
    assert ei.value.code == -3
    with pytest.raises(P.PimdError) as ei:
        P.pimd_create(cfg, reps, 0x100010, n)
    assert ei.value.code == -1
    with pytest.raises(P.PimdError):
        P.pimd_create(cfg, reps, 0, n)


def test_null_context_calls_fail_cleanly(lib):
    assert lib.pimd_step(None, 1) == -1
    assert lib.pimd_sync(None) == -1
    assert lib.pimd_estimators(None, None, 1) == -1
    assert P.pimd_last_error(None)
    lib.pimd_destroy(None)
