"""The bead-sharded ring polymer (beads split for the forces, atoms split for
the ring-polymer step, two all-to-alls per step) on the CPU: the oracle's
step cut at its force evaluation composes back to the whole step bit for
bit, and two gloo ranks running the sharded step through the package's
transposes reproduce a single-process oracle trajectory bit for bit."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2503_23728_gb300 import shard as SH
from paper_2503_23728_gb300 import synth as s

torch = pytest.importorskip("torch")


def _free_port():
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    p = sk.getsockname()[1]
    sk.close()
    return p


def test_split_covers_and_balances():
    for n, g in ((32, 1), (32, 3), (10, 4), (7, 7)):
        parts = SH.split(n, g)
        assert parts[0][0] == 0 and parts[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        sizes = [hi - lo for lo, hi in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        SH.ShardPlan(4, 10, 5)


def _fad_system(fad_model, P=4, **kw):
    w, r, m = fad_model
    rep = s.Replica(r.Z, r.x0, r.box, P, r.T, r.seed, r.name)
    return rep, m, O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m, **kw)


@pytest.mark.parametrize("splitting,transform", [("obabo", "normal_modes"), ("baoab", "normal_modes"),
                                                 ("obabo", "staging")])
def test_oracle_step_halves_compose_to_the_whole_step(fad_model, splitting, transform):
    """ring_start over atom ranges, forces of the new beads, ring_finish over
    the same ranges: q and p equal or_step's bit for bit (Sec. 2.1 splitting
    cut at the force evaluation; every coordinate sees the same operations
    and noise counters), the heat to rounding."""
    rep, m, ref = _fad_system(fad_model, splitting=splitting, transform=transform)
    _, _, cut = _fad_system(fad_model, splitting=splitting, transform=transform)
    ref.step(5)
    ranges = [(0, 3), (3, 7), (7, rep.n_atoms)]
    for _ in range(5):
        for lo, hi in ranges:
            cut.ring_start(lo, hi)
        _, F, _ = O.energy_forces_batch(m, rep.Z, cut.xb, rep.box)
        for lo, hi in ranges:
            cut.ring_finish(lo, hi, F)
        cut.f[:] = F
        cut.step_count.value += 1
    assert np.array_equal(cut.q, ref.q) and np.array_equal(cut.p, ref.p)
    assert abs(cut.Q.value - ref.Q.value) <= 1e-12 * max(1.0, abs(ref.Q.value))


class _OracleRing:
    """An atom slice's ring-polymer step on the oracle (full-size arrays,
    only the slice advanced)."""

    def __init__(self, system, atoms):
        self.s, (self.lo, self.hi) = system, atoms
        self.f = np.zeros_like(system.f)

    def positions(self):
        # bead positions as the oracle formed them for its last forces
        return torch.tensor(self.s.xb[:, self.lo:self.hi, :].copy())

    def set_forces(self, f):
        self.f[:, self.lo:self.hi, :] = f.numpy()

    def start(self):
        self.s.ring_start(self.lo, self.hi, self.f)
        return torch.tensor(self.s.xb[:, self.lo:self.hi, :].copy())

    def finish(self, f):
        self.f[:, self.lo:self.hi, :] = f.numpy()
        self.s.ring_finish(self.lo, self.hi, self.f)
        self.s.step_count.value += 1


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = s.workload("fad")
    r = w.replicas[0]
    m = s.xavier_model(s.elements_of(w.replicas), w.widths, seed=11)
    G = O.descriptors(m, r.x0, r.box)
    s.set_normalisation(m, G, r.Z)
    rep = s.Replica(r.Z, r.x0, r.box, 6, r.T, r.seed, r.name)
    plan = SH.ShardPlan(rep.n_beads, rep.n_atoms, world)
    sysm = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m)

    def forces(xb):
        _, F, _ = O.energy_forces_batch(m, rep.Z, xb.numpy(), rep.box)
        return torch.tensor(F)

    ring = _OracleRing(sysm, plan.atoms[rank])
    run = SH.ShardedRingPolymer(plan, rank, forces, ring)
    run.prime()
    run.step(6)
    lo, hi = plan.atoms[rank]
    mine = (lo, hi, sysm.q[:, lo:hi, :].copy(), sysm.p[:, lo:hi, :].copy(), sysm.Q.value)
    got = [None] * world
    dist.all_gather_object(got, mine)
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_trajectory():
    """FAD, P = 6, two ranks: 3 beads each for the forces, 5 atoms each for
    the ring-polymer step, six steps; the assembled q and p equal a
    single-process oracle run bit for bit, and the heats add up."""
    import torch.multiprocessing as mp
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    w = s.workload("fad")
    r = w.replicas[0]
    m = s.xavier_model(s.elements_of(w.replicas), w.widths, seed=11)
    s.set_normalisation(m, O.descriptors(m, r.x0, r.box), r.Z)
    rep = s.Replica(r.Z, r.x0, r.box, 6, r.T, r.seed, r.name)
    ref = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m)
    ref.step(6)
    q = np.zeros_like(ref.q)
    p = np.zeros_like(ref.p)
    Q = 0.0
    for lo, hi, qa, pa, Qa in out[0]:
        q[:, lo:hi, :] = qa
        p[:, lo:hi, :] = pa
        Q += Qa
    assert all(np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3]) for a, b in zip(out[0], out[1]))
    assert np.array_equal(q, ref.q) and np.array_equal(p, ref.p)
    assert abs(Q - ref.Q.value) <= 1e-12 * max(1.0, abs(ref.Q.value))
