"""Bead-sharded ring polymer over several GPUs (one process per GPU).

The beads of a ring polymer interact only through the springs of the
ring-polymer step (Sec. 2.1): the force evaluation of every bead is
independent of the others. A step is therefore split over G ranks as:

  * rank r evaluates the forces of its bead slice (P_r beads, all N atoms);
  * one all-to-all turns the bead-sliced forces [P_r][N][3] into atom-sliced
    forces [P][N_r][3] (every bead of the rank's atom slice);
  * each rank runs the ring-polymer step (normal-mode transform, PILE-L,
    free ring-polymer propagation) on its atom slice, which needs every bead
    of an atom but no other atom;
  * one all-to-all turns the new atom-sliced positions back into bead slices.

Two all-to-alls per step, each 3 P N / G values per rank, FP32 on the wire
(positions and forces are FP32 on the working precisions' force path). The
thermostat noise of each atom slice is drawn at the whole system's counter
indices, so the sharded run follows the single-GPU trajectory.

This module holds the decomposition, the two transposes (torch.distributed,
any backend: NCCL on GPUs, gloo on CPUs) and the GPU adapters around the C
ABI (`Context.energy_forces` for a bead slice, `Context.ring_start` /
`ring_finish` for an atom slice). Any force function and ring object with the
same methods can be plugged in.
"""
from __future__ import annotations

import numpy as np


def split(n: int, parts: int) -> list:
    """Contiguous, balanced ranges [lo, hi) of n items over `parts` owners."""
    base, extra = divmod(n, parts)
    out, lo = [], 0
    for r in range(parts):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


class ShardPlan:
    """Bead slices and atom slices of one ring polymer (P beads, N atoms)
    over `world` ranks."""

    def __init__(self, n_beads: int, n_atoms: int, world: int):
        if world < 1 or world > n_beads or world > n_atoms:
            raise ValueError("need 1 <= world <= min(P, N)")
        self.P, self.N, self.world = int(n_beads), int(n_atoms), int(world)
        self.beads = split(self.P, self.world)
        self.atoms = split(self.N, self.world)

    def n_beads(self, r: int) -> int:
        lo, hi = self.beads[r]
        return hi - lo

    def n_atoms(self, r: int) -> int:
        lo, hi = self.atoms[r]
        return hi - lo


def beads_to_atoms(t, plan: ShardPlan, rank: int, group=None, wire_dtype=None):
    """[P_rank][N][3] (this rank's beads, every atom) -> [P][N_rank][3]
    (every bead, this rank's atoms): one all-to-all."""
    import torch
    import torch.distributed as dist
    wd = wire_dtype or t.dtype
    send = torch.cat([t[:, lo:hi, :].reshape(-1) for (lo, hi) in plan.atoms]).to(wd).contiguous()
    in_sizes = [plan.n_beads(rank) * plan.n_atoms(s) * 3 for s in range(plan.world)]
    out_sizes = [plan.n_beads(s) * plan.n_atoms(rank) * 3 for s in range(plan.world)]
    recv = torch.empty(sum(out_sizes), dtype=wd, device=t.device)
    if plan.world == 1:
        recv.copy_(send)
    else:
        dist.all_to_all_single(recv, send, out_sizes, in_sizes, group=group)
    parts = torch.split(recv, out_sizes)
    na = plan.n_atoms(rank)
    return torch.cat([p.view(plan.n_beads(s), na, 3) for s, p in enumerate(parts)], dim=0).to(t.dtype)


def atoms_to_beads(t, plan: ShardPlan, rank: int, group=None, wire_dtype=None):
    """[P][N_rank][3] (every bead, this rank's atoms) -> [P_rank][N][3]
    (this rank's beads, every atom): one all-to-all."""
    import torch
    import torch.distributed as dist
    wd = wire_dtype or t.dtype
    send = torch.cat([t[lo:hi].reshape(-1) for (lo, hi) in plan.beads]).to(wd).contiguous()
    in_sizes = [plan.n_beads(s) * plan.n_atoms(rank) * 3 for s in range(plan.world)]
    out_sizes = [plan.n_beads(rank) * plan.n_atoms(s) * 3 for s in range(plan.world)]
    recv = torch.empty(sum(out_sizes), dtype=wd, device=t.device)
    if plan.world == 1:
        recv.copy_(send)
    else:
        dist.all_to_all_single(recv, send, out_sizes, in_sizes, group=group)
    parts = torch.split(recv, out_sizes)
    pb = plan.n_beads(rank)
    return torch.cat([p.view(pb, plan.n_atoms(s), 3) for s, p in enumerate(parts)], dim=1).to(t.dtype)


class ShardedRingPolymer:
    """One rank's part of the bead-sharded step.

    force_fn(x) -> f: bead forces of this rank's bead slice, x and f
        [P_rank][N][3].
    ring: this rank's atom slice with every bead; positions() -> [P][N_rank][3]
        (current beads), set_forces(f), start() -> [P][N_rank][3] (new beads),
        finish(f) with f [P][N_rank][3].
    """

    def __init__(self, plan: ShardPlan, rank: int, force_fn, ring, group=None, wire_dtype=None):
        self.plan, self.rank, self.force_fn, self.ring = plan, rank, force_fn, ring
        self.group, self.wire = group, wire_dtype
        self.steps = 0

    def _forces_of(self, x_atoms):
        xb = atoms_to_beads(x_atoms, self.plan, self.rank, self.group, self.wire)
        fb = self.force_fn(xb)
        return beads_to_atoms(fb, self.plan, self.rank, self.group, self.wire)

    def prime(self):
        """Forces of the current positions (before the first step)."""
        self.ring.set_forces(self._forces_of(self.ring.positions()))

    def step(self, n: int = 1):
        for _ in range(n):
            x_atoms = self.ring.start()
            self.ring.finish(self._forces_of(x_atoms))
            self.steps += 1


class GpuBeadForces:
    """Forces of a bead slice on this rank's GPU through the C ABI: a context
    holding the slice's beads of the whole system (its own ring-polymer
    state is not used)."""

    def __init__(self, replica, n_beads: int, model, dt_fs: float, gamma0_per_fs: float, precision="fp32",
                 widths=(128, 128, 128), deterministic=True, **kw):
        from . import pimd as P
        from .synth import Replica
        rep = Replica(replica.Z, replica.x0, replica.box, int(n_beads), replica.T, replica.seed, replica.name)
        self.N = rep.n_atoms
        self.ctx = P.Context([rep], dt_fs, gamma0_per_fs, precision=precision, widths=widths,
                             deterministic=deterministic, **kw)
        self.ctx.set_weights(model)

    def __call__(self, x):
        _, f, _ = self.ctx.energy_forces(x.reshape(-1, 3).contiguous(), want_virial=False)
        return f.view(-1, self.N, 3)


class GpuAtomRing:
    """The ring-polymer step of an atom slice (every bead) on this rank's
    GPU through the C ABI: a context of the slice's atoms with no potential
    of its own (harmonic, omega 0), its noise drawn at the whole system's
    indices."""

    def __init__(self, replica, atoms: tuple, dt_fs: float, gamma0_per_fs: float, precision="fp32",
                 deterministic=True, **kw):
        from . import pimd as P
        from .synth import Replica
        lo, hi = atoms
        rep = Replica(replica.Z[lo:hi], replica.x0[lo:hi], replica.box, replica.n_beads, replica.T, replica.seed,
                      replica.name)
        self.P, self.Na = replica.n_beads, hi - lo
        self.ctx = P.Context([rep], dt_fs, gamma0_per_fs, precision=precision, potential=P.POT_HARMONIC,
                             omega=0.0, deterministic=deterministic, **kw)
        self.ctx.set_noise_index(lo, replica.n_atoms)

    def positions(self):
        x, _, _ = self.ctx.get_forces()
        import torch
        return torch.tensor(np.asarray(x).reshape(self.P, self.Na, 3), device="cuda")

    def set_forces(self, f):
        self.ctx.set_forces(f.reshape(-1, 3).to(dtype=f.dtype).double())

    def start(self):
        return self.ctx.ring_start().view(self.P, self.Na, 3)

    def finish(self, f):
        self.ctx.ring_finish(f.reshape(-1, 3).double())
