"""The bead-sharded ring polymer on the GPU through the C ABI: two ranks'
worth of contexts (bead slices for the forces, atom slices with every bead
for the ring-polymer step) driven in one process, the two transposes done by
slicing (the collectives themselves are covered by the gloo test on the
CPU). In deterministic mode the slices reproduce the single-context
trajectory bit for bit, and the same trajectory as the FP64 oracle to the
FP32 path's bar."""
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


def test_two_slices_reproduce_the_single_context(water64_model):
    P = _P()
    from paper_2503_23728_gb300 import shard as SH
    w, r, m = water64_model
    rep = s.Replica(r.Z, r.x0, r.box, 4, r.T, r.seed, r.name)
    plan = SH.ShardPlan(rep.n_beads, rep.n_atoms, 2)
    whole = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="fp32", widths=w.widths, deterministic=True)
    whole.set_weights(m)
    forces = [SH.GpuBeadForces(rep, plan.n_beads(k), m, w.dt_fs, w.gamma0_per_fs, widths=w.widths)
              for k in range(2)]
    rings = [SH.GpuAtomRing(rep, plan.atoms[k], w.dt_fs, w.gamma0_per_fs) for k in range(2)]

    def forces_of(x_slices):
        x = torch.cat(x_slices, dim=1)                                   # every bead, every atom
        f = torch.cat([forces[k](x[lo:hi].contiguous()) for k, (lo, hi) in enumerate(plan.beads)], dim=0)
        return [f[:, lo:hi, :].contiguous() for lo, hi in plan.atoms]   # back to atom slices

    f0 = forces_of([g.positions() for g in rings])
    for g, f in zip(rings, f0):
        g.set_forces(f)
    n = 6
    for _ in range(n):
        fs = forces_of([g.start() for g in rings])
        for g, f in zip(rings, fs):
            g.finish(f)
    whole.step(n)
    q, p, st, Q = whole.get_state()
    q = q.reshape(rep.n_beads, rep.n_atoms, 3)
    p = p.reshape(rep.n_beads, rep.n_atoms, 3)
    Qs = 0.0
    for g, (lo, hi) in zip(rings, plan.atoms):
        qs, ps, sts, Qk = g.ctx.get_state()
        assert sts == st == n
        assert np.array_equal(qs.reshape(rep.n_beads, hi - lo, 3), q[:, lo:hi, :])
        assert np.array_equal(ps.reshape(rep.n_beads, hi - lo, 3), p[:, lo:hi, :])
        Qs += float(Qk[0])
    # the FP32 path forms heat increments and their block sums in FP32, and
    # the slices group coordinates into blocks differently from the whole
    assert abs(Qs - float(Q[0])) <= 1e-5 * max(1.0, abs(float(Q[0])))
    # and the whole trajectory against the FP64 oracle (FP32 path bar)
    so = O.System(rep, s.MASS, w.dt_fs, w.gamma0_per_fs, model=m)
    so.step(n)
    assert np.abs(q - so.q).max() < 1e-5 * max(1.0, np.abs(so.q).max())


def test_ring_calls_check_their_order(water64_model):
    P = _P()
    from paper_2503_23728_gb300 import shard as SH
    w, r, m = water64_model
    rep = s.Replica(r.Z, r.x0, r.box, 2, r.T, r.seed, r.name)
    g = SH.GpuAtomRing(rep, (0, 10), w.dt_fs, w.gamma0_per_fs)
    f = torch.zeros((2 * 10, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PimdError) as e:
        g.ctx.ring_finish(f)                      # no start before it
    assert e.value.code == -2
    g.ctx.set_forces(f)
    g.ctx.ring_start()
    with pytest.raises(P.PimdError) as e:
        g.ctx.ring_start()                        # the forces of the new positions are missing
    assert e.value.code == -2
    g.ctx.ring_finish(f)
    with pytest.raises(P.PimdError) as e:
        g.ctx.set_noise_index(5, 12)              # atoms 5 .. 14 do not fit in 12
    assert e.value.code == -1
