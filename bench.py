#!/usr/bin/env python
"""Throughput of the bead-batched PIMD step on one GB300 (per rank).

Workload: proton-disordered ice Ih, 432 H2O (1296 atoms), P = 32 beads,
T = 250 K, dt = 0.5 fs, 3 x 128 tanh network on 32 radial + 32 angular
symmetry functions, cutoff 6 A (synthetic, seeded; random-init weights).
A step is one full pass of the hot path: normal modes -> beads, neighbour
lists, descriptors, network forward + input gradient, adjoint forces and
virial, per-bead energies, OBABO ring-polymer update in normal-mode space.

Metric: bead-atom force evaluations per second (and ns/day) of the BF16
tensor-core path; the plain FP32 GPU path is measured beside it.
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "bead-atom force evals/sec & ns/day, ice P=32: BF16-TC fused vs plain FP32 GPU"
UNIT = "bead-atom force evals/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12    # SMs x FP32 lanes x 2 flop x max SM clock
# algorithmic FP32 flops of the adjoint (forces + virial) per unit.
# Pair sums: per unordered neighbour pair, plus per neighbour (radial terms,
# weights, chain rule, scatter).
ADJ_FLOP_PER_PAIR = 205
ADJ_FLOP_PER_NBR = 380
# Moment tensors: per neighbour the nested Horner evaluation of the 4 degree-8
# polynomials and their gradient (1340 FMA: 480 + 336 in x, 400 in y, 124 in
# z) on top of the per-neighbour work above; per bead-atom Q = dE/dM (165
# monomials x (16 FMA + 4 mul)).
MOM_ADJ_FLOP_PER_NBR = 380 + 2 * 1340
MOM_ADJ_FLOP_PER_ATOM = 165 * 36
# BF16 network path, reduced basis (the 81 monomials with x-degree <= 1):
# the 4 polynomials and their gradient by Horner in y within each z-level,
# the x-degree-1 term folded in first, then Horner in z: 628 FMA per
# neighbour (256 + 58 FP32x2 pairs; no multiply-add spent on a chain's zero
# starting value); per bead-atom
# Q = M Phi(s) 2 / (a! b! c!) (165 x 4 x 2 mul), Phi (36 x 4 FMA) and the
# fold onto the 81 (483 terms x 4 widths FMA)
MOM_RED_ADJ_FLOP_PER_NBR = 380 + 2 * 628
MOM_RED_ADJ_FLOP_PER_ATOM = 165 * 4 * 2 + 36 * 4 * 2 + 483 * 4 * 2
# DRAM bytes (read + write) of one adjoint launch from an ncu capture of the
# same kernel on the same workload (ice Ih, P = 32, BF16 network, reduced
# moment basis, desc_mom_adj_fast_kernel<12>): 139.9 MB read (mostly the
# 2.6 KB of moments per bead-atom written by the forward) + 3.4 MB written.
# Reported only for that configuration.
ADJ_TRAFFIC_NCU = {("ice", "bf16_tc", "moments"): 139.896832e6 + 3.420928e6}


def args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16_tc", choices=["bf16_tc", "fp32", "fp64"])
    ap.add_argument("--workload", default="ice", choices=["ice", "water64", "fad", "batch", "water4096"])
    ap.add_argument("--no-fp32", action="store_true", help="skip the plain FP32 comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default pair schedule")
    ap.add_argument("--no-extras", action="store_true", help="skip the analysis / metadynamics timings")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampler over the timed region."""

    def __init__(self, index: int):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def build_model(ctx, workload, precision_ctx_factory):
    """Random-init network; input normalisation and energy scale fixed from
    the library's own descriptors / forces of the initial configuration."""
    from paper_2503_23728_gb300 import synth as s
    rep = workload.replicas[0]
    m = s.xavier_model(s.elements_of(workload.replicas), workload.widths, seed=7)
    ctx.set_weights(m)
    G = ctx.descriptors().cpu().numpy()
    Z = np.concatenate([np.tile(r.Z, r.n_beads) for r in workload.replicas])
    s.set_normalisation(m, G, Z)
    ctx.set_weights(m)
    _, f, _ = ctx.energy_forces()
    rms = float(np.sqrt((f.cpu().numpy() ** 2).mean()))
    s.set_energy_scale(m, 1.0 / rms)
    ctx.set_weights(m)
    return m


def run_gpu(a, workload, precision, model=None):
    import torch
    from paper_2503_23728_gb300 import pimd as P
    ctx = P.Context(workload.replicas, workload.dt_fs, workload.gamma0_per_fs, precision=precision,
                    widths=workload.widths, timing=True)
    if model is None:
        model = build_model(ctx, workload, None)
    else:
        ctx.set_weights(model)
    if not a.no_tune:
        # angular method, pair schedule and overlapped parts, measured on
        # this workload during set-up (not timed); no cache, so every run
        # measures afresh
        from paper_2503_23728_gb300 import tuner
        ctx.tune_result = tuner.tune(ctx, cache=None)
    else:
        ctx.tune_result = None
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for _ in range(a.warmup):
        ctx.step(1)
    torch.cuda.synchronize()
    return ctx, model, stream, flush


def timed_steps(a, ctx, stream, flush, barrier, marked=False):
    """K steps, each one graph launch bracketed by CUDA events on the context
    stream, with the L2 flushed before each. marked: the steps carry the
    stage markers (event records inside the step's graph, which cost time of
    their own) and their stage times are returned; otherwise the steps run
    without markers, as a user's steps do."""
    import torch
    ctx.set_stage_timing(marked)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    stages = []
    barrier()
    torch.cuda.synchronize()
    for k in range(a.steps):
        flush.zero_()
        starts[k].record(stream)
        ctx.step(1)
        ends[k].record(stream)
        if marked:
            stages.append(ctx.stage_times())
    torch.cuda.synchronize()
    barrier()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return ms, stages


def adjoint_kernel_name(ctx) -> str:
    if ctx.angular == "moments":
        return "desc_mom_adj_fast_kernel" if ctx.precision == "bf16_tc" else "desc_mom_adj_kernel"
    return "desc_adj_kernel"


def adjoint_flops(ctx) -> float:
    nnb, _ = ctx.neighbours()
    n = nnb.astype(np.float64)
    if ctx.angular == "moments" and ctx.precision == "bf16_tc":
        return float(np.sum(MOM_RED_ADJ_FLOP_PER_NBR * n + MOM_RED_ADJ_FLOP_PER_ATOM))
    if ctx.angular == "moments":
        return float(np.sum(MOM_ADJ_FLOP_PER_NBR * n + MOM_ADJ_FLOP_PER_ATOM))
    return float(np.sum(ADJ_FLOP_PER_PAIR * n * (n - 1) / 2 + ADJ_FLOP_PER_NBR * n))


def forward_kernel_name(ctx) -> str:
    if ctx.angular == "moments":
        return "desc_mom_fwd_red_kernel" if ctx.precision == "bf16_tc" else "desc_mom_fwd_kernel"
    return "desc_fwd_kernel"


def forward_flops(ctx) -> float:
    """Algorithmic FP32 work of the descriptor forward. Moment path, reduced
    basis: per neighbour the 81 monomials x 4 widths multiply-adds into the
    moments plus geometry, the 32 radial Gaussians and the 4 angular weights
    (~200 flop); per bead-atom the rebuild of the 84 other moments (4 widths,
    2 flop each) and G from the squared moments (165 monomials x 4 widths x
    (1 square + 4 zeta x 2 lambda multiply-adds)). Pair sums: 81 flop per
    pair (see the design notes) plus the per-neighbour terms."""
    nnb, _ = ctx.neighbours()
    n = nnb.astype(np.float64)
    if ctx.angular == "moments":
        per_nbr = (81 if ctx.precision == "bf16_tc" else 165) * 4 * 2 + 200
        per_atom = 84 * 4 * 2 + 165 * 4 * (1 + 8) * 2
        return float(np.sum(per_nbr * n + per_atom))
    return float(np.sum(81 * n * (n - 1) / 2 + 200 * n))


def step_roofline_ms(fp32_flops: float, tc_flops: float, peaks: dict) -> float:
    """Bound of one step: the slower of its FP32 work on the derived FP32 peak
    and its tensor-core work on the measured BF16 peak (the HBM traffic of a
    step, ~0.3 GB, is below both)."""
    bf16 = peaks.get("bf16_tflops") or 1900.0
    return max(fp32_flops / (FP32_PEAK_TFLOPS * 1e12), tc_flops / (bf16 * 1e12)) * 1e3


def network_flops(ctx, widths) -> float:
    # forward + input gradient, 2 flop per MAC, over the padded element tiles
    macs = 0
    prev = 64
    for w in widths:
        macs += prev * w
        prev = w
    macs = 2 * macs + prev   # backward mirrors forward; output layer on CUDA cores
    return 2.0 * macs * ctx.B


def multistep_ms(ctx, stream, launches: int = 10) -> float:
    """Mean step time of 8-step launches (one graph each, whose inner step
    boundaries fuse the ring finish with the next ring start), back to back
    without L2 flushes: the regime of a long production run. Reported beside
    the headline, which times single flushed steps."""
    import torch
    st = torch.cuda.current_stream() if stream is None else stream
    ctx.set_stage_timing(False)   # a marked last step would split the graph
    ctx.step(8)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(launches):
        ctx.step(8)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (8 * launches)


def e2e_host(a, ctx, stream, barrier):
    """Force evaluation through the C ABI with host buffers: H2D of the bead
    positions from pinned memory, pimd_energy_forces, D2H of forces and
    energies, every step."""
    import torch
    _, f0, _ = ctx.energy_forces()
    x_dev0 = torch.empty(ctx.B, 3, dtype=torch.float64, device="cuda")
    xh, _, _ = ctx.get_forces()
    x_host = torch.tensor(xh, dtype=torch.float64).pin_memory()
    f_host = torch.empty(ctx.B, 3, dtype=torch.float64).pin_memory()
    e_host = torch.empty(ctx.S, dtype=torch.float64).pin_memory()
    e_dev = torch.empty(ctx.S, dtype=torch.float64, device="cuda")
    f_dev = torch.empty(ctx.B, 3, dtype=torch.float64, device="cuda")
    from paper_2503_23728_gb300 import pimd as P
    import ctypes as ct
    n = max(3, a.steps // 2)
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(n):
        x_dev0.copy_(x_host, non_blocking=True)
        P.pimd_energy_forces(ctx.h, ct.c_void_p(x_dev0.data_ptr()), ct.c_void_p(e_dev.data_ptr()),
                             ct.c_void_p(f_dev.data_ptr()), None)
        f_host.copy_(f_dev, non_blocking=True)
        e_host.copy_(e_dev, non_blocking=True)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = t0.elapsed_time(t1) / n
    return ms, ctx.B * 3 * 8, ctx.B * 3 * 8 + ctx.S * 8


# algorithmic FP32 operations per pair of the analysis kernels: the FP32
# pair rule (3 differences, 3 x (scale, round, scale, subtract), 3 squares,
# 2 adds) = 20, plus the bin choice (sqrt, scale) for the RDF
RDF_FLOP_PER_PAIR = 22
XRD_FLOP_PER_PAIR = 40   # pair vector 20, sqrt, sincos, sinc and sinc' 9, gradient 6, virial 9 (counted as 40)


def time_call(fn, stream, reps=5):
    import torch
    fn()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(reps):
        fn()
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / reps


def analysis_extras(ctx, w, stream):
    """Timed once per run, outside the step: RDF pair counts and the
    proton-transfer coordinate of every bead of the first replica, with
    their pair throughput against the FP32 ALU peak."""
    import torch
    rep = w.replicas[0]
    box = np.asarray(rep.box, dtype=float)
    r_max = min(8.0, 0.5 * box.min()) if box[0] > 0 else 8.0
    counts = torch.zeros((3, 400), dtype=torch.int64, device="cuda")
    ms = time_call(lambda: ctx.rdf_counts(r_max, 400, counts=counts), stream)
    pairs = rep.n_beads * rep.n_atoms * (rep.n_atoms - 1) / 2
    out = {"rdf": {"ms": ms, "pairs": pairs, "pairs_per_s": pairs / (ms / 1e3),
                   "achieved_tflops": RDF_FLOP_PER_PAIR * pairs / (ms / 1e3) / 1e12,
                   "frac_fp32_peak": RDF_FLOP_PER_PAIR * pairs / (ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                   "config": {"r_max_A": r_max, "bins": 400, "beads": rep.n_beads, "atoms": rep.n_atoms}}}
    if 1 in set(rep.Z.tolist()) and 8 in set(rep.Z.tolist()):
        x, L = rep.x0, box
        acc = np.where(rep.Z == 8)[0]
        bond = np.full(rep.n_atoms, -1, dtype=np.int32)
        for h in np.where(rep.Z == 1)[0]:
            d = x[acc] - x[h]
            d -= L * np.round(d / L)
            bond[h] = acc[np.argmin((d ** 2).sum(axis=1))]
        ms2 = time_call(lambda: ctx.pt_coordinate(bond, 8, (-2.5, 0.5), 60), stream)
        n_pairs = rep.n_beads * int((rep.Z == 1).sum()) * rep.n_atoms
        out["pt"] = {"ms": ms2, "pairs_scanned": n_pairs, "pairs_per_s": n_pairs / (ms2 / 1e3),
                     "note": "includes the host-side bond upload and one stream synchronisation per call"}
    return out


def metad_extras(w, stream):
    """WT-MetaD with the XRD CV (Sec. S3 settings: theta 11.95 deg, lambda
    1.54 A, bias factor 60, f = Z) on the same system: the per-step cost of
    the CV, bias and bias force, from the stage times of a biased and an
    unbiased context (BF16 network)."""
    import math
    from paper_2503_23728_gb300 import pimd as P
    Q = 4 * math.pi * math.sin(math.radians(11.95)) / 1.54
    rep = w.replicas[0]
    md = P.make_metad(("xrd", Q, {1: 1.0, 6: 6.0, 8: 8.0}), 0.0104, 0.5, 60.0, 100, 4096,
                      elements=sorted(set(rep.Z.tolist())))
    out = {}
    for name, m in (("plain", None), ("xrd_metad", md)):
        ctx = P.Context([rep], w.dt_fs, w.gamma0_per_fs, precision="bf16_tc", widths=w.widths, timing=True,
                        metad=m)
        model = s_model(w)
        ctx.set_weights(model)
        ctx.step(3)
        acc = []
        for _ in range(10):
            ctx.step(1)
            acc.append(ctx.stage_times())
        out[name] = float(np.median([a["energy"] for a in acc]))
        ctx.close()
    pairs = rep.n_beads * rep.n_atoms * (rep.n_atoms - 1)
    ms = out["xrd_metad"] - out["plain"]
    return {"xrd_metad_ms_per_step": ms, "energy_stage_ms": out, "pairs_per_step": pairs,
            "achieved_tflops": XRD_FLOP_PER_PAIR * pairs / max(ms, 1e-6) / 1e9,
            "frac_fp32_peak": XRD_FLOP_PER_PAIR * pairs / max(ms, 1e-6) / 1e9 / FP32_PEAK_TFLOPS}


def gfn_mac(F, L, edges, nodes):
    """Multiply-adds of one evaluation of the graph-field-network head: per
    directed edge the input layer (32 x F), per iteration the message layer
    (F x F) and the two node-to-edge layers (2 F x F), the readout (F x F);
    per node and iteration the update (2F x F + F x F)."""
    return edges * (32 * F + L * 3 * F * F + F * F) + nodes * L * 3 * F * F


def gfn_extras(w, stream, steps=5):
    """The graph-field-network force head (Sec. 2.2, Table S1 sizes: F = 128,
    L = 3) driving the same ring polymers: step time and the head's
    throughput, next to the energy model's step on the same workload."""
    from paper_2503_23728_gb300 import pimd as P
    from paper_2503_23728_gb300 import synth as s
    F, L = 128, 3
    m = s.gfn_model(s.elements_of(w.replicas), F, L, seed=7)
    out = {"features": F, "iterations": L}
    try:
        bf16_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops")
    except Exception:
        bf16_peak = None
    for prec in ("fp32", "bf16_tc"):
        ctx = P.Context(w.replicas, w.dt_fs, w.gamma0_per_fs, precision=prec, potential=P.POT_GFN, gfn=(F, L),
                        timing=True)
        ctx.set_gfn(m)
        ctx.step(2)
        acc = []
        for _ in range(steps):
            ctx.step(1)
            acc.append(ctx.stage_times())
        st = {k: float(np.median([a[k] for a in acc])) for k in acc[0]}
        nnb, _ = ctx.neighbours()
        mac = gfn_mac(F, L, float(nnb.sum()), ctx.B)
        tf = 2 * mac / (st["network"] / 1e3) / 1e12
        out[prec] = {"ms_per_step": float(sum(st.values())), "head_ms": st["network"], "head_tflops": tf,
                     "bead_atom_evals_per_s": ctx.B / (sum(st.values()) / 1e3)}
        if prec == "fp32":
            out[prec]["frac_fp32_peak"] = tf / FP32_PEAK_TFLOPS
        else:
            out[prec]["frac_bf16_peak_measured"] = tf / bf16_peak if bf16_peak else None
        ctx.close()
    return out


def s_model(w):
    from paper_2503_23728_gb300 import synth as s
    return s.xavier_model(s.elements_of(w.replicas), w.widths, seed=7)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_beads(O, workload, model, budget_s, seed):
    rep = workload.replicas[0]
    rng = np.random.default_rng(seed)
    done, beads, t0 = 0, 0, time.perf_counter()
    while beads < rep.n_beads:
        x = rep.x0 + rng.normal(scale=0.05, size=rep.x0.shape)
        O.energy_forces(model, rep.Z, x, rep.box)
        beads += 1
        done += rep.n_atoms
        if time.perf_counter() - t0 > budget_s:
            break
    return done, beads, time.perf_counter() - t0


def cpu_baseline(workload, model, budget_s=15.0, single_budget_s=8.0):
    """FP64 oracle on the host cores: force evaluations of whole beads of the
    same workload until ~budget_s of CPU work with OpenMP over all cores,
    then at least one bead on a single thread."""
    import oracle as O
    rep = workload.replicas[0]
    threads = O.threads()
    done, beads, dt = _oracle_beads(O, workload, model, budget_s, 5)
    O.set_threads(1)
    try:
        done1, beads1, dt1 = _oracle_beads(O, workload, model, single_budget_s, 6)
    finally:
        O.set_threads(threads)
    return {"value": done / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of %d beads of the %s workload (%d bead-atoms), full FP64 force evaluation, "
                      "OpenMP over atoms" % (beads, rep.n_beads, workload.name, done),
            "seconds": dt, "cpu_model": cpu_model(),
            "single_thread": {"value": done1 / dt1, "unit": UNIT, "cores": 1, "seconds": dt1,
                              "sample": "%d bead(s) (%d bead-atoms) on one thread" % (beads1, done1)}}


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks (the slowest rank's time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bead_atoms_per_rank: int, world: int, steps: int, max_ms: float) -> float:
    """Whole-job bead-atom evaluations per second: every rank advances its own
    replicas; the job takes as long as its slowest rank."""
    return world * bead_atoms_per_rank * steps / (max_ms / 1e3)


def workload_of(name, rank):
    from paper_2503_23728_gb300 import synth as s
    w = s.workload(name)
    if rank:
        seeds = s.replica_seeds(0xC0FFEE + rank, len(w.replicas))
        for r, sd in zip(w.replicas, seeds):
            r.seed = sd
    return w


def config_of(w, precision, world):
    desc = {"ice": "ice Ih 432 H2O (1296 atoms), P=32, T=250 K, dt=0.5 fs, 3x128 tanh, cutoff 6 A",
            "water64": "water 64 H2O (192 atoms), P=32, T=300 K, dt=0.5 fs, 3x128 tanh, cutoff 6 A",
            "fad": "formic-acid dimer (10 atoms), P=16, T=300 K, dt=0.25 fs, 2x64 tanh, cutoff 6 A",
            "batch": "256 gas-phase clusters of 6-24 atoms, P in {8,16,32,64}, 2x64 tanh",
            "water4096": "water 4096 H2O (12288 atoms), P=64, T=300 K, dt=0.5 fs, 4x256 tanh, cutoff 6 A"}[w.name]
    return {"workload": desc, "bead_atoms_per_gpu": w.bead_atoms, "replicas_per_gpu": len(w.replicas),
            "path": precision, "parallelism": "independent replicas per GPU" if world > 1 else "1 GPU",
            "l2": "flushed between timed steps (256 MB write)",
            "precision": {"network": {"bf16_tc": "bf16 tcgen05, fp32 accumulate", "fp32": "fp32",
                                      "fp64": "fp64"}[precision],
                          "descriptors_adjoint": "fp64" if precision == "fp64" else "fp32",
                          "ring_polymer_estimators": "fp64" if precision == "fp64" else
                          "fp64 state and estimators; fp32 deviates, heat increments and normal-mode sums of the fluctuation modes"}}


def main():
    a = args()
    rank, world, local = dist_env()
    if a.impl == "reference":
        return reference(a, rank, world)
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    import __graft_entry__ as ge
    ge.build()
    w = workload_of(a.workload, rank)
    ctx, model, stream, flush = run_gpu(a, w, a.precision)
    clk = Clocks(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    ms, _ = timed_steps(a, ctx, stream, flush, barrier)                      # the headline: no markers
    ms_marked, stages = timed_steps(a, ctx, stream, flush, barrier, True)    # stage and kernel times
    clocks = clk.stop()
    total_ms = max_over_ranks(float(np.sum(ms)), dist, "cuda")
    steps_per_s = a.steps / (total_ms / 1e3)
    value = job_throughput(w.bead_atoms, world, a.steps, total_ms)
    ns_day = steps_per_s * w.dt_fs * 86400 / 1e6
    st_mean = {k: float(np.mean([s[k] for s in stages])) for k in stages[0]}
    adj_flops = adjoint_flops(ctx)
    adj_ms = st_mean["adjoint"]
    achieved = adj_flops / (adj_ms / 1e3) / 1e12
    fwd_flops = forward_flops(ctx)
    net_flops = network_flops(ctx, w.widths)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    e2e_ms, h2d, d2h = e2e_host(a, ctx, stream, barrier)
    multi = {"ms_per_step": multistep_ms(ctx, stream), "launch": "8-step graphs, 10 back to back",
             "l2": "not flushed between steps"}
    extras = None
    if not a.no_extras and world == 1:
        extras = analysis_extras(ctx, w, stream)
        extras["metad"] = metad_extras(w, stream)
        extras["gfn"] = gfn_extras(w, stream)
    launches = ctx.kernels_per_step() * a.steps
    fp32 = None
    if not a.no_fp32 and a.precision != "fp32":
        ctx2, _, stream2, flush2 = run_gpu(a, w, "fp32", model)
        ms2, _ = timed_steps(a, ctx2, stream2, flush2, barrier)
        _, stages2 = timed_steps(a, ctx2, stream2, flush2, barrier, True)
        t2 = float(np.sum(ms2))
        st2 = {k: float(np.mean([s[k] for s in stages2])) for k in stages2[0]}
        fp32 = {"value": world * w.bead_atoms * a.steps / (t2 / 1e3), "ms_per_step": t2 / a.steps,
                "stages_ms": st2,
                "network_fp32": {"flops_per_launch": net_flops, "ms": st2["network"],
                                 "achieved_tflops": net_flops / (st2["network"] / 1e3) / 1e12,
                                 "frac_fp32_peak": net_flops / (st2["network"] / 1e3) / 1e12 / FP32_PEAK_TFLOPS},
                "adjoint": {"kernel": adjoint_kernel_name(ctx2), "flops_per_launch": adjoint_flops(ctx2),
                            "ms": st2["adjoint"],
                            "frac_fp32_peak": adjoint_flops(ctx2) / (st2["adjoint"] / 1e3) / 1e12 / FP32_PEAK_TFLOPS}}
        ctx2.close()
    if rank != 0:
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16_tc": "bf16", "fp32": "f32", "fp64": "f64"}[a.precision], "data": "synthetic",
        "config": config_of(w, a.precision, world),
        "ns_per_day": ns_day,
        "tuned_schedule": ctx.tune_result,
        "stages_ms": st_mean,
        "fp32_plain": fp32,
        "speedup_vs_fp32_plain": (value / fp32["value"]) if fp32 else None,
        "angular": ctx.angular,
        "roofline": {"bound": "alu", "kernel": adjoint_kernel_name(ctx) + " (angular+radial adjoint, forces, virial)",
                     "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": ADJ_TRAFFIC_NCU.get((w.name, a.precision, ctx.angular)),
                     "flops_per_launch": adj_flops,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                     # the whole step against its own bound: FP32 work of the
                     # descriptor forward and the adjoint on the FP32 pipes,
                     # network work on the tensor cores (measured BF16 peak)
                     "step_frac": step_roofline_ms(fwd_flops + adj_flops, net_flops, peaks) / (total_ms / a.steps),
                     "step_bound_ms": step_roofline_ms(fwd_flops + adj_flops, net_flops, peaks)},
        "descriptor_forward": {"kernel": forward_kernel_name(ctx), "flops_per_launch": fwd_flops,
                               "ms": st_mean["descriptors"],
                               "achieved_tflops": fwd_flops / (st_mean["descriptors"] / 1e3) / 1e12,
                               "frac_fp32_peak": fwd_flops / (st_mean["descriptors"] / 1e3) / 1e12 / FP32_PEAK_TFLOPS},
        "ms_per_step_with_stage_markers": float(np.sum(ms_marked)) / a.steps,
        "multistep": multi,
        "network_tensor": {"flops_per_launch": net_flops, "ms": st_mean["network"],
                           "achieved_tflops": net_flops / (st_mean["network"] / 1e3) / 1e12,
                           "peak_bf16_tflops_measured": peaks.get("bf16_tflops")},
        "clocks": clocks,
        "e2e": {"value": world * w.bead_atoms / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "what": "one force evaluation per step through pimd_energy_forces: bead positions H2D from "
                        "pinned memory, energies and forces D2H; no ring-polymer step and no L2 flush, "
                        "so it can exceed the device-timed full-step value"},
        "gpu_launches": launches,
        "next_rows": extras,
    }
    if world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, model)
    ctx.close()
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def reference(a, rank, world):
    """The FP64 CPU oracle as it stands: each step is the force evaluation of
    one bead of the workload (bounded sample)."""
    if rank != 0:
        return
    import oracle as O
    from paper_2503_23728_gb300 import synth as s
    w = s.workload(a.workload)
    rep = w.replicas[0]
    m = s.xavier_model(s.elements_of(w.replicas), w.widths, seed=7)
    G = O.descriptors(m, rep.x0, rep.box)
    s.set_normalisation(m, G, rep.Z)
    rng = np.random.default_rng(3)
    warm = max(1, min(a.warmup, 5))   # at most 5 untimed evaluations (~0.6 s each on 16 cores)
    tw = time.perf_counter()
    for _ in range(warm):
        O.energy_forces(m, rep.Z, rep.x0 + rng.normal(scale=0.05, size=rep.x0.shape), rep.box)
    per = (time.perf_counter() - tw) / warm
    # exactly the requested steps while they fit in ~4 minutes, else as many as fit
    steps = a.steps if a.steps * per <= 240.0 else max(1, int(240.0 / per))
    t0 = time.perf_counter()
    for _ in range(steps):
        O.energy_forces(m, rep.Z, rep.x0 + rng.normal(scale=0.05, size=rep.x0.shape), rep.box)
    dt = time.perf_counter() - t0
    value = steps * rep.n_atoms / dt
    sample = "%d steps x 1 bead (%d bead-atoms) of the %s workload, FP64 oracle force evaluation" % (
        steps, rep.n_atoms, w.name)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warm, "ms_per_step": dt / steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(w, "fp64", 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
