"""ctypes binding of libpimd.so (include/pimd.h), plus a small Context wrapper
that takes device memory and the stream from PyTorch.

Argument marshalling only: every step of the force evaluation and of the
ring-polymer dynamics runs in the library's CUDA kernels. There is no CPU
fallback; loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpimd.so")

PIMD_OK = 0
STATUS = {-9: "METAD_FULL", 0: "OK", -1: "INVALID_ARG", -2: "STATE", -3: "WORKSPACE_TOO_SMALL", -4: "CUDA", -5: "NONFINITE",
          -6: "TIMEOUT", -7: "NBR_OVERFLOW", -8: "UNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "bf16_tc": 2}
POT_MODEL, POT_HARMONIC, POT_GFN = 0, 1, 2
EXPORTS = ["pimd_abi_version", "pimd_workspace_size", "pimd_create", "pimd_set_weights", "pimd_step",
           "pimd_energy_forces", "pimd_descriptors", "pimd_estimators", "pimd_get_state", "pimd_set_state",
           "pimd_get_forces", "pimd_get_neighbours", "pimd_sync", "pimd_sizes", "pimd_destroy", "pimd_last_error",
           "pimd_stage_times", "pimd_kernels_per_step", "pimd_tune", "pimd_set_schedule", "pimd_set_angular", "pimd_get_angular",
           "pimd_element_types", "pimd_rdf_counts", "pimd_pt_coordinate",
           "pimd_metad_hills", "pimd_metad_set_hills", "pimd_metad_cv", "pimd_selftest_bounded_wait",
           "pimd_set_gfn", "pimd_set_stage_timing", "pimd_rdf_gr", "pimd_cv_histogram", "pimd_pi_fes",
           "pimd_metad_fes", "pimd_set_noise_index", "pimd_set_forces", "pimd_ring_start", "pimd_ring_finish",
           "pimd_set_overlap", "pimd_set_adjoint_warps", "pimd_get_adjoint_warps"]
ANGULAR = {"pairs": 0, "moments": 1}
STAGES = ["ring_start", "neighbours", "descriptors", "network", "adjoint", "energy", "ring_finish"]


class PimdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class pimd_metad_desc(ct.Structure):
    _fields_ = [("cv", ct.c_int), ("n_terms", ct.c_int), ("term_i", ct.c_int * 8), ("term_j", ct.c_int * 8),
                ("term_c", ct.c_double * 8), ("xrd_Q", ct.c_double), ("xrd_f", ct.c_double * 8),
                ("height_eV", ct.c_double), ("sigma", ct.c_double), ("bias_factor", ct.c_double),
                ("stride", ct.c_int), ("max_hills", ct.c_int)]


def make_metad(cv, height_eV: float, sigma: float, bias_factor: float, stride: int, max_hills: int,
               elements=None) -> pimd_metad_desc:
    """cv = ("distances", [(i, j, c), ...]) or ("xrd", Q, {Z: f}); for XRD the
    factors are laid out in ascending-Z order of `elements`."""
    m = pimd_metad_desc()
    if cv[0] == "distances":
        m.cv = 1
        m.n_terms = len(cv[1])
        for t, (i, j, c) in enumerate(cv[1]):
            m.term_i[t], m.term_j[t], m.term_c[t] = int(i), int(j), float(c)
    else:
        m.cv = 2
        m.xrd_Q = float(cv[1])
        for t, z in enumerate(sorted(elements)):
            m.xrd_f[t] = float(cv[2][int(z)])
    m.height_eV, m.sigma, m.bias_factor = float(height_eV), float(sigma), float(bias_factor)
    m.stride, m.max_hills = int(stride), int(max_hills)
    return m


class pimd_config(ct.Structure):
    _fields_ = [("dt_fs", ct.c_double), ("gamma0_per_fs", ct.c_double), ("pile_lambda", ct.c_double),
                ("cutoff_A", ct.c_double), ("precision", ct.c_int), ("thermostat", ct.c_int),
                ("potential", ct.c_int), ("max_neighbours", ct.c_int), ("omega_harm", ct.c_double),
                ("n_hidden", ct.c_int), ("widths", ct.c_int * 4), ("stream", ct.c_void_p), ("timing", ct.c_int),
                ("nbr_algo", ct.c_int), ("deterministic", ct.c_int), ("splitting", ct.c_int),
                ("free_rp", ct.c_int), ("metad", ct.POINTER(pimd_metad_desc)), ("nbr_skin_A", ct.c_double),
                ("transform", ct.c_int), ("gfn_features", ct.c_int), ("gfn_iterations", ct.c_int)]
TRANSFORM = {"normal_modes": 0, "staging": 1}
SPLITTING = {"obabo": 0, "baoab": 1}
FREE_RP = {"exact": 0, "cayley": 1}


class pimd_replica_desc(ct.Structure):
    _fields_ = [("n_atoms", ct.c_int), ("n_beads", ct.c_int), ("Z", ct.POINTER(ct.c_int)),
                ("x0", ct.POINTER(ct.c_double)), ("mass", ct.POINTER(ct.c_double)), ("box", ct.c_double * 3),
                ("T_K", ct.c_double), ("seed", ct.c_uint64)]


class pimd_model_desc(ct.Structure):
    _fields_ = [("n_elements", ct.c_int), ("Z", ct.POINTER(ct.c_int)), ("n_hidden", ct.c_int),
                ("widths", ct.POINTER(ct.c_int)), ("params", ct.POINTER(ct.POINTER(ct.c_double))),
                ("eta_R", ct.c_double), ("r_mu", ct.POINTER(ct.c_double)), ("zeta", ct.POINTER(ct.c_int)),
                ("lam", ct.POINTER(ct.c_double)), ("eta_A", ct.POINTER(ct.c_double))]


class pimd_gfn_desc(ct.Structure):
    _fields_ = [("n_elements", ct.c_int), ("Z", ct.c_int * 8), ("params", ct.POINTER(ct.c_double)),
                ("n_params", ct.c_size_t), ("r_mu", ct.c_double * 32), ("eta_R", ct.c_double)]


class pimd_est(ct.Structure):
    _fields_ = [("V_mean", ct.c_double), ("K_prim", ct.c_double), ("K_cv", ct.c_double), ("E_tot", ct.c_double),
                ("W", ct.c_double * 9), ("H_cons", ct.c_double), ("Q_thermo", ct.c_double),
                ("T_kin", ct.c_double), ("nbr_mean", ct.c_double), ("nbr_max", ct.c_double)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k in ("V_mean", "K_prim", "K_cv", "E_tot", "H_cons", "Q_thermo", "T_kin",
                                           "nbr_mean", "nbr_max")}
        d["W"] = np.array(list(self.W)).reshape(3, 3)
        return d


_lib = None


def load(path: str = LIB_PATH):
    """Load libpimd.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libpimd.so is not built (%s); run __graft_entry__.build()" % path)
    L = ct.CDLL(path)
    vp, dp, ip = ct.c_void_p, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int)
    L.pimd_abi_version.restype = ct.c_int
    L.pimd_workspace_size.argtypes = [ct.POINTER(pimd_config), ct.POINTER(pimd_replica_desc), ct.c_int,
                                      ct.POINTER(ct.c_size_t)]
    L.pimd_create.argtypes = [ct.POINTER(pimd_config), ct.POINTER(pimd_replica_desc), ct.c_int, vp, ct.c_size_t,
                              ct.POINTER(vp)]
    L.pimd_set_weights.argtypes = [vp, ct.POINTER(pimd_model_desc)]
    L.pimd_step.argtypes = [vp, ct.c_int]
    L.pimd_energy_forces.argtypes = [vp, vp, vp, vp, vp]
    L.pimd_descriptors.argtypes = [vp, vp, vp]
    L.pimd_estimators.argtypes = [vp, ct.POINTER(pimd_est), ct.c_int]
    L.pimd_get_state.argtypes = [vp, dp, dp, ct.POINTER(ct.c_uint64), dp]
    L.pimd_set_state.argtypes = [vp, dp, dp, ct.c_uint64, dp]
    L.pimd_get_forces.argtypes = [vp, dp, dp, dp]
    L.pimd_get_neighbours.argtypes = [vp, ip, ip]
    L.pimd_sync.argtypes = [vp]
    L.pimd_sizes.argtypes = [vp, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64), ip, ip]
    L.pimd_destroy.argtypes = [vp]
    L.pimd_destroy.restype = None
    L.pimd_last_error.argtypes = [vp]
    L.pimd_last_error.restype = ct.c_char_p
    L.pimd_stage_times.argtypes = [vp, ct.POINTER(ct.c_float)]
    L.pimd_kernels_per_step.argtypes = [vp]
    L.pimd_kernels_per_step.restype = ct.c_int
    L.pimd_tune.argtypes = [vp, ct.c_int, dp]
    L.pimd_set_schedule.argtypes = [vp, ct.c_int]
    L.pimd_set_angular.argtypes = [vp, ct.c_int]
    L.pimd_set_gfn.argtypes = [vp, vp]
    L.pimd_get_angular.argtypes = [vp]
    L.pimd_get_angular.restype = ct.c_int
    L.pimd_set_adjoint_warps.argtypes = [vp, ct.c_int]
    L.pimd_get_adjoint_warps.argtypes = [vp]
    L.pimd_get_adjoint_warps.restype = ct.c_int
    L.pimd_selftest_bounded_wait.argtypes = [vp, ct.c_double]
    L.pimd_metad_hills.argtypes = [vp, ct.c_int, dp, dp, ct.c_int]
    L.pimd_metad_hills.restype = ct.c_int
    L.pimd_metad_set_hills.argtypes = [vp, ct.c_int, dp, dp, ct.c_int]
    L.pimd_metad_cv.argtypes = [vp, dp, dp]
    L.pimd_element_types.argtypes = [vp, ct.POINTER(ct.c_int)]
    L.pimd_element_types.restype = ct.c_int
    L.pimd_rdf_counts.argtypes = [vp, ct.c_int, ct.c_double, ct.c_int, vp]
    L.pimd_pt_coordinate.argtypes = [vp, ct.c_int, vp, ct.c_int, ct.c_double, ct.c_double, ct.c_int, vp, vp]
    L.pimd_descriptors_noalloc.argtypes = [vp, ct.c_int, dp, ct.c_double, ct.c_double, dp, dp, vp, vp]
    L.pimd_set_stage_timing.argtypes = [vp, ct.c_int]
    L.pimd_rdf_gr.argtypes = [vp, ct.c_int, ct.c_double, ct.c_int, ct.c_double, vp, vp]
    L.pimd_cv_histogram.argtypes = [vp, ct.c_int, ct.c_double, ct.c_double, ct.c_int, ct.c_double, vp, vp]
    L.pimd_pi_fes.argtypes = [vp, ct.c_int, vp, vp, ct.c_double, ct.c_double, ct.c_int, vp, vp]
    L.pimd_metad_fes.argtypes = [vp, ct.c_int, vp, ct.c_int, vp]
    L.pimd_set_noise_index.argtypes = [vp, ct.c_int, ct.c_int, ct.c_int]
    L.pimd_set_overlap.argtypes = [vp, ct.c_int]
    L.pimd_set_overlap.restype = ct.c_int
    L.pimd_set_forces.argtypes = [vp, vp]
    L.pimd_ring_start.argtypes = [vp, vp]
    L.pimd_ring_finish.argtypes = [vp, vp]
    _lib = L
    return L


def _check(rc: int, ctx=None):
    if rc != PIMD_OK:
        msg = load().pimd_last_error(ctx)
        raise PimdError(rc, msg.decode() if msg else "")


def _dp(a):
    return None if a is None else a.ctypes.data_as(ct.POINTER(ct.c_double))


def _ip(a):
    return None if a is None else a.ctypes.data_as(ct.POINTER(ct.c_int))


# ---------------------------------------------------------------- C-ABI calls
def pimd_abi_version() -> int:
    return int(load().pimd_abi_version())


def pimd_workspace_size(cfg: pimd_config, reps) -> int:
    n = ct.c_size_t(0)
    _check(load().pimd_workspace_size(ct.byref(cfg), reps, len(reps), ct.byref(n)))
    return int(n.value)


def pimd_create(cfg: pimd_config, reps, workspace_ptr: int, ws_bytes: int):
    h = ct.c_void_p()
    _check(load().pimd_create(ct.byref(cfg), reps, len(reps), ct.c_void_p(workspace_ptr), ws_bytes, ct.byref(h)))
    return h


def pimd_set_weights(ctx, model: pimd_model_desc):
    _check(load().pimd_set_weights(ctx, ct.byref(model)), ctx)


def pimd_step(ctx, n_steps: int):
    _check(load().pimd_step(ctx, int(n_steps)), ctx)


def pimd_energy_forces(ctx, x_ptr, e_ptr, f_ptr, vir_ptr):
    _check(load().pimd_energy_forces(ctx, x_ptr, e_ptr, f_ptr, vir_ptr), ctx)


def pimd_descriptors(ctx, x_ptr, G_ptr):
    _check(load().pimd_descriptors(ctx, x_ptr, G_ptr), ctx)


def pimd_estimators(ctx, n_reps: int):
    out = (pimd_est * n_reps)()
    _check(load().pimd_estimators(ctx, out, n_reps), ctx)
    return [o.as_dict() for o in out]


def pimd_get_state(ctx, n_entries: int, n_reps: int):
    q = np.zeros(n_entries)
    p = np.zeros(n_entries)
    Q = np.zeros(n_reps)
    step = ct.c_uint64(0)
    _check(load().pimd_get_state(ctx, _dp(q), _dp(p), ct.byref(step), _dp(Q)), ctx)
    return q, p, int(step.value), Q


def pimd_set_state(ctx, q, p, step: int, Q=None):
    q = np.ascontiguousarray(q, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    Qa = None if Q is None else np.ascontiguousarray(Q, dtype=np.float64)
    _check(load().pimd_set_state(ctx, _dp(q), _dp(p), int(step), _dp(Qa)), ctx)


def pimd_get_forces(ctx, B: int, S: int):
    x = np.zeros((B, 3))
    f = np.zeros((B, 3))
    V = np.zeros(S)
    _check(load().pimd_get_forces(ctx, _dp(x), _dp(f), _dp(V)), ctx)
    return x, f, V


def pimd_get_neighbours(ctx, B: int, maxnb: int):
    nnb = np.zeros(B, dtype=np.int32)
    nbr = np.zeros((B, maxnb), dtype=np.int32)
    _check(load().pimd_get_neighbours(ctx, _ip(nnb), _ip(nbr)), ctx)
    return nnb, nbr


def pimd_stage_times(ctx) -> dict:
    ms = (ct.c_float * len(STAGES))()
    _check(load().pimd_stage_times(ctx, ms), ctx)
    return {k: float(v) for k, v in zip(STAGES, ms)}


def pimd_tune(ctx, reps: int = 3) -> dict:
    out = np.zeros(3)
    _check(load().pimd_tune(ctx, int(reps), _dp(out)), ctx)
    choice = int(out[1])
    return {"best_ms": float(out[0]), "band_length": max(choice, 0),
            "angular": "moments" if choice < 0 else "pairs", "default_ms": float(out[2]),
            "adjoint_warps": int(load().pimd_get_adjoint_warps(ctx))}


def pimd_set_schedule(ctx, band_length: int):
    _check(load().pimd_set_schedule(ctx, int(band_length)), ctx)


def pimd_set_angular(ctx, algo):
    """algo: "pairs" | "moments" (or PIMD_ANG_* value)."""
    _check(load().pimd_set_angular(ctx, ANGULAR.get(algo, algo) if isinstance(algo, str) else int(algo)), ctx)


def pimd_get_angular(ctx) -> str:
    return {0: "pairs", 1: "moments"}[int(load().pimd_get_angular(ctx))]


def pimd_selftest_bounded_wait(seconds: float = 0.2, stream=None) -> int:
    """Status of one bounded wait that nothing completes (PIMD_ERR_TIMEOUT = -6 expected)."""
    return int(load().pimd_selftest_bounded_wait(stream, float(seconds)))


def pimd_metad_hills(ctx, replica: int, capacity: int = 1 << 20):
    n = int(load().pimd_metad_hills(ctx, int(replica), None, None, 0))
    if n < 0:
        _check(n, ctx)
    s = np.zeros(n)
    h = np.zeros(n)
    if n:
        n2 = int(load().pimd_metad_hills(ctx, int(replica), _dp(s), _dp(h), n))
        if n2 < 0:
            _check(n2, ctx)
    return s, h


def pimd_metad_set_hills(ctx, replica: int, s, h):
    s = np.ascontiguousarray(s, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    _check(load().pimd_metad_set_hills(ctx, int(replica), _dp(s), _dp(h), len(s)), ctx)


def pimd_metad_cv(ctx, S: int):
    cv = np.zeros(S)
    vb = np.zeros(S)
    _check(load().pimd_metad_cv(ctx, _dp(cv), _dp(vb)), ctx)
    return cv, vb


def pimd_element_types(ctx) -> list:
    z = (ct.c_int * 8)()
    n = int(load().pimd_element_types(ctx, z))
    if n < 0:
        _check(n, ctx)
    return [int(z[k]) for k in range(n)]


def pimd_rdf_counts(ctx, replica: int, r_max: float, n_bins: int, counts_ptr):
    _check(load().pimd_rdf_counts(ctx, int(replica), float(r_max), int(n_bins), ct.c_void_p(counts_ptr)), ctx)


def pimd_pt_coordinate(ctx, replica: int, bond_ptr, acceptor_Z: int, v_min: float, v_max: float, n_bins: int,
                       v_ptr, hist_ptr):
    _check(load().pimd_pt_coordinate(ctx, int(replica), ct.c_void_p(bond_ptr), int(acceptor_Z), float(v_min),
                                     float(v_max), int(n_bins), ct.c_void_p(v_ptr) if v_ptr else None,
                                     ct.c_void_p(hist_ptr) if hist_ptr else None), ctx)


def pimd_kernels_per_step(ctx) -> int:
    return int(load().pimd_kernels_per_step(ctx))


def pimd_descriptors_noalloc(x_ptr, n_atoms: int, box, cutoff: float, eta_R: float, r_mu, eta_A, G_ptr,
                             stream=None):
    """Descriptors of one configuration using the library's static scratch
    array (no device allocation by the library; see include/pimd.h)."""
    b = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    rm = np.ascontiguousarray(r_mu, dtype=np.float64)
    ea = np.ascontiguousarray(eta_A, dtype=np.float64)
    # the library reads exactly 32, 4 and 3 values from these host arrays
    if rm.size != 32 or ea.size != 4 or (b is not None and b.size != 3):
        raise ValueError("r_mu needs 32 values, eta_A 4 and box 3 (or None)")
    _check(load().pimd_descriptors_noalloc(x_ptr, int(n_atoms), _dp(b), float(cutoff), float(eta_R), _dp(rm),
                                           _dp(ea), G_ptr, stream))


def pimd_sync(ctx):
    _check(load().pimd_sync(ctx), ctx)


def pimd_sizes(ctx):
    B, S = ct.c_int64(0), ct.c_int64(0)
    R, M = ct.c_int(0), ct.c_int(0)
    _check(load().pimd_sizes(ctx, ct.byref(B), ct.byref(S), ct.byref(R), ct.byref(M)), ctx)
    return int(B.value), int(S.value), int(R.value), int(M.value)


def pimd_destroy(ctx):
    load().pimd_destroy(ctx)


def pimd_last_error(ctx=None) -> str:
    m = load().pimd_last_error(ctx)
    return m.decode() if m else ""


# ---------------------------------------------------------------- helpers
def make_config(dt_fs, gamma0_per_fs, precision="fp32", cutoff=6.0, widths=(128, 128, 128), pile_lambda=1.0,
                thermostat=True, potential=POT_MODEL, omega=0.0, max_neighbours=128, stream=None,
                timing=False, nbr_algo=0, deterministic=False, splitting="obabo",
                free_rp="exact", metad=None, nbr_skin=-1.0, transform="normal_modes", gfn=(128, 3)) -> pimd_config:
    c = pimd_config()
    c.dt_fs = dt_fs
    c.gamma0_per_fs = gamma0_per_fs
    c.pile_lambda = pile_lambda
    c.cutoff_A = cutoff
    c.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    c.thermostat = 1 if thermostat else 0
    c.potential = potential
    c.max_neighbours = max_neighbours
    c.omega_harm = omega
    c.n_hidden = len(widths)
    for l, w in enumerate(widths):
        c.widths[l] = int(w)
    c.stream = stream
    c.timing = 1 if timing else 0
    c.nbr_algo = int(nbr_algo)
    c.deterministic = 1 if deterministic else 0
    c.splitting = SPLITTING[splitting] if isinstance(splitting, str) else int(splitting)
    c.free_rp = FREE_RP[free_rp] if isinstance(free_rp, str) else int(free_rp)
    if metad is not None:
        c.metad = ct.pointer(metad)
    c.nbr_skin_A = float(nbr_skin)
    c.transform = TRANSFORM[transform] if isinstance(transform, str) else int(transform)
    c.gfn_features, c.gfn_iterations = int(gfn[0]), int(gfn[1])
    return c


class _Keep:
    """Holds numpy arrays referenced by ctypes structures."""

    def __init__(self):
        self.items = []

    def add(self, a):
        self.items.append(a)
        return a


def make_replicas(replicas, keep: _Keep, masses=None):
    arr = (pimd_replica_desc * len(replicas))()
    for k, r in enumerate(replicas):
        Z = keep.add(np.ascontiguousarray(r.Z, dtype=np.int32))
        x0 = keep.add(np.ascontiguousarray(r.x0, dtype=np.float64))
        d = arr[k]
        d.n_atoms = len(Z)
        d.n_beads = int(r.n_beads)
        d.Z = _ip(Z)
        d.x0 = _dp(x0)
        if masses is not None:
            m = keep.add(np.ascontiguousarray([masses[int(z)] for z in Z], dtype=np.float64))
            d.mass = _dp(m)
        else:
            d.mass = None
        for a in range(3):
            d.box[a] = float(r.box[a])
        d.T_K = float(r.T)
        d.seed = int(r.seed)
    return arr


def make_gfn(model, keep: _Keep) -> pimd_gfn_desc:
    """pimd_gfn_desc of a synth.GfnModel (FP64 blob in the pimd.h layout)."""
    g = pimd_gfn_desc()
    g.n_elements = len(model.elements)
    for e, z in enumerate(model.elements):
        g.Z[e] = int(z)
    blob = keep.add(np.ascontiguousarray(model.blob, dtype=np.float64))
    g.params = _dp(blob)
    g.n_params = blob.size
    for k, r in enumerate(model.desc["r_mu"]):
        g.r_mu[k] = float(r)
    g.eta_R = float(model.desc["eta_R"])
    return g


def pimd_set_gfn(ctx, g: pimd_gfn_desc):
    _check(load().pimd_set_gfn(ctx, ct.byref(g)), ctx)


def make_model(model, keep: _Keep) -> pimd_model_desc:
    m = pimd_model_desc()
    els = list(model.elements)
    m.n_elements = len(els)
    m.Z = _ip(keep.add(np.array(els, dtype=np.int32)))
    m.n_hidden = len(model.widths)
    m.widths = _ip(keep.add(np.array(model.widths, dtype=np.int32)))
    ptrs = (ct.POINTER(ct.c_double) * len(els))()
    for e, z in enumerate(els):
        ptrs[e] = _dp(keep.add(np.ascontiguousarray(model.params[z], dtype=np.float64)))
    keep.add(ptrs)
    m.params = ct.cast(ptrs, ct.POINTER(ct.POINTER(ct.c_double)))
    d = model.desc
    m.eta_R = d["eta_R"]
    m.r_mu = _dp(keep.add(np.array(d["r_mu"], dtype=np.float64)))
    m.zeta = _ip(keep.add(np.array(d["zeta"], dtype=np.int32)))
    m.lam = _dp(keep.add(np.array(d["lam"], dtype=np.float64)))
    m.eta_A = _dp(keep.add(np.array(d["eta_A"], dtype=np.float64)))
    return m


class Context:
    """One library context on the current CUDA device; device workspace and
    the stream come from PyTorch."""

    def __init__(self, replicas, dt_fs, gamma0_per_fs, precision="fp32", widths=(128, 128, 128), cutoff=6.0,
                 pile_lambda=1.0, thermostat=True, potential=POT_MODEL, omega=0.0, max_neighbours=128,
                 masses=None, stream=None, timing=False, nbr_algo=0, deterministic=False, splitting="obabo",
                 free_rp="exact", metad=None, nbr_skin=-1.0, transform="normal_modes", gfn=(128, 3)):
        """gfn: (features, iterations) of the graph-field-network head, used
        with potential=POT_GFN (FP32 precision)."""
        import torch
        self.torch = torch
        self.keep = _Keep()
        self.replicas = list(replicas)
        self.widths = tuple(int(v) for v in widths)
        self.precision = precision if isinstance(precision, str) else {v: k for k, v in PRECISION.items()}[precision]
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.cfg = make_config(dt_fs, gamma0_per_fs, precision, cutoff, widths, pile_lambda, thermostat, potential,
                               omega, max_neighbours, ct.c_void_p(stream.cuda_stream), timing, nbr_algo,
                               deterministic, splitting, free_rp, metad, nbr_skin, transform, gfn)
        self.metad_desc = metad
        self.reps = make_replicas(self.replicas, self.keep, masses)
        self.ws_bytes = pimd_workspace_size(self.cfg, self.reps)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        self.h = pimd_create(self.cfg, self.reps, self.workspace.data_ptr(), self.ws_bytes)
        self.B, self.S, self.R, self.maxnb = pimd_sizes(self.h)

    def close(self):
        if self.h is not None:
            pimd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, model):
        keep = _Keep()
        desc = make_model(model, keep)
        pimd_set_weights(self.h, desc)

    def set_gfn(self, model):
        """Parameters of the graph-field-network head (synth.GfnModel)."""
        keep = _Keep()
        pimd_set_gfn(self.h, make_gfn(model, keep))

    def step(self, n: int = 1):
        pimd_step(self.h, n)

    def energy_forces(self, x=None, want_virial=True):
        """x: CUDA FP64 tensor [B, 3] or None (current beads). Returns per-bead
        energies [S], forces [B, 3] and virials [S, 3, 3] as CUDA tensors."""
        t = self.torch
        e = t.empty(self.S, dtype=t.float64, device="cuda")
        f = t.empty(self.B, 3, dtype=t.float64, device="cuda")
        v = t.empty(self.S, 9, dtype=t.float64, device="cuda") if want_virial else None
        xp = None
        if x is not None:
            x = x.to(device="cuda", dtype=t.float64).contiguous()
            xp = ct.c_void_p(x.data_ptr())
        pimd_energy_forces(self.h, xp, ct.c_void_p(e.data_ptr()), ct.c_void_p(f.data_ptr()),
                           ct.c_void_p(v.data_ptr()) if v is not None else None)
        return e, f, (v.view(self.S, 3, 3) if v is not None else None)

    def descriptors(self, x=None):
        t = self.torch
        G = t.empty(self.B, 64, dtype=t.float64, device="cuda")
        xp = None
        if x is not None:
            x = x.to(device="cuda", dtype=t.float64).contiguous()
            xp = ct.c_void_p(x.data_ptr())
        pimd_descriptors(self.h, xp, ct.c_void_p(G.data_ptr()))
        return G

    def estimators(self):
        return pimd_estimators(self.h, self.R)

    def get_state(self):
        return pimd_get_state(self.h, 3 * self.B, self.R)

    def set_state(self, q, p, step, Q=None):
        pimd_set_state(self.h, q, p, step, Q)

    def get_forces(self):
        return pimd_get_forces(self.h, self.B, self.S)

    def neighbours(self):
        return pimd_get_neighbours(self.h, self.B, self.maxnb)

    def sync(self):
        pimd_sync(self.h)

    def stage_times(self) -> dict:
        return pimd_stage_times(self.h)

    def set_noise_index(self, atom_offset: int, n_atoms_total: int, replica: int = 0):
        """Draw the replica's thermostat noise as atoms atom_offset .. of a
        system of n_atoms_total atoms (a slice of a larger ring polymer);
        resets the replica's initial state."""
        _check(load().pimd_set_noise_index(self.h, int(replica), int(atom_offset), int(n_atoms_total)), self.h)

    def set_forces(self, f):
        """Bead forces (CUDA FP64 [B, 3]) of the current positions, before the
        first ring_start."""
        f = f.contiguous()
        _check(load().pimd_set_forces(self.h, ct.c_void_p(f.data_ptr())), self.h)

    def ring_start(self):
        """First half of a step with the current forces; the new bead
        positions as a CUDA FP64 [B, 3] tensor."""
        x = self.torch.empty((self.B, 3), dtype=self.torch.float64, device="cuda")
        _check(load().pimd_ring_start(self.h, ct.c_void_p(x.data_ptr())), self.h)
        return x

    def ring_finish(self, f):
        """Second half of the step with the forces f (CUDA FP64 [B, 3]) of the
        positions ring_start returned."""
        f = f.contiguous()
        _check(load().pimd_ring_finish(self.h, ct.c_void_p(f.data_ptr())), self.h)

    def set_overlap(self, on: bool) -> bool:
        """Overlapped parts of the bead-atoms in the step's graph; returns
        whether this context has parts."""
        rc = load().pimd_set_overlap(self.h, 1 if on else 0)
        if rc < 0:
            _check(rc, self.h)
        return rc == 1

    def set_stage_timing(self, on: bool):
        _check(load().pimd_set_stage_timing(self.h, 1 if on else 0), self.h)

    def kernels_per_step(self) -> int:
        return pimd_kernels_per_step(self.h)

    def tune(self, reps: int = 3) -> dict:
        return pimd_tune(self.h, reps)

    def set_schedule(self, band_length: int):
        pimd_set_schedule(self.h, band_length)

    def set_angular(self, algo: str):
        pimd_set_angular(self.h, algo)

    def set_adjoint_warps(self, warps_per_sm: int):
        """Residency of the BF16 moment-tensor adjoint: 12 or 16 warps per SM."""
        _check(load().pimd_set_adjoint_warps(self.h, int(warps_per_sm)), self.h)

    @property
    def adjoint_warps(self) -> int:
        return int(load().pimd_get_adjoint_warps(self.h))

    def metad_hills(self, replica: int = 0):
        return pimd_metad_hills(self.h, replica)

    def metad_set_hills(self, s, h, replica: int = 0):
        pimd_metad_set_hills(self.h, replica, s, h)

    def metad_cv(self):
        """(CV, bias) of every bead-system at the last force evaluation"""
        return pimd_metad_cv(self.h, sum(r.n_beads for r in self.replicas))

    def element_types(self) -> list:
        return pimd_element_types(self.h)

    def rdf_counts(self, r_max: float, n_bins: int, replica: int = 0, counts=None):
        """Pair counts of every bead of one replica (device uint64 tensor
        [T (T + 1) / 2, n_bins], accumulated into counts if given)."""
        torch = self.torch
        T = len(self.element_types())
        if counts is None:
            counts = torch.zeros((T * (T + 1) // 2, n_bins), dtype=torch.int64, device="cuda")
        pimd_rdf_counts(self.h, replica, r_max, n_bins, counts.data_ptr())
        return counts

    def rdf_gr(self, counts, r_max: float, n_configs: float, replica: int = 0):
        """g(r) per element pair (device FP64 tensor, counts' shape) from the
        pair counts of rdf_counts summed over n_configs bead configurations."""
        torch = self.torch
        g = torch.empty(counts.shape, dtype=torch.float64, device="cuda")
        _check(load().pimd_rdf_gr(self.h, int(replica), float(r_max), int(counts.shape[1]), float(n_configs),
                                  ct.c_void_p(counts.data_ptr()), ct.c_void_p(g.data_ptr())), self.h)
        return g

    def cv_histogram(self, s_range, n_bins: int, hist=None, wsum=None, log_w_shift: float = 0.0,
                     replica: int = 0):
        """Adds the current configuration to the bead-resolved CV histogram
        (device FP64 [P, n_bins] and [1], created zeroed when None) with the
        weight that removes the bias; returns (hist, wsum)."""
        torch = self.torch
        if hist is None:
            hist = torch.zeros((self.replicas[replica].n_beads, n_bins), dtype=torch.float64, device="cuda")
        if wsum is None:
            wsum = torch.zeros(1, dtype=torch.float64, device="cuda")
        _check(load().pimd_cv_histogram(self.h, int(replica), float(s_range[0]), float(s_range[1]), int(n_bins),
                                        float(log_w_shift), ct.c_void_p(hist.data_ptr()),
                                        ct.c_void_p(wsum.data_ptr())), self.h)
        return hist, wsum

    def pi_fes(self, hist, wsum, s_range, replica: int = 0):
        """(F [n_bins], F_k [P, n_bins]) in eV on the device: the path-integral
        free energy and each bead's, from a cv_histogram histogram."""
        torch = self.torch
        P, n_bins = hist.shape
        F = torch.empty(n_bins, dtype=torch.float64, device="cuda")
        Fk = torch.empty((P, n_bins), dtype=torch.float64, device="cuda")
        _check(load().pimd_pi_fes(self.h, int(replica), ct.c_void_p(hist.data_ptr()), ct.c_void_p(wsum.data_ptr()),
                                  float(s_range[0]), float(s_range[1]), int(n_bins), ct.c_void_p(F.data_ptr()),
                                  ct.c_void_p(Fk.data_ptr())), self.h)
        return F, Fk

    def metad_fes(self, s, replica: int = 0):
        """F(s) = -(gamma / (gamma - 1)) V(s) of the replica's hills at the
        CV values s (device FP64 tensor), on the device."""
        torch = self.torch
        s = s.to(device="cuda", dtype=torch.float64).contiguous()
        F = torch.empty_like(s)
        _check(load().pimd_metad_fes(self.h, int(replica), ct.c_void_p(s.data_ptr()), int(s.numel()),
                                     ct.c_void_p(F.data_ptr())), self.h)
        return F

    def pt_coordinate(self, bond, acceptor_Z: int = 8, v_range=(-2.0, 1.0), n_bins: int = 60, replica: int = 0):
        """Proton-transfer coordinate of every bead of one replica: (v [P, N]
        float tensor, NaN for non-protons; histogram int64 tensor [n_bins]).
        bond: per atom the replica-local index of its bonding atom, -1 for
        atoms that are not protons."""
        torch = self.torch
        rep = self.replicas[replica]
        b = torch.as_tensor(np.asarray(bond, dtype=np.int32), device="cuda")
        v = torch.empty((rep.n_beads, rep.n_atoms), dtype=torch.float32, device="cuda")
        h = torch.zeros(n_bins, dtype=torch.int64, device="cuda")
        pimd_pt_coordinate(self.h, replica, b.data_ptr(), acceptor_Z, v_range[0], v_range[1], n_bins, v.data_ptr(),
                           h.data_ptr())
        self.torch.cuda.current_stream().synchronize() if self.stream is None else self.stream.synchronize()
        return v, h

    @property
    def angular(self) -> str:
        return pimd_get_angular(self.h)


def _autograd_function():
    import torch

    class PimdEnergy(torch.autograd.Function):
        """Per-bead energies V_k(x) with dV/dx from the library's adjoint
        kernel (forces are evaluated with the energies; backward scales them
        by the incoming gradient)."""

        @staticmethod
        def forward(fctx, x, context):
            e, f, _ = context.energy_forces(x.detach(), want_virial=False)
            fctx.save_for_backward(f)
            fctx.bead_of_atom = context._bead_index()
            return e

        @staticmethod
        def backward(fctx, grad_e):
            (f,) = fctx.saved_tensors
            g = grad_e[fctx.bead_of_atom].unsqueeze(1)
            return -(g * f), None

    return PimdEnergy


def _bead_index(self):
    t = self.torch
    if not hasattr(self, "_bidx"):
        idx = []
        s = 0
        for r in self.replicas:
            for k in range(int(r.n_beads)):
                idx.extend([s] * r.n_atoms)
                s += 1
        self._bidx = t.tensor(idx, dtype=t.long, device="cuda")
    return self._bidx


Context._bead_index = _bead_index


def pimd_energy(x, context):
    """Differentiable per-bead energies (torch.autograd)."""
    return _autograd_function().apply(x, context)
