"""FP64 CPU oracle for PIMD with a symmetry-function neural-network potential.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's cpu_baseline / reference legs are its only users. It is a plain,
slow restatement of the method (paper Sec. 2.1 ring-polymer Hamiltonian,
normal modes and estimators; descriptor-based energy model of Sec. 1 / ref.
[17] with forces as the energy gradient, Sec. 2.2; PILE-L of Tables S2-S3) in
C, loaded through ctypes. It shares no code with the CUDA library.

The graph-field-network force head (Sec. 2.2, direct forces) is the numpy
module ``oracle.gfn``.

Parity pins live in tests/test_oracle_*.py (the step cut at its force
evaluation, for bead-sharded runs: tests/test_shard.py, bit for bit against
the whole step; the free-energy and g(r) routines of Sec. 2.5 and Figs. 8-9:
tests/test_oracle_fes.py). Parts without an independent pin: long-time
trajectory physics of the random-init network (parity unpinned).
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

ND = 64
MAX_ELEM = 8
MAX_LAYERS = 8

_lib = None


class OrModel(ct.Structure):
    _fields_ = [
        ("n_elem", ct.c_int),
        ("Z", ct.c_int * MAX_ELEM),
        ("n_hidden", ct.c_int),
        ("width", ct.c_int * MAX_LAYERS),
        ("params", ct.POINTER(ct.c_double) * MAX_ELEM),
        ("rc", ct.c_double),
        ("eta_R", ct.c_double),
        ("r_mu", ct.c_double * 32),
        ("zeta", ct.c_int * 4),
        ("lam", ct.c_double * 2),
        ("eta_A", ct.c_double * 4),
    ]


class OrMetad(ct.Structure):
    _fields_ = [("cv", ct.c_int), ("n_terms", ct.c_int), ("ti", ct.c_int * 8), ("tj", ct.c_int * 8),
                ("tc", ct.c_double * 8), ("Q", ct.c_double), ("f_atom", ct.POINTER(ct.c_double)),
                ("h0", ct.c_double), ("sigma", ct.c_double), ("gamma", ct.c_double), ("stride", ct.c_int),
                ("max_hills", ct.c_int), ("hill_s", ct.POINTER(ct.c_double)), ("hill_h", ct.POINTER(ct.c_double)),
                ("n_hills", ct.c_int), ("cv_last", ct.POINTER(ct.c_double)), ("vb_last", ct.POINTER(ct.c_double))]


class Metad:
    """Well-tempered metadynamics state for one system (oracle side).
    cv = ("distances", [(i, j, c), ...]) or ("xrd", Q, f_atom)."""

    def __init__(self, cv, n_atoms: int, n_beads: int, h0: float, sigma: float, gamma: float, stride: int,
                 max_hills: int = 4096):
        m = OrMetad()
        if cv[0] == "distances":
            m.cv = 1
            m.n_terms = len(cv[1])
            for t, (i, j, c) in enumerate(cv[1]):
                m.ti[t], m.tj[t], m.tc[t] = int(i), int(j), float(c)
            self.f = None
        else:
            m.cv = 2
            m.Q = float(cv[1])
            self.f = _f64(cv[2])
            m.f_atom = _dp(self.f)
        m.h0, m.sigma, m.gamma, m.stride, m.max_hills = float(h0), float(sigma), float(gamma), int(stride), int(max_hills)
        self.hs = np.zeros(max_hills)
        self.hh = np.zeros(max_hills)
        self.cv_last = np.zeros(n_beads)
        self.vb_last = np.zeros(n_beads)
        m.hill_s, m.hill_h = _dp(self.hs), _dp(self.hh)
        m.cv_last, m.vb_last = _dp(self.cv_last), _dp(self.vb_last)
        m.n_hills = 0
        self.m = m
        self.n_atoms = n_atoms

    @property
    def hills(self):
        n = self.m.n_hills
        return self.hs[:n].copy(), self.hh[:n].copy()

    def cv(self, x, box, grad: bool = False):
        """(s, ds/dx [n,3] or None, vir [3,3] or None) of one configuration"""
        x = _f64(x)
        g = np.zeros((self.n_atoms, 3)) if grad else None
        v = np.zeros(9) if grad else None
        s = lib().or_cv(ct.byref(self.m), self.n_atoms, _dp(x), _dp(_box(box)), _dp(g) if grad else None,
                        _dp(v) if grad else None)
        return s, g, (v.reshape(3, 3) if grad else None)

    def deposit(self, cv_last, vb_last, T: float):
        """one deposition from given per-bead CVs and biases"""
        self.cv_last[:] = cv_last
        self.vb_last[:] = vb_last
        lib().or_metad_deposit(ct.byref(self.m), len(self.cv_last), float(T))

    def bias(self, s: float):
        dv = ct.c_double(0.0)
        v = lib().or_metad_bias(ct.byref(self.m), float(s), ct.byref(dv))
        return v, dv.value

    def set_hills(self, s, h):
        s, h = _f64(s), _f64(h)
        self.hs[:len(s)] = s
        self.hh[:len(h)] = h
        self.m.n_hills = len(s)

    def fes(self, s):
        """F(s) = -(gamma / (gamma - 1)) V(s) of the current hills"""
        s = _f64(np.atleast_1d(s))
        F = np.zeros(len(s))
        lib().or_metad_fes(ct.byref(self.m), len(s), _dp(s), _dp(F))
        return F


class OrSys(ct.Structure):
    _fields_ = [
        ("N", ct.c_int), ("P", ct.c_int),
        ("Z", ct.POINTER(ct.c_int)),
        ("mass", ct.POINTER(ct.c_double)),
        ("box", ct.c_double * 3),
        ("T", ct.c_double),
        ("seed", ct.c_uint64),
        ("replica", ct.c_int),
        ("dt", ct.c_double),
        ("gamma0", ct.c_double),
        ("pile_lambda", ct.c_double),
        ("thermostat", ct.c_int),
        ("potential", ct.c_int),
        ("omega_harm", ct.c_double),
        ("maxnb", ct.c_int),
        ("splitting", ct.c_int),
        ("free_rp", ct.c_int),
        ("metad", ct.POINTER(OrMetad)),
        ("transform", ct.c_int),
    ]


class OrEst(ct.Structure):
    _fields_ = [("V_mean", ct.c_double), ("K_prim", ct.c_double), ("K_cv", ct.c_double),
                ("E_tot", ct.c_double), ("W", ct.c_double * 9), ("H_cons", ct.c_double),
                ("Q_thermo", ct.c_double), ("T_kin", ct.c_double)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k in ("V_mean", "K_prim", "K_cv", "E_tot", "H_cons", "Q_thermo", "T_kin")}
        d["W"] = np.array(list(self.W)).reshape(3, 3)
        return d


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ct.CDLL(path)
        dp = ct.POINTER(ct.c_double)
        ip = ct.POINTER(ct.c_int)
        L.or_neighbours.argtypes = [ct.c_int, dp, dp, ct.c_double, ct.c_int, ip, ip]
        L.or_descriptors.argtypes = [ct.POINTER(OrModel), ct.c_int, dp, dp, ip, ip, ct.c_int, dp]
        L.or_mlp.argtypes = [ct.POINTER(OrModel), ct.c_int, dp, dp]
        L.or_mlp.restype = ct.c_double
        L.or_energy_forces.argtypes = [ct.POINTER(OrModel), ct.c_int, ip, dp, dp, ct.c_int, dp, dp, dp]
        L.or_energy_forces_batch.argtypes = [ct.POINTER(OrModel), ct.c_int, ct.c_int, ip, dp, dp,
                                             ct.c_int, dp, dp, dp]
        L.or_nm_matrix.argtypes = [ct.c_int, dp]
        L.or_nm_freqs.argtypes = [ct.c_int, ct.c_double, dp]
        u32p = ct.POINTER(ct.c_uint32)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_normal.argtypes = [ct.c_uint64, ct.c_uint32, ct.c_uint32, ct.c_uint32, ct.c_uint32]
        L.or_normal.restype = ct.c_double
        L.or_init.argtypes = [ct.POINTER(OrSys), dp, dp, dp]
        L.or_forces.argtypes = [ct.POINTER(OrSys), ct.POINTER(OrModel), dp, dp, dp, dp, dp]
        L.or_step.argtypes = [ct.POINTER(OrSys), ct.POINTER(OrModel), ct.c_int, ct.POINTER(ct.c_uint64),
                              dp, dp, dp, dp, dp, dp]
        L.or_estimators.argtypes = [ct.POINTER(OrSys), dp, dp, dp, dp, dp, ct.c_double, ct.POINTER(OrEst)]
        L.or_set_threads.argtypes = [ct.c_int]
        u64p = ct.POINTER(ct.c_uint64)
        L.or_rdf_counts.argtypes = [ct.c_int, dp, dp, ip, ct.c_int, ct.c_double, ct.c_int, u64p]
        L.or_pt_coordinate.argtypes = [ct.c_int, dp, dp, ip, ip, ct.c_double, ct.c_double, ct.c_int,
                                       ct.POINTER(ct.c_float), u64p]
        L.or_cv.argtypes = [ct.POINTER(OrMetad), ct.c_int, dp, dp, dp, dp]
        L.or_cv.restype = ct.c_double
        L.or_metad_bias.argtypes = [ct.POINTER(OrMetad), ct.c_double, ct.POINTER(ct.c_double)]
        L.or_metad_bias.restype = ct.c_double
        L.or_metad_deposit.argtypes = [ct.POINTER(OrMetad), ct.c_int, ct.c_double]
        L.or_staging_to_beads.argtypes = [ct.c_int, dp, dp]
        L.or_beads_to_staging.argtypes = [ct.c_int, dp, dp]
        L.or_staging_forces.argtypes = [ct.c_int, dp, dp]
        L.or_free_rp_step.argtypes = [ct.c_int, ct.c_double, ct.c_double, ct.c_double,
                                      ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
        L.or_get_threads.restype = ct.c_int
        L.or_rdf_gr.argtypes = [ct.c_int, ip, ct.c_double, ct.c_double, ct.c_int, ct.c_double, u64p, dp]
        L.or_cv_histogram.argtypes = [ct.c_int, dp, dp, ct.c_double, ct.c_double, ct.c_double, ct.c_int,
                                      ct.c_double, dp, dp]
        L.or_pi_fes.argtypes = [ct.c_int, ct.c_int, dp, ct.c_double, ct.c_double, ct.c_double, dp, dp]
        L.or_metad_fes.argtypes = [ct.POINTER(OrMetad), ct.c_int, dp, dp]
        L.or_ring_start.argtypes = [ct.POINTER(OrSys), ct.c_uint64, ct.c_int, ct.c_int, dp, dp, dp, dp,
                                    ct.POINTER(ct.c_double)]
        L.or_ring_finish.argtypes = [ct.POINTER(OrSys), ct.c_uint64, ct.c_int, ct.c_int, dp, dp,
                                     ct.POINTER(ct.c_double)]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _box(box) -> np.ndarray:
    return _f64(box if box is not None else (0.0, 0.0, 0.0))


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def threads() -> int:
    return int(lib().or_get_threads())


class ModelHandle:
    """ctypes view of a synth.Model (keeps its parameter blobs alive)."""

    def __init__(self, model):
        self.model = model
        s = OrModel()
        s.n_elem = len(model.elements)
        self._blobs = []
        for e, z in enumerate(model.elements):
            s.Z[e] = int(z)
            b = _f64(model.params[z])
            self._blobs.append(b)
            s.params[e] = _dp(b)
        s.n_hidden = len(model.widths)
        for l, w in enumerate(model.widths):
            s.width[l] = int(w)
        d = model.desc
        s.rc = d["cutoff"]
        s.eta_R = d["eta_R"]
        for m, r in enumerate(d["r_mu"]):
            s.r_mu[m] = r
        for k, z in enumerate(d["zeta"]):
            s.zeta[k] = int(z)
        for k, l in enumerate(d["lam"]):
            s.lam[k] = l
        for k, e in enumerate(d["eta_A"]):
            s.eta_A[k] = e
        self.s = s

    @property
    def ptr(self):
        return ct.byref(self.s)


def neighbours(x, box, rc: float, maxnb: int = 256):
    """Sorted neighbour sets under the exact FP32 inclusion rule."""
    x = _f64(x)
    n = len(x)
    nbr = np.zeros((n, maxnb), dtype=np.int32)
    nnb = np.zeros(n, dtype=np.int32)
    worst = lib().or_neighbours(n, _dp(x), _dp(_box(box)), rc, maxnb, _ip(nbr), _ip(nnb))
    if worst > maxnb:
        raise ValueError("neighbour overflow: %d > %d" % (worst, maxnb))
    return [nbr[i, :nnb[i]].copy() for i in range(n)], nbr, nnb


def descriptors(model, x, box, maxnb: int = 256) -> np.ndarray:
    mh = model if isinstance(model, ModelHandle) else ModelHandle(model)
    x = _f64(x)
    _, nbr, nnb = neighbours(x, box, mh.model.desc["cutoff"], maxnb)
    G = np.zeros((len(x), ND))
    lib().or_descriptors(mh.ptr, len(x), _dp(x), _dp(_box(box)), _ip(nbr), _ip(nnb), maxnb, _dp(G))
    return G


def mlp(model, z: int, G) -> tuple[float, np.ndarray]:
    mh = model if isinstance(model, ModelHandle) else ModelHandle(model)
    G = _f64(G)
    g = np.zeros(ND)
    E = lib().or_mlp(mh.ptr, int(z), _dp(G), _dp(g))
    return E, g


def energy_forces(model, Z, x, box, maxnb: int = 256):
    """Per-atom energies E_i (eV), forces -dV/dx (eV/A), virial W (eV)."""
    mh = model if isinstance(model, ModelHandle) else ModelHandle(model)
    x = _f64(x)
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    n = len(x)
    E = np.zeros(n)
    F = np.zeros((n, 3))
    W = np.zeros(9)
    r = lib().or_energy_forces(mh.ptr, n, _ip(Z), _dp(x), _dp(_box(box)), maxnb, _dp(E), _dp(F), _dp(W))
    if r < 0:
        raise ValueError("oracle energy_forces failed (%d)" % r)
    return E, F, W.reshape(3, 3)


def energy_forces_batch(model, Z, xs, box, maxnb: int = 256):
    mh = model if isinstance(model, ModelHandle) else ModelHandle(model)
    xs = _f64(xs)
    nconf, n = xs.shape[0], xs.shape[1]
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    E = np.zeros((nconf, n))
    F = np.zeros((nconf, n, 3))
    W = np.zeros((nconf, 9))
    r = lib().or_energy_forces_batch(mh.ptr, nconf, n, _ip(Z), _dp(xs), _dp(_box(box)), maxnb,
                                     _dp(E), _dp(F), _dp(W))
    if r < 0:
        raise ValueError("oracle energy_forces failed (%d)" % r)
    return E, F, W.reshape(nconf, 3, 3)


def nm_matrix(P: int) -> np.ndarray:
    C = np.zeros((P, P))
    lib().or_nm_matrix(P, _dp(C))
    return C


def nm_freqs(P: int, omega_P: float) -> np.ndarray:
    w = np.zeros(P)
    lib().or_nm_freqs(P, omega_P, _dp(w))
    return w


def rdf_counts(x, box, types, n_types: int, r_max: float, n_bins: int) -> np.ndarray:
    """RDF pair counts [n_types (n_types + 1) / 2, n_bins] of one configuration
    (FP32 distance rule; see or_rdf_counts)."""
    x = _f64(x)
    t = np.ascontiguousarray(types, dtype=np.int32)
    out = np.zeros(n_types * (n_types + 1) // 2 * n_bins, dtype=np.uint64)
    lib().or_rdf_counts(len(t), _dp(x), _dp(_box(box)), _ip(t), int(n_types), float(r_max), int(n_bins),
                        out.ctypes.data_as(ct.POINTER(ct.c_uint64)))
    return out.reshape(-1, n_bins)


def pt_coordinate(x, box, bond, acceptor, v_min: float, v_max: float, n_bins: int):
    """Proton-transfer coordinate per atom (NaN for non-protons) and its
    histogram (see or_pt_coordinate)."""
    x = _f64(x)
    b = np.ascontiguousarray(bond, dtype=np.int32)
    a = np.ascontiguousarray(acceptor, dtype=np.int32)
    v = np.zeros(len(b), dtype=np.float32)
    h = np.zeros(n_bins, dtype=np.uint64)
    lib().or_pt_coordinate(len(b), _dp(x), _dp(_box(box)), _ip(b), _ip(a), float(v_min), float(v_max),
                           int(n_bins), v.ctypes.data_as(ct.POINTER(ct.c_float)),
                           h.ctypes.data_as(ct.POINTER(ct.c_uint64)))
    return v, h


def rdf_gr(counts, n_per_type, volume: float, r_max: float, n_configs: float) -> np.ndarray:
    """g(r) per element pair from pair counts [T (T + 1) / 2, n_bins] summed
    over n_configs configurations (see or_rdf_gr)."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    n = np.ascontiguousarray(n_per_type, dtype=np.int32)
    g = np.zeros(c.shape, dtype=np.float64)
    lib().or_rdf_gr(len(n), _ip(n), float(volume), float(r_max), int(c.shape[1]), float(n_configs),
                    c.ctypes.data_as(ct.POINTER(ct.c_uint64)), _dp(g))
    return g


class CvHistogram:
    """Bead-resolved CV histogram of the path-integral FES (Sec. 2.5):
    add() takes the P beads' CVs and biases of one configuration."""

    def __init__(self, P: int, s_min: float, s_max: float, n_bins: int, T: float, log_w_shift: float = 0.0):
        self.P, self.n_bins, self.T = int(P), int(n_bins), float(T)
        self.s_min, self.s_max = float(s_min), float(s_max)
        self.inv_ds = n_bins / (s_max - s_min)
        self.shift = float(log_w_shift)
        self.hist = np.zeros((self.P, self.n_bins))
        self.wsum = np.zeros(1)

    def add(self, s, vb=None):
        s = _f64(s)
        vb = np.zeros(self.P) if vb is None else _f64(vb)
        lib().or_cv_histogram(self.P, _dp(s), _dp(vb), self.T, self.s_min, self.inv_ds, self.n_bins, self.shift,
                              _dp(self.hist), _dp(self.wsum))

    def fes(self):
        """(F [n_bins], F_k [P, n_bins]) in eV, +inf where a bin is empty"""
        F = np.zeros(self.n_bins)
        Fk = np.zeros((self.P, self.n_bins))
        lib().or_pi_fes(self.P, self.n_bins, _dp(self.hist), float(self.wsum[0]),
                        (self.s_max - self.s_min) / self.n_bins, self.T, _dp(F), _dp(Fk))
        return F, Fk


def staging_to_beads(u):
    """bead positions [P, N, 3] from staging coordinates [P, N, 3]"""
    u = _f64(u)
    P = u.shape[0]
    x = np.zeros_like(u)
    a, b = np.zeros(P), np.zeros(P)
    for i in range(u.shape[1]):
        for d in range(3):
            a[:] = u[:, i, d]
            lib().or_staging_to_beads(P, _dp(a), _dp(b))
            x[:, i, d] = b
    return x


def beads_to_staging(x):
    x = _f64(x)
    P = x.shape[0]
    u = np.zeros_like(x)
    a, b = np.zeros(P), np.zeros(P)
    for i in range(x.shape[1]):
        for d in range(3):
            a[:] = x[:, i, d]
            lib().or_beads_to_staging(P, _dp(a), _dp(b))
            u[:, i, d] = b
    return u


def staging_forces(f):
    f = _f64(f)
    P = len(f)
    out = np.zeros(P)
    lib().or_staging_forces(P, _dp(f), _dp(out))
    return out


def free_rp_step(free_rp: str, m: float, w: float, h: float, p: float, q: float) -> tuple:
    """One free ring-polymer step of one mode: (p, q) after time h."""
    pp, qq = ct.c_double(p), ct.c_double(q)
    lib().or_free_rp_step({"exact": 0, "cayley": 1}[free_rp], float(m), float(w), float(h), ct.byref(pp),
                          ct.byref(qq))
    return pp.value, qq.value


def philox(ctr, key) -> tuple:
    c = (ct.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ct.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ct.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def normal(seed: int, index: int, step: int, replica: int, stream: int) -> float:
    return float(lib().or_normal(seed, index, step, replica, stream))


class System:
    """One ring-polymer system advanced by the oracle integrator.

    potential = "model" (symmetry-function network) or "harmonic" with
    angular frequency omega (1/fs)."""

    def __init__(self, replica, masses: dict, dt: float, gamma0: float, pile_lambda: float = 1.0,
                 model=None, thermostat: bool = True, potential: str = "model", omega: float = 0.0,
                 replica_index: int = 0, maxnb: int = 256, splitting: str = "obabo",
                 free_rp: str = "exact", metad: "Metad" = None, transform: str = "normal_modes"):
        self.mh = None if model is None else (model if isinstance(model, ModelHandle) else ModelHandle(model))
        self.Z = np.ascontiguousarray(replica.Z, dtype=np.int32)
        self.mass = _f64([masses[int(z)] for z in replica.Z])
        N, P = len(self.Z), int(replica.n_beads)
        s = OrSys()
        s.N, s.P = N, P
        s.Z = _ip(self.Z)
        s.mass = _dp(self.mass)
        for a in range(3):
            s.box[a] = float(replica.box[a])
        s.T = float(replica.T)
        s.seed = int(replica.seed)
        s.replica = int(replica_index)
        s.dt = float(dt)
        s.gamma0 = float(gamma0)
        s.pile_lambda = float(pile_lambda)
        s.thermostat = 1 if thermostat else 0
        s.potential = 1 if potential == "harmonic" else 0
        s.omega_harm = float(omega)
        s.maxnb = int(maxnb)
        s.splitting = {"obabo": 0, "baoab": 1}[splitting]
        s.free_rp = {"exact": 0, "cayley": 1}[free_rp]
        s.transform = {"normal_modes": 0, "staging": 1}[transform]
        self.metad = metad
        if metad is not None:
            s.metad = ct.pointer(metad.m)
        self.s = s
        self.N, self.P = N, P
        self.q = np.zeros((P, N, 3))
        self.p = np.zeros((P, N, 3))
        self.f = np.zeros((P, N, 3))
        self.xb = np.zeros((P, N, 3))
        self.V = np.zeros(P)
        self.W = np.zeros((P, 9))
        self.Q = ct.c_double(0.0)
        self.step_count = ct.c_uint64(0)
        x0 = _f64(replica.x0)
        lib().or_init(ct.byref(s), _dp(x0), _dp(self.q), _dp(self.p))
        self.compute_forces()

    def _mptr(self):
        return self.mh.ptr if self.mh is not None else None

    def compute_forces(self):
        r = lib().or_forces(ct.byref(self.s), self._mptr(), _dp(self.q), _dp(self.xb), _dp(self.f),
                            _dp(self.V), _dp(self.W))
        if r < 0:
            raise ValueError("oracle forces failed (%d)" % r)

    def step(self, n: int = 1):
        r = lib().or_step(ct.byref(self.s), self._mptr(), int(n), ct.byref(self.step_count), _dp(self.q),
                          _dp(self.p), _dp(self.f), _dp(self.V), _dp(self.W), ct.byref(self.Q))
        if r < 0:
            raise ValueError("oracle step failed (%d)" % r)

    def ring_start(self, lo: int, hi: int, f=None):
        """First half of a step for atoms lo .. hi-1 with the bead forces f
        ([P, N, 3], default: the last evaluated ones); their new bead
        positions land in self.xb. The step counter is the caller's."""
        f = self.f if f is None else _f64(f)
        lib().or_ring_start(ct.byref(self.s), self.step_count.value, int(lo), int(hi), _dp(self.q), _dp(self.p),
                            _dp(f), _dp(self.xb), ct.byref(self.Q))

    def ring_finish(self, lo: int, hi: int, f):
        """Second half of the step for atoms lo .. hi-1 with the forces f
        ([P, N, 3]) of the new positions."""
        f = _f64(f)
        lib().or_ring_finish(ct.byref(self.s), self.step_count.value, int(lo), int(hi), _dp(self.p), _dp(f),
                             ct.byref(self.Q))

    def beads(self) -> np.ndarray:
        if self.s.transform == 1:
            return staging_to_beads(self.q)
        C = nm_matrix(self.P)
        return np.einsum("jk,kia->jia", C, self.q)

    def estimators(self) -> dict:
        e = OrEst()
        lib().or_estimators(ct.byref(self.s), _dp(self.q), _dp(self.p), _dp(self.f), _dp(self.V),
                            _dp(self.W), self.Q.value, ct.byref(e))
        return e.as_dict()
