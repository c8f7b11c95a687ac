"""Seeded synthetic inputs for the PIMD + symmetry-function MLFF hot path.

This module only draws numbers: atom positions, element lists, boxes, replica
sets and random-init MLP weights with the shapes of the paper's workloads
(formic-acid dimer, Sec. 3.1; 64-molecule water box, Sec. 3.2 and Table S2;
ice, Sec. 3.2; many independent trajectories, Sec. 2.3). It evaluates none of
the method's arithmetic (no descriptors, network, forces or integrator), so
both the CUDA path and the FP64 test oracle receive identical arrays from it.

Everything is deterministic for a given seed (numpy PCG64 streams; per-replica
seeds derived with splitmix64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# element numbers and masses (amu) used by the synthetic systems
H, C, O = 1, 6, 8
MASS = {H: 1.008, C: 12.011, O: 15.999}

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One step of the splitmix64 mixer (Steele, Lea, Flood 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & MASK64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def replica_seeds(seed: int, n: int) -> list[int]:
    out, s = [], seed & MASK64
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & MASK64
        out.append(splitmix64(s))
    return out


def f32(v: float) -> float:
    """Round to the nearest FP32 value (used for box lengths, so that the FP32
    and FP64 sides of a comparison see exactly the same periodic box)."""
    return float(np.float32(v))


@dataclass
class Replica:
    """One ring-polymer system: N atoms, P beads."""
    Z: np.ndarray            # int32 [N]
    x0: np.ndarray           # float64 [N, 3], Angstrom
    box: tuple               # (Lx, Ly, Lz); 0 = non-periodic
    n_beads: int
    T: float                 # K
    seed: int
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.Z.shape[0])


@dataclass
class Workload:
    name: str
    replicas: list
    dt_fs: float
    gamma0_per_fs: float     # centroid friction 1/tau0
    widths: tuple            # hidden-layer widths of the per-element MLP
    cutoff: float = 6.0
    pile_lambda: float = 1.0
    notes: dict = field(default_factory=dict)

    @property
    def bead_atoms(self) -> int:
        return sum(r.n_atoms * r.n_beads for r in self.replicas)


def _rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _wrap(x: np.ndarray, box) -> np.ndarray:
    L = np.asarray(box, dtype=np.float64)
    return x - L * np.floor(x / L)


# --------------------------------------------------------------------------
# formic-acid dimer (Sec. 3.1): planar C2h cyclic dimer template + jitter
# --------------------------------------------------------------------------
def fad_template() -> tuple[np.ndarray, np.ndarray]:
    """Planar centrosymmetric (C2h) formic-acid dimer with C=O 1.22, C-O 1.32,
    O-H 0.97, C-H 1.09 A, O-C-O 125 deg and hydrogen-bonded O...O 2.70 A.
    Atom order: C1 O1 O2 H1 Hc1 | C2 O3 O4 H2 Hc2 (monomer 2 is the inversion
    image of monomer 1); H1 is bonded to O1 and points at O4's partner."""
    half = math.radians(125.0) / 2
    s, c = math.sin(half), math.cos(half)
    # O1 (hydroxyl) and O2 (carbonyl) hang below carbon at (0, h)
    dx = 1.22 * s - 1.32 * s
    h = (math.sqrt(2.70 ** 2 - dx * dx) + (1.32 + 1.22) * c) / 2
    C1 = np.array([0.0, h, 0.0])
    O1 = C1 + 1.32 * np.array([-s, -c, 0.0])
    O2 = C1 + 1.22 * np.array([s, -c, 0.0])
    O2b = -O2                      # carbonyl O of monomer 2 (H-bond acceptor)
    u = (O2b - O1) / np.linalg.norm(O2b - O1)
    H1 = O1 + 0.97 * u
    Hc1 = C1 + np.array([0.0, 1.09, 0.0])
    mono = np.stack([C1, O1, O2, H1, Hc1])
    x = np.concatenate([mono, -mono])
    Z = np.array([C, O, O, H, H] * 2, dtype=np.int32)
    return Z, x


def fad_dimer_cv_terms() -> list:
    """Double-proton-transfer CV of the dimer (Sec. 3.1):
    s = d(O1,H1) - d(O2,H1) + d(O4,H2) - d(O3,H2), each proton's bonding
    oxygen with +1 and its hydrogen-bond acceptor with -1, as (i, j, c) over
    the template's atom order (H1 = 3 bonded to O 1, accepted by O 7; H2 = 8
    bonded to O 6, accepted by O 2)."""
    return [(1, 3, 1.0), (7, 3, -1.0), (6, 8, 1.0), (2, 8, -1.0)]


def fad(seed: int = 1001, n_beads: int = 16, T: float = 300.0, jitter: float = 0.05) -> Replica:
    rng = np.random.default_rng(seed)
    Z, x = fad_template()
    x = x + rng.normal(scale=jitter, size=x.shape)
    return Replica(Z, x, (0.0, 0.0, 0.0), n_beads, T, replica_seeds(seed, 1)[0], "fad")


# --------------------------------------------------------------------------
# liquid-water-like boxes (Sec. 3.2): oriented molecules on a cubic grid
# --------------------------------------------------------------------------
def water_box(n_side: int, spacing: float = 3.105, seed: int = 1002, n_beads: int = 32,
              T: float = 300.0, jitter: float = 0.05, name: str = "water") -> Replica:
    rng = np.random.default_rng(seed)
    L = f32(n_side * spacing)
    roh, ang = 0.9572, math.radians(104.52)
    # molecule frame: O at origin, H's in the xy plane symmetric about x
    hx, hy = roh * math.cos(ang / 2), roh * math.sin(ang / 2)
    frame = np.array([[0.0, 0.0, 0.0], [hx, hy, 0.0], [hx, -hy, 0.0]])
    xs, Z = [], []
    g = (np.arange(n_side) + 0.5) * spacing
    for ix in g:
        for iy in g:
            for iz in g:
                R = _rotation(rng)
                xs.append(frame @ R.T + np.array([ix, iy, iz]))
                Z += [O, H, H]
    x = np.concatenate(xs)
    x = x + rng.normal(scale=jitter, size=x.shape)
    x = _wrap(x, (L, L, L))
    return Replica(np.array(Z, dtype=np.int32), x, (L, L, L), n_beads, T,
                   replica_seeds(seed, 1)[0], name)


# --------------------------------------------------------------------------
# hexagonal ice Ih (Sec. 3.2) with ice-rule proton disorder
# --------------------------------------------------------------------------
def ice_ih_oxygens(nx: int, ny: int, nz: int, a: float = 4.514, c: float = 7.372):
    """Oxygen sites of an nx x ny x nz supercell of the orthorhombic
    (a, sqrt(3) a, c) ice Ih cell (8 O per cell; ideal tetrahedral z = 1/16)."""
    b = math.sqrt(3.0) * a
    z = 1.0 / 16.0
    hexf = [(1 / 3, 2 / 3, z), (2 / 3, 1 / 3, z + 0.5), (1 / 3, 2 / 3, 0.5 - z), (2 / 3, 1 / 3, -z)]
    cell = []
    for (u, v, w) in hexf:
        p = np.array([a * (u - v / 2), a * math.sqrt(3) / 2 * v, w * c])
        for shift in (np.zeros(3), np.array([a / 2, b / 2, 0.0])):
            cell.append(_wrap(p + shift, (a, b, c)))
    cell = np.array(cell)
    out = []
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                out.append(cell + np.array([i * a, j * b, k * c]))
    box = (f32(nx * a), f32(ny * b), f32(nz * c))
    return np.concatenate(out), box


def _min_image(d: np.ndarray, box) -> np.ndarray:
    L = np.asarray(box, dtype=np.float64)
    return d - L * np.round(d / L)


def ice_ih(nx: int = 6, ny: int = 3, nz: int = 3, seed: int = 1003, n_beads: int = 32,
           T: float = 250.0, jitter: float = 0.05) -> Replica:
    """Proton-disordered ice Ih. Each O-O hydrogen bond of the 4-regular
    oxygen graph is oriented along a seeded random Eulerian circuit, so every
    oxygen donates two and accepts two protons (the ice rules); each proton
    sits on its O->O line at 0.9572 A from the donor."""
    rng = np.random.default_rng(seed)
    Ox, box = ice_ih_oxygens(nx, ny, nz)
    n = len(Ox)
    adj = [[] for _ in range(n)]
    for i in range(n):
        d = np.linalg.norm(_min_image(Ox - Ox[i], box), axis=1)
        nb = np.nonzero((d > 0.1) & (d < 3.0))[0]
        if len(nb) != 4:
            raise RuntimeError("ice lattice: oxygen %d has %d neighbours" % (i, len(nb)))
        adj[i] = [int(j) for j in nb]
    # Hierholzer's algorithm over undirected edges, random edge choice
    unused = {(min(i, j), max(i, j)) for i in range(n) for j in adj[i]}
    avail = [list(a) for a in adj]
    directed = []
    stack, path_edges = [int(rng.integers(n))], []
    while stack:
        v = stack[-1]
        cand = [w for w in avail[v] if (min(v, w), max(v, w)) in unused]
        if cand:
            w = cand[int(rng.integers(len(cand)))]
            unused.discard((min(v, w), max(v, w)))
            stack.append(w)
            path_edges.append((v, w))
        else:
            stack.pop()
            if path_edges:
                directed.append(path_edges.pop())
    if unused or len(directed) != 2 * n:
        raise RuntimeError("ice lattice: Eulerian orientation failed")
    donors = [[] for _ in range(n)]
    for (u, v) in directed:
        donors[u].append(v)
    xs, Z = [], []
    for u in range(n):
        if len(donors[u]) != 2:
            raise RuntimeError("ice rules violated at oxygen %d" % u)
        xs.append(Ox[u])
        for v in donors[u]:
            d = _min_image(Ox[v] - Ox[u], box)
            xs.append(Ox[u] + 0.9572 * d / np.linalg.norm(d))
        Z += [O, H, H]
    x = np.array(xs)
    x = x + rng.normal(scale=jitter, size=x.shape)
    x = _wrap(x, box)
    return Replica(np.array(Z, dtype=np.int32), x, box, n_beads, T,
                   replica_seeds(seed, 1)[0], "ice_ih")


# --------------------------------------------------------------------------
# many independent small gas-phase systems (multi-trajectory mode, Sec. 2.3)
# --------------------------------------------------------------------------
def cluster(rng: np.random.Generator, n: int, d_min: float = 0.9, density: float = 0.1):
    side = (n / density) ** (1.0 / 3.0)
    Z = rng.choice([H, H, C, O], size=n).astype(np.int32)
    x = np.zeros((n, 3))
    k = 0
    while k < n:
        p = rng.uniform(0.0, side, size=3)
        if k == 0 or np.min(np.linalg.norm(x[:k] - p, axis=1)) >= d_min:
            x[k] = p
            k += 1
    return Z, x


def batch(n_rep: int = 256, seed: int = 1004, n_min: int = 6, n_max: int = 24,
          beads=(8, 16, 32, 64), T: float = 300.0) -> list:
    rng = np.random.default_rng(seed)
    seeds = replica_seeds(seed, n_rep)
    reps = []
    for r in range(n_rep):
        n = int(rng.integers(n_min, n_max + 1))
        Z, x = cluster(rng, n)
        P = int(rng.choice(beads))
        reps.append(Replica(Z, x, (0.0, 0.0, 0.0), P, T, seeds[r], "cluster%d" % r))
    return reps


# --------------------------------------------------------------------------
# model hyper-parameters and random-init weights
# --------------------------------------------------------------------------
N_RADIAL = 32
N_ANGULAR = 32
N_DESC = N_RADIAL + N_ANGULAR
ZETAS = (1, 2, 4, 8)
LAMBDAS = (1.0, -1.0)
ETA_A = (0.005, 0.02, 0.05, 0.1)


def descriptor_params(cutoff: float = 6.0) -> dict:
    """Symmetry-function hyper-parameters: 32 radial centres r_mu evenly from
    0.5 to 5.5 A with width eta_R = 1/(2 Delta^2); angular channels
    zeta x lambda x eta_A = 4 x 2 x 4, ordered zeta-major, eta-minor."""
    delta = 5.0 / (N_RADIAL - 1)
    return dict(cutoff=cutoff,
                r_mu=[0.5 + m * delta for m in range(N_RADIAL)],
                eta_R=1.0 / (2.0 * delta * delta),
                zeta=list(ZETAS), lam=list(LAMBDAS), eta_A=list(ETA_A))


@dataclass
class Model:
    """Per-element MLP parameters, FP64. Layout of one element's flat blob:
    for each hidden layer l: W_l [h_l, h_{l-1}] row-major then b_l [h_l];
    then w_out [h_L], b_out [1]; mu [64]; sigma [64]; s_E [1]; e_Z [1]."""
    elements: tuple
    widths: tuple
    params: dict             # Z -> flat float64 blob
    desc: dict

    def blob_size(self) -> int:
        return blob_size(self.widths)

    def offsets(self) -> dict:
        return blob_offsets(self.widths)


def blob_offsets(widths) -> dict:
    off, o, prev = {}, 0, N_DESC
    for l, h in enumerate(widths):
        off["W%d" % l] = (o, (h, prev)); o += h * prev
        off["b%d" % l] = (o, (h,)); o += h
        prev = h
    off["w_out"] = (o, (prev,)); o += prev
    off["b_out"] = (o, (1,)); o += 1
    off["mu"] = (o, (N_DESC,)); o += N_DESC
    off["sigma"] = (o, (N_DESC,)); o += N_DESC
    off["s_E"] = (o, (1,)); o += 1
    off["e_Z"] = (o, (1,)); o += 1
    off["_size"] = o
    return off


def blob_size(widths) -> int:
    return blob_offsets(widths)["_size"]


def view(blob: np.ndarray, widths, key: str) -> np.ndarray:
    o, shape = blob_offsets(widths)[key]
    n = int(np.prod(shape))
    return blob[o:o + n].reshape(shape)


def xavier_model(elements, widths, seed: int, cutoff: float = 6.0) -> Model:
    """Xavier-uniform weights U(+-sqrt(6/(fan_in+fan_out))), zero biases,
    identity normalisation (mu = 0, sigma = 1), s_E = 1, e_Z = 0."""
    rng = np.random.default_rng(seed)
    params = {}
    for z in sorted(elements):
        blob = np.zeros(blob_size(widths))
        prev = N_DESC
        for l, h in enumerate(widths):
            a = math.sqrt(6.0 / (prev + h))
            view(blob, widths, "W%d" % l)[:] = rng.uniform(-a, a, size=(h, prev))
            prev = h
        a = math.sqrt(6.0 / (prev + 1))
        view(blob, widths, "w_out")[:] = rng.uniform(-a, a, size=prev)
        view(blob, widths, "sigma")[:] = 1.0
        view(blob, widths, "s_E")[:] = 1.0
        params[int(z)] = blob
    return Model(tuple(sorted(int(z) for z in elements)), tuple(widths), params,
                 descriptor_params(cutoff))


def set_normalisation(model: Model, G: np.ndarray, Z: np.ndarray, floor: float = 1e-2) -> None:
    """Freeze per-element, per-channel mean and standard deviation of a set of
    descriptor rows G [n, 64] (element of each row in Z) into the model; the
    standard deviation is floored at `floor`. G comes from whichever
    implementation the caller trusts; this function only takes moments."""
    for z in model.elements:
        rows = G[Z == z]
        if len(rows) == 0:
            continue
        blob = model.params[z]
        view(blob, model.widths, "mu")[:] = rows.mean(axis=0)
        view(blob, model.widths, "sigma")[:] = np.maximum(rows.std(axis=0), floor)


def set_energy_scale(model: Model, s_E: float) -> None:
    for z in model.elements:
        view(model.params[z], model.widths, "s_E")[:] = s_E


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def workload(name: str) -> Workload:
    """fad | water64 | ice | batch | water4096 (system shapes of Sec. 3 and
    Tables S1-S2; P = 32 per the bead-convergence note of Sec. S3)."""
    if name == "fad":
        return Workload("fad", [fad()], 0.25, 1.0 / 100.0, (64, 64))
    if name == "water64":
        return Workload("water64", [water_box(4, seed=1002)], 0.5, 1.0 / 1000.0, (128, 128, 128))
    if name == "ice":
        return Workload("ice", [ice_ih()], 0.5, 1.0 / 1000.0, (128, 128, 128))
    if name == "batch":
        return Workload("batch", batch(), 0.25, 1.0 / 100.0, (64, 64))
    if name == "water4096":
        return Workload("water4096", [water_box(16, seed=1005, n_beads=64, name="water4096")],
                        0.5, 1.0 / 1000.0, (256, 256, 256, 256))
    raise KeyError(name)


def elements_of(replicas) -> tuple:
    s = set()
    for r in replicas:
        s.update(int(z) for z in r.Z)
    return tuple(sorted(s))


# --------------------------------------------------------------------------
# graph field network (direct-force head, Sec. 2.2): parameter shapes and
# random-init weights. Layout of the flat FP64 blob (row-major matrices,
# y = W x + b):
#   emb [n_el][F]; W_e [F][32], b_e [F];
#   per iteration l = 0 .. L-1: W_m [F][F], b_m [F], W_v1 [F][2F], b_v1 [F],
#       W_v2 [F][F], b_v2 [F], W_a1 [F][F], b_a1 [F], W_a2 [F][F], b_a2 [F];
#   W_f1 [F][F], b_f1 [F], w_f2 [F], b_f2 [1], s_F [1].
# --------------------------------------------------------------------------
GFN_ITER_KEYS = (("W_m", "FF"), ("b_m", "F"), ("W_v1", "F2F"), ("b_v1", "F"), ("W_v2", "FF"), ("b_v2", "F"),
                 ("W_a1", "FF"), ("b_a1", "F"), ("W_a2", "FF"), ("b_a2", "F"))


def gfn_offsets(F: int, L: int, n_el: int) -> dict:
    shapes = {"F": (F,), "FF": (F, F), "F2F": (F, 2 * F)}
    off, o = {}, 0

    def put(key, shape):
        nonlocal o
        off[key] = (o, shape)
        o += int(np.prod(shape))

    put("emb", (n_el, F))
    put("W_e", (F, N_RADIAL))
    put("b_e", (F,))
    for l in range(L):
        for k, s in GFN_ITER_KEYS:
            put("%s%d" % (k, l), shapes[s])
    put("W_f1", (F, F))
    put("b_f1", (F,))
    put("w_f2", (F,))
    put("b_f2", (1,))
    put("s_F", (1,))
    off["_size"] = o
    return off


@dataclass
class GfnModel:
    """Graph-field-network force head: feature width F, L message-passing
    iterations, one FP64 parameter blob (layout in gfn_offsets), the radial
    basis of the descriptors (r_mu, eta_R, cutoff)."""
    elements: tuple
    F: int
    L: int
    blob: np.ndarray
    desc: dict

    def view(self, key: str) -> np.ndarray:
        o, shape = gfn_offsets(self.F, self.L, len(self.elements))[key]
        return self.blob[o:o + int(np.prod(shape))].reshape(shape)


def gfn_model(elements, F: int = 128, L: int = 3, seed: int = 11, cutoff: float = 6.0) -> GfnModel:
    """Xavier-uniform matrices, small uniform biases (so that every term of
    the head is exercised), N(0, 1) embeddings, s_F = 1."""
    rng = np.random.default_rng(seed)
    els = tuple(sorted(int(z) for z in elements))
    off = gfn_offsets(F, L, len(els))
    blob = np.zeros(off["_size"])
    for key, val in off.items():
        if key == "_size":
            continue
        o, shape = val
        n = int(np.prod(shape))
        if key == "emb":
            blob[o:o + n] = rng.normal(size=n)
        elif len(shape) == 2:
            a = math.sqrt(6.0 / (shape[0] + shape[1]))
            blob[o:o + n] = rng.uniform(-a, a, size=n)
        elif key == "w_f2":
            a = math.sqrt(6.0 / (shape[0] + 1))
            blob[o:o + n] = rng.uniform(-a, a, size=n)
        elif key == "s_F":
            blob[o] = 1.0
        else:
            blob[o:o + n] = rng.uniform(-0.1, 0.1, size=n)
    return GfnModel(els, F, L, blob, descriptor_params(cutoff))


def set_force_scale(model: GfnModel, s_F: float) -> None:
    model.view("s_F")[:] = s_F
