"""FP64 oracle of the graph-field-network force head (paper Sec. 2.2).

TEST INFRASTRUCTURE ONLY (tests, smoke(), the benchmark's CPU legs). Plain
numpy in the order of the paper's equations; shares no code with the CUDA
library.

Sec. 2.2 gives the head as iterated node / edge updates and a force read
out from the final edge representation:

    m_i^(l)     = phi_m(e_ij^(l))                       (summed over j in N(i))
    n_i^(l+1)   = n_i^(l) + phi_v(n_i^(l), m_i^(l))
    e_ij^(l+1)  = e_ij^(l) + agg(n_i^(l), n_j^(l))
    F_ij        = c_ij * d_ij * phi_f(e_ij^(L))

Readings where the text leaves the form open (one line each; all are the
module's, none is printed in the paper):
  * node input n_i^(0): a learned embedding of the element (the backbone that
    would feed it is outside the head);
  * edge input e_ij^(0) = W_e rho(r_ij) + b_e, rho = the 32 radial functions
    exp(-eta_R (r - r_mu)^2) fc(r) of the descriptors;
  * m_i^(l) sums phi_m over the neighbours; phi_m = SiLU(W_m e + b_m);
  * phi_v(n, m) = W_v2 SiLU(W_v1 [n; m] + b_v1) + b_v2;
  * agg(n_i, n_j) = W_a2 SiLU(W_a1 (n_i + n_j) + b_a1) + b_a2 (symmetric, so
    e_ij = e_ji at every iteration), with the pre-update n^(l) as printed;
  * phi_f(e) = w_f2 . SiLU(W_f1 e + b_f1) + b_f2 (a scalar);
  * c_ij = s_F fc(r_ij) (vanishes with its slope at the cutoff), d_ij =
    (x_i - x_j) / |x_i - x_j|, F_i = sum_j F_ij; L = 3 and SiLU per Table S1;
  * virial of the pair forces W = 1/2 sum_i sum_j (x_i - x_j) (x) F_ij.
F_ij = -F_ji follows (d antisymmetric, e and c symmetric), so momentum is
conserved; the forces are equivariant under rotations and central, so the
torque vanishes for a free cluster. There is no energy: the head is
non-conservative by construction.
"""
from __future__ import annotations

import numpy as np

from . import neighbours


def silu(v):
    return v / (1.0 + np.exp(-v))


def _edges(model, x, box, maxnb: int):
    """Directed edges (i, j) of the neighbour lists (exact FP32 rule) with the
    FP64 minimum-image vectors r_ij = x_j - x_i."""
    rc = model.desc["cutoff"]
    _, nbr, nnb = neighbours(x, box, rc, maxnb)
    src = np.repeat(np.arange(len(x)), nnb)
    dst = np.concatenate([nbr[i, :nnb[i]] for i in range(len(x))]) if len(x) else np.zeros(0, int)
    r = x[dst] - x[src]
    if box is not None and box[0] > 0.0:
        L = np.asarray(box, dtype=np.float64)
        r = r - L * np.rint(r / L)
    return src, dst.astype(np.int64), r


def cutoff(r, rc):
    return np.where(r < rc, 0.5 * (np.cos(np.pi * r / rc) + 1.0), 0.0)


def forces(model, Z, x, box=None, maxnb: int = 256):
    """Forces F [N, 3] (eV/A) and the pair-force virial W [3, 3] (eV) of one
    configuration (one bead)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    Z = np.asarray(Z)
    F_, L_ = model.F, model.L
    rc = model.desc["cutoff"]
    r_mu = np.asarray(model.desc["r_mu"])
    eta_R = model.desc["eta_R"]
    src, dst, rij = _edges(model, x, box, maxnb)
    r = np.linalg.norm(rij, axis=1)
    fc = cutoff(r, rc)
    rho = np.exp(-eta_R * (r[:, None] - r_mu[None, :]) ** 2) * fc[:, None]
    # inputs
    idx = np.array([model.elements.index(int(z)) for z in Z], dtype=np.int64)
    n = model.view("emb")[idx].copy()
    e = rho @ model.view("W_e").T + model.view("b_e")
    # L message-passing iterations
    for l in range(L_):
        W = {k: model.view("%s%d" % (k, l)) for k in ("W_m", "b_m", "W_v1", "b_v1", "W_v2", "b_v2",
                                                       "W_a1", "b_a1", "W_a2", "b_a2")}
        m = np.zeros((len(x), F_))
        np.add.at(m, src, silu(e @ W["W_m"].T + W["b_m"]))
        n_new = n + silu(np.concatenate([n, m], axis=1) @ W["W_v1"].T + W["b_v1"]) @ W["W_v2"].T + W["b_v2"]
        e = e + silu((n[src] + n[dst]) @ W["W_a1"].T + W["b_a1"]) @ W["W_a2"].T + W["b_a2"]
        n = n_new
    # force readout
    phi = silu(e @ model.view("W_f1").T + model.view("b_f1")) @ model.view("w_f2") + model.view("b_f2")[0]
    d = -rij / r[:, None]
    Fij = (model.view("s_F")[0] * fc * phi)[:, None] * d
    Fo = np.zeros((len(x), 3))
    np.add.at(Fo, src, Fij)
    Wv = 0.5 * np.einsum("ea,eb->ab", -rij, Fij)
    return Fo, Wv


def forces_batch(model, Z, xs, box=None, maxnb: int = 256):
    out = [forces(model, Z, x, box, maxnb) for x in xs]
    return np.stack([o[0] for o in out]), np.stack([o[1] for o in out])
