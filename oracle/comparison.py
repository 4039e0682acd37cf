"""The two approximations GCA-H^2 improves on (oracle): pure Green
quadrature (Sect. 2) and single-level GCA (Sect. 3), with their products and
storage, for the error-versus-storage comparison of the paper's Fig. 1-3.

TEST INFRASTRUCTURE ONLY (see the package header).

* Green quadrature (``build_gq``): every admissible block is replaced by the
  quadrature of Green's representation formula on the box omega_tau (Eq. (2)),
      G|tau-hat x sigma-hat ~ A_tau B_{tau sigma}^*,
  A_tau = the Green quadrature matrix of tau (|tau-hat| x 2k; it depends on
  tau only) and B_{tau sigma} the matching factor of sigma on tau's box
  (|sigma-hat| x 2k, ``gca.green_factor_b``).  Storage: every needed A_tau
  once, one B per block.
* Single-level GCA (``build_gca1``): G|tau-hat x sigma-hat ~ V_tau
  G|tilde-tau x tilde-sigma V_sigma^* with V_tau from the cross approximation
  of A_tau on all of tau's triangles (``gca.build_bases(nested=False)``), no
  transfer matrices.  Storage: every V_tau, the couplings.
* Near field as in GCA-H^2 (exact blocks).

Pinned by tests (tests/test_oracle_comparison.py): products equal the dense
representation; the Green quadrature error falls as the box rule's order m
grows and the GCA errors as the tolerance falls; at equal tolerance the
single-level GCA and GCA-H^2 errors agree while GCA-H^2 stores less; V_tau
interpolates (V_tau[tilde-tau, :] = I).
"""

from dataclasses import dataclass

import numpy as np

from . import cluster
from .galerkin import Galerkin
from .gca import build_bases, green_factor_b, green_matrix, omega_rule


@dataclass
class GQ:
    tree: dict
    far: list
    near: list
    A: dict                  # tau -> |tau-hat| x 2k
    B: dict                  # (tau, sigma) -> |sigma-hat| x 2k
    N: dict
    n: int


def _rows(tree, c):
    return tree["perm"][tree["begin"][c]:tree["end"][c]]


def build_gq(vertices, triangles, params, tree=None):
    """Pure Green quadrature for the admissible blocks (Sect. 2)."""
    gal = Galerkin(vertices, triangles, params.sauter_q)
    if tree is None:
        tree = cluster.build_tree(vertices, triangles, params.leaf_size)
    lo, hi = cluster.cluster_boxes(vertices, triangles, tree)
    far, near = cluster.block_tree(tree, lo, hi, params.eta)
    diam = cluster.diameter(lo, hi)
    A, B, rules = {}, {}, {}
    for (t, s) in far:
        if t not in rules:
            rules[t] = omega_rule(lo[t], hi[t], diam[t], params.margin(), params.box_gauss_m)
            z, nrm, w = rules[t]
            A[t] = green_matrix(gal, _rows(tree, t), z, nrm, w, diam[t])
        z, nrm, w = rules[t]
        B[(t, s)] = green_factor_b(gal, _rows(tree, s), z, nrm, w, diam[t])
    N = {(t, s): gal.block(_rows(tree, t), _rows(tree, s)) for (t, s) in near}
    return GQ(tree, far, near, A, B, N, gal.n)


def gq_matvec(h, X, transpose=False):
    X = np.asarray(X, dtype=np.float64)
    vec = X.ndim == 1
    X = X[:, None] if vec else X
    Y = np.zeros_like(X)
    tree = h.tree
    for (t, s) in h.far:
        rt, rs = _rows(tree, t), _rows(tree, s)
        if transpose:
            Y[rs] += h.B[(t, s)] @ (h.A[t].T @ X[rt])
        else:
            Y[rt] += h.A[t] @ (h.B[(t, s)].T @ X[rs])
    for (t, s) in h.near:
        rt, rs = _rows(tree, t), _rows(tree, s)
        if transpose:
            Y[rs] += h.N[(t, s)].T @ X[rt]
        else:
            Y[rt] += h.N[(t, s)] @ X[rs]
    return Y[:, 0] if vec else Y


def gq_dense(h):
    G = np.zeros((h.n, h.n))
    tree = h.tree
    for (t, s) in h.far:
        G[np.ix_(_rows(tree, t), _rows(tree, s))] = h.A[t] @ h.B[(t, s)].T
    for (t, s) in h.near:
        G[np.ix_(_rows(tree, t), _rows(tree, s))] = h.N[(t, s)]
    return G


def gq_storage(h):
    a = sum(m.size for m in h.A.values())
    b = sum(m.size for m in h.B.values())
    nn = sum(m.size for m in h.N.values())
    return {"A": a, "B": b, "N": nn, "total": a + b + nn}


@dataclass
class GCA1:
    tree: dict
    bases: object            # gca.Bases with V_tau for every cluster in a block
    far: list
    near: list
    S: dict
    N: dict
    n: int


def build_gca1(vertices, triangles, params, tree=None):
    """Single-level Green cross approximation (Sect. 3)."""
    gal = Galerkin(vertices, triangles, params.sauter_q)
    if tree is None:
        tree = cluster.build_tree(vertices, triangles, params.leaf_size)
    lo, hi = cluster.cluster_boxes(vertices, triangles, tree)
    far, near = cluster.block_tree(tree, lo, hi, params.eta)
    bases = build_bases(gal, tree, lo, hi, params, far, nested=False)
    S = {(t, s): gal.block(bases.pivots[t], bases.pivots[s]) for (t, s) in far}
    N = {(t, s): gal.block(_rows(tree, t), _rows(tree, s)) for (t, s) in near}
    return GCA1(tree, bases, far, near, S, N, gal.n)


def gca1_matvec(h, X, transpose=False):
    X = np.asarray(X, dtype=np.float64)
    vec = X.ndim == 1
    X = X[:, None] if vec else X
    Y = np.zeros_like(X)
    tree = h.tree
    V = h.bases.V
    for (t, s) in h.far:
        rt, rs = _rows(tree, t), _rows(tree, s)
        if transpose:
            Y[rs] += V[s] @ (h.S[(t, s)].T @ (V[t].T @ X[rt]))
        else:
            Y[rt] += V[t] @ (h.S[(t, s)] @ (V[s].T @ X[rs]))
    for (t, s) in h.near:
        rt, rs = _rows(tree, t), _rows(tree, s)
        if transpose:
            Y[rs] += h.N[(t, s)].T @ X[rt]
        else:
            Y[rt] += h.N[(t, s)] @ X[rs]
    return Y[:, 0] if vec else Y


def gca1_dense(h):
    G = np.zeros((h.n, h.n))
    tree = h.tree
    V = h.bases.V
    for (t, s) in h.far:
        G[np.ix_(_rows(tree, t), _rows(tree, s))] = V[t] @ h.S[(t, s)] @ V[s].T
    for (t, s) in h.near:
        G[np.ix_(_rows(tree, t), _rows(tree, s))] = h.N[(t, s)]
    return G


def gca1_storage(h):
    inblock = {c for b in h.far for c in b}
    v = sum(h.bases.V[c].size for c in inblock)
    s = sum(m.size for m in h.S.values())
    nn = sum(m.size for m in h.N.values())
    return {"V": v, "S": s, "N": nn, "total": v + s + nn}
