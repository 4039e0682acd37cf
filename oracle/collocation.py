"""Collocation variant (oracle): the single-layer operator discretised by
collocation instead of Galerkin's method, and its GCA-H^2.

TEST INFRASTRUCTURE ONLY (see the package header).

Sect. 6 replaces the double integral of Eq. (1) by a single one,

    c_ij = int g(x_i, y) phi_j(y) dy,

with collocation points x_i, and regularises the one singular case (y at
x_i) by a Duffy transformation.  The paper pairs vertices with nodal linear
functions; with the piecewise constant basis used throughout here the
collocation point of row i is the centroid of triangle i (the point of the
7-point rule's centre), the reading of this module:

* ``entries``: disjoint and touching pairs j != i by the 7-point rule on T_j;
  j = i by the Duffy transformation around x_i: T_i splits into the three
  triangles (x_i, P_k, P_k+1); on each, y = x_i + s ((1 - t) P_k + t P_k+1
  - x_i) has Jacobian s |(P_k - x_i) x (P_k+1 - x_i)| and |x_i - y| = s rho(t),
  so the integrand J / rho(t) does not depend on s: the s-integral is 1 and
  t takes a Gauss-Legendre rule of 4 q points (q = sauter_q; 1 / rho(t) is
  analytic on [0, 1], with complex singularities at a distance of about
  the inradius over the edge length, so the rule converges geometrically).
* GCA-H^2 (Sect. 2 - Sect. 4): rows: for y outside omega_tau the function
  x -> g(x, y) is harmonic, so Green's formula separates it with the factors
  g(x_i, z_nu) and dg/dn_z(x_i, z_nu) evaluated at the collocation points:
      a_{i nu} = sqrt(w_nu) g(x_i, z_nu),  a_{i nu+k} = -d_tau sqrt(w_nu) dg/dn_z(x_i, z_nu),
  cross-approximated and nested into the row bases; columns: the y-factors
  are the integrals against phi_j of the Galerkin single layer, so the
  column bases are the Galerkin ones (``gca``); couplings C|tilde-tau x
  tilde-sigma, near field C|tau-hat x sigma-hat; C x forwards x through the
  column bases and returns through the row bases.

Pinned by tests (tests/test_oracle_collocation.py): the Duffy value against
the closed-form potential of a flat triangle; the unit-density potential on
the unit sphere (sum_j c_ij -> 1 at O(h^2)); the collocation Green matrix
reproducing Green's formula; fast product = explicit bases; the spectral
error falling with the tolerance.
"""

from dataclasses import dataclass
from types import SimpleNamespace

import numpy as np

from . import cluster, h2
from .galerkin import FOUR_PI, Galerkin, dg_dn, g
from .gca import Bases, build_bases
from .rules import gauss_legendre_01, triangle_points


class Collocation:
    """Entries c_ij of the collocated single layer on one mesh."""

    def __init__(self, vertices, triangles, q=5):
        self.v = np.asarray(vertices, dtype=np.float64)
        self.t = np.asarray(triangles, dtype=np.int64)
        self.q = int(q)
        self.pts, self.wts = triangle_points(self.v, self.t)
        self.xc = self.pts[:, 0, :]     # the 7-point rule's centre: the centroid

    @property
    def n(self):
        return self.t.shape[0]

    def regular(self, i, j):
        """7-point rule on T_j for the point x_i."""
        x = self.xc[i][:, None, :]
        return (self.wts[j] * g(x, self.pts[j])).sum(axis=1)

    def duffy(self, i):
        """c_ii by the Duffy transformation around the centroid."""
        t, w = gauss_legendre_01(4 * self.q)
        out = np.zeros(len(i))
        for m, a in enumerate(i):
            P = self.v[self.t[a]]
            x = self.xc[a]
            for k in range(3):
                A, B = P[k], P[(k + 1) % 3]
                jac = np.linalg.norm(np.cross(A - x, B - x))
                e = (1.0 - t)[:, None] * A + t[:, None] * B - x
                out[m] += jac * np.sum(w / np.linalg.norm(e, axis=1))
        return out / FOUR_PI

    def entries(self, i, j, chunk=1 << 16):
        i = np.asarray(i, dtype=np.int64).ravel()
        j = np.asarray(j, dtype=np.int64).ravel()
        out = np.empty(len(i))
        for s in range(0, len(i), chunk):
            ii, jj = i[s:s + chunk], j[s:s + chunk]
            res = np.empty(len(ii))
            same = ii == jj
            if (~same).any():
                res[~same] = self.regular(ii[~same], jj[~same])
            if same.any():
                res[same] = self.duffy(ii[same])
            out[s:s + chunk] = res
        return out

    def block(self, rows, cols):
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        return self.entries(np.repeat(rows, len(cols)), np.tile(cols, len(rows))).reshape(len(rows), len(cols))

    def dense_matrix(self):
        idx = np.arange(self.n)
        return self.block(idx, idx)


def collocation_green_matrix(col, rows, z, nrm, w, d_tau):
    """The rows' Green quadrature matrix at the collocation points (len(rows) x 2k)."""
    x = col.xc[rows][:, None, :]     # (r, 1, 3)
    sw = np.sqrt(w)
    k = z.shape[0]
    A = np.empty((len(rows), 2 * k))
    A[:, :k] = sw[None, :] * g(x, z[None, :, :])
    A[:, k:] = -d_tau * sw[None, :] * dg_dn(x, z[None, :, :], nrm[None, :, :])
    return A


@dataclass
class ColH2:
    tree: dict
    rows: Bases                    # collocation row bases
    cols: Bases                    # the Galerkin single layer's bases
    far: list
    near: list
    S: dict                        # (tau, sigma) -> r_tau x r'_sigma
    N: dict
    n: int


def build_col_h2(vertices, triangles, params, tree=None):
    """The GCA-H^2 construction of the collocation matrix C on one mesh."""
    gal = Galerkin(vertices, triangles, params.sauter_q)
    col = Collocation(vertices, triangles, params.sauter_q)
    if tree is None:
        tree = cluster.build_tree(vertices, triangles, params.leaf_size)
    lo, hi = cluster.cluster_boxes(vertices, triangles, tree)
    far, near = cluster.block_tree(tree, lo, hi, params.eta)
    rows = build_bases(col, tree, lo, hi, params, far, green=collocation_green_matrix)
    cols = build_bases(gal, tree, lo, hi, params, far)
    S = {(t, s): col.block(rows.pivots[t], cols.pivots[s]) for (t, s) in far}
    perm = tree["perm"]
    N = {(t, s): col.block(perm[tree["begin"][t]:tree["end"][t]], perm[tree["begin"][s]:tree["end"][s]])
         for (t, s) in near}
    return ColH2(tree, rows, cols, far, near, S, N, col.n)


def _side(h, bases):
    return SimpleNamespace(tree=h.tree, bases=bases)


def matvec(h, X, transpose=False):
    """C_H2 x (or C_H2^T x): column bases forward, couplings, row bases back."""
    X, vec = h2._as2d(X)
    src, dst = (h.rows, h.cols) if transpose else (h.cols, h.rows)
    xh = h2.forward(_side(h, src), X)
    R = X.shape[1]
    yh = {c: np.zeros((dst.rank[c], R)) for c in xh}
    for (t, s) in h.far:
        if transpose:
            yh[s] += h.S[(t, s)].T @ xh[t]
        else:
            yh[t] += h.S[(t, s)] @ xh[s]
    Y = np.zeros_like(X)
    h2.backward(_side(h, dst), yh, Y)
    tree = h.tree
    for (t, s) in h.near:
        rt = tree["perm"][tree["begin"][t]:tree["end"][t]]
        rs = tree["perm"][tree["begin"][s]:tree["end"][s]]
        if transpose:
            Y[rs] += h.N[(t, s)].T @ X[rt]
        else:
            Y[rt] += h.N[(t, s)] @ X[rs]
    return Y[:, 0] if vec else Y


def matvec_t(h, X):
    return matvec(h, X, transpose=True)


def dense(h):
    Vr = h2.explicit_bases(_side(h, h.rows))
    Wc = h2.explicit_bases(_side(h, h.cols))
    tree = h.tree
    C = np.zeros((h.n, h.n))
    for (t, s) in h.far:
        rt = tree["perm"][tree["begin"][t]:tree["end"][t]]
        rs = tree["perm"][tree["begin"][s]:tree["end"][s]]
        C[np.ix_(rt, rs)] = Vr[t] @ h.S[(t, s)] @ Wc[s].T
    for (t, s) in h.near:
        rt = tree["perm"][tree["begin"][t]:tree["end"][t]]
        rs = tree["perm"][tree["begin"][s]:tree["end"][s]]
        C[np.ix_(rt, rs)] = h.N[(t, s)]
    return C
