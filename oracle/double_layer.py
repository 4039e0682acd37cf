"""Double-layer operator (oracle): Galerkin entries and its GCA-H^2.

TEST INFRASTRUCTURE ONLY (see the package header).

The boundary integral equation of Sect. 1 holds, beside the single-layer
kernel g, the double-layer kernel: the derivative of g(x, y) with respect to
y in the direction of the unit outer normal n_y,

    dg/dn_y(x, y) = <n_y, x - y> / (4 pi |x - y|^3)

(grad_y |x - y|^-1 = (x - y) / |x - y|^3).  Galerkin discretisation with the
piecewise constant basis of Eq. (1) gives

    k_ij = int_{T_i} int_{T_j} dg/dn_y(x, y) dy dx,

a non-symmetric matrix K.  On a flat triangle x - y lies in the plane of T_j,
so k_ii = 0; pairs with a common edge or vertex use the Sauter-Schwab
substitutions of ``sauter`` (Sect. 8) with this kernel, disjoint pairs the
7-point rule on both triangles.

GCA-H^2 of K (Sect. 2 - Sect. 4 applied to this kernel):

* rows: for y outside omega_tau, x -> dg/dn_y(x, y) is harmonic in omega_tau,
  so Green's representation formula in x separates it with the factors
  g(x, z_nu) and dg/dn_z(x, z_nu), those of the single layer: the row bases
  V_tau, E_tau and pivots tilde-tau are the single layer's (``gca``).
* columns: for x outside omega_sigma, y -> g(x, y) is harmonic in
  omega_sigma; applying <n_y, grad_y> to its representation formula gives
      dg/dn_y(x, y) = int_{d omega} dg/dn_y(y, z) dg/dn_z(x, z)
                                  - d2g/dn_y dn_z(y, z) g(x, z) dz,
  with d2g/dn_y dn_z(y, z) = (<n_y, n_z> / r^3 - 3 <n_y, d> <n_z, d> / r^5)
  / (4 pi), d = z - y, r = |d|.  Its y-factors, quadratured on the box rule,
  give the column Green matrix (``column_green_matrix``)
      a'_{j nu}     =          sqrt(w_nu) int dg/dn_y(y, z_nu)         phi_j(y) dy
      a'_{j, nu+k}  = -d_sigma sqrt(w_nu) int d2g/dn_y dn_z(y, z_nu)  phi_j(y) dy
  (d_sigma = diam(sigma) balances the two kinds of columns as d_tau does in
  Sect. 2); cross approximation of it, nested as in Sect. 4, gives the
  column pivots tilde-sigma', bases W_sigma and transfer matrices F.
* couplings K|tilde-tau x tilde-sigma', near field K|tau-hat x sigma-hat, and
      K|tau-hat x sigma-hat ~ V_tau K|tilde-tau x tilde-sigma' W_sigma^*.
* products: K x forwards x through the column bases, applies the couplings
  and returns through the row bases; K^T x the other way round.

Pinned by tests (tests/test_oracle_double_layer.py): k_ii = 0; Gauss's law
on the closed polyhedron (the solid angle of a face-interior point is half
the full angle, so sum_j k_ij = -|T_i| / 2) against a semi-analytic K; the
touching entries against the solid-angle closed form of the inner integral
with a graded outer rule; disjoint entries against refined product rules;
the column representation formula converging in m; the unit-sphere identity
dg/dn_y = -g / 2 (K + G / 2 shrinking under refinement); fast product =
explicit bases, the adjoint identity, and the spectral error of the H^2
approximation falling with the tolerance.
"""

from dataclasses import dataclass
from types import SimpleNamespace

import numpy as np

from . import cluster, h2, sauter
from .galerkin import FOUR_PI, order_pair, shared_vertices
from .gca import Bases, build_bases, omega_rule
from .galerkin import Galerkin
from .rules import triangle_points


def unit_normals(vertices, triangles):
    """Outer unit normal of every triangle, (b - a) x (c - a) normalised."""
    a = vertices[triangles[:, 0]]
    b = vertices[triangles[:, 1]]
    c = vertices[triangles[:, 2]]
    n = np.cross(b - a, c - a)
    return n / np.linalg.norm(n, axis=1)[:, None]


def dg_dny(x, y, ny):
    """dg/dn_y(x, y) = <n_y, x - y> / (4 pi |x - y|^3)."""
    d = x - y
    r2 = (d * d).sum(axis=-1)
    return (ny * d).sum(axis=-1) / (FOUR_PI * r2 * np.sqrt(r2))


def d2g_dny_dnz(y, z, ny, nz):
    """d2g/dn_y dn_z(y, z) = (<n_y, n_z> / r^3 - 3 <n_y, d> <n_z, d> / r^5) / (4 pi), d = z - y."""
    d = z - y
    r2 = (d * d).sum(axis=-1)
    r = np.sqrt(r2)
    a = (ny * d).sum(axis=-1)
    b = (nz * d).sum(axis=-1)
    nn = (ny * nz).sum(axis=-1)
    return (nn / (r2 * r) - 3.0 * a * b / (r2 * r2 * r)) / FOUR_PI


class DoubleLayer:
    """Galerkin entries k_ij of the double-layer kernel on one mesh."""

    def __init__(self, vertices, triangles, sauter_q=5):
        self.v = np.asarray(vertices, dtype=np.float64)
        self.t = np.asarray(triangles, dtype=np.int64)
        self.q = int(sauter_q)
        self.pts, self.wts = triangle_points(self.v, self.t)
        self.nrm = unit_normals(self.v, self.t)

    @property
    def n(self):
        return self.t.shape[0]

    def regular(self, i, j):
        """7 x 7 point rule for disjoint pairs."""
        x = self.pts[i][:, :, None, :]
        y = self.pts[j][:, None, :, :]
        ny = self.nrm[j][:, None, None, :]
        w = self.wts[i][:, :, None] * self.wts[j][:, None, :]
        return (w * dg_dny(x, y, ny)).sum(axis=(1, 2))

    def singular(self, i, j, case):
        """Sauter-Schwab rules for a common vertex (1) or edge (2); 0 for
        identical flat triangles (3)."""
        if case == 3:
            return np.zeros(len(i))
        P = np.empty((len(i), 3, 3))
        Q = np.empty((len(i), 3, 3))
        for m, (a, b) in enumerate(zip(i, j)):
            oi, oj = order_pair(self.t[a], self.t[b], case)
            P[m] = self.v[oi]
            Q[m] = self.v[oj]
        ny = self.nrm[np.asarray(j)]
        out = np.empty(len(i))
        chunk = 256
        for s in range(0, len(i), chunk):
            n_s = ny[s:s + chunk]
            kern = lambda x, y, n_s=n_s: dg_dny(x, y, n_s[:, None, :])  # noqa: E731
            out[s:s + chunk] = sauter.integrate(case, P[s:s + chunk], Q[s:s + chunk], kern, self.q)
        return out

    def entries(self, i, j, chunk=1 << 16):
        """k_ij for index arrays i, j."""
        i = np.asarray(i, dtype=np.int64).ravel()
        j = np.asarray(j, dtype=np.int64).ravel()
        out = np.empty(len(i))
        for s in range(0, len(i), chunk):
            ii = i[s:s + chunk]
            jj = j[s:s + chunk]
            case = shared_vertices(self.t, ii, jj)
            res = np.empty(len(ii))
            reg = case == 0
            if reg.any():
                res[reg] = self.regular(ii[reg], jj[reg])
            for c in (1, 2, 3):
                sel = case == c
                if sel.any():
                    res[sel] = self.singular(ii[sel], jj[sel], c)
            out[s:s + chunk] = res
        return out

    def block(self, rows, cols):
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        ii = np.repeat(rows, len(cols))
        jj = np.tile(cols, len(rows))
        return self.entries(ii, jj).reshape(len(rows), len(cols))

    def dense_matrix(self):
        idx = np.arange(self.n)
        return self.block(idx, idx)


def column_green_matrix(dl, cols, z, nrm, w, d_sigma):
    """The column Green matrix of the double layer on the triangles `cols`
    (len(cols) x 2k), from the y-factors of the differentiated
    representation formula (module header)."""
    y = dl.pts[cols]                 # (c, 7, 3)
    wy = dl.wts[cols]                # (c, 7)
    ny = dl.nrm[cols][:, None, :]    # (c, 1, 3)
    sw = np.sqrt(w)
    k = z.shape[0]
    A = np.empty((len(cols), 2 * k))
    for nu in range(k):
        zz = z[nu][None, None, :]
        nz = nrm[nu][None, None, :]
        A[:, nu] = sw[nu] * (wy * dg_dny(zz, y, ny)).sum(axis=1)
        A[:, nu + k] = -d_sigma * sw[nu] * (wy * d2g_dny_dnz(y, zz, ny, nz)).sum(axis=1)
    return A


@dataclass
class DLH2:
    tree: dict
    rows: Bases                    # row bases (the single layer's)
    cols: Bases                    # column bases of the double layer
    far: list
    near: list
    S: dict                        # (tau, sigma) -> r_tau x r'_sigma
    N: dict                        # (tau, sigma) -> |tau-hat| x |sigma-hat|
    n: int


def build_dl_h2(vertices, triangles, params, tree=None):
    """The GCA-H^2 construction of the double-layer matrix K on one mesh."""
    gal = Galerkin(vertices, triangles, params.sauter_q)
    dl = DoubleLayer(vertices, triangles, params.sauter_q)
    if tree is None:
        tree = cluster.build_tree(vertices, triangles, params.leaf_size)
    lo, hi = cluster.cluster_boxes(vertices, triangles, tree)
    far, near = cluster.block_tree(tree, lo, hi, params.eta)
    rows = build_bases(gal, tree, lo, hi, params, far)
    cols = build_bases(dl, tree, lo, hi, params, far, green=column_green_matrix)
    S = {(t, s): dl.block(rows.pivots[t], cols.pivots[s]) for (t, s) in far}
    perm = tree["perm"]
    N = {(t, s): dl.block(perm[tree["begin"][t]:tree["end"][t]], perm[tree["begin"][s]:tree["end"][s]])
         for (t, s) in near}
    return DLH2(tree, rows, cols, far, near, S, N, dl.n)


def _side(h, bases):
    return SimpleNamespace(tree=h.tree, bases=bases)


def matvec(h, X, transpose=False):
    """Fast product K_H2 x (or K_H2^T x): forward transform through the
    column bases (row bases for the transpose), couplings, backward
    transform through the row bases (column bases), near field."""
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
    """The represented matrix: V_tau S W_sigma^T on the far blocks, N near."""
    Vr = h2.explicit_bases(_side(h, h.rows))
    Wc = h2.explicit_bases(_side(h, h.cols))
    tree = h.tree
    K = np.zeros((h.n, h.n))
    for (t, s) in h.far:
        rt = tree["perm"][tree["begin"][t]:tree["end"][t]]
        rs = tree["perm"][tree["begin"][s]:tree["end"][s]]
        K[np.ix_(rt, rs)] = Vr[t] @ h.S[(t, s)] @ Wc[s].T
    for (t, s) in h.near:
        rt = tree["perm"][tree["begin"][t]:tree["end"][t]]
        rs = tree["perm"][tree["begin"][s]:tree["end"][s]]
        K[np.ix_(rt, rs)] = h.N[(t, s)]
    return K
