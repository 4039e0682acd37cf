"""Curved triangles for the nodal basis (oracle; test infrastructure).

Sect. 6 replaces the flat parametrisation of every triangle by a quadratic
one: Phi_t maps the reference triangle onto the curved triangle t by
interpolating its three vertices and three surface points at the midpoints
of its edges.  The basis functions are mapped nodal ones (phi_i o Phi_t is
linear on the reference triangle, i.e. a barycentric coordinate), and every
integral over t picks up the Gramian gamma_t = |d1 Phi_t x d2 Phi_t|:

    int_t phi_i int_s g phi_j
        = int_ref gamma_t lambda_a int_ref g(Phi_t(x), Phi_s(y)) gamma_s lambda_b dy dx.

Pieces (the reference coordinates are the barycentric lambda_0..2, with
x^ = (lambda_1, lambda_2)):

* ``shape``: the six quadratic Lagrange functions lambda_a (2 lambda_a - 1)
  (vertices) and 4 lambda_a lambda_b (edge midpoints), and their
  derivatives by lambda;
* ``quadratic_map``, ``gramian``: Phi(lambda) and |d1 Phi x d2 Phi| from the
  derivative of the map; ``gramian_interpolated``: the same from the normal
  n = d1 Phi x d2 Phi interpolated through its values at the six nodes (the
  recipe of Sect. 6: n is a quadratic polynomial);
* ``curved_points``: the 7-point rule on every curved triangle (nodes
  Phi(lambda_q), weights w_q gamma(lambda_q) / 2);
* ``local_singular_curved``: touching pairs by the Sauter-Schwab maps of
  ``sauter`` on the reference coordinates (u1, u2) -> lambda = (1 - u1,
  u1 - u2, u2) in the vertex order of ``galerkin.order_pair``; the map is
  not affine, so all four variables (xi included) are sampled by the
  q-point Gauss rule;
* ``P1CurvedGalerkin``, ``cluster_boxes_curved``, ``build_p1c_h2``: the
  nodal Galerkin matrix and its GCA-H^2 (Sect. 2-5) on curved triangles.

Pinned by tests: flat midpoints reproduce the flat nodal matrix, the
interpolated Gramian equals the derivative one, the area of the curved
sphere converges at fourth order (second for flat triangles), the
constant-density identity on the unit sphere, symmetry and positive
definiteness, convergence of the singular rules in q, and the H^2
product against the dense matrix.
"""

import numpy as np

from . import cluster, sauter
from .galerkin import FOUR_PI, order_pair
from .gca import H2, build_bases
from .p1 import P1Galerkin, build_tree_points, green_matrix_p1, shared
from .rules import RADON7

# stored node order of a curved triangle: vertices 0, 1, 2, then the
# midpoints of the edges (0, 1), (1, 2), (2, 0)
_EDGE_NODE = {(0, 1): 3, (1, 0): 3, (1, 2): 4, (2, 1): 4, (0, 2): 5, (2, 0): 5}


def shape(lam):
    """Quadratic Lagrange functions N (..., 6) and dN/dlambda (..., 6, 3)."""
    lam = np.asarray(lam, dtype=np.float64)
    l0, l1, l2 = lam[..., 0], lam[..., 1], lam[..., 2]
    N = np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                  4 * l0 * l1, 4 * l1 * l2, 4 * l2 * l0], axis=-1)
    z = np.zeros_like(l0)
    dN = np.stack([
        np.stack([4 * l0 - 1, z, z], axis=-1),
        np.stack([z, 4 * l1 - 1, z], axis=-1),
        np.stack([z, z, 4 * l2 - 1], axis=-1),
        np.stack([4 * l1, 4 * l0, z], axis=-1),
        np.stack([z, 4 * l2, 4 * l1], axis=-1),
        np.stack([4 * l2, z, 4 * l0], axis=-1),
    ], axis=-2)
    return N, dN


def quadratic_map(X6, lam):
    """Phi(lambda) for nodes X6 (..., 6, 3) at lambda (..., 3)."""
    N, _ = shape(lam)
    return np.einsum("...k,...kd->...d", N, X6)


def tangents(X6, lam):
    """d Phi / d x^_1 and d Phi / d x^_2 (x^ = (lambda_1, lambda_2), lambda_0 = 1 - x^_1 - x^_2)."""
    _, dN = shape(lam)
    d1 = dN[..., 1] - dN[..., 0]
    d2 = dN[..., 2] - dN[..., 0]
    return np.einsum("...k,...kd->...d", d1, X6), np.einsum("...k,...kd->...d", d2, X6)


def gramian(X6, lam):
    t1, t2 = tangents(X6, lam)
    n = np.cross(t1, t2)
    return np.sqrt((n * n).sum(axis=-1))


def gramian_interpolated(X6, lam):
    """The Gramian from the normal interpolated through the six nodes."""
    nodes = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [.5, .5, 0], [0, .5, .5], [.5, 0, .5]])
    X6 = np.asarray(X6, dtype=np.float64)
    t1, t2 = tangents(X6[..., None, :, :], nodes)
    n_nodes = np.cross(t1, t2)                       # (..., 6, 3)
    N, _ = shape(lam)
    n = np.einsum("...k,...kd->...d", N, n_nodes)
    return np.sqrt((n * n).sum(axis=-1))


def curved_nodes(vertices, triangles, midpoints):
    """X6 per triangle: (nt, 6, 3)."""
    v = np.asarray(vertices, dtype=np.float64)
    t = np.asarray(triangles, dtype=np.int64)
    m = np.asarray(midpoints, dtype=np.float64).reshape(-1, 3, 3)
    return np.concatenate([v[t], m], axis=1)


def curved_points(X6, rule=RADON7):
    """7-point rule on curved triangles: points (nt, 7, 3), weights (nt, 7)."""
    bary, wts = rule
    pts = quadratic_map(X6[:, None, :, :], bary[None, :, :])
    gam = gramian(X6[:, None, :, :], bary[None, :, :])
    return pts, wts[None, :] * gam * 0.5


def ordered_nodes(X6, tri, order):
    """Nodes of a triangle in the vertex order `order` (vertex ids): the
    ordered vertices, then the midpoints of the ordered edges (0, 1),
    (1, 2), (2, 0); with the stored corner of each ordered vertex."""
    c = [list(tri).index(a) for a in order]
    idx = [c[0], c[1], c[2], _EDGE_NODE[(c[0], c[1])], _EDGE_NODE[(c[1], c[2])], _EDGE_NODE[(c[2], c[0])]]
    return X6[idx], c


def local_singular_curved(X6, tri_t, tri_s, Xt, Xs, case, q):
    """3 x 3 matrix of one touching pair of curved triangles (Sauter-Schwab,
    order q in all four variables); Xt, Xs are the pair's stored nodes."""
    oi, oj = order_pair(tri_t, tri_s, case)
    P, ci = ordered_nodes(Xt, tri_t, oi)
    Q, cj = ordered_nodes(Xs, tri_s, oj)
    xi, e1, e2, e3, wt = sauter.cube_rule(q)
    acc = np.zeros((3, 3))
    for (u1, u2), (v1, v2), w in sauter.sub_maps(case, xi, e1, e2, e3):
        lu = np.stack([1.0 - u1, u1 - u2, u2], axis=-1)      # (s, 3)
        lv = np.stack([1.0 - v1, v1 - v2, v2], axis=-1)
        x = quadratic_map(P, lu)
        y = quadratic_map(Q, lv)
        d = x - y
        kv = wt * w * gramian(P, lu) * gramian(Q, lv) / np.sqrt((d * d).sum(axis=1))
        acc += (lu * kv[:, None]).T @ lv
    out = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            out[ci[a], cj[b]] = acc[a, b]
    return out / FOUR_PI


class P1CurvedGalerkin(P1Galerkin):
    """Galerkin entries of the single-layer matrix in the mapped nodal basis
    on curved triangles."""

    def __init__(self, vertices, triangles, midpoints, sauter_q=5):
        super().__init__(vertices, triangles, sauter_q)
        self.X6 = curved_nodes(vertices, triangles, midpoints)
        self.pts, self.wts = curved_points(self.X6)

    def regular_pairs(self, ti, si):
        bary, _ = RADON7
        xp, wx = self.pts[ti], self.wts[ti]
        yp, wy = self.pts[si], self.wts[si]
        d = xp[:, :, None, :] - yp[:, None, :, :]
        kw = wx[:, :, None] / np.sqrt((d * d).sum(axis=-1)) * wy[:, None, :]
        return np.einsum("pa,mpq,qb->mab", bary, kw, bary) / FOUR_PI

    def pair(self, ti, si):
        key = (ti, si)
        if key not in self._pair:
            a, b = self.t[ti], self.t[si]
            c = shared(a, b)
            if c == 0:
                self._pair[key] = self.regular_pairs(np.array([ti]), np.array([si]))[0]
            else:
                self._pair[key] = local_singular_curved(self.X6, a, b, self.X6[ti], self.X6[si], c, self.q)
        return self._pair[key]


def cluster_boxes_curved(gal, tree):
    """Box of a cluster: the bounding box of the six nodes of every curved
    triangle in the supports of its basis functions."""
    ptr, tri, _ = gal.supports
    nc = len(tree["begin"])
    lo = np.empty((nc, 3))
    hi = np.empty((nc, 3))
    for c in range(nc):
        idx = tree["perm"][tree["begin"][c]:tree["end"][c]]
        ts = np.concatenate([tri[ptr[i]:ptr[i + 1]] for i in idx])
        pts = gal.X6[ts].reshape(-1, 3)
        lo[c] = pts.min(axis=0)
        hi[c] = pts.max(axis=0)
    return lo, hi


def build_p1c_h2(vertices, triangles, midpoints, params, tree=None, follow=None):
    """GCA-H^2 of the single-layer matrix in the mapped nodal basis on
    curved triangles (``follow`` as in ``p1.build_p1_h2``)."""
    gal = P1CurvedGalerkin(vertices, triangles, midpoints, params.sauter_q)
    if tree is None:
        tree = build_tree_points(vertices, params.leaf_size)
    lo, hi = cluster_boxes_curved(gal, tree)
    far, near = cluster.block_tree(tree, lo, hi, params.eta)
    bases = build_bases(gal, tree, lo, hi, params, far, green=green_matrix_p1, follow=follow)
    S = {}
    for (t, s) in far:
        S[(t, s)] = gal.block(bases.pivots[t], bases.pivots[s])
    N = {}
    perm = tree["perm"]
    for (t, s) in near:
        N[(t, s)] = gal.block(perm[tree["begin"][t]:tree["end"][t]],
                              perm[tree["begin"][s]:tree["end"][s]])
    return H2(tree, bases, far, near, S, N, gal.n, lo, hi)
