"""Kernel function and Galerkin entries (oracle).

* ``g(x, y) = 1 / (4 pi |x - y|)``, the fundamental solution of Laplace's
  equation (Sect. 1).
* ``dg_dn(x, z, n) = <n, x - z> / (4 pi |x - z|^3)``: the derivative of
  g(x, z) with respect to z in direction n, as it appears in Green's
  representation formula (Sect. 2).  The paper uses it without a formula;
  it follows from grad_z |x - z|^-1 = (x - z) / |x - z|^3.  The same
  function gives dg/dn_z(z, y) = dg_dn(y, z, n).
* ``entries(i, j)``: Galerkin entries g_ij of Eq. (1) for piecewise
  constant basis functions (the indicator of triangle i, Sect. 2).  Pairs
  are classified by the number of shared vertex ids (Sect. 8): 3 identical,
  2 common edge, 1 common vertex (Sauter-Schwab, ``sauter``), 0 disjoint
  (7-point rule on both triangles, 49 kernel evaluations).
* ``dense_matrix``: the full G for small n.

Pinned by tests: symmetry, positive definiteness, the single-layer potential
of unit density on the unit sphere (row sums of G approach the triangle
areas at O(h^2)), and the l = 1 spherical-harmonic eigenvalue 1/3.
"""

import numpy as np

from . import sauter
from .rules import triangle_points

FOUR_PI = 4.0 * np.pi


def g(x, y):
    d = x - y
    return 1.0 / (FOUR_PI * np.sqrt((d * d).sum(axis=-1)))


def dg_dn(x, z, n):
    d = x - z
    r2 = (d * d).sum(axis=-1)
    return (n * d).sum(axis=-1) / (FOUR_PI * r2 * np.sqrt(r2))


def inv_dist(x, y):
    d = x - y
    return 1.0 / np.sqrt((d * d).sum(axis=-1))


def shared_vertices(triangles, i, j):
    """Number of vertex ids shared by triangles i and j (arrays)."""
    ti = triangles[i]
    tj = triangles[j]
    return (ti[:, :, None] == tj[:, None, :]).sum(axis=(1, 2))


def order_pair(ti, tj, case):
    """Vertex orders of a touching pair for the Sauter-Schwab maps.

    identical: both in stored order.  Common edge: (s1, s2, other) with
    s1, s2 the shared ids in the order they occur in ti.  Common vertex:
    the shared id first, then the remaining two in cyclic order.
    """
    ti = [int(a) for a in ti]
    tj = [int(a) for a in tj]
    if case == 3:
        return ti, list(ti)
    if case == 2:
        s = [a for a in ti if a in tj]
        oi = [a for a in ti if a not in s][0]
        oj = [a for a in tj if a not in s][0]
        return [s[0], s[1], oi], [s[0], s[1], oj]
    if case == 1:
        s = [a for a in ti if a in tj][0]
        pi = ti.index(s)
        pj = tj.index(s)
        return ([ti[pi], ti[(pi + 1) % 3], ti[(pi + 2) % 3]],
                [tj[pj], tj[(pj + 1) % 3], tj[(pj + 2) % 3]])
    raise ValueError(case)


class Galerkin:
    """Galerkin entries of the single-layer matrix on one mesh."""

    def __init__(self, vertices, triangles, sauter_q=5):
        self.v = np.asarray(vertices, dtype=np.float64)
        self.t = np.asarray(triangles, dtype=np.int64)
        self.q = int(sauter_q)
        self.pts, self.wts = triangle_points(self.v, self.t)

    @property
    def n(self):
        return self.t.shape[0]

    def regular(self, i, j):
        """7 x 7 point rule for disjoint pairs (49 kernel evaluations)."""
        x = self.pts[i]
        y = self.pts[j]
        d = x[:, :, None, :] - y[:, None, :, :]
        r = np.sqrt((d * d).sum(axis=-1))
        w = self.wts[i][:, :, None] * self.wts[j][:, None, :]
        return (w / r).sum(axis=(1, 2)) / FOUR_PI

    def singular(self, i, j, case):
        P = np.empty((len(i), 3, 3))
        Q = np.empty((len(i), 3, 3))
        for m, (a, b) in enumerate(zip(i, j)):
            oi, oj = order_pair(self.t[a], self.t[b], case)
            P[m] = self.v[oi]
            Q[m] = self.v[oj]
        out = np.empty(len(i))
        chunk = 256
        for s in range(0, len(i), chunk):
            out[s:s + chunk] = sauter.integrate(case, P[s:s + chunk], Q[s:s + chunk],
                                                inv_dist, self.q)
        return out / FOUR_PI

    def entries(self, i, j, chunk=1 << 16):
        """g_ij for index arrays i, j (Eq. (1), piecewise constant basis)."""
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
        """G restricted to rows x cols (triangle ids)."""
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        ii = np.repeat(rows, len(cols))
        jj = np.tile(cols, len(rows))
        return self.entries(ii, jj).reshape(len(rows), len(cols))

    def dense_matrix(self):
        idx = np.arange(self.n)
        return self.block(idx, idx)
