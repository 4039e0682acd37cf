"""Continuous piecewise linear basis functions (oracle; test infrastructure).

Sect. 5 replaces the piecewise constant basis by the nodal basis phi_i of
the vertices: phi_i is continuous, linear on every triangle, 1 in vertex i
and 0 in all other vertices, so its support is the set T_i of triangles
around vertex i and

    g_ij = sum_{t in T_i} sum_{s in T_j} int_t phi_i(x) int_s g(x, y) phi_j(y) dy dx.

Pieces, in the order of that section:

* ``vertex_supports``: T_i for every vertex, triangles in ascending order,
  with the corner (0, 1, 2) at which vertex i sits in each.
* ``support_union``: the union of the T_i over a list of vertices
  tau-hat = (i_0, i_1, ...), each triangle once, with the local number of
  each of its three corners (-1 where the corner is not in tau-hat).  This
  is the mergesort of Sect. 5: every vertex contributes a list of rows
  (triangle, three local numbers, its own number at its corner), the lists
  are merged pairwise until one is left, and two rows of the same triangle
  meeting in a merge are combined corner by corner.
* ``local_regular`` / ``local_singular``: the 3 x 3 matrix of one triangle
  pair, M[a, b] = int_t lambda_a(x) int_s g(x, y) lambda_b(y) dy dx with
  lambda_a the barycentric coordinates (the restrictions of the basis
  functions of the corners).  Disjoint pairs use the 7-point rule on both
  triangles (49 kernel evaluations shared by all nine entries: the
  pair-by-pair assembly of Sect. 5); touching pairs the Sauter-Schwab rules
  of ``sauter`` with the barycentric weights of both sample points.
* ``P1Galerkin.block``: G restricted to vertex lists rows x cols, assembled
  pair by pair over the two support unions.
* ``green_matrix_p1``: the Green quadrature matrix A_tau of Sect. 2 for
  nodal rows, a_{i nu} = sqrt(w_nu) int g(x, z_nu) phi_i(x) dx and
  a_{i, nu+k} = -d_tau sqrt(w_nu) int dg/dn_z(x, z_nu) phi_i(x) dx.
* ``build_p1_h2``: the GCA-H^2 construction of ``gca`` with vertices as
  indices: a cluster tree over the vertex positions, cluster boxes that
  contain the supports of their basis functions (Sect. 2), nested bases,
  couplings G|tilde-tau x tilde-sigma and near-field blocks.

Pinned by tests: the worked example of the support union in Sect. 5
(``tests/golden/p1_support_union.txt``), the union against a brute-force
set union, the 3 x 3 matrices against the piecewise constant entries (the
barycentric coordinates sum to one) and against brute-force subdivision,
symmetry and positive definiteness of the dense matrix, the unit-sphere
identity for a constant density (sum_j g_ij -> int phi_i = |T_i| / 3) and
the first spherical harmonic, and the H^2 product against the dense matrix.
"""

import numpy as np

from . import cluster, sauter
from .galerkin import FOUR_PI, dg_dn, g, order_pair
from .gca import H2, aca, build_bases, omega_rule  # noqa: F401  (aca re-exported for tests)
from .rules import RADON7, triangle_areas, triangle_points


def vertex_supports(nv, triangles):
    """CSR of the supports: for vertex i, ptr[i]..ptr[i+1] index tri (the
    triangles containing i, ascending) and corner (the position of i in
    each)."""
    t = np.asarray(triangles, dtype=np.int64)
    cnt = np.zeros(nv + 1, dtype=np.int64)
    for c in range(3):
        np.add.at(cnt, t[:, c] + 1, 1)
    ptr = np.cumsum(cnt)
    tri = np.empty(ptr[-1], dtype=np.int64)
    corner = np.empty(ptr[-1], dtype=np.int64)
    fill = ptr[:-1].copy()
    for k in range(t.shape[0]):          # triangles in ascending order
        for c in range(3):
            i = t[k, c]
            tri[fill[i]] = k
            corner[fill[i]] = c
            fill[i] += 1
    return ptr, tri, corner


def _merge(a, b):
    """Merge two row lists sorted by triangle, combining equal triangles."""
    out = []
    i = j = 0
    while i < len(a) and j < len(b):
        ta, tb = a[i][0], b[j][0]
        if ta < tb:
            out.append(a[i])
            i += 1
        elif tb < ta:
            out.append(b[j])
            j += 1
        else:
            loc = tuple(x if x >= 0 else y for x, y in zip(a[i][1], b[j][1]))
            out.append((ta, loc))
            i += 1
            j += 1
    out.extend(a[i:])
    out.extend(b[j:])
    return out


def support_union(supports, tau):
    """Rows (triangle, (l0, l1, l2)) of the union of the supports of the
    vertices tau (local numbers 0, 1, ... in the order of tau; -1 marks a
    corner outside tau), ascending by triangle (Sect. 5)."""
    ptr, tri, corner = supports
    lists = []
    for a, i in enumerate(tau):
        rows = []
        for k in range(ptr[i], ptr[i + 1]):
            loc = [-1, -1, -1]
            loc[corner[k]] = a
            rows.append((int(tri[k]), tuple(loc)))
        lists.append(rows)
    if not lists:
        return []
    while len(lists) > 1:
        nxt = []
        for k in range(0, len(lists) - 1, 2):
            nxt.append(_merge(lists[k], lists[k + 1]))
        if len(lists) % 2:
            nxt.append(lists[-1])
        lists = nxt
    return lists[0]


def local_regular(v, tri_t, tri_s):
    """3 x 3 matrices of disjoint triangle pairs (7-point rule on both).

    tri_t, tri_s: (m, 3) vertex ids.  Returns (m, 3, 3)."""
    bary, wts = RADON7
    v = np.asarray(v, dtype=np.float64)
    tt = np.asarray(tri_t, dtype=np.int64).reshape(-1, 3)
    ss = np.asarray(tri_s, dtype=np.int64).reshape(-1, 3)
    xp, wx = triangle_points(v, tt)      # (m, 7, 3), (m, 7)
    yp, wy = triangle_points(v, ss)
    d = xp[:, :, None, :] - yp[:, None, :, :]
    k = 1.0 / np.sqrt((d * d).sum(axis=-1))          # (m, 7, 7)
    kw = wx[:, :, None] * k * wy[:, None, :]
    return np.einsum("pa,mpq,qb->mab", bary, kw, bary) / FOUR_PI


def local_singular(v, tri_t, tri_s, case, q):
    """3 x 3 matrices of touching triangle pairs (Sauter-Schwab, order q).

    ``case``: 3 identical, 2 common edge, 1 common vertex.  The pair is put
    in the vertex order the rules need (``galerkin.order_pair``); the sample
    points carry the barycentric coordinates of that order, which are mapped
    back to the corners of the stored triangles.  Returns (m, 3, 3)."""
    v = np.asarray(v, dtype=np.float64)
    tt = np.asarray(tri_t, dtype=np.int64).reshape(-1, 3)
    ss = np.asarray(tri_s, dtype=np.int64).reshape(-1, 3)
    m = tt.shape[0]
    out = np.zeros((m, 3, 3))
    xi, e1, e2, e3, wt = sauter.cube_rule(q)
    for p in range(m):
        oi, oj = order_pair(tt[p], ss[p], case)
        P = v[oi]
        Q = v[oj]
        ci = [list(tt[p]).index(a) for a in oi]     # stored corner of each ordered vertex
        cj = [list(ss[p]).index(a) for a in oj]
        jp = np.cross(P[1] - P[0], P[2] - P[1])
        jq = np.cross(Q[1] - Q[0], Q[2] - Q[1])
        jac = np.sqrt(jp @ jp) * np.sqrt(jq @ jq)
        acc = np.zeros((3, 3))
        for (u1, u2), (v1, v2), w in sauter.sub_maps(case, xi, e1, e2, e3):
            x = P[0] + u1[:, None] * (P[1] - P[0]) + u2[:, None] * (P[2] - P[1])
            y = Q[0] + v1[:, None] * (Q[1] - Q[0]) + v2[:, None] * (Q[2] - Q[1])
            d = x - y
            kv = wt * w / np.sqrt((d * d).sum(axis=1))
            lu = np.stack([1.0 - u1, u1 - u2, u2])      # barycentric, ordered vertices
            lv = np.stack([1.0 - v1, v1 - v2, v2])
            acc += (lu * kv[None, :]) @ lv.T
        for a in range(3):
            for b in range(3):
                out[p, ci[a], cj[b]] += acc[a, b] * jac
    return out / FOUR_PI


def shared(tri_t, tri_s):
    """Number of vertex ids two triangles share."""
    return sum(1 for a in tri_t if a in tri_s)


class P1Galerkin:
    """Galerkin entries of the single-layer matrix in the nodal basis."""

    def __init__(self, vertices, triangles, sauter_q=5):
        self.v = np.asarray(vertices, dtype=np.float64)
        self.t = np.asarray(triangles, dtype=np.int64)
        self.q = int(sauter_q)
        self.supports = vertex_supports(self.v.shape[0], self.t)
        self.pts, self.wts = triangle_points(self.v, self.t)
        self._pair = {}

    @property
    def n(self):
        return self.v.shape[0]

    def regular_pairs(self, ti, si):
        """3 x 3 matrices of disjoint triangle pairs (triangle ids)."""
        return local_regular(self.v, self.t[ti], self.t[si])

    def pair(self, ti, si):
        """3 x 3 matrix of the triangle pair (ti, si), cached."""
        key = (ti, si)
        if key not in self._pair:
            a, b = self.t[ti], self.t[si]
            c = shared(a, b)
            if c == 0:
                self._pair[key] = local_regular(self.v, a, b)[0]
            else:
                self._pair[key] = local_singular(self.v, a, b, c, self.q)[0]
        return self._pair[key]

    def block(self, rows, cols):
        """G restricted to the vertex lists rows x cols, assembled pair by
        pair over the two support unions (Sect. 5)."""
        rows = [int(i) for i in rows]
        cols = [int(j) for j in cols]
        ur = support_union(self.supports, rows)
        uc = support_union(self.supports, cols)
        out = np.zeros((len(rows), len(cols)))
        if not ur or not uc:
            return out
        rt = np.array([r[0] for r in ur])
        rl = np.array([r[1] for r in ur])          # (m1, 3) local rows, -1: none
        ct = np.array([c[0] for c in uc])
        cl = np.array([c[1] for c in uc])
        tc = self.t[ct]
        step = max(1, (1 << 16) // len(ct))
        for s0 in range(0, len(rt), step):
            ti = rt[s0:s0 + step]
            tr = self.t[ti]
            nsh = (tr[:, None, :, None] == tc[None, :, None, :]).sum(axis=(2, 3))
            ii, jj = np.nonzero(nsh == 0)
            if len(ii):
                M = self.regular_pairs(ti[ii], ct[jj])
                self._scatter(out, rl[s0 + ii], cl[jj], M)
            for i, j in zip(*np.nonzero(nsh > 0)):
                M = self.pair(int(ti[i]), int(ct[j]))[None]
                self._scatter(out, rl[s0 + i][None], cl[j][None], M)
        return out

    @staticmethod
    def _scatter(out, lr, lc, M):
        """out[lr[p, a], lc[p, b]] += M[p, a, b] where both local numbers exist."""
        for a in range(3):
            for b in range(3):
                ok = (lr[:, a] >= 0) & (lc[:, b] >= 0)
                if ok.any():
                    np.add.at(out, (lr[ok, a], lc[ok, b]), M[ok, a, b])

    def dense_matrix(self):
        idx = np.arange(self.n)
        return self.block(idx, idx)


def load_integrals(gal):
    """int phi_i = |T_i| / 3 summed over the support (the 7-point rule is
    exact for linear integrands)."""
    area = triangle_areas(gal.v, gal.t)
    out = np.zeros(gal.n)
    for c in range(3):
        np.add.at(out, gal.t[:, c], area / 3.0)
    return out


def green_matrix_p1(gal, rows, z, nrm, w, d_tau):
    """A_tau of Sect. 2 for the vertex rows (len(rows) x 2k)."""
    bary, _ = RADON7
    ptr, tri, corner = gal.supports
    sw = np.sqrt(w)
    k = z.shape[0]
    A = np.zeros((len(rows), 2 * k))
    for r, i in enumerate(rows):
        ts = tri[ptr[i]:ptr[i + 1]]
        cs = corner[ptr[i]:ptr[i + 1]]
        x = gal.pts[ts]                            # (s, 7, 3)
        wx = gal.wts[ts] * bary[:, cs].T           # (s, 7): weight * lambda_corner
        for nu in range(k):
            gv = g(x, z[nu][None, None, :])
            dv = dg_dn(x, z[nu][None, None, :], nrm[nu][None, None, :])
            A[r, nu] = sw[nu] * (wx * gv).sum()
            A[r, nu + k] = -d_tau * sw[nu] * (wx * dv).sum()
    return A


def build_tree_points(points, leaf_size):
    """The cluster tree of ``cluster.build_tree`` on points (the vertex
    positions) instead of triangle centroids."""
    p = np.asarray(points, dtype=np.float64)
    return cluster.build_tree_from_centers(p, leaf_size)


def cluster_boxes_p1(vertices, triangles, supports, tree):
    """Box of a cluster: the bounding box of the vertices of all triangles
    in the supports of its basis functions (Sect. 2)."""
    v = np.asarray(vertices, dtype=np.float64)
    t = np.asarray(triangles, dtype=np.int64)
    ptr, tri, _ = supports
    nc = len(tree["begin"])
    lo = np.empty((nc, 3))
    hi = np.empty((nc, 3))
    for c in range(nc):
        idx = tree["perm"][tree["begin"][c]:tree["end"][c]]
        ts = np.concatenate([tri[ptr[i]:ptr[i + 1]] for i in idx])
        pts = v[t[ts].ravel()]
        lo[c] = pts.min(axis=0)
        hi[c] = pts.max(axis=0)
    return lo, hi


def build_p1_h2(vertices, triangles, params, tree=None, follow=None):
    """GCA-H^2 of the single-layer matrix in the nodal basis.  ``follow``
    (test infrastructure): cluster -> pivot vertex ids to replay in the cross
    approximations (``gca.aca``)."""
    gal = P1Galerkin(vertices, triangles, params.sauter_q)
    if tree is None:
        tree = build_tree_points(vertices, params.leaf_size)
    lo, hi = cluster_boxes_p1(vertices, triangles, gal.supports, tree)
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
