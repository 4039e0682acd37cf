"""Oracle of the continuous piecewise linear basis (Sect. 5) against what the
paper and the mathematics fix: the worked example of the support union,
brute-force unions, the piecewise constant entries (the barycentric
coordinates sum to one), linear densities through the Sauter-Schwab rules,
brute-force subdivision, symmetry, positive definiteness, the unit-sphere
identities and the dense matrix for the H^2 product."""

import os

import numpy as np
import pytest

import synth
from oracle import cluster, gca, h2, p1, sauter
from oracle.galerkin import FOUR_PI, Galerkin
from oracle.params import Params
from oracle.rules import RADON7, triangle_areas

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "p1_support_union.txt")


def _golden():
    tris, tau, sup, rows, merged = [], None, {}, [], []
    val = lambda s: -1 if s == "_" else int(s) - 1  # noqa: E731 (1-based -> 0-based, bottom -> -1)
    with open(GOLDEN) as f:
        for line in f:
            w = line.split()
            if not w or w[0].startswith("#"):
                continue
            if w[0] == "triangle":
                tris.append([int(a) - 1 for a in w[2:5]])
            elif w[0] == "tau":
                tau = [int(a) - 1 for a in w[1:]]
            elif w[0] == "support":
                sup[int(w[1]) - 1] = [int(a) - 1 for a in w[2:]]
            elif w[0] == "row":
                rows.append((int(w[1]) - 1, tuple(val(a) for a in w[2:5])))
            elif w[0] == "merged":
                merged.append((int(w[1]) - 1, tuple(val(a) for a in w[2:5])))
    return np.array(tris), tau, sup, rows, merged


def test_worked_example_of_the_paper():
    tris, tau, sup, rows, merged = _golden()
    nv = int(tris.max()) + 1
    S = p1.vertex_supports(nv, tris)
    ptr, tri, corner = S
    for i, ts in sup.items():
        assert list(tri[ptr[i]:ptr[i + 1]]) == ts
    # the rows before the merge, vertex after vertex
    before = []
    for a, i in enumerate(tau):
        for k in range(ptr[i], ptr[i + 1]):
            loc = [-1, -1, -1]
            loc[corner[k]] = a
            before.append((int(tri[k]), tuple(loc)))
    assert before == rows
    assert p1.support_union(S, tau) == merged


def _mesh(level):
    return synth.icosphere(level)


def test_support_union_against_brute_force():
    v, t = _mesh(2)
    S = p1.vertex_supports(len(v), t)
    rng = np.random.default_rng(3)
    for trial in range(20):
        tau = list(rng.choice(len(v), size=int(rng.integers(1, 40)), replace=False))
        got = p1.support_union(S, tau)
        pos = {int(i): a for a, i in enumerate(tau)}
        want = []
        for k in range(len(t)):
            loc = tuple(pos.get(int(c), -1) for c in t[k])
            if any(x >= 0 for x in loc):
                want.append((k, loc))
        assert got == want, trial


def _far_pair():
    v, t = _mesh(2)
    c = v[t].mean(axis=1)
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2)
    i, j = np.unravel_index(np.argmax(d), d.shape)
    return v, t, int(i), int(j)


def test_regular_matrix_sums_to_the_constant_entry():
    v, t = _mesh(2)
    gal = Galerkin(v, t)
    rng = np.random.default_rng(0)
    for _ in range(20):
        i, j = rng.integers(0, len(t), size=2)
        if len(set(t[i]) & set(t[j])):
            continue
        M = p1.local_regular(v, t[i], t[j])[0]
        assert abs(M.sum() - gal.regular(np.array([i]), np.array([j]))[0]) <= 1e-14 * abs(M.sum())


def _subdivide(P, levels):
    """Sub-triangles (vertex triples) of triangle P after `levels` midpoint refinements."""
    tris = [np.array(P)]
    for _ in range(levels):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array(x) for x in ([a, ab, ca], [ab, b, bc], [ca, bc, c], [ab, bc, ca])]
        tris = nxt
    return tris


def _bary(P, x):
    """Barycentric coordinates of points x (m, 3) in triangle P, from a least-squares solve."""
    A = np.stack([P[1] - P[0], P[2] - P[0]], axis=1)
    uv = np.linalg.lstsq(A, (x - P[0]).T, rcond=None)[0].T
    return np.stack([1 - uv[:, 0] - uv[:, 1], uv[:, 0], uv[:, 1]], axis=1)


def test_regular_matrix_against_subdivision():
    """Far triangles: the 7-point rule against 64 sub-triangles per side."""
    v, t, i, j = _far_pair()
    P, Q = v[t[i]], v[t[j]]
    bary, wts = RADON7
    xs, wx, ys, wy = [], [], [], []
    for sub in _subdivide(P, 3):
        xs.append(bary @ sub)
        wx.append(wts * triangle_areas(sub, np.array([[0, 1, 2]]))[0])
    for sub in _subdivide(Q, 3):
        ys.append(bary @ sub)
        wy.append(wts * triangle_areas(sub, np.array([[0, 1, 2]]))[0])
    x, wx, y, wy = np.concatenate(xs), np.concatenate(wx), np.concatenate(ys), np.concatenate(wy)
    lx, ly = _bary(P, x), _bary(Q, y)
    K = 1.0 / (FOUR_PI * np.linalg.norm(x[:, None] - y[None], axis=2))
    want = (lx * wx[:, None]).T @ K @ (ly * wy[:, None])
    got = p1.local_regular(v, t[i], t[j])[0]
    # the 7-point rule errs by about 5e-9 here; a misassigned corner would err
    # by the spread of the entries (about 2e-3)
    assert np.abs(got - want).max() <= 1e-7 * np.abs(want).max()


@pytest.mark.parametrize("case", [3, 2, 1])
def test_singular_matrix_against_linear_densities(case):
    """Sum_ab f(P_a) h(Q_b) M_ab = int int f(x) h(y) g(x, y) for linear f, h
    (the barycentric coordinates reproduce linear functions), computed by the
    plain Sauter-Schwab integral of the weighted kernel; and the total against
    the piecewise constant entry."""
    v, t = _mesh(2)
    gal = Galerkin(v, t)
    sh = np.array([[len(set(a) & set(b)) for b in t] for a in t[:40]])
    i, j = map(int, np.argwhere(sh == case)[0])
    M = p1.local_singular(v, t[i], t[j], case, 6)[0]
    M5 = p1.local_singular(v, t[i], t[j], case, 5)[0]
    assert abs(M5.sum() - gal.singular(np.array([i]), np.array([j]), case)[0]) <= 1e-13 * abs(M5.sum())
    f = np.array([0.3, -1.2, 0.7])
    hh = np.array([1.1, 0.4, -0.5])
    from oracle.galerkin import order_pair
    oi, oj = order_pair(t[i], t[j], case)
    kern = lambda x, y: (0.2 + x @ f) * (-0.1 + y @ hh) / np.linalg.norm(x - y, axis=-1)  # noqa: E731
    want = sauter.integrate(case, v[oi][None], v[oj][None], kern, 6)[0] / FOUR_PI
    fa = 0.2 + v[t[i]] @ f
    hb = -0.1 + v[t[j]] @ hh
    got = fa @ M @ hb
    assert abs(got - want) <= 1e-12 * abs(want)


def test_pair_matrices_transpose():
    """M(t, s) = M(s, t)^T: exactly for the identical and common-vertex
    rules (symmetric in the two triangles), for the common-edge rule up to
    its quadrature error, which falls geometrically with q."""
    v, t = _mesh(2)
    sh = np.array([[len(set(a) & set(b)) for b in t] for a in t[:40]])
    for case, q, tol in ((3, 4, 1e-13), (1, 4, 1e-13), (2, 4, 1e-5), (2, 6, 1e-8), (2, 8, 1e-10)):
        i, j = map(int, np.argwhere(sh == case)[0])
        A = p1.local_singular(v, t[i], t[j], case, q)[0]
        B = p1.local_singular(v, t[j], t[i], case, q)[0]
        assert np.abs(A - B.T).max() <= tol * np.abs(A).max(), (case, q)


@pytest.fixture(scope="module")
def dense2():
    v, t = _mesh(2)
    gal = p1.P1Galerkin(v, t, 5)
    return v, t, gal, gal.dense_matrix()


def test_dense_symmetric_positive_definite(dense2):
    _, _, _, G = dense2
    # exact up to the common-edge rule, whose two orders of a pair agree to
    # its quadrature error (about 1e-7 of the largest entry at q = 5)
    assert np.abs(G - G.T).max() <= 1e-6 * np.abs(G).max()
    np.linalg.cholesky(G)


def test_block_is_dense_submatrix(dense2):
    _, _, gal, G = dense2
    rng = np.random.default_rng(5)
    rows = rng.choice(gal.n, 17, replace=False)
    cols = rng.choice(gal.n, 23, replace=False)
    assert np.abs(gal.block(rows, cols) - G[np.ix_(rows, cols)]).max() <= 1e-15 * np.abs(G).max()


@pytest.fixture(scope="module")
def dense3():
    v, t = _mesh(3)
    gal = p1.P1Galerkin(v, t, 5)
    return v, t, gal, gal.dense_matrix()


def _identity_errors(dense):
    v, t, gal, G = dense
    ones = p1.load_integrals(gal)
    e_const = np.linalg.norm(G.sum(axis=1) - ones) / np.linalg.norm(ones)
    # density z: potential z / 3 on the unit sphere (first spherical harmonic)
    bary, wts = RADON7
    x = np.einsum("qc,tcd->tqd", bary, v[t])
    w = wts[None, :] * triangle_areas(v, t)[:, None]
    rhs = np.zeros(len(v))
    for c in range(3):
        np.add.at(rhs, t[:, c], (w * bary[None, :, c] * x[:, :, 2]).sum(axis=1) / 3.0)
    e_z = np.linalg.norm(G @ v[:, 2] - rhs) / np.linalg.norm(rhs)
    return e_const, e_z


def test_unit_sphere_identities_converge(dense2, dense3):
    e2 = _identity_errors(dense2)
    e3 = _identity_errors(dense3)
    for a, b in zip(e2, e3):
        assert b < a / 3.0, (a, b)      # O(h^2): about a quarter per refinement
    assert e3[0] < 1e-2 and e3[1] < 2e-2


def test_green_rows_sum_to_constant_rows():
    """sum_i phi_i = 1, so the nodal rows of A_tau summed over all vertices
    equal the piecewise constant rows summed over all triangles."""
    v, t = _mesh(2)
    gal1 = p1.P1Galerkin(v, t)
    gal0 = Galerkin(v, t)
    lo, hi = v.min(axis=0), v.max(axis=0)
    z, nrm, w = gca.omega_rule(lo, hi, np.linalg.norm(hi - lo), 0.125, 3)
    A1 = p1.green_matrix_p1(gal1, np.arange(len(v)), z, nrm, w, 2.0)
    A0 = gca.green_matrix(gal0, np.arange(len(t)), z, nrm, w, 2.0)
    assert np.abs(A1.sum(axis=0) - A0.sum(axis=0)).max() <= 1e-12 * np.abs(A0.sum(axis=0)).max()


def test_vertex_tree_is_the_point_bisection():
    v, _ = _mesh(3)
    tree = p1.build_tree_points(v, 32)
    pseudo = np.repeat(np.arange(len(v))[:, None], 3, axis=1)
    ref = cluster.build_tree_from_centers(v, 32)
    for k in ("perm", "begin", "end", "child0", "child1", "level"):
        assert np.array_equal(tree[k], ref[k])
    assert sorted(tree["perm"]) == list(range(len(v)))
    assert pseudo.shape == (len(v), 3)


def test_p1_h2_product_against_dense(dense3):
    v, t, _, G = dense3
    prm = Params(leaf_size=16, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    H = p1.build_p1_h2(v, t, prm)
    assert H.n == len(v) and len(H.far) > 0
    x = np.random.default_rng(1).standard_normal((len(v), 2))
    y = h2.matvec(H, x)
    err = np.linalg.norm(y - G @ x, axis=0) / np.linalg.norm(G @ x, axis=0)
    assert err.max() < 1e-4
    # interpolation: V restricted to the pivots is the identity
    for c, piv in enumerate(H.bases.pivots):
        if piv is not None and len(piv) and cluster.is_leaf(H.tree, c):
            rows = list(H.tree["perm"][H.tree["begin"][c]:H.tree["end"][c]])
            V = H.bases.V[c]
            assert np.abs(V[[rows.index(p) for p in piv]] - np.eye(len(piv))).max() <= 1e-12
