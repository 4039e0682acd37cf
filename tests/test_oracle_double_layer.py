"""Pins of the double-layer oracle (oracle/double_layer.py) against what the
mathematics fixes, independently of its own code:

* the solid angle Omega_T(x) = int_T <n_y, y - x> / |y - x|^3 dy of a flat
  triangle (Van Oosterom and Strackee's closed form, checked here against
  brute force), so that int_T dg/dn_y(x, y) dy = -Omega_T(x) / (4 pi);
* Gauss's law on a closed polyhedron: the solid angles of all faces seen
  from a point inside a face add up to 2 pi, so sum_j k_ij = -|T_i| / 2;
* touching entries against the closed-form inner integral with a graded
  outer rule (identical flat triangles and coplanar neighbours give 0);
* the unit-sphere identity <n_y, x - y> = -|x - y|^2 / 2, i.e. dg/dn_y =
  -g / 2, so K + G / 2 shrinks as the polyhedron refines;
* the differentiated representation formula behind the column Green matrix
  converging in the box rule's order;
* the H^2 approximation: fast product = explicit bases, adjoint identity,
  spectral error falling with the tolerance, row bases equal to the single
  layer's.
"""

import numpy as np
import pytest

import synth
from oracle import double_layer as odl, gca as ogca, h2 as oh2, sauter
from oracle.galerkin import Galerkin, dg_dn, g
from oracle.params import Params
from oracle.rules import box_rule, triangle_areas


def solid_angle(x, V):
    """Signed solid angle of the flat triangle V seen from x (..., 3):
    tan(Omega / 2) = a . (b x c) / (|a||b||c| + (a.b)|c| + (a.c)|b| + (b.c)|a|)."""
    a = V[0] - x
    b = V[1] - x
    c = V[2] - x
    la, lb, lc = (np.linalg.norm(u, axis=-1) for u in (a, b, c))
    num = (a * np.cross(b, c)).sum(-1)
    den = la * lb * lc + (a * b).sum(-1) * lc + (a * c).sum(-1) * lb + (b * c).sum(-1) * la
    return 2.0 * np.arctan2(num, den)


def brute_flux(x, V, q=40, levels=5):
    """int_T <n, y - x> / |y - x|^3 dy by a collapsed Gauss rule on a uniform
    4^levels refinement of V (x away from the triangle)."""
    V = np.asarray(V, dtype=np.float64)
    if levels > 0:
        a, b, c = V
        ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
        return sum(brute_flux(x, np.array(T), q, levels - 1)
                   for T in ([a, ab, ca], [ab, b, bc], [ca, bc, c], [ab, bc, ca]))
    n = np.cross(V[1] - V[0], V[2] - V[0])
    jac = np.linalg.norm(n)
    n = n / jac
    t, w = np.polynomial.legendre.leggauss(q)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    s, r = np.meshgrid(t, t, indexing="ij")
    wt = (np.outer(w, w) * s).ravel()
    y = V[0] + s.ravel()[:, None] * (V[1] - V[0]) + (s * r).ravel()[:, None] * (V[2] - V[1])
    d = y - x
    return jac * np.sum(wt * (d @ n) / np.linalg.norm(d, axis=1) ** 3)


def graded(levels, p, sigma, ends):
    t, w = np.polynomial.legendre.leggauss(p)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    if ends == {1}:
        cuts = np.concatenate([1.0 - sigma ** np.arange(levels + 1), [1.0]])
    else:
        half = 0.5 * sigma ** np.arange(levels + 1)
        cuts = np.unique(np.concatenate([[0.0], half, 1.0 - half, [1.0]]))
    a, b = cuts[:-1], cuts[1:]
    return (a[:, None] + (b - a)[:, None] * t).ravel(), ((b - a)[:, None] * w).ravel()


def outer(f, P, levels=26, p=12, sigma=0.3):
    """int_{T_P} f(x) dx, refined towards the edges and vertices of T_P."""
    P = np.asarray(P, dtype=np.float64)
    c = P.mean(axis=0)
    s, ws = graded(levels, p, sigma, {1})
    t, wt = graded(levels, p, sigma, {0, 1})
    S, T = np.meshgrid(s, t, indexing="ij")
    W = np.outer(ws, wt) * S
    tot = 0.0
    for k in range(3):
        a, b = P[k], P[(k + 1) % 3]
        area2 = np.linalg.norm(np.cross(a - c, b - c))
        x = c + S[..., None] * (((1.0 - T)[..., None] * a + T[..., None] * b) - c)
        tot += area2 * np.sum(W * f(x))
    return tot


def reference_entry(P, Q):
    """k for the pair (T_P, T_Q): -(1 / 4 pi) int_{T_P} Omega_{T_Q}(x) dx."""
    Q = np.asarray(Q, dtype=np.float64)
    return -outer(lambda x: solid_angle(x, Q), P) / (4.0 * np.pi)


A = np.array([0.1, 0.0, 0.05])
B = np.array([1.0, 0.2, -0.1])
C = np.array([0.3, 0.9, 0.2])
D = np.array([0.8, -0.7, 0.3])
E = np.array([-0.6, 0.4, 0.5])
F = np.array([-0.5, -0.6, -0.2])
Dp = A + 1.3 * (B - A) - 0.9 * (C - A)
Ep = A - 0.7 * (B - A) + 0.2 * (C - A)
Fp = A - 0.4 * (B - A) - 0.8 * (C - A)


@pytest.mark.parametrize("x", [[0.4, 0.3, 0.6], [2.0, -1.0, 0.3], [0.45, 0.35, 0.062], [-0.3, 0.1, -0.2]])
def test_solid_angle_closed_form(x):
    x = np.asarray(x, dtype=np.float64)
    V = np.array([A, B, C])
    assert abs(solid_angle(x, V) - brute_flux(x, V)) <= 1e-12 * abs(solid_angle(x, V))


def test_solid_angles_of_closed_polyhedron():
    # from a point inside a face, the other faces of a closed surface fill
    # half the full solid angle (and the own face none)
    v, t = synth.mesh_for_config("perturbed320")
    rng = np.random.default_rng(4)
    for i in rng.choice(len(t), 6, replace=False):
        bc = rng.dirichlet([1.0, 1.0, 1.0])
        x = bc @ v[t[i]]
        # the own face contributes nothing (x - y lies in its plane; the
        # closed form jumps by +-2 pi across it and is not used there)
        tot = sum(solid_angle(x, v[t[j]]) for j in range(len(t)) if j != i)
        assert abs(tot - 2.0 * np.pi) <= 1e-12


def test_identical_pairs_vanish():
    v, t = synth.mesh_for_config("sphere80")
    dl = odl.DoubleLayer(v, t, 5)
    idx = np.arange(len(t))
    assert np.all(dl.entries(idx, idx) == 0.0)


@pytest.mark.parametrize("case,P,Q,zero", [(2, [A, B, C], [A, B, D], False), (1, [A, B, C], [A, E, F], False),
                                           (2, [A, B, C], [A, B, Dp], True), (1, [A, B, C], [A, Ep, Fp], True)])
def test_touching_kernel_matches_semi_analytic(case, P, Q, zero):
    nq = odl.unit_normals(np.array(Q), np.array([[0, 1, 2]]))[0]
    kern = lambda x, y: odl.dg_dny(x, y, nq[None, None, :])  # noqa: E731
    got = sauter.integrate(case, np.array([P]), np.array([Q]), kern, 14)[0]
    ref = reference_entry(P, Q)
    if zero:
        assert abs(got) <= 1e-15 and abs(ref) <= 1e-15
    else:
        assert abs(got - ref) <= 1e-10 * abs(ref), (got, ref)


@pytest.mark.parametrize("case", [1, 2])
def test_mesh_touching_entries(case):
    """Touching entries of a mesh through DoubleLayer.entries (vertex order by
    order_pair, the normal of the stored triangle) against the reference."""
    v, t = synth.mesh_for_config("perturbed1280")
    dl = odl.DoubleLayer(v, t, sauter_q=14)
    from oracle.galerkin import shared_vertices
    rng = np.random.default_rng(case + 10)
    found = 0
    for a in rng.integers(0, len(t), 50):
        js = np.nonzero(shared_vertices(t, np.full(len(t), a), np.arange(len(t))) == case)[0]
        b = int(js[0])
        got = dl.entries(np.array([a]), np.array([b]))[0]
        ref = reference_entry(v[t[a]], v[t[b]])
        assert abs(got - ref) <= 1e-10 * abs(ref), (a, b, got, ref)
        found += 1
        if found == 3:
            break


def test_regular_entries_against_reference():
    v, t = synth.mesh_for_config("perturbed320")
    dl = odl.DoubleLayer(v, t, 5)
    from oracle.galerkin import shared_vertices
    cen = v[t].mean(axis=1)
    i = 7
    js = [j for j in np.argsort(np.linalg.norm(cen - cen[i], axis=1))
          if shared_vertices(t, np.array([i]), np.array([j]))[0] == 0]
    prev = None
    for j in (js[0], js[5], js[40], js[200]):
        got = dl.entries(np.array([i]), np.array([j]))[0]
        ref = reference_entry(v[t[i]], v[t[j]])
        err = abs(got - ref) / abs(ref)
        assert err <= 2e-3
        prev = err
    assert prev <= 1e-9  # far pairs: the 7 x 7 rule is exact to rounding


def test_gauss_law_row_sums():
    """sum_j k_ij = -|T_i| / 2 on a closed polyhedron; the oracle's K meets it
    within the accuracy of its 7 x 7 rule on close disjoint pairs."""
    v, t = synth.mesh_for_config("sphere320")
    K = odl.DoubleLayer(v, t, 5).dense_matrix()
    area = triangle_areas(v, t)
    err = np.abs(K.sum(axis=1) + area / 2) / area
    assert err.max() <= 2e-3


def test_unit_sphere_identity_under_refinement():
    # on the unit sphere <n_y, x - y> = -|x - y|^2 / 2, so dg/dn_y = -g / 2
    # and K = -G / 2 in the limit; on smooth densities (constant and the l = 1
    # harmonic z) the polyhedral discretisations converge to each other
    errs = []
    for name in ("sphere80", "sphere320", "sphere1280"):
        v, t = synth.mesh_for_config(name)
        cen = v[t].mean(axis=1)
        f = np.stack([np.ones(len(t)), cen[:, 2]], axis=1)
        dl = odl.DoubleLayer(v, t, 5)
        gal = Galerkin(v, t, 5)
        idx = np.arange(len(t))
        Kf = np.zeros_like(f)
        Gf = np.zeros_like(f)
        for s in range(0, len(t), 256):
            rows = idx[s:s + 256]
            Kf[rows] = dl.block(rows, idx) @ f
            Gf[rows] = gal.block(rows, idx) @ f
        errs.append(np.linalg.norm(Kf + Gf / 2, axis=0) / np.linalg.norm(Gf / 2, axis=0))
    errs = np.array(errs)
    assert np.all(errs[1] < 0.5 * errs[0]) and np.all(errs[2] < 0.5 * errs[1])
    assert np.all(errs[2] < 5e-3)


def test_column_representation_formula_converges():
    """dg/dn_y(x, y) = sum_nu w_nu [dg/dn_y(y, z) dg/dn_z(x, z) - d2g(y, z) g(x, z)]
    for y inside omega, x outside, as the box rule's order grows."""
    lo, hi = np.array([-0.5, -0.4, -0.3]), np.array([0.5, 0.4, 0.3])
    y = np.array([0.05, -0.05, 0.02])
    ny = np.array([0.3, 0.5, -0.8])
    ny /= np.linalg.norm(ny)
    x = np.array([2.1, 1.3, -1.7])
    exact = odl.dg_dny(x, y, ny)
    errs = []
    for m in (2, 4, 6, 8, 10, 12, 14):
        z, nz, w = box_rule(lo, hi, m)
        approx = np.sum(w * (odl.dg_dny(z, y[None, :], ny[None, :]) * dg_dn(x[None, :], z, nz)
                             - odl.d2g_dny_dnz(y[None, :], z, ny[None, :], nz) * g(x[None, :], z)))
        errs.append(abs(approx - exact) / abs(exact))
    assert errs[-1] < 5e-5
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_column_factors_reproduce_the_quadrature():
    # the column Green matrix times the x-side factors is the quadrature of
    # the differentiated representation formula, entry for entry
    v, t = synth.mesh_for_config("sphere80")
    dl = odl.DoubleLayer(v, t, 5)
    cols = np.arange(0, 6)
    lo, hi = v[t[cols]].reshape(-1, 3).min(0), v[t[cols]].reshape(-1, 3).max(0)
    d = np.linalg.norm(hi - lo)
    z, nz, w = box_rule(lo - 0.2 * d, hi + 0.2 * d, 3)
    Ac = odl.column_green_matrix(dl, cols, z, nz, w, d)
    x = np.array([3.0, -2.0, 1.0])
    bx = np.concatenate([np.sqrt(w) * dg_dn(x[None, :], z, nz), np.sqrt(w) / d * g(x[None, :], z)])
    got = Ac @ bx
    y, wy, ny = dl.pts[cols], dl.wts[cols], dl.nrm[cols][:, None, :]
    want = np.zeros(len(cols))
    for nu in range(len(w)):
        f = (odl.dg_dny(z[nu][None, None, :], y, ny) * dg_dn(x, z[nu], nz[nu])
             - odl.d2g_dny_dnz(y, z[nu][None, None, :], ny, nz[nu][None, None, :]) * g(x, z[nu]))
        want += w[nu] * (wy * f).sum(axis=1)
    assert np.allclose(got, want, rtol=1e-13, atol=0)


@pytest.fixture(scope="module")
def dl320():
    # the 1280-triangle workload's parameters (leaf 32, m = 3, tol 1e-6)
    v, t = synth.mesh_for_config("sphere1280")
    p = Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    h = odl.build_dl_h2(v, t, p)
    assert len(h.far) > 0
    return v, t, p, h


def test_row_bases_are_the_single_layers(dl320):
    v, t, p, h = dl320
    hs = ogca.build_h2(v, t, p)
    for c in range(len(h.tree["begin"])):
        assert np.array_equal(h.rows.pivots[c], hs.bases.pivots[c])


def test_fast_product_equals_explicit(dl320):
    v, t, p, h = dl320
    K = odl.dense(h)
    x = synth.uniform_rhs(len(t), 3, seed=2)
    assert np.abs(odl.matvec(h, x) - K @ x).max() <= 1e-13 * np.abs(K @ x).max()
    assert np.abs(odl.matvec_t(h, x) - K.T @ x).max() <= 1e-13 * np.abs(K.T @ x).max()
    # non-symmetric: the transpose differs
    assert np.linalg.norm(odl.matvec_t(h, x) - odl.matvec(h, x)) > 1e-3 * np.linalg.norm(odl.matvec(h, x))


def test_adjoint_identity(dl320):
    v, t, p, h = dl320
    a = synth.normal_rhs(len(t), 2, seed=3)
    b = synth.normal_rhs(len(t), 2, seed=4)
    lhs = (a * odl.matvec(h, b)).sum(0)
    rhs = (odl.matvec_t(h, a) * b).sum(0)
    assert np.all(np.abs(lhs - rhs) <= 1e-13 * np.linalg.norm(a, axis=0) * np.linalg.norm(odl.matvec(h, b), axis=0))


def test_spectral_error_falls_with_tolerance(dl320):
    v, t, p, h6 = dl320
    K = odl.DoubleLayer(v, t, 5).dense_matrix()
    nk = np.linalg.norm(K, 2)
    h3 = odl.build_dl_h2(v, t, Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-3, sauter_q=5))
    e3 = np.linalg.norm(K - odl.dense(h3), 2) / nk
    e6 = np.linalg.norm(K - odl.dense(h6), 2) / nk
    assert 0.0 < e6 < 0.1 * e3
    assert e6 < 1e-5
