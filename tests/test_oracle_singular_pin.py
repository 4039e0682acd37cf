"""Independent pin of the touching-pair (Sauter-Schwab) integrals of the
oracle (Sect. 8: identical triangles, a common edge, a common vertex).

The reference value of I = int_{T_i} int_{T_j} 1 / |x - y| dy dx is formed
without any Sauter-Schwab substitution:

* the inner integral phi(x) = int_T 1 / |x - y| dy over a flat triangle has a
  closed form (the potential of a uniform triangle): split T into the three
  signed sub-triangles (x0, a, b) spanned by the projection x0 of x onto T's
  plane and each edge (a, b), and integrate in polar coordinates around x0;
  per edge with in-plane distance p from x0 to the edge line, edge
  coordinates l- <= l+ of its end points, height h of x above the plane and
  R+- = |x - b|, |x - a|:
      p ln((R+ + l+) / (R- + l-))
        - |h| [atan(p l+ / (p^2 + h^2 + |h| R+)) - atan(p l- / (p^2 + h^2 + |h| R-))];
  the formula is itself checked here against brute-force quadrature at
  points off the triangle;
* the outer integral over T_i uses a geometrically graded tensor Gauss rule
  on the three sub-triangles (centroid, edge) of T_i, refined towards T_i's
  edges and vertices, where phi loses smoothness.

The oracle's Sauter-Schwab value at high order must agree to 1e-10, for
each case, on coplanar and non-coplanar pairs and on pairs taken from a
mesh through ``Galerkin.entries`` (which also exercises the vertex order of
``order_pair``).  The oracle's default order q = 5 is held to its measured
error bound.
"""

import numpy as np
import pytest

import synth
from oracle import sauter
from oracle.galerkin import Galerkin, shared_vertices


def triangle_potential(x, V):
    """phi(x) = int_T 1 / |x - y| dy for the flat triangle V (3 x 3), x (..., 3)."""
    V = np.asarray(V, dtype=np.float64)
    nrm = np.cross(V[1] - V[0], V[2] - V[0])
    nrm = nrm / np.linalg.norm(nrm)
    h = (x - V[0]) @ nrm
    x0 = x - h[..., None] * nrm
    ah = np.abs(h)
    out = np.zeros(x.shape[:-1])
    for k in range(3):
        a, b = V[k], V[(k + 1) % 3]
        s = (b - a) / np.linalg.norm(b - a)
        m = np.cross(s, nrm)                     # outward in-plane normal of the edge
        p = (a - x0) @ m                         # signed distance of x0 to the edge line
        lm = (a - x0) @ s
        lp = (b - x0) @ s
        r0 = p * p + h * h
        Rm = np.sqrt(r0 + lm * lm)
        Rp = np.sqrt(r0 + lp * lp)

        def rl(R, l):                            # R + l without cancellation
            with np.errstate(divide="ignore", invalid="ignore"):
                return np.where(l >= 0, R + l, r0 / (R - l))
        with np.errstate(divide="ignore", invalid="ignore"):
            logt = np.where(np.abs(p) > 0, p * np.log(rl(Rp, lp) / rl(Rm, lm)), 0.0)
        at = np.arctan2(p * lp, r0 + ah * Rp) - np.arctan2(p * lm, r0 + ah * Rm)
        out += logt - ah * at
    return out


def graded_nodes(levels, p, sigma, ends):
    """Composite Gauss rule on [0, 1], geometrically refined towards the
    end points listed in `ends` (subsets of {0, 1})."""
    t, w = np.polynomial.legendre.leggauss(p)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    if ends == {1}:
        cuts = np.concatenate([1.0 - sigma ** np.arange(levels + 1), [1.0]])
    elif ends == {0, 1}:
        half = 0.5 * sigma ** np.arange(levels + 1)
        cuts = np.unique(np.concatenate([[0.0], half, 1.0 - half, [1.0]]))
    else:
        raise ValueError(ends)
    a, b = cuts[:-1], cuts[1:]
    nodes = (a[:, None] + (b - a)[:, None] * t[None, :]).ravel()
    wts = ((b - a)[:, None] * w[None, :]).ravel()
    return nodes, wts


def outer_integral(f, P, levels=26, p=12, sigma=0.3):
    """int_{T_P} f(x) dx, graded towards the edges and vertices of T_P."""
    P = np.asarray(P, dtype=np.float64)
    c = P.mean(axis=0)
    s, ws = graded_nodes(levels, p, sigma, {1})
    t, wt = graded_nodes(levels, p, sigma, {0, 1})
    S, T = np.meshgrid(s, t, indexing="ij")
    W = np.outer(ws, wt) * S
    total = 0.0
    for k in range(3):
        a, b = P[k], P[(k + 1) % 3]
        area2 = np.linalg.norm(np.cross(a - c, b - c))
        edge = (1.0 - T)[..., None] * a + T[..., None] * b
        x = c + S[..., None] * (edge - c)
        total += area2 * np.sum(W * f(x))
    return total


def reference_integral(P, Q):
    return outer_integral(lambda x: triangle_potential(x, Q), P)


A = np.array([0.1, 0.0, 0.05])
B = np.array([1.0, 0.2, -0.1])
C = np.array([0.3, 0.9, 0.2])
D = np.array([0.8, -0.7, 0.3])
E = np.array([-0.6, 0.4, 0.5])
F = np.array([-0.5, -0.6, -0.2])
Dp = A + 1.3 * (B - A) - 0.9 * (C - A) + 0.0 * np.cross(B - A, C - A)   # in the plane of ABC
Ep = A - 0.7 * (B - A) + 0.2 * (C - A)                                    # in the plane of ABC
Fp = A - 0.4 * (B - A) - 0.8 * (C - A)

PAIRS = {
    "identical": (3, [A, B, C], [A, B, C]),
    "edge": (2, [A, B, C], [A, B, D]),
    "edge_coplanar": (2, [A, B, C], [A, B, Dp]),
    "vertex": (1, [A, B, C], [A, E, F]),
    "vertex_coplanar": (1, [A, B, C], [A, Ep, Fp]),
}


def brute_potential(x, V, q=40, levels=5):
    """phi(x) by a collapsed tensor Gauss rule on each of the 4^levels
    triangles of a uniform refinement of V (x off the triangle)."""
    V = np.asarray(V, dtype=np.float64)
    if levels > 0:
        a, b, c = V
        ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
        return sum(brute_potential(x, T, q, levels - 1)
                   for T in ([a, ab, ca], [ab, b, bc], [ca, bc, c], [ab, bc, ca]))
    t, w = np.polynomial.legendre.leggauss(q)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    s, r = np.meshgrid(t, t, indexing="ij")
    wt = (np.outer(w, w) * s).ravel()
    y = V[0] + s.ravel()[:, None] * (V[1] - V[0]) + (s * r).ravel()[:, None] * (V[2] - V[1])
    jac = np.linalg.norm(np.cross(V[1] - V[0], V[2] - V[1]))
    d = np.linalg.norm(x[None, :] - y, axis=1)
    return jac * np.sum(wt / d)


@pytest.mark.parametrize("x", [[0.4, 0.3, 0.6], [2.0, -1.0, 0.3], [0.45, 0.35, 0.062],
                               [-0.3, 0.1, -0.2], [0.5, 0.4, 1e-3 + 0.07]])
def test_triangle_potential_closed_form(x):
    x = np.asarray(x)
    V = [A, B, C]
    got = triangle_potential(x[None, :], V)[0]
    want = brute_potential(x, V)
    assert abs(got - want) <= 1e-12 * abs(want)


def test_triangle_potential_in_plane_centroid_symmetry():
    # equilateral triangle, x at its centroid: the three edges contribute
    # equally, p ln((R + l)/(R - l)) with p = inradius, l = half side
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, np.sqrt(3) / 2, 0.0]])
    c = V.mean(axis=0)
    rin = np.sqrt(3) / 6
    want = 3 * rin * np.log((np.hypot(rin, 0.5) + 0.5) / (np.hypot(rin, 0.5) - 0.5))
    assert abs(triangle_potential(c[None, :], V)[0] - want) <= 1e-14 * want


@pytest.mark.parametrize("name", list(PAIRS))
def test_sauter_schwab_matches_semi_analytic(name):
    case, P, Q = PAIRS[name]
    ref = reference_integral(P, Q)
    got = sauter.integrate(case, np.array([P]), np.array([Q]),
                           lambda x, y: 1.0 / np.sqrt(((x - y) ** 2).sum(-1)), 14)[0]
    assert abs(got - ref) <= 1e-10 * abs(ref), (name, got, ref)


def test_outer_rule_is_converged():
    # the reference itself: refining the graded outer rule changes nothing
    case, P, Q = PAIRS["identical"]
    a = outer_integral(lambda x: triangle_potential(x, Q), P, levels=26, p=12)
    b = outer_integral(lambda x: triangle_potential(x, Q), P, levels=34, p=16, sigma=0.25)
    assert abs(a - b) <= 1e-12 * abs(b)


@pytest.mark.parametrize("case", [3, 2, 1])
def test_mesh_entries_match_semi_analytic(case):
    """Galerkin entries of touching pairs of a mesh (vertex order chosen by
    order_pair inside Galerkin.entries) against the semi-analytic value."""
    v, t = synth.mesh_for_config("perturbed1280")
    gal = Galerkin(v, t, sauter_q=14)
    rng = np.random.default_rng(case)
    i = rng.integers(0, len(t), 400)
    cand = []
    for a in i:
        for b in range(len(t)):
            if shared_vertices(t, np.array([a]), np.array([b]))[0] == case:
                cand.append((a, b))
                break
    cand = cand[:3]
    assert len(cand) == 3
    for a, b in cand:
        got = gal.entries(np.array([a]), np.array([b]))[0]
        ref = reference_integral(v[t[a]], v[t[b]]) / (4 * np.pi)
        assert abs(got - ref) <= 1e-10 * abs(ref), (case, a, b)


@pytest.mark.parametrize("name,bound", [("identical", 2e-6), ("edge", 1e-7), ("vertex", 1e-6),
                                        ("edge_coplanar", 3e-6), ("vertex_coplanar", 3e-7)])
def test_default_order_error_bound(name, bound):
    # the order used by the build (q = 5): its error against the reference
    # (measured 1e-6, 4e-8, 4e-7, 1.6e-6, 1.1e-7; it falls by about three
    # orders of magnitude for every three orders of q, to 1e-15 at q = 14)
    case, P, Q = PAIRS[name]
    ref = reference_integral(P, Q)
    got = sauter.integrate(case, np.array([P]), np.array([Q]),
                           lambda x, y: 1.0 / np.sqrt(((x - y) ** 2).sum(-1)), 5)[0]
    assert abs(got - ref) <= bound * abs(ref), (name, abs(got - ref) / abs(ref))
