"""Pins for the oracle's Galerkin matrix (Eq. (1), piecewise constant basis).

Closed forms on the unit sphere: the single-layer potential of unit density
is 1 on the sphere, so the row sums of G approach the triangle areas, and
the first spherical harmonic is an eigenfunction with eigenvalue 1/3; both
errors fall by about 4 per refinement (O(h^2)).
"""

import numpy as np
import pytest

import synth
from oracle import galerkin
from oracle.galerkin import Galerkin
from oracle.rules import gauss_legendre_01, triangle_areas


@pytest.fixture(scope="module")
def dense_by_level():
    out = {}
    for level in (1, 2, 3):
        v, t = synth.icosphere(level)
        out[level] = (v, t, Galerkin(v, t, 5).dense_matrix())
    return out


def test_unit_density_potential_is_one(dense_by_level):
    errs = []
    for level in (1, 2, 3):
        v, t, G = dense_by_level[level]
        area = triangle_areas(v, t)
        errs.append(np.abs(G.sum(axis=1) / area - 1.0).max())
    assert errs[-1] < 3e-3
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5


def test_first_harmonic_eigenvalue(dense_by_level):
    errs = []
    for level in (1, 2, 3):
        v, t, G = dense_by_level[level]
        area = triangle_areas(v, t)
        zc = ((v[t[:, 0]] + v[t[:, 1]] + v[t[:, 2]]) / 3.0)[:, 2]
        ref = area * zc / 3.0
        errs.append(np.abs(G @ zc - ref).max() / np.abs(ref).max())
    assert errs[-1] < 5e-3
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5


def test_symmetric_up_to_singular_quadrature(dense_by_level):
    v, t, G = dense_by_level[2]
    asym5 = np.abs(G - G.T).max() / np.abs(G).max()
    assert asym5 < 1e-7
    G8 = Galerkin(v, t, 8).dense_matrix()
    asym8 = np.abs(G8 - G8.T).max() / np.abs(G8).max()
    assert asym8 < asym5 / 10
    # regular (disjoint) entries are symmetric to rounding
    case = galerkin.shared_vertices(np.asarray(t, dtype=np.int64),
                                    *np.nonzero(np.ones_like(G, dtype=bool)))
    reg = (case == 0).reshape(G.shape)
    assert np.abs((G - G.T)[reg]).max() <= 1e-15 * np.abs(G).max()


def test_positive_definite(dense_by_level):
    _, _, G = dense_by_level[2]
    np.linalg.cholesky(0.5 * (G + G.T))


def test_classification_brute_force():
    v, t = synth.icosphere(1)
    n = len(t)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    got = galerkin.shared_vertices(np.asarray(t, dtype=np.int64), i.ravel(), j.ravel())
    want = np.array([len(set(t[a]) & set(t[b])) for a, b in zip(i.ravel(), j.ravel())])
    assert np.array_equal(got, want)
    # conforming closed mesh: n identical, 3n ordered edge-neighbour pairs
    assert (got == 3).sum() == n and (got == 2).sum() == 3 * n


def test_regular_rule_against_brute_force():
    """Far pairs: the 7 x 7 rule agrees with a high-order product rule."""
    v, t = synth.icosphere(2)
    gal = Galerkin(v, t, 5)
    c = (v[t[:, 0]] + v[t[:, 1]] + v[t[:, 2]]) / 3.0
    rng = np.random.default_rng(0)
    pairs = []
    while len(pairs) < 20:
        a, b = rng.integers(0, len(t), size=2)
        if np.linalg.norm(c[a] - c[b]) > 1.0:
            pairs.append((a, b))
    tq, wq = gauss_legendre_01(12)
    s, r = np.meshgrid(tq, tq, indexing="ij")
    w = (np.outer(wq, wq) * s).ravel()
    u1, u2 = s.ravel(), (s * r).ravel()
    for a, b in pairs:
        P, Q = v[t[a]], v[t[b]]
        x = P[0] + u1[:, None] * (P[1] - P[0]) + u2[:, None] * (P[2] - P[1])
        y = Q[0] + u1[:, None] * (Q[1] - Q[0]) + u2[:, None] * (Q[2] - Q[1])
        jp = np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[1]))
        jq = np.linalg.norm(np.cross(Q[1] - Q[0], Q[2] - Q[1]))
        ref = np.einsum("a,b,ab->", w, w, 1.0 / np.linalg.norm(
            x[:, None, :] - y[None, :, :], axis=-1)) * jp * jq / (4 * np.pi)
        got = gal.regular(np.array([a]), np.array([b]))[0]
        assert abs(got - ref) < 1e-7 * ref
