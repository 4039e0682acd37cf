"""Pins of the collocation oracle (oracle/collocation.py), independent of
its own code:

* the Duffy value c_ii against the closed-form potential of a flat triangle
  at its centroid (the formula pinned in test_oracle_singular_pin.py);
* the unit-density potential on the unit sphere equals 1, so sum_j c_ij
  approaches 1 at O(h^2) as the icosphere refines;
* the rows' Green matrix at collocation points times the Galerkin factor B
  converging to the entry (Green's formula, Eq. (2)) as m grows;
* H^2: fast product = explicit bases, adjoint identity, spectral error
  falling with the tolerance; the column bases are the Galerkin ones.
"""

import numpy as np
import pytest

import synth
from oracle import collocation as ocol, gca as ogca
from oracle.params import Params
from oracle.rules import box_rule
from test_oracle_singular_pin import triangle_potential


@pytest.mark.parametrize("name", ["sphere80", "perturbed320"])
def test_duffy_matches_closed_form(name):
    v, t = synth.mesh_for_config(name)
    col = ocol.Collocation(v, t, q=12)
    for i in (0, 7, 33):
        got = col.duffy([i])[0] * 4 * np.pi
        want = triangle_potential(col.xc[i][None, :], v[t[i]])[0]
        assert abs(got - want) <= 1e-12 * want


def test_duffy_default_order():
    v, t = synth.mesh_for_config("perturbed320")
    col = ocol.Collocation(v, t, q=5)
    errs = [abs(col.duffy([i])[0] * 4 * np.pi - triangle_potential(col.xc[i][None, :], v[t[i]])[0])
            / triangle_potential(col.xc[i][None, :], v[t[i]])[0] for i in range(0, 320, 40)]
    assert max(errs) <= 1e-8  # q = 5 (20 points a edge)


def test_unit_density_on_the_sphere():
    errs = []
    for name in ("sphere80", "sphere320", "sphere1280"):
        v, t = synth.mesh_for_config(name)
        col = ocol.Collocation(v, t, 5)
        idx = np.arange(len(t))
        rows = idx[::max(1, len(t) // 64)]
        s = col.block(rows, idx).sum(axis=1)
        errs.append(np.abs(s - 1.0).max())
    assert errs[1] < 0.35 * errs[0] and errs[2] < 0.35 * errs[1]
    assert errs[2] < 5e-3


def test_collocation_green_matrix_reproduces_entries():
    v, t = synth.mesh_for_config("sphere320")
    col = ocol.Collocation(v, t, 5)
    from oracle.galerkin import Galerkin
    gal = Galerkin(v, t, 5)
    rows = np.array([0, 1, 2, 3])
    cen = v[t].mean(axis=1)
    far = int(np.argmax(np.linalg.norm(cen - cen[0], axis=1)))
    cols = np.array([far])
    pts = v[t[rows]].reshape(-1, 3)
    lo, hi = pts.min(0), pts.max(0)
    d = np.linalg.norm(hi - lo)
    want = col.block(rows, cols)[:, 0]
    errs = []
    for m in (2, 4, 6, 8, 10):
        z, nz, w = box_rule(lo - 0.25 * d, hi + 0.25 * d, m)
        A = ocol.collocation_green_matrix(col, rows, z, nz, w, d)
        B = ogca.green_factor_b(gal, cols, z, nz, w, d)
        errs.append(np.abs(A @ B.T[:, 0] - want).max() / np.abs(want).max())
    assert errs[-1] < 1e-5
    assert all(b < a for a, b in zip(errs, errs[1:]))


@pytest.fixture(scope="module")
def col1280():
    v, t = synth.mesh_for_config("sphere1280")
    p = Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    h = ocol.build_col_h2(v, t, p)
    assert len(h.far) > 0
    return v, t, p, h


def test_columns_are_the_galerkin_bases(col1280):
    v, t, p, h = col1280
    hs = ogca.build_h2(v, t, p)
    for c in range(len(h.tree["begin"])):
        assert np.array_equal(h.cols.pivots[c], hs.bases.pivots[c])
    differ = sum(not np.array_equal(h.rows.pivots[c], hs.bases.pivots[c]) for c in range(len(h.tree["begin"])))
    assert differ > 0


def test_fast_product_equals_explicit_and_adjoint(col1280):
    v, t, p, h = col1280
    C = ocol.dense(h)
    x = synth.uniform_rhs(len(t), 3, seed=2)
    assert np.abs(ocol.matvec(h, x) - C @ x).max() <= 1e-13 * np.abs(C @ x).max()
    assert np.abs(ocol.matvec_t(h, x) - C.T @ x).max() <= 1e-13 * np.abs(C.T @ x).max()


def test_spectral_error_falls_with_tolerance(col1280):
    v, t, p, h6 = col1280
    C = ocol.Collocation(v, t, 5).dense_matrix()
    nc = np.linalg.norm(C, 2)
    h3 = ocol.build_col_h2(v, t, Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-3, sauter_q=5))
    e3 = np.linalg.norm(C - ocol.dense(h3), 2) / nc
    e6 = np.linalg.norm(C - ocol.dense(h6), 2) / nc
    assert 0.0 < e6 < 0.1 * e3
    assert e6 < 1e-5
