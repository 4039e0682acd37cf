"""Oracle of curved triangles for the nodal basis (Sect. 6) against what the
paper and the mathematics fix: flat midpoints give back the flat nodal
matrix, the Gramian interpolated through the six nodes (the paper's recipe)
equals the one from the derivative of the map, the curved unit sphere's area
and the constant-density identity converge at fourth order (second for flat
triangles, the paper's reason for curving them), symmetry and positive
definiteness, the singular rules converging in q, and the H^2 product
against the dense matrix."""

import numpy as np
import pytest

import synth
from oracle import cluster, curved, h2, p1
from oracle.params import Params
from oracle.rules import RADON7, triangle_areas

SPHERES = {1: "sphere80", 2: "sphere320", 3: "sphere1280", 4: "sphere5120"}


def _curved(level):
    name = SPHERES[level]
    v, t = synth.mesh_for_config(name)
    return v, t, synth.edge_midpoints_for_config(name)


def test_flat_midpoints_give_the_flat_matrix():
    v, t, _ = _curved(1)
    flat = 0.5 * (v[t] + v[t][:, [1, 2, 0], :])
    A = p1.P1Galerkin(v, t, 5).dense_matrix()
    B = curved.P1CurvedGalerkin(v, t, flat, 5).dense_matrix()
    assert np.abs(A - B).max() <= 1e-13 * np.abs(A).max()


def test_midpoints_follow_their_edges():
    """A midpoint assigned to the wrong edge changes the curved entries."""
    v, t, m = _curved(1)
    good = curved.P1CurvedGalerkin(v, t, m, 5)
    bad = curved.P1CurvedGalerkin(v, t, m[:, [1, 2, 0], :], 5)
    idx = np.arange(len(v))[:6]
    assert np.abs(good.block(idx, idx) - bad.block(idx, idx)).max() > 1e-4 * np.abs(good.block(idx, idx)).max()


def test_gramian_by_interpolated_normal():
    v, t, m = _curved(2)
    X6 = curved.curved_nodes(v, t, m)
    lam = np.random.default_rng(0).dirichlet([1, 1, 1], size=40)
    for k in range(0, len(t), 37):
        a = curved.gramian(X6[k], lam)
        b = curved.gramian_interpolated(X6[k], lam)
        assert np.abs(a - b).max() <= 1e-14 * a.max()
    # flat nodes: twice the triangle area everywhere
    flat = np.concatenate([v[t], 0.5 * (v[t] + v[t][:, [1, 2, 0], :])], axis=1)
    assert np.allclose(curved.gramian(flat[:, None], lam[None, :3]), 2 * triangle_areas(v, t)[:, None],
                       rtol=1e-13, atol=0)


def test_sphere_area_converges_at_fourth_order():
    err_c, err_f = [], []
    for L in (1, 2, 3, 4):
        v, t, m = _curved(L)
        _, w = curved.curved_points(curved.curved_nodes(v, t, m))
        err_c.append(abs(w.sum() - 4 * np.pi))
        err_f.append(abs(triangle_areas(v, t).sum() - 4 * np.pi))
    rc = np.array(err_c[:-1]) / np.array(err_c[1:])
    rf = np.array(err_f[:-1]) / np.array(err_f[1:])
    assert np.all(rc > 14.0) and np.all(rc < 17.0), rc
    assert np.all(rf > 3.5) and np.all(rf < 4.5), rf


@pytest.fixture(scope="module")
def dense_curved():
    out = {}
    for L in (1, 2):
        v, t, m = _curved(L)
        gal = curved.P1CurvedGalerkin(v, t, m, 5)
        out[L] = (v, t, gal, gal.dense_matrix())
    return out


def _load(gal):
    """int phi_i over the curved triangles (7-point rule with the Gramian)."""
    bary, _ = RADON7
    load = np.zeros(gal.n)
    for c in range(3):
        np.add.at(load, gal.t[:, c], (gal.wts * bary[None, :, c]).sum(axis=1))
    return load


def test_constant_density_identity_converges_at_fourth_order(dense_curved):
    """On the unit sphere the single-layer potential of density 1 is 1, so
    sum_j g_ij -> int phi_i; with curved triangles the error falls by about
    16 per refinement (flat triangles: 4)."""
    errs = []
    for L in (1, 2):
        v, t, gal, G = dense_curved[L]
        load = _load(gal)
        errs.append(np.abs(G.sum(axis=1) - load).max() / load.max())
    assert errs[1] < 1e-4
    assert errs[0] / errs[1] > 12.0, errs


def test_dense_symmetric_positive_definite(dense_curved):
    _, _, _, G = dense_curved[2]
    # exact up to the touching pairs, whose two orders agree to the quadrature error
    assert np.abs(G - G.T).max() <= 1e-6 * np.abs(G).max()
    assert np.linalg.eigvalsh(0.5 * (G + G.T)).min() > 0.0


@pytest.mark.parametrize("case", [1, 2, 3])
def test_singular_rules_converge_in_q(case):
    v, t, m = _curved(2)
    X6 = curved.curved_nodes(v, t, m)
    ti = 5
    if case == 3:
        si = ti
    else:
        sh = [(t[s] == t[ti][:, None]).any(axis=0).sum() for s in range(len(t))]
        si = int(np.nonzero(np.array(sh) == case)[0][0])
    vals = [curved.local_singular_curved(X6, t[ti], t[si], X6[ti], X6[si], case, q) for q in (4, 6, 8, 12)]
    d = [np.abs(vals[k] - vals[-1]).max() / np.abs(vals[-1]).max() for k in range(3)]
    assert d[2] < 1e-8 and d[0] > d[1] > d[2], d


def test_curved_h2_product_against_dense(dense_curved):
    v, t, gal, G = dense_curved[2]
    m = synth.edge_midpoints_for_config(SPHERES[2])
    prm = Params(leaf_size=8, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    H = curved.build_p1c_h2(v, t, m, prm)
    assert H.n == len(v) and len(H.far) > 0
    x = np.random.default_rng(1).standard_normal((len(v), 2))
    y = h2.matvec(H, x)
    err = np.linalg.norm(y - G @ x, axis=0) / np.linalg.norm(G @ x, axis=0)
    assert err.max() < 1e-4
    # the cluster boxes hold every node of the curved supports
    ptr, tri, _ = gal.supports
    for c in range(len(H.tree["begin"])):
        idx = H.tree["perm"][H.tree["begin"][c]:H.tree["end"][c]]
        ts = np.concatenate([tri[ptr[i]:ptr[i + 1]] for i in idx])
        pts = gal.X6[ts].reshape(-1, 3)
        assert np.all(pts >= H.lo[c]) and np.all(pts <= H.hi[c])
    assert cluster.is_leaf(H.tree, int(np.argmax(H.tree["level"])))
