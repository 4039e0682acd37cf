"""Pins of the comparison approximations (oracle/comparison.py) on the
1280-triangle sphere against the dense Galerkin matrix G:

* the fast products equal the dense representation (and its transpose);
* pure Green quadrature converges as the box rule's order m grows (Eq. (2)
  is an exact identity discretised by quadrature, Sect. 2);
* single-level GCA: V_tau[tilde-tau, :] = I, the error falls with the
  tolerance, and at equal tolerance it matches GCA-H^2's error while storing
  more (the nested bases' saving, Sect. 4);
* at a comparable error Green quadrature needs far more storage than GCA
  (the paper's observation on Fig. 1-2).
"""

import numpy as np
import pytest

from oracle import comparison as ocmp, gca as ogca, h2 as oh2
from oracle.params import Params


def _err(G, D):
    return np.linalg.norm(G - D, 2) / np.linalg.norm(G, 2)


@pytest.fixture(scope="module")
def gq_runs(sphere1280):
    v, t = sphere1280
    return {m: ocmp.build_gq(v, t, Params(leaf_size=32, eta=2.0, box_gauss_m=m, aca_tol=1e-6, sauter_q=5))
            for m in (2, 3, 4)}


@pytest.fixture(scope="module")
def gca1_runs(sphere1280):
    # leaf 16: admissible blocks on several levels, so that nesting matters
    v, t = sphere1280
    return {tol: ocmp.build_gca1(v, t, Params(leaf_size=16, eta=2.0, box_gauss_m=3, aca_tol=tol, sauter_q=5))
            for tol in (1e-3, 1e-6)}


def test_gq_products_match_dense(gq_runs, sphere1280):
    h = gq_runs[3]
    D = ocmp.gq_dense(h)
    x = np.random.default_rng(0).standard_normal((len(sphere1280[1]), 3))
    assert np.abs(ocmp.gq_matvec(h, x) - D @ x).max() <= 1e-13 * np.abs(D @ x).max()
    assert np.abs(ocmp.gq_matvec(h, x, transpose=True) - D.T @ x).max() <= 1e-13 * np.abs(D.T @ x).max()


def test_gq_converges_in_m(gq_runs, dense_1280):
    errs = [_err(dense_1280, ocmp.gq_dense(gq_runs[m])) for m in (2, 3, 4)]
    assert errs[2] < 0.5 * errs[1] < 0.25 * errs[0]


def test_gca1_products_and_interpolation(gca1_runs, sphere1280):
    h = gca1_runs[1e-6]
    D = ocmp.gca1_dense(h)
    x = np.random.default_rng(1).standard_normal((len(sphere1280[1]), 2))
    assert np.abs(ocmp.gca1_matvec(h, x) - D @ x).max() <= 1e-13 * np.abs(D @ x).max()
    assert np.abs(ocmp.gca1_matvec(h, x, transpose=True) - D.T @ x).max() <= 1e-13 * np.abs(D.T @ x).max()
    tree = h.tree
    for c, V in h.bases.V.items():
        if V.size == 0:
            continue
        rows = tree["perm"][tree["begin"][c]:tree["end"][c]]
        pos = [int(np.nonzero(rows == p)[0][0]) for p in h.bases.pivots[c]]
        assert np.abs(V[pos, :] - np.eye(V.shape[1])).max() <= 1e-13


def test_gca1_against_h2(gca1_runs, sphere1280, dense_1280):
    v, t = sphere1280
    e3 = _err(dense_1280, ocmp.gca1_dense(gca1_runs[1e-3]))
    e6 = _err(dense_1280, ocmp.gca1_dense(gca1_runs[1e-6]))
    assert e6 < 0.1 * e3
    h2 = ogca.build_h2(v, t, Params(leaf_size=16, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5))
    e_h2 = _err(dense_1280, oh2.dense(h2))
    assert e_h2 < 10 * e6 and e6 < 10 * e_h2
    # on this small mesh every child basis has full rank (|tau-hat| <= 2k),
    # so V_tau and [E_1; E_2] have the same size
    assert oh2.storage(h2)["total"] <= ocmp.gca1_storage(gca1_runs[1e-6])["total"]


def test_nesting_saves_storage_once_ranks_saturate():
    # 5120 triangles: clusters above the leaves hold more than 2k triangles,
    # their children's ranks saturate and [E_1; E_2] is smaller than V_tau
    import synth
    from oracle import cluster
    from oracle.galerkin import Galerkin
    v, t = synth.mesh_for_config("sphere5120")
    p = Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    gal = Galerkin(v, t, 5)
    tree = cluster.build_tree(v, t, p.leaf_size)
    lo, hi = cluster.cluster_boxes(v, t, tree)
    far, near = cluster.block_tree(tree, lo, hi, p.eta)
    nested = ogca.build_bases(gal, tree, lo, hi, p, far)
    single = ogca.build_bases(gal, tree, lo, hi, p, far, nested=False)
    s_nested = sum(m.size for m in nested.V.values()) + sum(m.size for m in nested.E.values())
    inblock = {c for b in far for c in b}
    s_single = sum(single.V[c].size for c in inblock)
    assert s_nested < 0.9 * s_single  # measured 0.86 at this size; the saving grows with n


def test_gq_needs_more_storage(gq_runs, gca1_runs, dense_1280):
    # Green quadrature at m = 4 is less accurate than single-level GCA at
    # tolerance 1e-6 and stores more
    e_gq = _err(dense_1280, ocmp.gq_dense(gq_runs[4]))
    e_gca = _err(dense_1280, ocmp.gca1_dense(gca1_runs[1e-6]))
    assert e_gq > e_gca
    assert ocmp.gq_storage(gq_runs[4])["total"] > ocmp.gca1_storage(gca1_runs[1e-6])["total"]
