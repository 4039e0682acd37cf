"""GPU parity of the collocation variant (gca_build_collocation) against the
float64 oracle (oracle/collocation.py) on the 1280-triangle sphere and an
ellipsoid: row ranks and pivots (collocation Green matrices) and column
ranks and pivots (the Galerkin single layer's) exactly; V, E, W, F,
couplings and near field (Duffy diagonal included) within 1e-10; C x and
C^T x within 1e-10 (f64), 1e-6 (f32), 1.6e-2 (bf16); at the bench size,
sampled entries and rows of the dense C against the float64 product.
"""

import numpy as np
import pytest

import sampling
import synth
from oracle import collocation as ocol
from oracle.params import Params as OParams
from test_gpu_double_layer import _check_bases, _rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32, TOL16 = 1e-10, 1e-6, 1.6e-2


@pytest.fixture(scope="module")
def lib():
    import paper_1810_08429_b300 as gca
    assert torch.cuda.is_available()
    return gca


@pytest.fixture(scope="module", params=[("sphere1280", 32), ("ellipsoid1280", 16)])
def col_pair(lib, request):
    name, leaf = request.param
    v, t = synth.mesh_for_config(name)
    p = OParams(leaf_size=leaf, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    ref = ocol.build_col_h2(v, t, p)
    tree = lib.tree_build(v, t, leaf)
    h = lib.build_collocation(v, t, tree, lib.Params(leaf_size=leaf, eta=2.0, box_gauss_m=3, aca_tol=1e-6,
                                                      sauter_q=5))
    return v, t, tree, ref, h, h.export(), h.export_columns()


def test_bases_match_oracle(col_pair):
    v, t, tree, ref, h, d, dc = col_pair
    _check_bases(ref.rows, d["rank"], d["pivots"], d["V"], d["E"], tree, TOL64)
    _check_bases(ref.cols, dc["rank"], dc["pivots"], dc["W"], dc["F"], tree, TOL64)
    assert set(map(tuple, d["far"].tolist())) == set(ref.far)
    assert set(map(tuple, d["near"].tolist())) == set(ref.near)
    assert h.column_stats()["op"] == 2


def test_entries_match_oracle(col_pair):
    v, t, tree, ref, h, d, dc = col_pair
    r, r2 = d["rank"], dc["rank"]
    at = 0
    scale = max(np.abs(m).max() for m in ref.S.values())
    for (a, b) in map(tuple, d["far"].tolist()):
        blk = d["S"][at:at + r[a] * r2[b]].reshape(r[a], r2[b])
        at += r[a] * r2[b]
        assert np.abs(blk - ref.S[(a, b)]).max() <= TOL64 * scale, f"coupling {(a, b)}"
    sz = lambda c: tree["end"][c] - tree["begin"][c]  # noqa: E731
    at = 0
    scale = max(np.abs(m).max() for m in ref.N.values())
    for (a, b) in map(tuple, d["near"].tolist()):
        blk = d["N"][at:at + sz(a) * sz(b)].reshape(sz(a), sz(b))
        at += sz(a) * sz(b)
        assert np.abs(blk - ref.N[(a, b)]).max() <= TOL64 * scale, f"near {(a, b)}"
    assert h.stats()["n_singular"][3] == len(t)  # one Duffy entry per row


@pytest.mark.parametrize("prec,tol", [("f64", TOL64), ("f32", TOL32), ("bf16", TOL16)])
def test_products_match_oracle(col_pair, prec, tol):
    v, t, tree, ref, h, d, dc = col_pair
    x = synth.normal_rhs(len(t), 5, seed=9)
    dt = torch.float64 if prec == "f64" else torch.float32
    xd = torch.from_numpy(x).to(dt).cuda()
    assert _rel(h.matvec(xd, prec).double().cpu().numpy(), ocol.matvec(ref, x)) <= tol
    assert _rel(h.matvec(xd, prec, transpose=True).double().cpu().numpy(), ocol.matvec_t(ref, x)) <= tol
    h.check()


def test_bench_size_samples(lib):
    CFG = dict(leaf_size=64, eta=2.0, box_gauss_m=4, aca_tol=1e-8, sauter_q=5)
    v, t = synth.mesh_for_config("sphere20480")
    p = OParams(**CFG)
    tree = lib.tree_build(v, t, 64)
    h = lib.build_collocation(v, t, tree, lib.Params(**CFG))
    d, dc = h.export(), h.export_columns()
    otree, lo, hi, far, near = sampling.oracle_geometry(v, t, p)
    sampling.check_tree(tree, otree)
    sampling.check_blocks(d, far, near)
    col = ocol.Collocation(v, t, 5)
    rng = np.random.default_rng(5)
    # near entries, the Duffy diagonal included
    nr = d["near"]
    szc = otree["end"] - otree["begin"]
    noff = np.concatenate([[0], np.cumsum(szc[nr[:, 0]] * szc[nr[:, 1]])])
    pick = np.unique(np.concatenate([rng.choice(len(nr), 48, replace=False),
                                     np.nonzero(nr[:, 0] == nr[:, 1])[0][:8]]))
    ii, jj, got = [], [], []
    for b in pick:
        a, s = nr[b]
        ia = rng.integers(0, szc[a], 16)
        ic = rng.integers(0, szc[s], 16)
        if a == s:
            ia[:4] = ic[:4]
        ii.append(otree["perm"][otree["begin"][a] + ia])
        jj.append(otree["perm"][otree["begin"][s] + ic])
        got.append(d["N"][noff[b] + ia * szc[s] + ic])
    ii, jj, got = np.concatenate(ii), np.concatenate(jj), np.concatenate(got)
    want = col.entries(ii, jj)
    assert (np.abs(got - want) / np.abs(want)).max() <= 1e-10
    # couplings
    r, r2 = d["rank"], dc["rank"]
    poff = np.concatenate([[0], np.cumsum(r)])
    poff2 = np.concatenate([[0], np.cumsum(r2)])
    fr = d["far"]
    soff = np.concatenate([[0], np.cumsum(r[fr[:, 0]] * r2[fr[:, 1]])])
    ii, jj, got = [], [], []
    for b in rng.choice(len(fr), 48, replace=False):
        a, s = fr[b]
        ia = rng.integers(0, r[a], 8)
        ic = rng.integers(0, r2[s], 8)
        ii.append(d["pivots"][poff[a] + ia])
        jj.append(dc["pivots"][poff2[s] + ic])
        got.append(d["S"][soff[b] + ia * r2[s] + ic])
    ii, jj, got = np.concatenate(ii), np.concatenate(jj), np.concatenate(got)
    want = col.entries(ii, jj)
    assert (np.abs(got - want) / np.abs(want)).max() <= 1e-10
    # rows of the dense C against the float64 product
    x = synth.normal_rhs(len(t), 2, seed=4)
    y = h.matvec(torch.from_numpy(x).cuda(), "f64").cpu().numpy()
    for i in rng.choice(len(t), 3, replace=False):
        c = col.block(np.array([i]), np.arange(len(t)))[0]
        err = np.abs(y[i] - c @ x) / (np.abs(c) @ np.abs(x))
        assert err.max() <= 1e-5, (i, err)
