"""GPU parity of the double-layer operator K (gca_build_double_layer)
against the float64 oracle (oracle/double_layer.py) on the 1280-triangle
sphere and an ellipsoid (leaf 32 / 16, eta 2, m = 3, tol 1e-6, q = 5):

* integer results exactly: the row ranks and pivots (the single layer's),
  the column ranks and pivots tilde-sigma', the block lists;
* float64 coefficients within a relative 1e-10: row bases V, E, column
  bases W, F, couplings K|tilde-tau x tilde-sigma', near field (including
  the Sauter-Schwab entries of touching pairs);
* products K x and K^T x (different: K is not symmetric) in float64 within
  1e-10 of the oracle's, float32 within 1e-6, bfloat16 within 1.6e-2 per
  right-hand side; the adjoint identity;
* at the bench size (20480 triangles, leaf 64, m = 4, tol 1e-8): sampled
  entries, column leaf bases from the oracle's own column Green matrix and
  cross approximation, and sampled rows of the dense K against the product.
"""

import numpy as np
import pytest

import sampling
import synth
from oracle import cluster, double_layer as odl, gca as ogca
from oracle.params import Params as OParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32, TOL16 = 1e-10, 1e-6, 1.6e-2


@pytest.fixture(scope="module")
def lib():
    import paper_1810_08429_b300 as gca
    assert torch.cuda.is_available()
    return gca


def _gpu_params(lib, p):
    return lib.Params(leaf_size=p.leaf_size, eta=p.eta, box_gauss_m=p.box_gauss_m, aca_tol=p.aca_tol,
                      sauter_q=p.sauter_q)


@pytest.fixture(scope="module", params=[("sphere1280", 32), ("ellipsoid1280", 16)])
def dl_pair(lib, request):
    name, leaf = request.param
    v, t = synth.mesh_for_config(name)
    p = OParams(leaf_size=leaf, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    ref = odl.build_dl_h2(v, t, p)
    tree = lib.tree_build(v, t, leaf)
    h = lib.build_double_layer(v, t, tree, _gpu_params(lib, p))
    return v, t, tree, ref, h, h.export(), h.export_columns()


def _check_bases(bases, rank, pivots, Vflat, Eflat, tree, tol):
    nc = len(tree["begin"])
    assert np.array_equal(rank, bases.rank.astype(np.int32))
    at = 0
    for c in range(nc):
        got = pivots[at:at + rank[c]]
        at += rank[c]
        if c:
            assert np.array_equal(got, bases.pivots[c]), f"pivots of cluster {c}"
    sz = lambda c: tree["end"][c] - tree["begin"][c]  # noqa: E731
    par = cluster.parents({k: np.asarray(v) for k, v in tree.items()})
    at = 0
    scale = max([np.abs(m).max() for m in bases.V.values() if m.size] + [1.0])
    for c in range(1, nc):
        if tree["child0"][c] >= 0:
            continue
        blk = Vflat[at:at + sz(c) * rank[c]].reshape(sz(c), rank[c])
        at += sz(c) * rank[c]
        if blk.size:
            assert np.abs(blk - bases.V[c]).max() <= tol * scale, f"basis of leaf {c}"
    assert at == len(Vflat)
    at = 0
    scale = max([np.abs(m).max() for m in bases.E.values() if m.size] + [1.0])
    for c in range(1, nc):
        if par[c] <= 0:
            continue
        blk = Eflat[at:at + rank[c] * rank[par[c]]].reshape(rank[c], rank[par[c]])
        at += rank[c] * rank[par[c]]
        if blk.size:
            assert np.abs(blk - bases.E[c]).max() <= tol * scale, f"transfer of cluster {c}"
    assert at == len(Eflat)


def test_bases_match_oracle(dl_pair):
    v, t, tree, ref, h, d, dc = dl_pair
    _check_bases(ref.rows, d["rank"], d["pivots"], d["V"], d["E"], tree, TOL64)
    _check_bases(ref.cols, dc["rank"], dc["pivots"], dc["W"], dc["F"], tree, TOL64)
    assert set(map(tuple, d["far"].tolist())) == set(ref.far)
    assert set(map(tuple, d["near"].tolist())) == set(ref.near)
    assert h.column_stats()["op"] == 1


def test_entries_match_oracle(dl_pair):
    v, t, tree, ref, h, d, dc = dl_pair
    r, r2 = d["rank"], dc["rank"]
    at = 0
    scale = max(np.abs(m).max() for m in ref.S.values())
    for (a, b) in map(tuple, d["far"].tolist()):
        blk = d["S"][at:at + r[a] * r2[b]].reshape(r[a], r2[b])
        at += r[a] * r2[b]
        assert np.abs(blk - ref.S[(a, b)]).max() <= TOL64 * scale, f"coupling {(a, b)}"
    assert at == len(d["S"])
    sz = lambda c: tree["end"][c] - tree["begin"][c]  # noqa: E731
    at = 0
    scale = max(np.abs(m).max() for m in ref.N.values())
    for (a, b) in map(tuple, d["near"].tolist()):
        blk = d["N"][at:at + sz(a) * sz(b)].reshape(sz(a), sz(b))
        at += sz(a) * sz(b)
        assert np.abs(blk - ref.N[(a, b)]).max() <= TOL64 * scale, f"near {(a, b)}"
    st = h.stats()
    assert st["n_singular"][3] == len(t)  # identical pairs, all zero


def _rel(y, want):
    y = np.asarray(y).reshape(len(y), -1)
    want = np.asarray(want).reshape(len(want), -1)
    return (np.linalg.norm(y - want, axis=0) / np.linalg.norm(want, axis=0)).max()


@pytest.mark.parametrize("prec,tol", [("f64", TOL64), ("f32", TOL32), ("bf16", TOL16)])
def test_products_match_oracle(dl_pair, prec, tol):
    v, t, tree, ref, h, d, dc = dl_pair
    x = synth.normal_rhs(len(t), 5, seed=7)
    dt = torch.float64 if prec == "f64" else torch.float32
    xd = torch.from_numpy(x).to(dt).cuda()
    y = h.matvec(xd, prec).double().cpu().numpy()
    yt = h.matvec(xd, prec, transpose=True).double().cpu().numpy()
    want, want_t = odl.matvec(ref, x), odl.matvec_t(ref, x)
    assert _rel(y, want) <= tol
    assert _rel(yt, want_t) <= tol
    assert _rel(want_t, want) > 1e-3  # the transpose is a different operator
    if prec != "bf16":
        assert _rel(h.matvec_noalloc(xd, prec).double().cpu().numpy(), want) <= tol
    h.check()


def test_adjoint_identity(dl_pair):
    v, t, tree, ref, h, d, dc = dl_pair
    a = torch.from_numpy(synth.normal_rhs(len(t), 3, seed=1)).cuda()
    b = torch.from_numpy(synth.normal_rhs(len(t), 3, seed=2)).cuda()
    lhs = (a * h.matvec(b, "f64")).sum(0)
    rhs = (h.matvec(a, "f64", transpose=True) * b).sum(0)
    scale = a.norm(dim=0) * h.matvec(b, "f64").norm(dim=0)
    assert ((lhs - rhs).abs() / scale).max() <= 1e-13


def test_bench_size_samples(lib):
    """20480-triangle sphere with the bench parameters: sampled couplings
    and near entries (touching pairs included), column leaf bases from the
    oracle's column Green matrix and cross approximation on that leaf, and
    sampled rows of the dense K against the float64 product."""
    CFG = dict(leaf_size=64, eta=2.0, box_gauss_m=4, aca_tol=1e-8, sauter_q=5)
    v, t = synth.mesh_for_config("perturbed20480")
    p = OParams(**CFG)
    tree = lib.tree_build(v, t, 64)
    h = lib.build_double_layer(v, t, tree, lib.Params(**CFG))
    d = h.export()
    dc = h.export_columns()
    otree, lo, hi, far, near = sampling.oracle_geometry(v, t, p)
    sampling.check_tree(tree, otree)
    sampling.check_blocks(d, far, near)
    dl = odl.DoubleLayer(v, t, 5)
    rng = np.random.default_rng(20480)
    # near entries (touching pairs and identical triangles included), relative
    # to the largest sampled entry: identical flat triangles give exactly 0
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
    want = dl.entries(ii, jj)
    assert np.all(got[want == 0.0] == 0.0)
    assert (np.abs(got - want) / np.abs(want).max()).max() <= 1e-10
    # couplings: rows of tilde-tau against columns of tilde-sigma'
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
    want = dl.entries(ii, jj)
    assert (np.abs(got - want) / np.abs(want).max()).max() <= 1e-10
    # column leaf bases (the column analogue of sampling.check_leaf_bases)
    diam = cluster.diameter(lo, hi)
    needed = ogca.needed_clusters(otree, [tuple(b) for b in fr.tolist()])
    voff, at = {}, 0
    for c in range(1, len(otree["begin"])):
        if otree["child0"][c] < 0:
            voff[c] = at
            at += (otree["end"][c] - otree["begin"][c]) * r2[c]
    cand = [c for c in voff if needed[c]]
    for c in rng.choice(cand, 4, replace=False):
        rows = otree["perm"][otree["begin"][c]:otree["end"][c]]
        z, nrm, w = ogca.omega_rule(lo[c], hi[c], diam[c], p.margin(), p.box_gauss_m)
        A = odl.column_green_matrix(dl, rows, z, nrm, w, diam[c])
        res = ogca.aca(A, p.aca_tol, p.tie_rel)
        piv = dc["pivots"][poff2[c]:poff2[c] + r2[c]]
        W = dc["W"][voff[c]:voff[c] + len(rows) * r2[c]].reshape(len(rows), r2[c])
        if len(res.rows) == r2[c] and np.array_equal(piv, rows[res.rows]):
            assert np.abs(W - res.V).max() <= 1e-8 * max(np.abs(res.V).max(), 1.0)
        else:  # a late pivot flipped under rounding: W must still interpolate A
            pos = np.array([int(np.nonzero(rows == q)[0][0]) for q in piv])
            assert np.abs(W[pos, :] - np.eye(r2[c])).max() <= 1e-12
            assert np.abs(A - W @ A[pos, :]).max() <= 10 * p.aca_tol * np.abs(A).max()
    # dense rows of K against the float64 product
    x = synth.normal_rhs(len(t), 2, seed=4)
    y = h.matvec(torch.from_numpy(x).cuda(), "f64").cpu().numpy()
    for i in rng.choice(len(t), 3, replace=False):
        k = dl.block(np.array([i]), np.arange(len(t)))[0]
        err = np.abs(y[i] - k @ x) / (np.abs(k) @ np.abs(x))
        assert err.max() <= 1e-5, (i, err)
