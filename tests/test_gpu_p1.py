"""GPU parity of the nodal (continuous piecewise linear) basis of Sect. 5
(gca_build_p1, gca_support_union) against the float64 oracle (oracle/p1.py):

* integer results exactly: the support unions of the device's mergesort
  (the paper's worked example, random vertex subsets, cluster ranges), the
  vertex tree and the block lists; the pivots replayed by the oracle's cross
  approximation (each within 1e-7 of its largest residual, the ranks
  agreeing with its stopping rule);
* float64 coefficients within a relative 1e-10: leaf bases V, transfers E,
  couplings G|tilde-tau x tilde-sigma and the near field (touching pairs by
  Sauter-Schwab with barycentric weights included) on the 1280-triangle
  sphere (642 vertices, leaf 32) and ellipsoid (leaf 16), eta 2, m = 3,
  tol 1e-6, q = 5, against the oracle built on the GPU's pivots;
* products in float64 within 1e-10 of the oracle's H^2 product, float32
  within 1e-6, bfloat16 within 1.6e-2 per right-hand side; the transpose
  (G is symmetric) and the no-allocation product; the oracle's H^2
  imported (construction bypassed);
* at the bench size (the 20480-triangle sphere: 10242 vertices, leaf 64,
  m = 4, tol 1e-8): the oracle's vertex tree and block tree, sampled near
  and coupling entries, leaf bases from the oracle's own Green matrix and
  cross approximation, and rows of the dense nodal matrix against the
  float64 product.
"""

import os

import numpy as np
import pytest

import sampling
import synth
from oracle import cluster, gca as ogca, h2 as oh2, p1 as op1
from oracle.params import Params as OParams
from oracle_dump import oracle_dump

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32, TOL16 = 1e-10, 1e-6, 1.6e-2
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "p1_support_union.txt")


@pytest.fixture(scope="module")
def lib():
    import paper_1810_08429_b300 as gca
    assert torch.cuda.is_available()
    return gca


def _gpu_params(lib, p):
    return lib.Params(leaf_size=p.leaf_size, eta=p.eta, box_gauss_m=p.box_gauss_m, aca_tol=p.aca_tol,
                      sauter_q=p.sauter_q)


def _golden_example():
    tris, tau = [], None
    with open(GOLDEN) as f:
        for line in f:
            w = line.split()
            if w and w[0] == "triangle":
                tris.append([int(a) - 1 for a in w[2:5]])
            elif w and w[0] == "tau":
                tau = [int(a) - 1 for a in w[1:]]
    return np.array(tris), tau


def test_support_union_worked_example(lib):
    """The worked example of Sect. 5 through the device's mergesort."""
    tris, tau = _golden_example()
    nv = int(tris.max()) + 1
    # any coordinates: the union depends on the connectivity only
    rng = np.random.default_rng(0)
    v = rng.normal(size=(nv, 3))
    sup = op1.vertex_supports(nv, tris)
    got = lib.support_union(v, tris, [tau])[0]
    assert got == op1.support_union(sup, tau)


def test_support_union_matches_oracle(lib):
    v, t = synth.mesh_for_config("perturbed20480")
    sup = op1.vertex_supports(len(v), t)
    rng = np.random.default_rng(5)
    tree = lib.tree_build_points(v, 64)
    lists = [np.array([], dtype=np.int64), np.array([17])]
    for c in rng.choice(len(tree["begin"]), 12, replace=False):  # cluster ranges (near-field rows)
        lists.append(tree["perm"][tree["begin"][c]:tree["end"][c]][:400])
    for size in (3, 40, 97, 192, 431):  # scattered subsets (pivot lists)
        lists.append(rng.choice(len(v), size, replace=False))
    got = lib.support_union(v, t, lists)
    for a, g in zip(lists, got):
        assert g == op1.support_union(sup, [int(i) for i in a])


def test_support_union_rejects_bad_lists(lib):
    v, t = synth.mesh_for_config("sphere320")
    with pytest.raises(lib.GCAError):
        lib.support_union(v, t, [np.array([3, 3])])
    with pytest.raises(lib.GCAError):
        lib.support_union(v, t, [np.array([len(v)])])


@pytest.fixture(scope="module", params=[("sphere1280", 32), ("ellipsoid1280", 16)])
def p1_pair(lib, request):
    """The GPU handle and the oracle's H^2 built on the GPU's pivot
    sequences (late pivots whose residuals agree to rounding may come in
    either order; the replay measures how far each pivot lies below the
    largest residual of the oracle's own residual matrix)."""
    name, leaf = request.param
    v, t = synth.mesh_for_config(name)
    p = OParams(leaf_size=leaf, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    tree = lib.tree_build_points(v, leaf)
    h = lib.build_p1(v, t, tree, _gpu_params(lib, p))
    d = h.export()
    poff = np.concatenate([[0], np.cumsum(d["rank"])])
    follow = {c: d["pivots"][poff[c]:poff[c + 1]] for c in range(1, len(tree["begin"])) if d["rank"][c]}
    ref = op1.build_p1_h2(v, t, p, follow=follow)
    return v, t, tree, ref, h, d


def test_structure_matches_oracle(p1_pair):
    v, t, tree, ref, h, d = p1_pair
    otree = ref.tree
    for k in ("perm", "begin", "end", "child0", "child1", "level"):
        assert np.array_equal(np.asarray(otree[k]), tree[k]), k
    assert [tuple(b) for b in d["far"].tolist()] == sorted(ref.far)
    assert [tuple(b) for b in d["near"].tolist()] == sorted(ref.near)
    assert np.array_equal(d["rank"], ref.bases.rank.astype(np.int32))
    # every cluster the oracle needs has a GPU pivot sequence, and each GPU
    # pivot is the oracle's largest residual up to rounding: at most 1e-7
    # relative below it, the stopping rule agreeing on the rank
    needed = ogca.needed_clusters(otree, ref.far)
    assert set(ref.bases.replay) == {c for c in range(1, len(otree["begin"])) if needed[c]}
    for c, (gap, (low, after)) in ref.bases.replay.items():
        assert gap <= 1e-7, (c, gap)
        assert low > 1.0 - 1e-7 and after <= 1.0 + 1e-7, (c, low, after)
    assert h.stats()["n"] == len(v)


def test_coefficients_match_oracle(p1_pair):
    v, t, tree, ref, h, d = p1_pair
    r = d["rank"]
    nc = len(tree["begin"])
    sz = lambda c: tree["end"][c] - tree["begin"][c]  # noqa: E731
    par = cluster.parents({k: np.asarray(a) for k, a in tree.items()})
    at = 0
    scale = max([np.abs(m).max() for m in ref.bases.V.values() if m.size] + [1.0])
    for c in range(1, nc):
        if tree["child0"][c] >= 0:
            continue
        blk = d["V"][at:at + sz(c) * r[c]].reshape(sz(c), r[c])
        at += sz(c) * r[c]
        if blk.size:
            assert np.abs(blk - ref.bases.V[c]).max() <= TOL64 * scale, f"basis of leaf {c}"
    at = 0
    scale = max([np.abs(m).max() for m in ref.bases.E.values() if m.size] + [1.0])
    for c in range(1, nc):
        if par[c] <= 0:
            continue
        blk = d["E"][at:at + r[c] * r[par[c]]].reshape(r[c], r[par[c]])
        at += r[c] * r[par[c]]
        if blk.size:
            assert np.abs(blk - ref.bases.E[c]).max() <= TOL64 * scale, f"transfer of cluster {c}"
    at = 0
    scale = max(np.abs(m).max() for m in ref.S.values())
    for (a, b) in map(tuple, d["far"].tolist()):
        blk = d["S"][at:at + r[a] * r[b]].reshape(r[a], r[b])
        at += r[a] * r[b]
        assert np.abs(blk - ref.S[(a, b)]).max() <= TOL64 * scale, f"coupling {(a, b)}"
    at = 0
    scale = max(np.abs(m).max() for m in ref.N.values())
    for (a, b) in map(tuple, d["near"].tolist()):
        blk = d["N"][at:at + sz(a) * sz(b)].reshape(sz(a), sz(b))
        at += sz(a) * sz(b)
        assert np.abs(blk - ref.N[(a, b)]).max() <= TOL64 * scale, f"near {(a, b)}"
    st = h.stats()
    assert st["n_singular"][3] > 0 and st["n_singular"][2] > 0 and st["n_singular"][1] > 0


def _rel(y, want):
    y = np.asarray(y).reshape(len(y), -1)
    want = np.asarray(want).reshape(len(want), -1)
    return (np.linalg.norm(y - want, axis=0) / np.linalg.norm(want, axis=0)).max()


@pytest.mark.parametrize("prec,tol", [("f64", TOL64), ("f32", TOL32), ("bf16", TOL16)])
def test_products_match_oracle(p1_pair, prec, tol):
    v, t, tree, ref, h, d = p1_pair
    x = synth.normal_rhs(len(v), 5, seed=7)
    dt = torch.float64 if prec == "f64" else torch.float32
    xd = torch.from_numpy(x).to(dt).cuda()
    want, want_t = oh2.matvec(ref, x), oh2.matvec_t(ref, x)
    assert _rel(h.matvec(xd, prec).double().cpu().numpy(), want) <= tol
    # G is symmetric up to the quadrature error of the touching pairs (their
    # rules follow the order of the pair): the transpose matches the
    # oracle's transposed product, and the product itself to that error
    assert _rel(h.matvec(xd, prec, transpose=True).double().cpu().numpy(), want_t) <= tol
    assert _rel(want_t, want) <= 1e-6
    if prec != "bf16":
        assert _rel(h.matvec_noalloc(xd, prec).double().cpu().numpy(), want) <= tol
    h.check()


def test_imported_oracle_h2(lib, p1_pair):
    """The oracle's nodal H^2 imported (construction bypassed), multiplied."""
    v, t, tree, ref, h, d = p1_pair
    hi = lib.import_h2(tree, len(v), oracle_dump(ref))
    x = synth.normal_rhs(len(v), 3, seed=3)
    y = hi.matvec(torch.from_numpy(x).cuda(), "f64").cpu().numpy()
    assert _rel(y, oh2.matvec(ref, x)) <= TOL64


def test_bench_size_samples(lib):
    """The 20480-triangle sphere (10242 vertices) with the bench parameters."""
    CFG = dict(leaf_size=64, eta=2.0, box_gauss_m=4, aca_tol=1e-8, sauter_q=5)
    v, t = synth.mesh_for_config("sphere20480")
    p = OParams(**CFG)
    tree = lib.tree_build_points(v, 64)
    h = lib.build_p1(v, t, tree, lib.Params(**CFG))
    d = h.export()
    gal = op1.P1Galerkin(v, t, 5)
    otree = op1.build_tree_points(v, 64)
    sampling.check_tree(tree, otree)
    lo, hi = op1.cluster_boxes_p1(v, t, gal.supports, otree)
    far, near = cluster.block_tree(otree, lo, hi, p.eta)
    sampling.check_blocks(d, far, near)
    rng = np.random.default_rng(10242)
    szc = otree["end"] - otree["begin"]
    # near entries: sampled rows x columns of sampled blocks (diagonal blocks
    # included: every touching case), relative to the largest entry
    nr = d["near"]
    noff = np.concatenate([[0], np.cumsum(szc[nr[:, 0]] * szc[nr[:, 1]])])
    pick = np.unique(np.concatenate([rng.choice(len(nr), 24, replace=False),
                                     np.nonzero(nr[:, 0] == nr[:, 1])[0][:6]]))
    worst, top = 0.0, 0.0
    for b in pick:
        a, s = nr[b]
        ia = np.unique(rng.integers(0, szc[a], 6))
        ic = np.unique(rng.integers(0, szc[s], 6))
        if a == s:
            ic = np.unique(np.concatenate([ic, ia]))
        want = gal.block(otree["perm"][otree["begin"][a] + ia], otree["perm"][otree["begin"][s] + ic])
        full = d["N"][noff[b]:noff[b + 1]].reshape(szc[a], szc[s])
        got = full[np.ix_(ia, ic)]
        worst = max(worst, np.abs(got - want).max())
        top = max(top, np.abs(want).max())
    assert worst <= 1e-10 * top
    # couplings between pivot vertices
    r = d["rank"]
    poff = np.concatenate([[0], np.cumsum(r)])
    fr = d["far"]
    soff = np.concatenate([[0], np.cumsum(r[fr[:, 0]] * r[fr[:, 1]])])
    worst, top = 0.0, 0.0
    for b in rng.choice(len(fr), 24, replace=False):
        a, s = fr[b]
        ia = np.unique(rng.integers(0, r[a], 5))
        ic = np.unique(rng.integers(0, r[s], 5))
        want = gal.block(d["pivots"][poff[a] + ia], d["pivots"][poff[s] + ic])
        got = d["S"][soff[b]:soff[b + 1]].reshape(r[a], r[s])[np.ix_(ia, ic)]
        worst = max(worst, np.abs(got - want).max())
        top = max(top, np.abs(want).max())
    assert worst <= 1e-10 * top
    # leaf bases from the oracle's nodal Green matrix and cross approximation
    diam = cluster.diameter(lo, hi)
    needed = ogca.needed_clusters(otree, [tuple(b) for b in fr.tolist()])
    voff, at = {}, 0
    for c in range(1, len(otree["begin"])):
        if otree["child0"][c] < 0:
            voff[c] = at
            at += szc[c] * r[c]
    cand = [c for c in voff if needed[c]]
    for c in rng.choice(cand, 4, replace=False):
        rows = otree["perm"][otree["begin"][c]:otree["end"][c]]
        z, nrm, w = ogca.omega_rule(lo[c], hi[c], diam[c], p.margin(), p.box_gauss_m)
        A = op1.green_matrix_p1(gal, rows, z, nrm, w, diam[c])
        res = ogca.aca(A, p.aca_tol, p.tie_rel)
        piv = d["pivots"][poff[c]:poff[c] + r[c]]
        V = d["V"][voff[c]:voff[c] + len(rows) * r[c]].reshape(len(rows), r[c])
        if len(res.rows) == r[c] and np.array_equal(piv, rows[res.rows]):
            assert np.abs(V - res.V).max() <= 1e-8 * max(np.abs(res.V).max(), 1.0)
        else:  # a late pivot flipped under rounding: V must still interpolate A
            pos = np.array([int(np.nonzero(rows == q)[0][0]) for q in piv])
            assert np.abs(V[pos, :] - np.eye(r[c])).max() <= 1e-12
            assert np.abs(A - V @ A[pos, :]).max() <= 10 * p.aca_tol * np.abs(A).max()
    # rows of the dense nodal matrix against the float64 product
    x = synth.normal_rhs(len(v), 2, seed=4)
    y = h.matvec(torch.from_numpy(x).cuda(), "f64").cpu().numpy()
    for i in rng.choice(len(v), 3, replace=False):
        g = gal.block(np.array([i]), np.arange(len(v)))[0]
        err = np.abs(y[i] - g @ x) / (np.abs(g) @ np.abs(x))
        assert err.max() <= 1e-5, (i, err)
    h.check()
