"""Pins for the oracle's GCA construction (Sect. 2, Sect. 3, Sect. 4)."""

import numpy as np
import pytest

import synth
from oracle import cluster, gca, h2
from oracle.galerkin import Galerkin, dg_dn, g
from oracle.params import Params


# ---------------------------------------------------------------- Sect. 2

@pytest.fixture(scope="module")
def leaf_setup():
    v, t = synth.icosphere(3)
    tr = cluster.build_tree(v, t, 32)
    lo, hi = cluster.cluster_boxes(v, t, tr)
    far, _ = cluster.block_tree(tr, lo, hi, 2.0)
    gal = Galerkin(v, t, 5)
    return v, t, tr, lo, hi, far, gal


def test_factorisation_reproduces_eq2(leaf_setup):
    """A B^* equals the Eq. (2) quadrature integrated against phi_i, phi_j."""
    v, t, tr, lo, hi, far, gal = leaf_setup
    tau, sigma = far[0]
    diam = cluster.diameter(lo, hi)
    z, n, w = gca.omega_rule(lo[tau], hi[tau], diam[tau], 0.125, 3)
    rows = tr["perm"][tr["begin"][tau]:tr["end"][tau]][:6]
    cols = tr["perm"][tr["begin"][sigma]:tr["end"][sigma]][:5]
    A = gca.green_matrix(gal, rows, z, n, w, diam[tau])
    B = gca.green_factor_b(gal, cols, z, n, w, diam[tau])
    AB = A @ B.T
    for a, i in enumerate(rows):
        for b, j in enumerate(cols):
            x, wx = gal.pts[i], gal.wts[i]
            y, wy = gal.pts[j], gal.wts[j]
            direct = 0.0
            for p in range(7):
                for q in range(7):
                    term = (w * (g(x[p][None], z) * dg_dn(y[q][None], z, n)
                                 - dg_dn(x[p][None], z, n) * g(z, y[q][None]))).sum()
                    direct += wx[p] * wy[q] * term
            assert abs(AB[a, b] - direct) <= 1e-13 * abs(direct)


def test_green_factorisation_approximates_block(leaf_setup):
    """For an admissible block, A B^* approximates G, better for larger m."""
    v, t, tr, lo, hi, far, gal = leaf_setup
    diam = cluster.diameter(lo, hi)
    tau, sigma = far[len(far) // 2]
    rows = tr["perm"][tr["begin"][tau]:tr["end"][tau]]
    cols = tr["perm"][tr["begin"][sigma]:tr["end"][sigma]]
    Gb = gal.block(rows, cols)
    errs = []
    for m in (2, 4, 8, 12):
        z, n, w = gca.omega_rule(lo[tau], hi[tau], diam[tau], 0.125, m)
        A = gca.green_matrix(gal, rows, z, n, w, diam[tau])
        B = gca.green_factor_b(gal, cols, z, n, w, diam[tau])
        errs.append(np.linalg.norm(A @ B.T - Gb) / np.linalg.norm(Gb))
    # slow but steady: the pure Green quadrature needs many points (Fig. 1)
    assert errs[-1] < 1e-4
    assert all(b < a / 4 for a, b in zip(errs, errs[1:]))


def test_green_matrix_scaling(leaf_setup):
    """Under x -> s x both halves of A scale by s^2 (d_tau balances them)."""
    v, t, tr, lo, hi, far, gal = leaf_setup
    tau = far[0][0]
    rows = tr["perm"][tr["begin"][tau]:tr["end"][tau]]
    diam = cluster.diameter(lo, hi)
    z, n, w = gca.omega_rule(lo[tau], hi[tau], diam[tau], 0.125, 3)
    A1 = gca.green_matrix(gal, rows, z, n, w, diam[tau])
    s = 3.0
    gal3 = Galerkin(v * s, t, 5)
    z3, n3, w3 = gca.omega_rule(lo[tau] * s, hi[tau] * s, diam[tau] * s, 0.125, 3)
    A3 = gca.green_matrix(gal3, rows, z3, n3, w3, diam[tau] * s)
    assert np.abs(A3 - s * s * A1).max() <= 1e-13 * np.abs(A3).max()
    r1 = gca.aca(A1, 1e-6)
    r3 = gca.aca(A3, 1e-6)
    assert np.array_equal(r1.rows, r3.rows)


# ---------------------------------------------------------------- Sect. 3

def _complete_pivoting_reference(A, tol, tie_rel=2.0 ** -40):
    """Gaussian elimination with complete pivoting, scalar Python loops."""
    R = [list(map(float, row)) for row in A]
    nr, nc = len(R), len(R[0])
    piv = []
    first = None
    while len(piv) < min(nr, nc):
        big = max(abs(R[i][j]) for i in range(nr) for j in range(nc))
        if first is None:
            first = big
        if big == 0.0 or (piv and big <= tol * first):
            break
        best = None
        for j in range(nc):
            for i in range(nr):
                if abs(R[i][j]) >= big * (1.0 - tie_rel):
                    best = (i, j)
                    break
            if best:
                break
        i0, j0 = best
        p = R[i0][j0]
        u = [R[i][j0] / p for i in range(nr)]
        v = list(R[i0])
        for i in range(nr):
            for j in range(nc):
                R[i][j] = R[i][j] - u[i] * v[j]
        piv.append(best)
    return piv


def test_aca_pivots_brute_force():
    rng = np.random.default_rng(7)
    for shape in [(6, 9), (9, 4), (12, 12)]:
        A = rng.standard_normal(shape)
        res = gca.aca(A, 1e-12)
        ref = _complete_pivoting_reference(A, 1e-12)
        assert list(zip(res.rows.tolist(), res.cols.tolist())) == ref


def test_aca_tie_break():
    A = np.array([[1.0, 3.0, -3.0],
                  [3.0, 0.5, 0.0],
                  [-3.0, 2.0, 1.0]])
    res = gca.aca(A, 1e-12)
    # |3| appears at (1,0), (2,0), (0,1), (0,2): smallest column, then row
    assert (res.rows[0], res.cols[0]) == (1, 0)


def test_aca_recovers_low_rank():
    rng = np.random.default_rng(11)
    for (m, n, k) in [(40, 30, 7), (64, 192, 20), (100, 12, 12)]:
        A = rng.standard_normal((m, k)) @ rng.standard_normal((k, n))
        res = gca.aca(A, 1e-12)
        assert len(res.rows) == k
        err = np.abs(res.V @ A[res.rows, :] - A).max() / np.abs(A).max()
        assert err < 1e-12
        assert np.abs(res.V[res.rows, :] - np.eye(k)).max() < 1e-14
        # V^ = A[:, Q] A[P, Q]^{-1}
        Vd = np.linalg.solve(A[np.ix_(res.rows, res.cols)].T, A[:, res.cols].T).T
        assert np.abs(Vd - res.V).max() < 1e-9 * max(1.0, np.abs(res.V).max())


def test_aca_stopping_rule():
    rng = np.random.default_rng(5)
    # singular values 10^-i: the rank grows by about one per decade of tol
    m, n = 30, 30
    Uq, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Vq, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Uq @ np.diag(10.0 ** -np.arange(m, dtype=float)) @ Vq.T
    ranks = [len(gca.aca(A, tol).rows) for tol in (1e-2, 1e-4, 1e-6, 1e-8)]
    assert ranks == sorted(ranks) and ranks[0] < ranks[-1]
    res = gca.aca(A, 1e-6)
    assert np.abs(res.V @ A[res.rows, :] - A).max() < 1e-4


def test_interpolation_sensitivity_at_tight_tolerance(monkeypatch):
    """Why bases are compared more loosely than products at tol 1e-8.

    One rounding error of noise on the Green matrices (relative 2e-16) moves
    the transfer matrices E by up to ~1e-9, while the pivots stay the same and
    the H^2 product moves by ~1e-15: V^ = A[:, Q] A[P, Q]^{-1} is
    ill-conditioned along directions that A[P, :] maps to almost nothing.
    """
    v, t = synth.mesh_for_config("ellipsoid1280")
    p = Params(leaf_size=24, eta=2.0, box_gauss_m=3, aca_tol=1e-8, sauter_q=4)
    H0 = gca.build_h2(v, t, p)
    orig = gca.green_matrix
    rng = np.random.default_rng(0)
    monkeypatch.setattr(gca, "green_matrix",
                        lambda *a, **k: (lambda A: A * (1 + 2e-16 * rng.standard_normal(A.shape)))(
                            orig(*a, **k)))
    H1 = gca.build_h2(v, t, p)
    for c in range(1, len(H0.bases.pivots)):
        assert np.array_equal(H0.bases.pivots[c], H1.bases.pivots[c])
    dE = max(np.abs(H0.bases.E[c] - H1.bases.E[c]).max() for c in H0.bases.E if H0.bases.E[c].size)
    x = synth.normal_rhs(len(t), 4, 1)
    y0, y1 = h2.matvec(H0, x), h2.matvec(H1, x)
    dy = (np.linalg.norm(y0 - y1, axis=0) / np.linalg.norm(y0, axis=0)).max()
    assert dy < 1e-13
    assert dE < 1e-8
    assert dE > 100 * dy


# ---------------------------------------------------------------- Sect. 4

def test_nested_bases_interpolate(h2_1280):
    H = h2_1280
    V = h2.explicit_bases(H)
    tr = H.tree
    for c, Vc in V.items():
        if H.bases.rank[c] == 0:  # a cluster the H^2 matrix does not use
            continue
        rows = tr["perm"][tr["begin"][c]:tr["end"][c]]
        pos = {int(r): a for a, r in enumerate(rows)}
        piv = [pos[int(p)] for p in H.bases.pivots[c]]
        assert np.abs(Vc[piv, :] - np.eye(len(piv))).max() < 1e-12
        assert H.bases.rank[c] <= min(len(rows), 2 * 54)
        if not cluster.is_leaf(tr, c):
            c0, c1 = tr["child0"][c], tr["child1"][c]
            pool = set(H.bases.pivots[c0].tolist()) | set(H.bases.pivots[c1].tolist())
            assert set(H.bases.pivots[c].tolist()) <= pool


def test_coupling_exact_on_pivots(h2_1280, dense_1280):
    H, G = h2_1280, dense_1280
    D = h2.dense(H)
    for (t, s) in H.far[::7]:
        pt, ps = H.bases.pivots[t], H.bases.pivots[s]
        assert np.abs(D[np.ix_(pt, ps)] - G[np.ix_(pt, ps)]).max() <= 1e-13 * np.abs(G).max()
    for (t, s) in H.near[::5]:
        rt = H.tree["perm"][H.tree["begin"][t]:H.tree["end"][t]]
        rs = H.tree["perm"][H.tree["begin"][s]:H.tree["end"][s]]
        assert np.array_equal(D[np.ix_(rt, rs)], G[np.ix_(rt, rs)])


def test_spectral_error_small(h2_1280, dense_1280):
    D = h2.dense(h2_1280)
    G = dense_1280
    err = np.linalg.norm(G - D, 2) / np.linalg.norm(G, 2)
    assert err < 1e-6


def test_error_falls_with_tolerance(sphere1280, dense_1280, h2_1280):
    v, t = sphere1280
    G = dense_1280
    nG = np.linalg.norm(G, 2)
    errs = []
    for tol in (1e-2, 1e-3, 1e-4):
        p = Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=tol, sauter_q=5)
        H = gca.build_h2(v, t, p)
        errs.append(np.linalg.norm(G - h2.dense(H), 2) / nG)
    errs.append(np.linalg.norm(G - h2.dense(h2_1280), 2) / nG)   # tol 1e-6
    assert all(b < a / 5 for a, b in zip(errs, errs[1:]))
    # the achieved accuracy tracks the requested tolerance
    for tol, e in zip((1e-2, 1e-3, 1e-4, 1e-6), errs):
        assert e < tol


def test_needed_clusters_brute_force(h2_1280):
    """needed(c) against its definition (Sect. 4: a basis enters the matrix
    only through V_tau S V_sigma^T and, nested, through its ancestors'): c or
    one of its ancestors is a row or column cluster of an admissible block.
    The clusters without a basis are exactly the unneeded ones, and the
    product still matches the one with every basis (checked elsewhere
    against the dense G)."""
    tree = h2_1280.tree
    nc = len(tree["begin"])
    parent = np.full(nc, -1)
    for c in range(nc):
        for ch in (tree["child0"][c], tree["child1"][c]):
            if ch >= 0:
                parent[ch] = c
    in_far = set()
    for (t, s) in h2_1280.far:
        in_far.add(int(t))
        in_far.add(int(s))
    ref = np.zeros(nc, dtype=bool)
    for c in range(nc):
        a = c
        while a >= 0:
            if a in in_far:
                ref[c] = True
                break
            a = parent[a]
    got = gca.needed_clusters(tree, h2_1280.far)
    assert np.array_equal(got, ref)
    assert not got[0]                       # the root is in no admissible block
    assert (~got).sum() > 1                 # the sphere's upper levels are unused
    rank = h2_1280.bases.rank
    assert np.all(rank[~got] == 0)
    assert np.all(rank[got] > 0)


def test_aca_replay_of_its_own_pivots():
    """The replay mode (test infrastructure for rounding-level pivot ties):
    replaying the cross approximation's own pivot rows reproduces it exactly
    with no gap and a consistent stop; another order shows up as a gap."""
    rng = np.random.default_rng(3)
    sv = 10.0 ** -np.arange(12)
    A = (rng.normal(size=(40, 12)) * sv) @ rng.normal(size=(12, 30))
    res = gca.aca(A, 1e-6)
    rep = gca.aca(A, 1e-6, follow=res.rows)
    assert np.array_equal(rep.rows, res.rows) and np.array_equal(rep.cols, res.cols)
    assert np.array_equal(rep.V, res.V)
    assert rep.gap == 0.0
    low, after = rep.stop
    assert low > 1.0 and after <= 1.0
    swapped = list(res.rows)
    swapped[0], swapped[1] = swapped[1], swapped[0]
    assert gca.aca(A, 1e-6, follow=swapped).gap > 0.5
    assert gca.aca(A, 1e-6, follow=list(res.rows) + [int(np.setdiff1d(np.arange(40), res.rows)[0])]).stop[0] <= 1.0
