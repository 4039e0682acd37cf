"""Checks of full-size GPU results on samples the oracle computes one by one.

At the benchmark sizes the oracle cannot build the whole H^2 matrix, but
each of these pieces depends on a few triangles only and is cheap for it:

* the cluster tree and block tree (oracle's own, compared exactly),
* near-field entries g_ij at sampled positions of sampled near blocks
  (Eq. (1); Sauter-Schwab for touching pairs, Sect. 8),
* leaf bases: the Green matrix of a leaf (Sect. 2) and its cross
  approximation (Sect. 3) depend only on the leaf's triangles and box,
* rows of the dense G: (G x)_i for sampled i, against which the H^2
  product must agree within the compression error.

Nothing here reads a GPU result as an oracle input: the GPU's arrays are
only compared with what the oracle computes from the mesh alone.
"""

import numpy as np

from oracle import cluster, gca as ogca
from oracle.galerkin import Galerkin


def oracle_geometry(v, t, params):
    tree = cluster.build_tree(v, t, params.leaf_size)
    lo, hi = cluster.cluster_boxes(v, t, tree)
    far, near = cluster.block_tree(tree, lo, hi, params.eta)
    return tree, lo, hi, far, near


def check_tree(ours, tree):
    for k in ("perm", "begin", "end", "child0", "child1", "level"):
        assert np.array_equal(np.asarray(ours[k]), np.asarray(tree[k])), k


def check_blocks(dump, far, near):
    assert sorted(map(tuple, dump["far"].tolist())) == sorted(far)
    assert sorted(map(tuple, dump["near"].tolist())) == sorted(near)


def near_offsets(dump, tree):
    sz = tree["end"] - tree["begin"]
    pairs = dump["near"]
    counts = sz[pairs[:, 0]] * sz[pairs[:, 1]]
    return np.concatenate([[0], np.cumsum(counts)])


def check_near_entries(dump, tree, gal, rng, blocks=64, per_block=16, tol=1e-10):
    """Sampled N entries against the oracle's Galerkin entries; every block
    that holds a touching pair contributes one of them."""
    pairs = dump["near"]
    off = near_offsets(dump, tree)
    perm = tree["perm"]
    pick = rng.choice(len(pairs), size=min(blocks, len(pairs)), replace=False)
    # diagonal blocks hold the identical / edge / vertex cases
    diag = np.nonzero(pairs[:, 0] == pairs[:, 1])[0]
    pick = np.unique(np.concatenate([pick, diag[:8]]))
    ii, jj, got = [], [], []
    for b in pick:
        t, s = pairs[b]
        mt = tree["end"][t] - tree["begin"][t]
        ms = tree["end"][s] - tree["begin"][s]
        a = rng.integers(0, mt, per_block)
        c = rng.integers(0, ms, per_block)
        if t == s:
            a[:4] = c[:4]  # identical triangles
        ii.append(perm[tree["begin"][t] + a])
        jj.append(perm[tree["begin"][s] + c])
        got.append(dump["N"][off[b] + a * ms + c])
    ii, jj, got = np.concatenate(ii), np.concatenate(jj), np.concatenate(got)
    ref = gal.entries(ii, jj)
    err = np.abs(got - ref) / np.abs(ref)
    assert err.max() <= tol, (err.max(), ii[err.argmax()], jj[err.argmax()])
    return float(err.max())


def check_coupling_entries(dump, gal, rng, blocks=64, per_block=16, tol=1e-10):
    """Sampled S entries against the oracle's Galerkin entries of the pivot
    triangles, S_{tau sigma}[a, b] = g(tilde-tau_a, tilde-sigma_b) (Sect. 4);
    relative per entry (all entries are positive)."""
    rank = dump["rank"]
    poff = np.concatenate([[0], np.cumsum(rank)])
    far = dump["far"]
    soff = np.concatenate([[0], np.cumsum(rank[far[:, 0]] * rank[far[:, 1]])])
    assert soff[-1] == len(dump["S"])
    pick = rng.choice(len(far), size=min(blocks, len(far)), replace=False)
    ii, jj, got = [], [], []
    for b in pick:
        t, s = far[b]
        a = rng.integers(0, rank[t], per_block)
        c = rng.integers(0, rank[s], per_block)
        ii.append(dump["pivots"][poff[t] + a])
        jj.append(dump["pivots"][poff[s] + c])
        got.append(dump["S"][soff[b] + a * rank[s] + c])
    ii, jj, got = np.concatenate(ii), np.concatenate(jj), np.concatenate(got)
    ref = gal.entries(ii, jj)
    err = np.abs(got - ref) / np.abs(ref)
    assert err.max() <= tol, (err.max(), ii[err.argmax()], jj[err.argmax()])
    return float(err.max())


def check_leaf_bases(dump, tree, lo, hi, gal, params, rng, leaves=6, tol=1e-8):
    """Leaf pivots and V from the oracle's own Green matrix and ACA.

    Pivots must agree as an ordered list.  Late pivots of a long cross
    approximation are chosen from a residual whose relative rounding noise
    grows with the rank, so a pivot can differ there; such a leaf is
    accepted if the GPU's basis is a valid interpolation of the oracle's
    matrix (V[tilde-tau, :] = I and A ~ V A[tilde-tau, :] within the ACA
    tolerance) and the two ranks agree within one."""
    nc = len(tree["begin"])
    rank = dump["rank"]
    voff = {}
    at = 0
    for c in range(1, nc):
        if tree["child0"][c] < 0:
            voff[c] = at
            at += (tree["end"][c] - tree["begin"][c]) * rank[c]
    poff = np.concatenate([[0], np.cumsum(rank)])
    diam = cluster.diameter(lo, hi)
    # leaves whose basis the H^2 matrix uses (they or an ancestor in an
    # admissible block); the others must have none
    needed = ogca.needed_clusters(tree, [tuple(b) for b in dump["far"].tolist()])
    for c in voff:
        if not needed[c]:
            assert rank[c] == 0, f"basis of unused leaf {c}"
    cand = [c for c in voff if needed[c]]
    flips = 0
    for c in rng.choice(cand, size=min(leaves, len(cand)), replace=False):
        rows = tree["perm"][tree["begin"][c]:tree["end"][c]]
        z, nrm, w = ogca.omega_rule(lo[c], hi[c], diam[c], params.margin(), params.box_gauss_m)
        A = ogca.green_matrix(gal, rows, z, nrm, w, diam[c])
        res = ogca.aca(A, params.aca_tol, params.tie_rel)
        piv = dump["pivots"][poff[c]:poff[c] + rank[c]]
        m = len(rows)
        V = dump["V"][voff[c]:voff[c] + m * rank[c]].reshape(m, rank[c])
        if len(res.rows) == rank[c] and np.array_equal(piv, rows[res.rows]):
            scale = np.abs(res.V).max()
            assert np.abs(V - res.V).max() <= tol * max(scale, 1.0), f"V of leaf {c}"
            continue
        flips += 1
        assert abs(len(res.rows) - rank[c]) <= 1, f"rank of leaf {c}"
        pos = np.array([int(np.nonzero(rows == p)[0][0]) for p in piv])
        assert np.abs(V[pos, :] - np.eye(rank[c])).max() <= 1e-12, f"interpolation of leaf {c}"
        approx = V @ A[pos, :]
        assert np.abs(A - approx).max() <= 10 * params.aca_tol * np.abs(A).max(), f"leaf {c}"
    return flips


def check_dense_rows(y, x, v, t, gal, rng, rows=4, tol=1e-5):
    """(G_H2 x)_i against (G x)_i for sampled rows i, relative to
    sum_j |g_ij| |x_j| (the compression error bound of the representation)."""
    n = len(t)
    idx = rng.choice(n, size=rows, replace=False)
    cols = np.arange(n)
    for i in idx:
        g = gal.block(np.array([i]), cols)[0]
        ref = g @ x
        scale = np.abs(g) @ np.abs(x)
        err = np.abs(y[i] - ref) / scale
        assert err.max() <= tol, (i, err.max())
