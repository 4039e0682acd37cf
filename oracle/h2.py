"""H^2 matrix-vector products and error estimates (oracle).

The paper stops at the representation (Sect. 4):
    G|tau-hat x sigma-hat ~ V_tau S_{tau sigma} V_sigma^*  (admissible),
    V_tau = [V_{tau_1} E_{tau_1}; V_{tau_2} E_{tau_2}]    (nested bases),
plus exact near-field blocks.  The product with a vector is fixed by that
representation; the fast evaluation is the standard H^2 recursion of the
H^2 literature the paper cites (forward transform up the cluster tree,
coupling, backward transform down the tree, near field):

* ``matvec``          the fast recursion,
* ``matvec_explicit`` the definition with explicitly assembled V_tau,
* ``matvec_t`` / ``matvec_explicit_t`` the transposed products,
* ``dense``           the represented matrix as a dense array,
* ``spectral_error``  ||G - G_H2||_2 / ||G||_2 by power iteration (the
                      paper's error measure, Sect. 2) or by SVD.

Pinned by tests: fast = explicit to 1e-13, the adjoint identity
<y, H x> = <H^T y, x>, dense(H) equal to G on pivot rows/columns of every
coupling block, and the spectral error falling with the ACA tolerance.
"""

import numpy as np

from . import cluster


def _leaves(tree):
    return [c for c in range(len(tree["begin"])) if cluster.is_leaf(tree, c)]


def _rows(tree, c):
    return tree["perm"][tree["begin"][c]:tree["end"][c]]


def forward(h, X):
    """x-hat_tau = V_tau^* x|tau-hat for every non-root cluster (recursive)."""
    tree = h.tree
    xh = {}
    order = np.argsort(-tree["level"], kind="stable")
    for c in order:
        if c == 0:
            continue
        if cluster.is_leaf(tree, c):
            xh[c] = h.bases.V[c].T @ X[_rows(tree, c)]
        else:
            c0, c1 = tree["child0"][c], tree["child1"][c]
            xh[c] = h.bases.E[c0].T @ xh[c0] + h.bases.E[c1].T @ xh[c1]
    return xh


def backward(h, yh, Y):
    """y|tau-hat += V_tau y-hat_tau for every non-root cluster (recursive)."""
    tree = h.tree
    order = np.argsort(tree["level"], kind="stable")
    yh = {c: v.copy() for c, v in yh.items()}
    for c in order:
        if c == 0:
            continue
        if cluster.is_leaf(tree, c):
            Y[_rows(tree, c)] += h.bases.V[c] @ yh[c]
        else:
            for ch in (tree["child0"][c], tree["child1"][c]):
                yh[ch] = yh[ch] + h.bases.E[ch] @ yh[c]
    return Y


def _as2d(X):
    X = np.asarray(X, dtype=np.float64)
    return (X[:, None], True) if X.ndim == 1 else (X, False)


def matvec(h, X, transpose=False):
    """Fast H^2 product (or its transpose) with X (n or n x R)."""
    X, vec = _as2d(X)
    tree = h.tree
    xh = forward(h, X)
    R = X.shape[1]
    yh = {c: np.zeros((h.bases.rank[c], R)) for c in xh}
    for (t, s) in h.far:
        if transpose:
            yh[s] += h.S[(t, s)].T @ xh[t]
        else:
            yh[t] += h.S[(t, s)] @ xh[s]
    Y = np.zeros_like(X)
    backward(h, yh, Y)
    for (t, s) in h.near:
        if transpose:
            Y[_rows(tree, s)] += h.N[(t, s)].T @ X[_rows(tree, t)]
        else:
            Y[_rows(tree, t)] += h.N[(t, s)] @ X[_rows(tree, s)]
    return Y[:, 0] if vec else Y


def matvec_t(h, X):
    return matvec(h, X, transpose=True)


def explicit_bases(h):
    """V_tau for every non-root cluster, assembled from the transfer matrices."""
    tree = h.tree
    V = {}
    order = np.argsort(-tree["level"], kind="stable")
    for c in order:
        if c == 0:
            continue
        if cluster.is_leaf(tree, c):
            V[c] = h.bases.V[c]
        else:
            c0, c1 = tree["child0"][c], tree["child1"][c]
            V[c] = np.vstack([V[c0] @ h.bases.E[c0], V[c1] @ h.bases.E[c1]])
    return V


def matvec_explicit(h, X, transpose=False):
    """sum_adm V_tau S V_sigma^* x|sigma-hat + sum_near N x (the definition)."""
    X, vec = _as2d(X)
    tree = h.tree
    V = explicit_bases(h)
    Y = np.zeros_like(X)
    for (t, s) in h.far:
        blk = V[t] @ h.S[(t, s)] @ V[s].T
        if transpose:
            Y[_rows(tree, s)] += blk.T @ X[_rows(tree, t)]
        else:
            Y[_rows(tree, t)] += blk @ X[_rows(tree, s)]
    for (t, s) in h.near:
        if transpose:
            Y[_rows(tree, s)] += h.N[(t, s)].T @ X[_rows(tree, t)]
        else:
            Y[_rows(tree, t)] += h.N[(t, s)] @ X[_rows(tree, s)]
    return Y[:, 0] if vec else Y


def matvec_explicit_t(h, X):
    return matvec_explicit(h, X, transpose=True)


def dense(h):
    tree = h.tree
    V = explicit_bases(h)
    D = np.zeros((h.n, h.n))
    for (t, s) in h.far:
        D[np.ix_(_rows(tree, t), _rows(tree, s))] = V[t] @ h.S[(t, s)] @ V[s].T
    for (t, s) in h.near:
        D[np.ix_(_rows(tree, t), _rows(tree, s))] = h.N[(t, s)]
    return D


def spectral_error(apply_err, apply_ref, n, iters=50, seed=1):
    """||E||_2 / ||G||_2 by power iteration on E^T E and G^T G (Sect. 2).

    apply_err / apply_ref map a vector x to E x / G x for symmetric E, G.
    """
    rng = np.random.default_rng(seed)

    def norm2(apply):
        x = rng.standard_normal(n)
        x /= np.linalg.norm(x)
        lam = 0.0
        for _ in range(iters):
            y = apply(apply(x))
            lam = np.linalg.norm(y)
            if lam == 0.0:
                return 0.0
            x = y / lam
        return np.sqrt(lam)

    return norm2(apply_err) / norm2(apply_ref)


def storage(h):
    """Number of stored coefficients: leaf bases, transfers, couplings, near."""
    v = sum(m.size for m in h.bases.V.values())
    e = sum(m.size for m in h.bases.E.values())
    s = sum(m.size for m in h.S.values())
    nn = sum(m.size for m in h.N.values())
    return {"V": v, "E": e, "S": s, "N": nn, "total": v + e + s + nn}
