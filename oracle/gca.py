"""GCA-H^2 construction (oracle): Green quadrature, cross approximation,
nested bases, coupling and near-field blocks.

Steps, in the paper's order:

1. ``omega_rule`` (Sect. 2): omega = box(tau) widened by margin * diam(tau)
   on each side; quadrature points z_nu, outward normals n_nu and weights
   w_nu on its boundary (``rules.box_rule``).
2. ``green_matrix`` (Sect. 2, the coefficients of A_{tau sigma}):
       a_{i nu}     =           sqrt(w_nu) int g(x, z_nu)        phi_i(x) dx
       a_{i, nu+k}  = -d_tau    sqrt(w_nu) int dg/dn_z(x, z_nu)  phi_i(x) dx
   with d_tau = diam(tau), integrals by the 7-point rule on triangle i.
   ``green_factor_b`` gives the matching B_{tau sigma} (only for the check
   that A B^* reproduces Eq. (2)).
3. ``aca`` (Sect. 3): cross approximation of the thin matrix with complete
   pivoting: at each step the entry of largest modulus in the residual is
   the pivot (ties within a relative ``tie_rel`` go to the smallest column,
   then smallest row); the residual loses the rank-one cross through it;
   stop before a pivot of modulus <= tol * |first pivot|, or at rank
   min(rows, cols).  The interpolation matrix V^ = A[:, Q] A[P, Q]^{-1} is
   obtained as U L^{-1} from the column factors U of the elimination
   (L = U[P, :] is unit lower triangular), so V^[P, :] = I.
4. ``build_bases`` (Sect. 3, Sect. 4): leaves run ACA on A_tau (all their
   triangles); a parent runs ACA on A^_tau = A_tau restricted to the rows
   tilde-tau_1 u tilde-tau_2 of its children (child 0 first), giving
   tilde-tau and V^_tau, which splits into the transfer matrices
   E_{tau_1} = V^_tau|tilde-tau_1 x tilde-tau and E_{tau_2}.  Leaves keep
   V_tau = V^_tau.  Only clusters whose basis the H^2 matrix uses get one:
   the bases enter through the admissible blocks, G|tau-hat x sigma-hat ~
   V_tau G|tilde-tau x tilde-sigma V_sigma^* (Sect. 4), and a parent's basis
   is built from its children's, so a cluster needs a basis iff it or one of
   its ancestors is in an admissible block.  The others (the root, and the
   coarse levels of a closed surface) get an empty one: rank 0, no pivots,
   zero-size V and E, which add nothing to the products.
5. ``build_h2`` (Sect. 4): coupling matrices S_{tau sigma} = G|tilde-tau x
   tilde-sigma for admissible blocks and near-field blocks G|tau-hat x
   sigma-hat for inadmissible leaf pairs, all from ``galerkin.entries``.

Pinned by tests: Gauss's law and Green's formula for the box rule, A B^*
equals the Eq. (2) quadrature, scaling covariance of A, exact recovery of
random low-rank matrices by ``aca``, brute-force pivot order, interpolation
V[tilde-tau, :] = I, V_tau = blockdiag(V_1, V_2) V^_tau, exactness on pivot
rows/columns of every coupling block, and the global spectral error of the
H^2 matrix decreasing with the tolerance.
"""

from dataclasses import dataclass, field

import numpy as np

from . import cluster
from .galerkin import Galerkin, dg_dn, g
from .rules import box_rule


def omega_rule(lo, hi, diam, margin, m):
    """Quadrature on the boundary of omega = box widened by margin * diam."""
    delta = margin * diam
    return box_rule(lo - delta, hi + delta, m)


def green_matrix(gal, rows, z, nrm, w, d_tau):
    """A_{tau sigma} restricted to the triangles ``rows`` (len(rows) x 2k)."""
    x = gal.pts[rows]            # (r, 7, 3)
    wx = gal.wts[rows]           # (r, 7)
    sw = np.sqrt(w)
    k = z.shape[0]
    A = np.empty((len(rows), 2 * k))
    for nu in range(k):
        gv = g(x, z[nu][None, None, :])                 # (r, 7)
        dv = dg_dn(x, z[nu][None, None, :], nrm[nu][None, None, :])
        A[:, nu] = sw[nu] * (wx * gv).sum(axis=1)
        A[:, nu + k] = -d_tau * sw[nu] * (wx * dv).sum(axis=1)
    return A


def green_factor_b(gal, cols, z, nrm, w, d_tau):
    """B_{tau sigma} restricted to the triangles ``cols`` (len(cols) x 2k)."""
    y = gal.pts[cols]
    wy = gal.wts[cols]
    sw = np.sqrt(w)
    k = z.shape[0]
    B = np.empty((len(cols), 2 * k))
    for nu in range(k):
        # dg/dn_z(z, y) = <n, y - z> / (4 pi |y - z|^3)
        dv = dg_dn(y, z[nu][None, None, :], nrm[nu][None, None, :])
        gv = g(z[nu][None, None, :], y)
        B[:, nu] = sw[nu] * (wy * dv).sum(axis=1)
        B[:, nu + k] = sw[nu] / d_tau * (wy * gv).sum(axis=1)
    return B


@dataclass
class ACAResult:
    rows: np.ndarray      # pivot row positions, in selection order
    cols: np.ndarray      # pivot column positions, in selection order
    U: np.ndarray         # column factors (nrows x r)
    V: np.ndarray         # interpolation matrix V^ (nrows x r)
    gap: float = 0.0      # replay: largest 1 - |R_ij| / max|R| over the steps
    stop: tuple = None    # replay: (smallest max|R| / (tol first) before a step,
                          #          max|R| / (tol first) after the last step)


def aca(A, tol, tie_rel=2.0 ** -40, follow=None):
    """Cross approximation with complete pivoting (Sect. 3).

    ``follow`` (test infrastructure): a sequence of row positions to take
    as the pivot rows instead of the argmax, each with the column that
    complete pivoting would take within that row.  It replays a pivot
    sequence found elsewhere (late pivots whose residuals are equal to
    rounding can be taken in either order); ``gap`` and ``stop`` then tell
    how far each replayed pivot fell below the largest residual and whether
    the stopping rule agrees with the replayed rank."""
    R = np.array(A, dtype=np.float64, copy=True)
    nr, nc = R.shape
    rmax = min(nr, nc) if follow is None else len(follow)
    prow, pcol, ucols = [], [], []
    first = None
    gap, low = 0.0, np.inf
    while len(prow) < rmax:
        absR = np.abs(R)
        big = absR.max()
        if first is None:
            first = big
        if follow is None and (big == 0.0 or (prow and big <= tol * first)):
            break
        if follow is None:
            cand = absR >= big * (1.0 - tie_rel)
            j = int(np.nonzero(cand.any(axis=0))[0][0])
            i = int(np.nonzero(cand[:, j])[0][0])
        else:
            i = int(follow[len(prow)])
            rowbig = absR[i].max()
            j = int(np.nonzero(absR[i] >= rowbig * (1.0 - tie_rel))[0][0])
            gap = max(gap, 1.0 - absR[i, j] / big)
            if prow:
                low = min(low, big / (tol * first))
        p = R[i, j]
        u = R[:, j] / p
        v = R[i, :].copy()
        R = R - np.outer(u, v)
        prow.append(i)
        pcol.append(j)
        ucols.append(u)
    r = len(prow)
    U = np.array(ucols).T if r else np.zeros((nr, 0))
    if r:
        L = U[prow, :]
        # V^ L = U  <=>  L^T V^T = U^T, L^T upper triangular, unit diagonal
        import scipy.linalg
        Vh = scipy.linalg.solve_triangular(L.T, U.T, lower=False, unit_diagonal=True).T
    else:
        Vh = np.zeros((nr, 0))
    stop = None
    if follow is not None and first:
        stop = (low, np.abs(R).max() / (tol * first) if r < min(nr, nc) else 0.0)
    return ACAResult(np.array(prow, dtype=np.int64), np.array(pcol, dtype=np.int64), U, Vh, gap, stop)


@dataclass
class Bases:
    pivots: list = field(default_factory=list)   # per cluster: triangle ids (tilde tau)
    V: dict = field(default_factory=dict)        # leaf -> (|tau-hat| x r)
    E: dict = field(default_factory=dict)        # child -> (r_child x r_parent)
    omega: dict = field(default_factory=dict)    # cluster -> (z, n, w)
    rank: np.ndarray = None
    replay: dict = field(default_factory=dict)   # cluster -> (gap, stop) of a replayed ACA


def needed_clusters(tree, far):
    """needed[c]: c or one of its ancestors is in an admissible block."""
    nc = len(tree["begin"])
    needed = np.zeros(nc, dtype=bool)
    for (t, s) in far:
        needed[t] = needed[s] = True
    for c in np.argsort(tree["level"], kind="stable"):   # top-down
        for ch in (tree["child0"][c], tree["child1"][c]):
            if ch >= 0 and needed[c]:
                needed[ch] = True
    return needed


def build_bases(gal, tree, lo, hi, params, far=None, green=None, nested=True, follow=None):
    """Nested cluster bases by Green cross approximation (Sect. 3, Sect. 4),
    for the clusters that need one (all non-root clusters when `far` is
    None); the others get empty bases.  `green(gal, rows, z, nrm, w, d)`
    forms the thin matrix of a cluster (default: the Green quadrature matrix
    A_tau of the single-layer kernel).  With nested=False every cluster that
    is in an admissible block gets a basis V_tau of its own from the cross
    approximation of A_tau on all of its triangles (the single-level GCA of
    Sect. 3), and no transfer matrices.  ``follow`` (test infrastructure):
    cluster -> pivot ids to replay in the cross approximations (see ``aca``);
    the largest gap and the stopping ratios are collected in
    ``bases.replay``."""
    if green is None:
        green = green_matrix
    if not nested:
        return _single_level_bases(gal, tree, lo, hi, params, far, green)
    nc = len(tree["begin"])
    diam = cluster.diameter(lo, hi)
    bases = Bases(pivots=[None] * nc, rank=np.zeros(nc, dtype=np.int64))
    margin = params.margin()
    needed = np.ones(nc, dtype=bool) if far is None else needed_clusters(tree, far)
    needed[0] = False
    order = np.argsort(-tree["level"], kind="stable")   # deepest level first
    for c in order:
        if not needed[c]:
            bases.pivots[c] = np.zeros(0, dtype=tree["perm"].dtype)
            if cluster.is_leaf(tree, c):
                bases.V[c] = np.zeros((tree["end"][c] - tree["begin"][c], 0))
            elif c != 0:
                for ch in (tree["child0"][c], tree["child1"][c]):
                    bases.E[ch] = np.zeros((bases.rank[ch], 0))
            continue
        z, nrm, w = omega_rule(lo[c], hi[c], diam[c], margin, params.box_gauss_m)
        bases.omega[c] = (z, nrm, w)
        if cluster.is_leaf(tree, c):
            rows = tree["perm"][tree["begin"][c]:tree["end"][c]]
        else:
            c0, c1 = tree["child0"][c], tree["child1"][c]
            rows = np.concatenate([bases.pivots[c0], bases.pivots[c1]])
        A = green(gal, rows, z, nrm, w, diam[c])
        fol = None
        if follow is not None:
            pos = {int(q): a for a, q in enumerate(rows)}
            fol = [pos[int(q)] for q in follow[c]]
        res = aca(A, params.aca_tol, params.tie_rel, follow=fol)
        if fol is not None:
            bases.replay[c] = (res.gap, res.stop)
        bases.pivots[c] = rows[res.rows]
        bases.rank[c] = len(res.rows)
        if cluster.is_leaf(tree, c):
            bases.V[c] = res.V
        else:
            r0 = bases.rank[tree["child0"][c]]
            bases.E[tree["child0"][c]] = res.V[:r0, :]
            bases.E[tree["child1"][c]] = res.V[r0:, :]
    return bases


def _single_level_bases(gal, tree, lo, hi, params, far, green):
    nc = len(tree["begin"])
    diam = cluster.diameter(lo, hi)
    bases = Bases(pivots=[None] * nc, rank=np.zeros(nc, dtype=np.int64))
    inblock = np.zeros(nc, dtype=bool)
    for (t, s) in far:
        inblock[t] = inblock[s] = True
    for c in range(nc):
        rows = tree["perm"][tree["begin"][c]:tree["end"][c]]
        if not inblock[c]:
            bases.pivots[c] = np.zeros(0, dtype=tree["perm"].dtype)
            bases.V[c] = np.zeros((len(rows), 0))
            continue
        z, nrm, w = omega_rule(lo[c], hi[c], diam[c], params.margin(), params.box_gauss_m)
        bases.omega[c] = (z, nrm, w)
        res = aca(green(gal, rows, z, nrm, w, diam[c]), params.aca_tol, params.tie_rel)
        bases.pivots[c] = rows[res.rows]
        bases.rank[c] = len(res.rows)
        bases.V[c] = res.V
    return bases


@dataclass
class H2:
    tree: dict
    bases: Bases
    far: list                      # admissible blocks (tau, sigma)
    near: list                     # inadmissible leaf blocks (tau, sigma)
    S: dict                        # (tau, sigma) -> r_tau x r_sigma
    N: dict                        # (tau, sigma) -> |tau-hat| x |sigma-hat|
    n: int
    lo: np.ndarray = None
    hi: np.ndarray = None


def build_h2(vertices, triangles, params, tree=None):
    """The whole GCA-H^2 construction on one mesh."""
    gal = Galerkin(vertices, triangles, params.sauter_q)
    if tree is None:
        tree = cluster.build_tree(vertices, triangles, params.leaf_size)
    lo, hi = cluster.cluster_boxes(vertices, triangles, tree)
    far, near = cluster.block_tree(tree, lo, hi, params.eta)
    bases = build_bases(gal, tree, lo, hi, params, far)
    S = {}
    for (t, s) in far:
        S[(t, s)] = gal.block(bases.pivots[t], bases.pivots[s])
    N = {}
    perm = tree["perm"]
    for (t, s) in near:
        N[(t, s)] = gal.block(perm[tree["begin"][t]:tree["end"][t]],
                              perm[tree["begin"][s]:tree["end"][s]])
    return H2(tree, bases, far, near, S, N, gal.n, lo, hi)
