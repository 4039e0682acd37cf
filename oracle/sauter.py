"""Sauter-Schwab quadrature for touching triangle pairs (oracle).

Sect. 8 integrates the singular kernel on pairs of triangles with Sauter's
rules and keeps one task list per case: identical triangles, a common edge,
a common vertex, disjoint triangles.  The rules themselves are not printed
in the paper; they are restated here from the underlying mathematics.

Both triangles are parametrised over the reference triangle
    T_ref = {(u1, u2) : 0 <= u2 <= u1 <= 1}
by x(u) = P0 + u1 (P1 - P0) + u2 (P2 - P1), with |det| = 2 |T|.  For the
common-edge case both parametrisations send the reference edge u2 = 0 to
the shared edge with the same orientation; for the common-vertex case both
send (0, 0) to the shared vertex.  Relative coordinates and Duffy-type
substitutions split T_ref x T_ref into 6 (identical), 5 (common edge) or
2 (common vertex) images of the unit cube [0,1]^4 in the variables
(xi, eta1, eta2, eta3); on each image the singularity sits at xi = 0 (or
eta1 = 0) and is cancelled by the Jacobian (xi^3 eta1^2 eta2, xi^3 eta1^2
and xi^3 eta1^2 eta2, xi^3 eta2 respectively), so a tensor Gauss-Legendre
rule of order q in all four variables converges exponentially.

Pinned by tests: each decomposition integrates smooth kernels (polynomials,
exponentials, a softened 1/r) to the value of a plain product rule (so the
pieces tile T x T exactly once with the right Jacobians), and the 1/r
integrals converge geometrically in q.
"""

import numpy as np

from .rules import gauss_legendre_01


def sub_maps(case, xi, e1, e2, e3):
    """Reference coordinates (u, v) of both triangles and the Jacobian weight.

    ``case`` is 3 (identical), 2 (common edge) or 1 (common vertex).
    Returns a list of ((u1, u2), (v1, v2), weight) per piece.
    """
    if case == 3:
        w = xi ** 3 * e1 ** 2 * e2
        a = 1.0 - e1 + e1 * e2
        return [
            ((xi, xi * a), (xi * (1.0 - e1 * e2 * e3), xi * (1.0 - e1)), w),
            ((xi * (1.0 - e1 * e2 * e3), xi * (1.0 - e1)), (xi, xi * a), w),
            ((xi, xi * e1 * (1.0 - e2 + e2 * e3)),
             (xi * (1.0 - e1 * e2), xi * e1 * (1.0 - e2)), w),
            ((xi * (1.0 - e1 * e2), xi * e1 * (1.0 - e2)),
             (xi, xi * e1 * (1.0 - e2 + e2 * e3)), w),
            ((xi * (1.0 - e1 * e2 * e3), xi * e1 * (1.0 - e2 * e3)),
             (xi, xi * e1 * (1.0 - e2)), w),
            ((xi, xi * e1 * (1.0 - e2)),
             (xi * (1.0 - e1 * e2 * e3), xi * e1 * (1.0 - e2 * e3)), w),
        ]
    if case == 2:
        w0 = xi ** 3 * e1 ** 2
        w = xi ** 3 * e1 ** 2 * e2
        return [
            ((xi, xi * e1 * e3), (xi * (1.0 - e1 * e2), xi * e1 * (1.0 - e2)), w0),
            ((xi, xi * e1), (xi * (1.0 - e1 * e2 * e3), xi * e1 * e2 * (1.0 - e3)), w),
            ((xi * (1.0 - e1 * e2), xi * e1 * (1.0 - e2)), (xi, xi * e1 * e2 * e3), w),
            ((xi * (1.0 - e1 * e2 * e3), xi * e1 * e2 * (1.0 - e3)), (xi, xi * e1), w),
            ((xi * (1.0 - e1 * e2 * e3), xi * e1 * (1.0 - e2 * e3)), (xi, xi * e1 * e2), w),
        ]
    if case == 1:
        w = xi ** 3 * e2
        return [
            ((xi, xi * e1), (xi * e2, xi * e2 * e3), w),
            ((xi * e2, xi * e2 * e3), (xi, xi * e1), w),
        ]
    raise ValueError("case must be 1, 2 or 3")


def cube_rule(q):
    """Tensor Gauss-Legendre rule of order q on [0,1]^4 (flattened)."""
    t, w = gauss_legendre_01(q)
    xi, e1, e2, e3 = np.meshgrid(t, t, t, t, indexing="ij")
    wt = np.einsum("a,b,c,d->abcd", w, w, w, w)
    return xi.ravel(), e1.ravel(), e2.ravel(), e3.ravel(), wt.ravel()


def integrate(case, P, Q, kernel, q):
    """Integral of kernel(x, y) over T_P x T_Q (touching pair, ordered).

    P, Q: arrays (m, 3, 3) of the vertex triples of m triangle pairs, ordered
    as required by ``case`` (see module header).  kernel maps arrays of
    points (..., 3), (..., 3) to values.  Returns an array of m integrals.
    """
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    xi, e1, e2, e3, wt = cube_rule(q)
    jp = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 1])
    jq = np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 1])
    jac = np.sqrt((jp * jp).sum(axis=1)) * np.sqrt((jq * jq).sum(axis=1))
    total = np.zeros(P.shape[0])
    for (u1, u2), (v1, v2), w in sub_maps(case, xi, e1, e2, e3):
        x = (P[:, None, 0, :] + u1[None, :, None] * (P[:, None, 1, :] - P[:, None, 0, :])
             + u2[None, :, None] * (P[:, None, 2, :] - P[:, None, 1, :]))
        y = (Q[:, None, 0, :] + v1[None, :, None] * (Q[:, None, 1, :] - Q[:, None, 0, :])
             + v2[None, :, None] * (Q[:, None, 2, :] - Q[:, None, 1, :]))
        total += (kernel(x, y) * (wt * w)[None, :]).sum(axis=1)
    return total * jac
