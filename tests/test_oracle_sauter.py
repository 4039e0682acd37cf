"""Pins for the Sauter-Schwab rules (Sect. 8, touching triangle pairs).

A substitution is correct iff it integrates every integrand correctly; the
smooth-kernel tests check that each case's pieces tile T x T exactly once
with the right Jacobians (against a plain product rule that needs no
singular treatment).  The 1/r tests then check geometric convergence in q.
"""

import numpy as np
import pytest

from oracle import sauter
from oracle.rules import gauss_legendre_01

A = np.array([0.1, 0.0, 0.05])
B = np.array([1.0, 0.2, -0.1])
C = np.array([0.3, 0.9, 0.2])
D = np.array([0.8, -0.7, 0.3])
E = np.array([-0.6, 0.4, 0.5])
F = np.array([-0.5, -0.6, -0.2])

PAIRS = {
    3: ([A, B, C], [A, B, C]),
    2: ([A, B, C], [A, B, D]),
    1: ([A, B, C], [A, E, F]),
}

KERNELS = {
    "poly": lambda x, y: 1 + (x[..., 0] - 2 * y[..., 1]) ** 2 + x[..., 2] * y[..., 0] ** 3,
    "exp": lambda x, y: np.exp(0.3 * x[..., 0] - 0.7 * y[..., 2] + 0.2 * x[..., 1] * y[..., 0]),
    "soft": lambda x, y: 1.0 / np.sqrt(((x - y) ** 2).sum(-1) + 0.3 ** 2),
}


def product_rule(P, Q, kernel, q):
    """Collapsed tensor Gauss rule on each triangle (no singular treatment)."""
    t, wt = gauss_legendre_01(q)
    s, r = np.meshgrid(t, t, indexing="ij")
    w = (np.outer(wt, wt) * s).ravel()
    u1, u2 = s.ravel(), (s * r).ravel()
    P = [np.asarray(p) for p in P]
    Q = [np.asarray(p) for p in Q]
    x = P[0] + u1[:, None] * (P[1] - P[0]) + u2[:, None] * (P[2] - P[1])
    y = Q[0] + u1[:, None] * (Q[1] - Q[0]) + u2[:, None] * (Q[2] - Q[1])
    K = kernel(x[:, None, :], y[None, :, :])
    jp = np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[1]))
    jq = np.linalg.norm(np.cross(Q[1] - Q[0], Q[2] - Q[1]))
    return np.einsum("a,b,ab->", w, w, K) * jp * jq


@pytest.mark.parametrize("case", [3, 2, 1])
@pytest.mark.parametrize("kname", ["poly", "exp", "soft"])
def test_substitution_is_exact_change_of_variables(case, kname):
    P, Q = PAIRS[case]
    k = KERNELS[kname]
    got = sauter.integrate(case, np.array([P]), np.array([Q]), k, 12)[0]
    ref = product_rule(P, Q, k, 30)
    tol = 1e-13 if kname != "soft" else 1e-8
    assert abs(got - ref) <= tol * abs(ref)


@pytest.mark.parametrize("case", [3, 2, 1])
def test_total_measure(case):
    # the Jacobian weights of all pieces add up to |T_ref|^2 = 1/4
    xi, e1, e2, e3, wt = sauter.cube_rule(4)
    tot = sum((wt * w).sum() for _, _, w in sauter.sub_maps(case, xi, e1, e2, e3))
    assert abs(tot - 0.25) < 1e-15


@pytest.mark.parametrize("case", [3, 2, 1])
def test_singular_kernel_converges_geometrically(case):
    P, Q = PAIRS[case]
    inv = lambda x, y: 1.0 / np.sqrt(((x - y) ** 2).sum(-1))  # noqa: E731
    qs = [3, 5, 7, 9, 16]
    vals = [sauter.integrate(case, np.array([P]), np.array([Q]), inv, q)[0] for q in qs]
    ref = vals[-1]
    errs = [abs(v - ref) / ref for v in vals[:-1]]
    assert errs[-1] < 1e-9
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_maps_stay_in_reference_triangle():
    xi, e1, e2, e3, _ = sauter.cube_rule(5)
    for case in (1, 2, 3):
        for (u1, u2), (v1, v2), w in sauter.sub_maps(case, xi, e1, e2, e3):
            for a, b in ((u1, u2), (v1, v2)):
                assert np.all(b >= -1e-15) and np.all(b <= a + 1e-15) and np.all(a <= 1 + 1e-15)
            assert np.all(w >= 0.0)
