"""Pins for the oracle's quadrature rules (Sect. 2): exactness on
polynomials, the surface measure of the box, Gauss's law for the normal
derivative of the fundamental solution, and convergence of Green's
representation formula as discretised by Eq. (2)."""

from math import factorial

import numpy as np
import pytest

from oracle import rules
from oracle.galerkin import dg_dn, g


@pytest.mark.parametrize("q", [1, 2, 3, 5, 8])
def test_gauss_legendre_exact_to_degree_2q_minus_1(q):
    t, w = rules.gauss_legendre_01(q)
    for p in range(2 * q):
        assert abs((w * t ** p).sum() - 1.0 / (p + 1)) < 1e-14
    # and not beyond: degree 2q is integrated with a visible error
    assert abs((w * t ** (2 * q)).sum() - 1.0 / (2 * q + 1)) > 1e-6 / q ** 4


def _monomial_exact(a, b):
    # integral of x^a y^b over the triangle (0,0), (1,0), (0,1)
    return factorial(a) * factorial(b) / factorial(a + b + 2)


def test_radon7_exact_to_degree_5():
    v = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    t = np.array([[0, 1, 2]])
    pts, wts = rules.triangle_points(v, t)
    x, y = pts[0, :, 0], pts[0, :, 1]
    for a in range(6):
        for b in range(6 - a):
            assert abs((wts[0] * x ** a * y ** b).sum() - _monomial_exact(a, b)) < 1e-15
    # degree 6 is not exact for every monomial: this is the degree-5 rule
    err6 = max(abs((wts[0] * x ** a * y ** (6 - a)).sum() - _monomial_exact(a, 6 - a))
               for a in range(7))
    assert err6 > 1e-6


def test_radon7_affine_invariance():
    # exactness carries over to an arbitrary triangle in space
    rng = np.random.default_rng(3)
    v = rng.standard_normal((3, 3))
    t = np.array([[0, 1, 2]])
    pts, wts = rules.triangle_points(v, t)
    area = rules.triangle_areas(v, t)[0]
    assert abs(wts.sum() - area) < 1e-14
    # the centroid is the first moment
    c = v.mean(axis=0)
    assert np.allclose((wts[0, :, None] * pts[0]).sum(axis=0) / area, c, atol=1e-14)


def test_box_rule_measure_and_normals():
    lo = np.array([-0.3, 0.1, 0.2])
    hi = np.array([0.5, 0.4, 1.7])
    z, n, w = rules.box_rule(lo, hi, 4)
    e = hi - lo
    area = 2.0 * (e[0] * e[1] + e[1] * e[2] + e[0] * e[2])
    assert z.shape == (96, 3) and n.shape == (96, 3) and w.shape == (96,)
    assert abs(w.sum() - area) < 1e-13
    assert np.allclose((w[:, None] * n).sum(axis=0), 0.0, atol=1e-13)
    # every point lies on the face named by its normal
    for zi, ni in zip(z, n):
        d = int(np.nonzero(ni)[0][0])
        assert zi[d] == (hi[d] if ni[d] > 0 else lo[d])
        assert np.all(zi >= lo - 1e-15) and np.all(zi <= hi + 1e-15)
    # the rule integrates a quadratic exactly on the box surface
    f = z[:, 0] ** 2
    exact = 0.0
    for d in range(3):
        d1, d2 = [a for a in range(3) if a != d]
        for side in (lo, hi):
            # face at x_d = side[d]; integrate x^2 over [lo_d1, hi_d1] x [lo_d2, hi_d2]
            def int_x2(lo_, hi_):
                return (hi_ ** 3 - lo_ ** 3) / 3.0
            if d == 0:
                exact += side[0] ** 2 * e[1] * e[2]
            elif d1 == 0:
                exact += int_x2(lo[0], hi[0]) * e[d2]
    assert abs((w * f).sum() - exact) < 1e-13


@pytest.mark.parametrize("inside", [True, False])
def test_gauss_law(inside):
    """Flux of the fundamental solution: -1 inside omega, 0 outside."""
    lo = np.array([0.0, 0.0, 0.0])
    hi = np.array([1.0, 0.7, 0.5])
    x = np.array([0.4, 0.3, 0.2]) if inside else np.array([2.3, 1.1, -0.9])
    target = -1.0 if inside else 0.0
    errs = []
    for m in (2, 4, 8, 16, 24):
        z, n, w = rules.box_rule(lo, hi, m)
        flux = (w * dg_dn(x[None, :], z, n)).sum()
        errs.append(abs(flux - target))
    assert errs[-1] < 1e-8
    assert all(b < a or b < 1e-15 for a, b in zip(errs, errs[1:]))


def test_green_representation_converges():
    """Eq. (2) converges to g(x, y) for x in tau, y outside omega (Sect. 2)."""
    lo = np.array([0.0, 0.0, 0.0])
    hi = np.array([1.0, 1.0, 1.0])
    delta = 0.25
    xs = np.array([[0.5, 0.5, 0.5], [0.1, 0.9, 0.3], [1.0, 0.0, 1.0]])
    ys = np.array([[3.0, 0.5, 0.5], [-1.5, 2.0, 2.2], [0.5, 0.5, -2.0]])
    errs = []
    for m in (3, 5, 8, 12, 16, 24):
        z, n, w = rules.box_rule(lo - delta, hi + delta, m)
        e = 0.0
        for x in xs:
            for y in ys:
                approx = (w * (g(x[None, :], z) * dg_dn(y[None, :], z, n)
                               - dg_dn(x[None, :], z, n) * g(z, y[None, :]))).sum()
                exact = g(x, y)
                e = max(e, abs(approx - exact) / exact)
        errs.append(e)
    assert errs[-1] < 1e-7
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_green_representation_vanishes_outside():
    """The same boundary integral is 0 for x outside omega."""
    lo = np.array([0.0, 0.0, 0.0])
    hi = np.array([1.0, 1.0, 1.0])
    x = np.array([-1.0, 0.4, 0.5])
    y = np.array([3.0, 0.5, 0.5])
    z, n, w = rules.box_rule(lo, hi, 16)
    val = (w * (g(x[None, :], z) * dg_dn(y[None, :], z, n)
                - dg_dn(x[None, :], z, n) * g(z, y[None, :]))).sum()
    assert abs(val) < 1e-6 * g(x, y)
