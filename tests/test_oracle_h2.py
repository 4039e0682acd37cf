"""Pins for the oracle's H^2 products: the fast recursion equals the
definition with explicit bases (Sect. 4), transposes satisfy the adjoint
identity, and the power-iteration error estimate of Sect. 2 matches SVD."""

import numpy as np

import synth
from oracle import h2


def test_fast_equals_explicit(h2_1280):
    x = synth.uniform_rhs(h2_1280.n, 3, seed=0)
    y_fast = h2.matvec(h2_1280, x)
    y_def = h2.matvec_explicit(h2_1280, x)
    assert np.abs(y_fast - y_def).max() <= 1e-13 * np.abs(y_def).max()
    yt_fast = h2.matvec_t(h2_1280, x)
    yt_def = h2.matvec_explicit_t(h2_1280, x)
    assert np.abs(yt_fast - yt_def).max() <= 1e-13 * np.abs(yt_def).max()


def test_dense_equals_products(h2_1280):
    D = h2.dense(h2_1280)
    x = synth.normal_rhs(h2_1280.n, 2, seed=4)
    assert np.abs(D @ x - h2.matvec(h2_1280, x)).max() <= 1e-13 * np.abs(D @ x).max()
    assert np.abs(D.T @ x - h2.matvec_t(h2_1280, x)).max() <= 1e-13 * np.abs(D.T @ x).max()


def test_adjoint_identity(h2_1280):
    x = synth.normal_rhs(h2_1280.n, 1, seed=1)[:, 0]
    y = synth.normal_rhs(h2_1280.n, 1, seed=2)[:, 0]
    lhs = y @ h2.matvec(h2_1280, x)
    rhs = h2.matvec_t(h2_1280, y) @ x
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_transpose_close_to_product(h2_1280):
    # G is symmetric up to the singular quadrature; so is its H^2 approximation
    x = synth.normal_rhs(h2_1280.n, 1, seed=3)
    a = h2.matvec(h2_1280, x)
    b = h2.matvec_t(h2_1280, x)
    assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)


def test_power_iteration_matches_svd(h2_1280, dense_1280):
    D = h2.dense(h2_1280)
    E = dense_1280 - D
    Es = 0.5 * (E + E.T)
    Gs = 0.5 * (dense_1280 + dense_1280.T)
    est = h2.spectral_error(lambda x: Es @ x, lambda x: Gs @ x, h2_1280.n, iters=200)
    ref = np.linalg.norm(Es, 2) / np.linalg.norm(Gs, 2)
    assert abs(est - ref) <= 0.05 * ref
