"""Seeded right-hand sides and field points.

Right-hand sides are column-major (n x R) float64 arrays in the original
triangle order, as the C-ABI expects them.
"""

import numpy as np


def uniform_rhs(n, nrhs=1, seed=0):
    """x ~ U(-1, 1), float64, Fortran order (n x nrhs)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.uniform(-1.0, 1.0, size=(n, nrhs)))


def normal_rhs(n, nrhs=1, seed=0):
    """x ~ N(0, 1), float64, Fortran order (n x nrhs)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal(size=(n, nrhs)))


def exterior_points(count, radius=3.0, seed=0):
    """Points uniform on the sphere of the given radius (normalised Gaussians)."""
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(size=(count, 3))
    p /= np.sqrt((p * p).sum(axis=1))[:, None]
    return radius * p
