"""Shared fixtures.  GPU tests are marked ``gpu``; everything else runs on CPU."""

import numpy as np
import pytest

import synth
from oracle import gca
from oracle.params import Params


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300)")


@pytest.fixture(scope="session")
def sphere1280():
    return synth.mesh_for_config("sphere1280")


@pytest.fixture(scope="session")
def sphere320():
    return synth.mesh_for_config("sphere320")


@pytest.fixture(scope="session")
def small_params():
    """Build parameters of the 1280-triangle workload (leaf 32, eta 2, m 3, tol 1e-6)."""
    return Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)


@pytest.fixture(scope="session")
def h2_1280(sphere1280, small_params):
    v, t = sphere1280
    return gca.build_h2(v, t, small_params)


@pytest.fixture(scope="session")
def dense_1280(sphere1280, small_params):
    from oracle.galerkin import Galerkin
    v, t = sphere1280
    return Galerkin(v, t, small_params.sauter_q).dense_matrix()


@pytest.fixture(scope="session")
def rng():
    return np.random.default_rng(1234)
