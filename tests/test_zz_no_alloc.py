"""h2_matvec_noalloc (the product whose workspace is a fixed array in the
library's device data) against h2_matvec, the allocating entry point, through
the C ABI.  Two calls in a row with different right-hand sides check that the
state one call leaves in the shared array does not reach the next; sizes over
the array's capacity must be rejected before anything runs.

The file is named to be collected last, so that it also runs after every
other GPU test in the same process.
"""

import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# float64 agrees up to the order of the atomic accumulation; reduced
# precisions share storage and accumulator types with h2_matvec
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-5}


@pytest.fixture(scope="module")
def setup():
    import paper_1810_08429_b300 as gca
    assert torch.cuda.is_available()
    v, t = synth.mesh_for_config("sphere1280")
    tree = gca.tree_build(v, t, 32)
    h = gca.build(v, t, tree, gca.Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6,
                                         sauter_q=5))
    return gca, h


def _noalloc(gca, h, prec, x, y):
    n, R = x.shape
    stream = torch.cuda.current_stream().cuda_stream
    return gca.lib.h2_matvec_noalloc(h._h, gca._PREC[prec], R, ctypes.c_void_p(x.data_ptr()), n,
                                     ctypes.c_void_p(y.data_ptr()), n, ctypes.c_void_p(stream))


def _colmajor(a, dt):
    return torch.from_numpy(np.asfortranarray(a)).to(dt).cuda().t().contiguous().t()


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("nrhs", [1, 3, 17])
def test_matches_h2_matvec_twice(setup, prec, nrhs):
    gca, h = setup
    dt = torch.float64 if prec == "f64" else torch.float32
    n = h.n
    for call, seed in enumerate((11, 12)):
        x = _colmajor(synth.uniform_rhs(n, nrhs, seed=seed + nrhs), dt)
        ref = h.matvec(x, prec)
        y = torch.full((nrhs, n), float("nan"), dtype=dt, device="cuda").t()
        rc = _noalloc(gca, h, prec, x, y)
        assert rc == 0, gca.lib.gca_last_error()
        torch.cuda.synchronize()
        err = _rel(y, ref)
        assert np.all(np.isfinite(err)) and err.max() <= TOL[prec], (call, err.max())
    st = ctypes.c_int32(-99)
    assert gca.lib.gca_h2_status(h._h, ctypes.byref(st)) == 0 and st.value == 0


def test_rejects_oversize(setup):
    gca, h = setup
    n, R = h.n, 4096  # x and y in cluster order alone need 2 n R 8 bytes > 32 MiB
    x = torch.zeros((R, n), dtype=torch.float64, device="cuda").t()
    y = torch.zeros((R, n), dtype=torch.float64, device="cuda").t()
    rc = _noalloc(gca, h, "f64", x, y)
    assert rc == -6  # GCA_ERR_UNSUPPORTED
    assert b"scratch" in gca.lib.gca_last_error()
    # the rejected call left nothing behind: the next product is still right
    xs = _colmajor(synth.uniform_rhs(n, 2, seed=5), torch.float64)
    ys = torch.empty((2, n), dtype=torch.float64, device="cuda").t()
    assert _noalloc(gca, h, "f64", xs, ys) == 0
    assert _rel(ys, h.matvec(xs, "f64")).max() <= TOL["f64"]


def test_invalid_arguments(setup):
    gca, h = setup
    n = h.n
    x = torch.zeros((1, n), dtype=torch.float64, device="cuda").t()
    y = torch.zeros((1, n), dtype=torch.float64, device="cuda").t()
    null = ctypes.c_void_p(0)
    assert gca.lib.h2_matvec_noalloc(None, 0, 1, ctypes.c_void_p(x.data_ptr()), n,
                                     ctypes.c_void_p(y.data_ptr()), n, null) == -1
    assert gca.lib.h2_matvec_noalloc(h._h, 0, 0, ctypes.c_void_p(x.data_ptr()), n,
                                     ctypes.c_void_p(y.data_ptr()), n, null) == -1
    assert gca.lib.h2_matvec_noalloc(h._h, 0, 1, ctypes.c_void_p(x.data_ptr()), n - 1,
                                     ctypes.c_void_p(y.data_ptr()), n, null) == -1


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_allocates_no_device_memory(setup, prec):
    """The point of the entry point: a product on a handle that never ran an
    allocating product leaves the device's free memory unchanged.  A first
    call on another handle loads the kernels (lazy module loading may place
    code in device memory); the measured call is on a fresh handle."""
    gca, h = setup
    dt = torch.float64 if prec == "f64" else torch.float32
    n = h.n
    x = _colmajor(synth.uniform_rhs(n, 4, seed=21), dt)
    y = torch.empty((4, n), dtype=dt, device="cuda").t()
    assert _noalloc(gca, h, prec, x, y) == 0
    v, t = synth.mesh_for_config("sphere1280")
    fresh = gca.build(v, t, gca.tree_build(v, t, 32),
                      gca.Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5))
    y2 = torch.empty((4, n), dtype=dt, device="cuda").t()
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    assert _noalloc(gca, fresh, prec, x, y2) == 0
    torch.cuda.synchronize()
    after = torch.cuda.mem_get_info()[0]
    assert after == before
    assert _rel(y2, h.matvec(x, prec)).max() <= TOL[prec]
