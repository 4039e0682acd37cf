"""Failure paths of the products and the build, reached without faulting the
GPU (the library's test hooks):

* a product whose dependency waits can never be satisfied (a count nothing
  reaches) with a short wait bound: the launch must return on its own, the
  status must report the expired wait (bit 1, GCA_ERR_TIMEOUT through
  gca_h2_check), and after clearing the status the next product on the
  same handle and context must be right again;
* a device allocation that fails at every position inside gca_build and
  gca_build_batch: the call returns GCA_ERR_OOM and leaves the device's free
  memory where it was;
* a handle used while another device is current is refused before any launch.
"""

import gc
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1810_08429_b300 as gca
    assert torch.cuda.is_available()
    yield gca
    for name in ("wait_cycles", "stall_chain", "fail_alloc", "device_skew"):
        gca.test_hook(name, 0)


@pytest.fixture(scope="module")
def small(lib):
    v, t = synth.mesh_for_config("sphere1280")
    tree = lib.tree_build(v, t, 32)
    prm = lib.Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    return v, t, tree, prm


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return (np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)).max()


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_expired_wait_returns_and_reports_timeout(lib, small, prec):
    v, t, tree, prm = small
    h = lib.build(v, t, tree, prm)
    dt = torch.float64 if prec == "f64" else torch.float32
    x = torch.from_numpy(synth.normal_rhs(len(t), 4, seed=2)).to(dt).cuda()
    ref = h.matvec(x, prec)
    h.check()
    lib.test_hook("wait_cycles", 1 << 22)  # about 2 ms
    lib.test_hook("stall_chain", 1)
    try:
        t0 = time.perf_counter()
        h.matvec(x, prec)
        with pytest.raises(lib.GCAError) as e:
            h.check()
        elapsed = time.perf_counter() - t0
    finally:
        lib.test_hook("stall_chain", 0)
        lib.test_hook("wait_cycles", 0)
    assert e.value.status == lib.ERR_TIMEOUT
    assert h.status() & 1
    assert elapsed < 5.0
    h.clear_status()
    assert h.status() == 0
    assert _rel(h.matvec(x, prec), ref) <= (1e-12 if prec == "f64" else 1e-5)
    h.check()


def test_expired_wait_in_a_batch(lib, small):
    v, t, tree, prm = small
    b = lib.build_batch([(v, t), (v, t)], [tree, tree], prm)
    xs = [torch.from_numpy(synth.normal_rhs(len(t), 3, seed=s)).float().cuda() for s in (1, 2)]
    ref = b.matvec(xs, "f32")
    lib.test_hook("wait_cycles", 1 << 22)
    lib.test_hook("stall_chain", 1)
    try:
        b.matvec(xs, "f32")
        with pytest.raises(lib.GCAError) as e:
            b.check()
    finally:
        lib.test_hook("stall_chain", 0)
        lib.test_hook("wait_cycles", 0)
    assert e.value.status == lib.ERR_TIMEOUT
    b.clear_status()
    out = b.matvec(xs, "f32")
    b.check()
    for a, r in zip(out, ref):
        assert _rel(a, r) <= 1e-5


def _free_bytes():
    # handles of earlier tests can still sit in reference cycles (exception
    # tracebacks): collect them, and return torch's cached blocks, so that
    # only this test's allocations move the device's free memory
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def test_allocation_failure_in_build_frees_everything(lib, small):
    v, t, tree, prm = small
    lib.build(v, t, tree, prm).free()  # loads every kernel of the build
    before = _free_bytes()
    failed = 0
    for n in range(1, 400):
        lib.test_hook("fail_alloc", n)
        try:
            h = lib.build(v, t, tree, prm)
        except lib.GCAError as e:
            assert e.status == lib.ERR_OOM, str(e)
            failed += 1
            assert _free_bytes() == before, n
            continue
        finally:
            lib.test_hook("fail_alloc", 0)
        h.free()
        break
    assert failed >= 10  # every allocation of the build was made to fail once
    assert _free_bytes() == before


def test_allocation_failure_in_batch_build(lib, small):
    v, t, tree, prm = small
    lib.build_batch([(v, t)] * 2, [tree] * 2, prm).free()
    before = _free_bytes()
    for n in (1, 7, 40, 75):
        lib.test_hook("fail_alloc", n)
        try:
            with pytest.raises(lib.GCAError) as e:
                lib.build_batch([(v, t)] * 2, [tree] * 2, prm)
        finally:
            lib.test_hook("fail_alloc", 0)
        assert e.value.status == lib.ERR_OOM
        assert _free_bytes() == before, n


def test_handle_on_another_device_is_refused(lib):
    v, t = synth.mesh_for_config("sphere320")
    tree = lib.tree_build(v, t, 16)
    lib.test_hook("device_skew", 1)
    try:
        h = lib.build(v, t, tree, lib.Params(leaf_size=16))
    finally:
        lib.test_hook("device_skew", 0)
    x = torch.zeros((len(t), 2), dtype=torch.float64).cuda()
    for call in (lambda: h.matvec(x, "f64"), lambda: h.matvec(x, "f64", transpose=True),
                 lambda: h.matvec_noalloc(x, "f64"), lambda: h.check()):
        with pytest.raises(lib.GCAError) as e:
            call()
        assert e.value.status == lib.ERR_INVALID_ARG
        cur = torch.cuda.current_device()
        assert f"built on device {cur + 1}, but device {cur} is current" in str(e.value)
