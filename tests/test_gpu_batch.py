"""Batched construction and products: meshes of different sizes and shapes
with different numbers of right-hand sides in one persistent launch give the
same results as the single-mesh products and the oracle."""

import numpy as np
import pytest

import synth
from oracle import gca as ogca, h2 as oh2
from oracle.params import Params as OParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel_cols(a, b):
    a = np.asarray(a).reshape(len(a), -1)
    b = np.asarray(b).reshape(len(b), -1)
    return (np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)).max()


@pytest.fixture(scope="module")
def batch_case():
    import paper_1810_08429_b300 as gca
    cases = [("sphere320", 16), ("perturbed320", 16), ("ellipsoid1280", 24)]
    p = OParams(leaf_size=16, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=4)
    meshes, trees, refs = [], [], []
    for name, leaf in cases:
        v, t = synth.mesh_for_config(name)
        meshes.append((v, t))
        trees.append(gca.tree_build(v, t, leaf))
        refs.append(ogca.build_h2(v, t, OParams(leaf_size=leaf, eta=2.0, box_gauss_m=3,
                                                aca_tol=1e-6, sauter_q=4)))
    b = gca.build_batch(meshes, trees, gca.Params(leaf_size=16, eta=2.0, box_gauss_m=3,
                                                  aca_tol=1e-6, sauter_q=4))
    return gca, b, meshes, refs


@pytest.mark.parametrize("transpose", [False, True])
def test_batch_f64_matches_oracle(batch_case, transpose):
    gca, b, meshes, refs = batch_case
    nrhs = [1, 5, 17]
    xs = [synth.normal_rhs(len(t), r, seed=i) for i, ((_, t), r) in enumerate(zip(meshes, nrhs))]
    ys = b.matvec([torch.from_numpy(x).cuda() for x in xs], "f64", transpose=transpose)
    for y, x, ref in zip(ys, xs, refs):
        want = oh2.matvec_t(ref, x) if transpose else oh2.matvec(ref, x)
        assert rel_cols(y.cpu().numpy(), want) <= 1e-10
    assert b.status() == 0


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("prec,R", [("f64", 12), ("f32", 32)])
def test_batch_equal_chunks(batch_case, prec, R, transpose):
    """Every mesh with the same number of right-hand-side chunks (3 of width 4
    in float64, 2 of width 16 in float32): the claim orders come from the
    batch's one-chunk orders, each claim repeated per chunk."""
    gca, b, meshes, refs = batch_case
    dt = torch.float64 if prec == "f64" else torch.float32
    xs = [synth.normal_rhs(len(t), R, seed=21 + i) for i, (_, t) in enumerate(meshes)]
    ys = b.matvec([torch.from_numpy(x).to(dt).cuda() for x in xs], prec, transpose=transpose)
    for y, x, ref in zip(ys, xs, refs):
        want = oh2.matvec_t(ref, x) if transpose else oh2.matvec(ref, x)
        assert rel_cols(y.double().cpu().numpy(), want) <= (1e-10 if prec == "f64" else 1e-6)
    assert b.status() == 0


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_batch_matches_single(batch_case, prec):
    gca, b, meshes, refs = batch_case
    nrhs = [16, 3, 16]
    xs = [torch.from_numpy(synth.normal_rhs(len(t), r, seed=7 + i)).float().cuda()
          for i, ((_, t), r) in enumerate(zip(meshes, nrhs))]
    ys = b.matvec(xs, prec)
    for h, x, y in zip(b.handles, xs, ys):
        single = h.matvec(x, prec)
        # same arithmetic; only the order of the atomic accumulations differs
        assert rel_cols(y.double().cpu().numpy(), single.double().cpu().numpy()) <= 1e-5
    assert b.status() == 0


def test_batch_host_io(batch_case):
    """A batched product with x and y in page-locked host memory (ragged R)
    equals the same product on device buffers."""
    gca, b, meshes, _ = batch_case
    nrhs = [2, 16, 5]
    xs = [synth.normal_rhs(len(t), r, seed=11 + i) for i, ((_, t), r) in enumerate(zip(meshes, nrhs))]
    yd = b.matvec([torch.from_numpy(x).cuda() for x in xs], "f64")
    yh = b.matvec([torch.from_numpy(x).pin_memory() for x in xs], "f64")
    torch.cuda.synchronize()
    for a, c in zip(yh, yd):
        assert not a.is_cuda
        c = c.cpu()
        assert float((a - c).norm() / c.norm()) <= 1e-13
