"""Full-size configurations on the GPU.

* The benchmark's workload in the benchmark's launch configuration: the
  20480-triangle sphere and its perturbed copy built together
  (gca_build_batch; leaf 64, eta 2, m 4, tol 1e-8) and applied in one
  persistent launch with 16 right-hand sides N(0, 1).  Tree and block tree
  equal the oracle's; sampled coupling and near-field entries and leaf
  bases match the oracle's; sampled rows of the float64 product match the dense G within
  the compression error; the adjoint identity holds; float32 and bfloat16
  products stay within their bounds of the float64 product.
* The 81920-triangle sphere (bench parameters): the oracle's tree and block
  tree, sampled coupling and near-field entries, leaf bases and dense rows;
  with 64 right-hand sides, float32 and bfloat16 products (and transposes)
  against float64 per right-hand side.
* 256 meshes of uneven size and type (1280-20480 triangles, 1-32
  right-hand sides each) in one persistent float32 launch, also replayed
  from a CUDA graph, against each mesh's own product; the float64 product
  of one mesh and the oracle's H^2 of the smallest mesh bound the float32
  error.

Float32 bound 1e-6 and bfloat16 bound 1.6e-2: relative 2-norm per
right-hand side.
"""

import numpy as np
import pytest

import sampling
import synth
from oracle import gca as ogca, h2 as oh2
from oracle.galerkin import Galerkin
from oracle.params import Params as OParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFG2 = dict(leaf_size=64, eta=2.0, box_gauss_m=4, aca_tol=1e-8, sauter_q=5)
TOL32 = 1e-6
TOL16 = 1.6e-2


@pytest.fixture(scope="module")
def lib():
    import paper_1810_08429_b300 as gca
    assert torch.cuda.is_available()
    return gca


def cols(a, b):
    a = a.double().cpu().numpy().reshape(a.shape[0], -1)
    b = b.double().cpu().numpy().reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


def colmajor(a, dt):
    return torch.from_numpy(np.asfortranarray(a)).to(dt).cuda().t().contiguous().t()


@pytest.fixture(scope="module")
def bench_batch(lib):
    meshes = [synth.mesh_for_config(nm) for nm in ("sphere20480", "perturbed20480")]
    trees = [lib.tree_build(v, t, CFG2["leaf_size"]) for v, t in meshes]
    b = lib.build_batch(meshes, trees, lib.Params(**CFG2))
    return meshes, trees, b


def test_bench_workload_samples_match_oracle(bench_batch):
    meshes, trees, b = bench_batch
    p = OParams(**CFG2)
    rng = np.random.default_rng(0)
    for (v, t), tr, h in zip(meshes, trees, b.handles):
        tree, lo, hi, far, near = sampling.oracle_geometry(v, t, p)
        sampling.check_tree(tr, tree)
        dump = h.export()
        sampling.check_blocks(dump, far, near)
        gal = Galerkin(v, t, p.sauter_q)
        sampling.check_near_entries(dump, tree, gal, rng)
        sampling.check_coupling_entries(dump, gal, rng)
        sampling.check_leaf_bases(dump, tree, lo, hi, gal, p, rng)


def test_bench_workload_products(bench_batch):
    meshes, trees, b = bench_batch
    xs = [synth.normal_rhs(len(t), 16, seed=0) for _, t in meshes]
    x64 = [colmajor(x, torch.float64) for x in xs]
    x32 = [colmajor(x, torch.float32) for x in xs]
    y64 = b.matvec(x64, "f64")
    y32 = b.matvec(x32, "f32")
    y16 = b.matvec(x32, "bf16")
    yt64 = b.matvec(x64, "f64", transpose=True)
    yt32 = b.matvec(x32, "f32", transpose=True)
    rng = np.random.default_rng(1)
    for i, (v, t) in enumerate(meshes):
        assert cols(y32[i], y64[i]).max() <= TOL32
        assert cols(y16[i], y64[i]).max() <= TOL16
        assert cols(yt32[i], yt64[i]).max() <= TOL32
        # rows of the float64 product against the dense Galerkin matrix
        gal = Galerkin(v, t, CFG2["sauter_q"])
        sampling.check_dense_rows(y64[i].cpu().numpy(), xs[i], v, t, gal, rng, rows=3)
    assert b.status() == 0


def test_adjoint_identity_full_size(bench_batch):
    meshes, trees, b = bench_batch
    n = len(meshes[0][1])
    a = [colmajor(synth.normal_rhs(len(t), 4, seed=5), torch.float64) for _, t in meshes]
    c = [colmajor(synth.normal_rhs(len(t), 4, seed=6), torch.float64) for _, t in meshes]
    hc = b.matvec(c, "f64")
    hta = b.matvec(a, "f64", transpose=True)
    for i in range(len(meshes)):
        lhs = (a[i] * hc[i]).sum(0)
        rhs = (hta[i] * c[i]).sum(0)
        scale = a[i].norm(dim=0) * hc[i].norm(dim=0)
        assert ((lhs - rhs).abs() / scale).max() <= 1e-13, n


@pytest.fixture(scope="module")
def sphere81920(lib):
    v, t = synth.mesh_for_config("sphere81920")
    tree = lib.tree_build(v, t, CFG2["leaf_size"])
    h = lib.build(v, t, tree, lib.Params(**CFG2))
    return v, t, tree, h


def test_sphere81920_samples_match_oracle(sphere81920):
    """The precision configuration (81920 triangles, built with the bench
    parameters) on samples the oracle computes one by one: its tree and block
    tree, coupling and near-field entries, leaf bases, and rows of the dense
    G against the float64 product."""
    v, t, tr, h = sphere81920
    p = OParams(**CFG2)
    rng = np.random.default_rng(81920)
    tree, lo, hi, far, near = sampling.oracle_geometry(v, t, p)
    sampling.check_tree(tr, tree)
    dump = h.export()
    sampling.check_blocks(dump, far, near)
    gal = Galerkin(v, t, p.sauter_q)
    sampling.check_near_entries(dump, tree, gal, rng)
    sampling.check_coupling_entries(dump, gal, rng)
    sampling.check_leaf_bases(dump, tree, lo, hi, gal, p, rng)
    del dump
    x = synth.normal_rhs(len(t), 4, seed=3)
    y = h.matvec(colmajor(x, torch.float64), "f64").cpu().numpy()
    sampling.check_dense_rows(y, x, v, t, gal, rng, rows=3)


def test_sphere81920_precision(sphere81920):
    v, t, tree, h = sphere81920
    X = synth.normal_rhs(len(t), 64, seed=0)
    x64 = colmajor(X, torch.float64)
    x32 = colmajor(X, torch.float32)
    for transpose in (False, True):
        y64 = h.matvec(x64, "f64", transpose=transpose)
        e32 = cols(h.matvec(x32, "f32", transpose=transpose), y64)
        e16 = cols(h.matvec(x32, "bf16", transpose=transpose), y64)
        assert e32.max() <= TOL32, e32.max()
        assert e16.max() <= TOL16, e16.max()
    assert h.status() == 0


@pytest.fixture(scope="module")
def ragged(lib):
    meshes = synth.batch_meshes(256, seed=0)
    rng = np.random.default_rng(0)
    R = [int(r) for r in rng.integers(1, 33, size=len(meshes))]
    trees = [lib.tree_build(v, t, CFG2["leaf_size"]) for v, t in meshes]
    flags = lib.DROP_F64 | lib.DROP_BF16 | lib.DROP_EXPORT
    b = lib.build_batch(meshes, trees, lib.Params(**CFG2, flags=flags))
    xs = [colmajor(synth.uniform_rhs(len(t), r, seed=i), torch.float32)
          for i, ((_, t), r) in enumerate(zip(meshes, R))]
    return meshes, trees, R, b, xs


def test_ragged_batch_one_launch(lib, ragged):
    meshes, trees, R, b, xs = ragged
    ys = b.matvec(xs, "f32")
    worst = 0.0
    for i, h in enumerate(b.handles):
        single = h.matvec(xs[i], "f32")
        worst = max(worst, cols(ys[i], single).max())
    assert worst <= 1e-5
    assert b.status() == 0
    # a dropped precision is refused, not computed
    with pytest.raises(lib.GCAError):
        b.handles[0].matvec(xs[0].double(), "f64")


def test_ragged_batch_float32_error(lib, ragged):
    meshes, trees, R, b, xs = ragged
    ys = b.matvec(xs, "f32")
    # the smallest mesh against the oracle's float64 H^2
    i = int(np.argmin([len(t) for _, t in meshes]))
    v, t = meshes[i]
    Ho = ogca.build_h2(v, t, OParams(**CFG2))
    ref = oh2.matvec(Ho, xs[i].double().cpu().numpy())
    assert cols(ys[i], torch.from_numpy(ref)).max() <= TOL32
    # the largest mesh against its own float64 product
    j = int(np.argmax([len(t) for _, t in meshes]))
    v, t = meshes[j]
    h64 = lib.build(v, t, trees[j], lib.Params(**CFG2, flags=lib.DROP_BF16 | lib.DROP_EXPORT))
    assert cols(ys[j], h64.matvec(xs[j].double(), "f64")).max() <= TOL32


def test_ragged_batch_graph_replay(lib, ragged):
    meshes, trees, R, b, xs = ragged
    outs = [torch.empty((x.shape[1], x.shape[0]), dtype=torch.float32, device="cuda").t() for x in xs]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        b.matvec(xs, "f32", outs=outs)  # sizes the workspace and uploads the descriptors
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.matvec(xs, "f32", outs=outs)
    for seed in (11, 12):
        for i, x in enumerate(xs):
            x.copy_(colmajor(synth.uniform_rhs(x.shape[0], x.shape[1], seed=seed + 1000 * i),
                             torch.float32))
        g.replay()
        torch.cuda.synchronize()
        for i, h in enumerate(b.handles[:16]):
            assert cols(outs[i], h.matvec(xs[i], "f32")).max() <= 1e-5
    assert b.status() == 0
