"""GPU parity: the CUDA construction and products against the FP64 oracle,
on the 1280-triangle sphere (leaf 32, eta 2, m = 3, tol 1e-6, q = 5) and
small edge cases.  Integer results (ranks, pivots, block lists) must match
exactly; float64 entries of G (coupling and near-field blocks) and float64
products within a relative 1e-10; float32 products within 1e-6 and bfloat16
products within 1.6e-2 (relative 2-norm per right-hand side against the
oracle's float64 product).

Bases V and transfer matrices E are interpolation operators
A[:, Q] A[P, Q]^{-1}; at tight ACA tolerances they move by up to ~1e-9
when A moves by one rounding error (pinned in test_oracle_gca.py), so they
are held to 1e-10 at tolerance 1e-6 and to TOL_BASIS_TIGHT below that.
"""

import numpy as np
import pytest

import synth
from oracle import cluster, gca as ogca, h2 as oh2
from oracle.params import Params as OParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-6
TOL16 = 1.6e-2
TOL_BASIS_TIGHT = 1e-8


@pytest.fixture(scope="module")
def lib():
    import paper_1810_08429_b300 as gca
    assert torch.cuda.is_available()
    return gca


def _params(lib, p):
    return lib.Params(leaf_size=p.leaf_size, eta=p.eta, box_gauss_m=p.box_gauss_m,
                      aca_tol=p.aca_tol, sauter_q=p.sauter_q)


@pytest.fixture(scope="module")
def gpu_1280(lib, sphere1280, small_params):
    v, t = sphere1280
    tree = lib.tree_build(v, t, small_params.leaf_size)
    h = lib.build(v, t, tree, _params(lib, small_params))
    return h, h.export(), tree


def _split(tree, rank, flat, sizes):
    out, at = {}, 0
    for key, sz in sizes:
        out[key] = flat[at:at + sz]
        at += sz
    assert at == len(flat)
    return out


def compare_structure(h2o, dump, tree):
    nc = len(tree["begin"])
    assert np.array_equal(dump["rank"], h2o.bases.rank.astype(np.int32))
    at = 0
    for c in range(nc):
        r = dump["rank"][c]
        got = dump["pivots"][at:at + r]
        at += r
        if c == 0:
            continue
        assert np.array_equal(got, h2o.bases.pivots[c]), f"pivots of cluster {c}"
    assert set(map(tuple, dump["far"].tolist())) == set(h2o.far)
    assert set(map(tuple, dump["near"].tolist())) == set(h2o.near)


def compare_coefficients(h2o, dump, tree, tol, tol_basis=None):
    tol_basis = tol if tol_basis is None else tol_basis
    nc = len(tree["begin"])
    rank = dump["rank"]
    sz = lambda c: tree["end"][c] - tree["begin"][c]  # noqa: E731
    par = cluster.parents({k: np.asarray(v) for k, v in tree.items()})
    # leaf bases
    at = 0
    scale = max(np.abs(m).max() for m in h2o.bases.V.values() if m.size)
    for c in range(1, nc):
        if tree["child0"][c] >= 0:
            continue
        blk = dump["V"][at:at + sz(c) * rank[c]].reshape(sz(c), rank[c])
        at += sz(c) * rank[c]
        if blk.size == 0:
            assert h2o.bases.V[c].size == 0
            continue
        assert np.abs(blk - h2o.bases.V[c]).max() <= tol_basis * scale, f"V of leaf {c}"
    assert at == len(dump["V"])
    # transfer matrices
    at = 0
    scale = max([np.abs(m).max() for m in h2o.bases.E.values() if m.size] + [1.0])
    for c in range(1, nc):
        if par[c] <= 0:
            continue
        blk = dump["E"][at:at + rank[c] * rank[par[c]]].reshape(rank[c], rank[par[c]])
        at += rank[c] * rank[par[c]]
        if blk.size == 0:  # a transfer into a cluster the H^2 matrix does not use
            assert h2o.bases.E[c].size == 0
            continue
        assert np.abs(blk - h2o.bases.E[c]).max() <= tol_basis * scale, f"E of cluster {c}"
    assert at == len(dump["E"])
    # coupling blocks
    at = 0
    scale = max(np.abs(m).max() for m in h2o.S.values()) if h2o.S else 1.0
    for (t, s) in map(tuple, dump["far"].tolist()):
        blk = dump["S"][at:at + rank[t] * rank[s]].reshape(rank[t], rank[s])
        at += rank[t] * rank[s]
        assert np.abs(blk - h2o.S[(t, s)]).max() <= tol * scale, f"S of block {(t, s)}"
    # near-field blocks
    at = 0
    scale = max(np.abs(m).max() for m in h2o.N.values())
    for (t, s) in map(tuple, dump["near"].tolist()):
        blk = dump["N"][at:at + sz(t) * sz(s)].reshape(sz(t), sz(s))
        at += sz(t) * sz(s)
        assert np.abs(blk - h2o.N[(t, s)]).max() <= tol * scale, f"N of block {(t, s)}"


def rel_cols(a, b):
    a = np.asarray(a).reshape(len(a), -1)
    b = np.asarray(b).reshape(len(b), -1)
    return (np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)).max()


def test_structure_matches_oracle(gpu_1280, h2_1280):
    h, dump, tree = gpu_1280
    compare_structure(h2_1280, dump, tree)


def test_coefficients_match_oracle(gpu_1280, h2_1280):
    h, dump, tree = gpu_1280
    compare_coefficients(h2_1280, dump, tree, TOL64)


def test_stats_consistent(gpu_1280, h2_1280):
    h, dump, tree = gpu_1280
    s = h.stats()
    st = oh2.storage(h2_1280)
    assert (s["v_entries"], s["e_entries"], s["s_entries"], s["n_entries"]) == \
        (st["V"], st["E"], st["S"], st["N"])
    # touching ordered pairs of a closed conforming mesh: n identical, 3n edges
    assert s["n_singular"][3] == 1280 and s["n_singular"][2] == 3 * 1280


def test_single_layer_couplings_mirrored(gpu_1280):
    """The transposed product of the single layer runs the product's own plan
    and coupling panels (the handle keeps no S^T).  That rests on the
    coupling blocks coming in mirrored pairs with transposed entries: G is
    symmetric (Eq. 1, g(x, y) = g(y, x), the same 7-point rule on both
    triangles) and a mirrored pair is evaluated once.  The near field keeps
    its transposed entries (Sauter-Schwab rules are not symmetric in the two
    triangles), checked by the transposed products against the oracle."""
    h, dump, tree = gpu_1280
    rank = dump["rank"]
    blocks, at = {}, 0
    for (t, s) in map(tuple, dump["far"].tolist()):
        blocks[(t, s)] = dump["S"][at:at + rank[t] * rank[s]].reshape(rank[t], rank[s])
        at += rank[t] * rank[s]
    for (t, s), b in blocks.items():
        assert np.array_equal(b, blocks[(s, t)].T), f"S of {(t, s)} and its mirror"


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 1e-6)])
def test_symmetric_transpose_adjoint(gpu_1280, prec, tol):
    """<G^T x, z> = <x, G z> (float64), and the float32 transposed product
    against the float64 one, for the symmetric handle whose transposed
    product reuses the product's plan."""
    h, _, _ = gpu_1280
    x = torch.from_numpy(synth.normal_rhs(1280, 4, seed=3)).cuda()
    z = torch.from_numpy(synth.normal_rhs(1280, 4, seed=4)).cuda()
    ref = h.matvec(x, "f64", transpose=True)
    if prec == "f64":
        lhs = (ref * z).sum(0)
        rhs = (x * h.matvec(z, "f64")).sum(0)
        assert ((lhs - rhs).abs() / rhs.abs()).max().item() <= tol
    else:
        yt = h.matvec(x.float(), prec, transpose=True).double()
        assert ((yt - ref).norm(dim=0) / ref.norm(dim=0)).max().item() <= tol


@pytest.mark.parametrize("nrhs", [1, 3, 17])
def test_matvec_f64(gpu_1280, h2_1280, nrhs):
    h, _, _ = gpu_1280
    x = synth.uniform_rhs(1280, nrhs, seed=0)
    ref = oh2.matvec(h2_1280, x)
    xt = torch.from_numpy(x).cuda()
    y = h.matvec(xt, "f64").cpu().numpy()
    assert rel_cols(y, ref) <= TOL64
    yt = h.matvec(xt, "f64", transpose=True).cpu().numpy()
    assert rel_cols(yt, oh2.matvec_t(h2_1280, x)) <= TOL64
    assert h.status() == 0


@pytest.mark.parametrize("prec,tol", [("f32", TOL32), ("bf16", TOL16)])
def test_matvec_reduced(gpu_1280, h2_1280, prec, tol):
    h, _, _ = gpu_1280
    x = synth.normal_rhs(1280, 16, seed=0)
    ref = oh2.matvec(h2_1280, x)
    refT = oh2.matvec_t(h2_1280, x)
    xt = torch.from_numpy(x).float().cuda()
    y = h.matvec(xt, prec).double().cpu().numpy()
    yt = h.matvec(xt, prec, transpose=True).double().cpu().numpy()
    assert rel_cols(y, ref) <= tol
    assert rel_cols(yt, refT) <= tol
    assert h.status() == 0


def test_matvec_leading_dimension(gpu_1280, h2_1280):
    h, _, _ = gpu_1280
    x = synth.uniform_rhs(1280, 2, seed=5)
    big = torch.zeros((2, 1300), dtype=torch.float64, device="cuda")
    big[:, :1280] = torch.from_numpy(x.T.copy()).cuda()
    xin = big.t()[:1280]                     # column-major, ldx = 1300
    out = torch.full((2, 1310), 7.0, dtype=torch.float64, device="cuda")
    yv = out.t()[:1280]                      # ldy = 1310
    h.matvec(xin, "f64", out=yv)
    assert rel_cols(yv.cpu().numpy(), oh2.matvec(h2_1280, x)) <= TOL64
    assert (out[:, 1280:] == 7.0).all()       # padding untouched


def test_single_leaf_mesh(lib):
    """n <= leaf size: no bases, the whole matrix is one near-field block."""
    v, t = synth.icosahedron()
    p = OParams(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    ref = ogca.build_h2(v, t, p)
    tree = lib.tree_build(v, t, 32)
    h = lib.build(v, t, tree, _params(lib, p))
    dump = h.export()
    compare_structure(ref, dump, tree)
    assert np.abs(dump["N"].reshape(20, 20) - ref.N[(0, 0)]).max() <= TOL64 * np.abs(ref.N[(0, 0)]).max()
    x = synth.uniform_rhs(20, 2, seed=3)
    y = h.matvec(torch.from_numpy(x).cuda(), "f64").cpu().numpy()
    assert rel_cols(y, oh2.matvec(ref, x)) <= TOL64


@pytest.mark.parametrize("name,leaf,m,tol", [("perturbed320", 16, 2, 1e-4),
                                             ("ellipsoid1280", 24, 3, 1e-8)])
def test_other_surfaces(lib, name, leaf, m, tol):
    """Ragged leaves, other box orders and tolerances, non-spherical surfaces."""
    v, t = synth.mesh_for_config(name)
    p = OParams(leaf_size=leaf, eta=2.0, box_gauss_m=m, aca_tol=tol, sauter_q=4)
    ref = ogca.build_h2(v, t, p)
    tree = lib.tree_build(v, t, leaf)
    h = lib.build(v, t, tree, _params(lib, p))
    dump = h.export()
    compare_structure(ref, dump, tree)
    compare_coefficients(ref, dump, tree, TOL64, TOL64 if tol >= 1e-6 else TOL_BASIS_TIGHT)
    x = synth.normal_rhs(len(t), 5, seed=1)
    y = h.matvec(torch.from_numpy(x).cuda(), "f64").cpu().numpy()
    assert rel_cols(y, oh2.matvec(ref, x)) <= TOL64


def test_close_disjoint_pair_uses_float64(lib):
    """Two disjoint triangles 5e-5 apart inside the icosahedron: their nodes are
    far closer than the float-pair floor 2^(E-8) of the near field (E = 1
    here), so their entries must have float64 accuracy (the float-pair rule
    would be about 1e-9 off); the other disjoint entries stay within the
    float-pair bound."""
    v0, t0 = synth.icosahedron()
    tiny = np.array([[0.0, 0.0, 0.0], [1e-3, 0.0, 0.0], [0.0, 1e-3, 0.0]])
    v = np.vstack([v0, tiny, tiny + [0.0, 0.0, 5e-5]])
    nv = len(v0)
    t = np.vstack([t0, [[nv, nv + 1, nv + 2], [nv + 3, nv + 4, nv + 5]]]).astype(np.int32)
    p = OParams(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    ref = ogca.build_h2(v, t, p)
    tree = lib.tree_build(v, t, 32)
    h = lib.build(v, t, tree, _params(lib, p))
    dump = h.export()
    compare_structure(ref, dump, tree)
    N = dump["N"].reshape(22, 22)
    perm = np.asarray(tree["perm"])
    R = ref.N[(0, 0)]
    err = np.abs(N - R) / np.abs(R)
    assert err.max() <= 1e-11
    a, b = (int(np.nonzero(perm == k)[0][0]) for k in (20, 21))
    assert err[a, b] <= 1e-13 and err[b, a] <= 1e-13


def test_translated_scaled_mesh(lib):
    """The 1280-triangle sphere scaled by 1000 and moved far from the origin:
    the float-pair grid follows the mesh's box (origin at its centre, step
    2^(E-22) from its half width), so the entries keep their accuracy."""
    v, t = synth.mesh_for_config("sphere1280")
    v = v * 1000.0 + np.array([3.0e4, -2.0e4, 5.0e3])
    p = OParams(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    ref = ogca.build_h2(v, t, p)
    tree = lib.tree_build(v, t, 32)
    h = lib.build(v, t, tree, _params(lib, p))
    dump = h.export()
    compare_structure(ref, dump, tree)
    compare_coefficients(ref, dump, tree, TOL64)
    x = synth.normal_rhs(len(t), 3, seed=2)
    y = h.matvec(torch.from_numpy(x).cuda(), "f64").cpu().numpy()
    assert rel_cols(y, oh2.matvec(ref, x)) <= TOL64


def test_mesh_scale_outside_float_range_refused(lib):
    """A mesh 1e-14 wide would underflow the float-pair quadrature: the build
    refuses it with an error instead of returning wrong entries."""
    v, t = synth.icosahedron()
    v = v * 1e-14
    p = OParams(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
    tree = lib.tree_build(v, t, 32)
    with pytest.raises(Exception, match="half width"):
        lib.build(v, t, tree, _params(lib, p))


def test_invalid_matvec_arguments(gpu_1280):
    import paper_1810_08429_b300 as gca
    h, _, _ = gpu_1280
    x = torch.zeros(1280, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(gca.GCAError):
        h.matvec_raw(0, 0, x.data_ptr(), 1280, x.data_ptr(), 1280, None)
    with pytest.raises(gca.GCAError):
        h.matvec_raw(0, 2, x.data_ptr(), 100, x.data_ptr(), 1280, None)
    with pytest.raises(gca.GCAError):
        h.matvec_raw(7, 2, x.data_ptr(), 1280, x.data_ptr(), 1280, None)


def test_pageable_host_memory_refused(gpu_1280):
    import paper_1810_08429_b300 as gca
    h, _, _ = gpu_1280
    x = np.zeros((2, 1280))  # pageable host memory: refused before any launch
    y = torch.zeros(1280, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(gca.GCAError):
        h.matvec_raw(0, 2, x.ctypes.data, 1280, y.data_ptr(), 1280, None)
    with pytest.raises(gca.GCAError):
        h.matvec_raw(0, 2, y.data_ptr(), 1280, x.ctypes.data, 1280, None)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_host_io_matches_device_io(gpu_1280, h2_1280, prec):
    """x and y in page-locked host memory, read and written in place by the
    product, give the product of device x and y (and the oracle's)."""
    h, _, _ = gpu_1280
    dt = torch.float64 if prec == "f64" else torch.float32
    x = synth.normal_rhs(1280, 3, seed=4)
    xd = torch.from_numpy(x).to("cuda", dt)
    xh = torch.from_numpy(x).to(dt).pin_memory()
    yd = h.matvec(xd, prec).cpu()
    yh = h.matvec(xh, prec)
    torch.cuda.synchronize()
    assert not yh.is_cuda and yh.is_pinned()
    assert rel_cols(yh.double().numpy(), yd.double().numpy()) <= (1e-13 if prec == "f64" else 1e-6)
    if prec == "f64":
        assert rel_cols(yh.numpy(), oh2.matvec(h2_1280, x)) <= TOL64
    yt = h.matvec(xh, prec, transpose=True)
    torch.cuda.synchronize()
    assert rel_cols(yt.double().numpy(), h.matvec(xd, prec, transpose=True).cpu().double().numpy()) <= \
        (1e-13 if prec == "f64" else 1e-6)


def test_float64_entries(lib, gpu_1280, h2_1280, sphere1280, small_params):
    """GCA_F64_ENTRIES: couplings, near field and Sauter-Schwab samples in
    float64 (the paper's precision) instead of float-pair arithmetic.  The
    bases are the same (the entries do not enter the cross approximation);
    the float64 entries match the oracle to 1e-12 of the largest entry and
    the float-pair ones to 1e-12 of each other's."""
    v, t = sphere1280
    h, d, tree = gpu_1280
    p = small_params
    h64 = lib.build(v, t, tree, lib.Params(leaf_size=p.leaf_size, eta=p.eta, box_gauss_m=p.box_gauss_m,
                                           aca_tol=p.aca_tol, sauter_q=p.sauter_q, flags=lib.F64_ENTRIES))
    d64 = h64.export()
    for k in ("rank", "pivots", "far", "near", "V", "E"):
        assert np.array_equal(d64[k], d[k]), k
    compare_coefficients(h2_1280, d64, tree, 1e-12, tol_basis=TOL64)
    for k in ("S", "N"):
        assert np.abs(d64[k] - d[k]).max() <= 1e-12 * np.abs(d64[k]).max(), k
    st, st64 = h.stats(), h64.stats()
    assert st["n_singular"] == st64["n_singular"]
    x = torch.from_numpy(synth.normal_rhs(len(t), 3, seed=5)).cuda()
    assert rel_cols(h64.matvec(x, "f64").cpu().numpy(), oh2.matvec(h2_1280, x.cpu().numpy())).max() <= 1e-10
