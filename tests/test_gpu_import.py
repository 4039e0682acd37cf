"""gca_h2_import: the oracle's GCA-H^2 representation (its bases, transfer
matrices, couplings and near field) imported through the C ABI and applied
by the GPU products, with the GPU construction bypassed.  The products must
equal the oracle's own H^2 products (Sect. 4 representation): float64 within
a relative 1e-10, float32 within 1e-6, bfloat16 within 1.6e-2 per
right-hand side.  A handle exported by the GPU build and imported again must
reproduce that handle's products."""

import numpy as np
import pytest

import synth
from oracle import gca as ogca, h2 as oh2
from oracle.params import Params as OParams
from oracle_dump import oracle_dump

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-6, "bf16": 1.6e-2}


@pytest.fixture(scope="module")
def lib():
    import paper_1810_08429_b300 as gca
    assert torch.cuda.is_available()
    return gca


def _rel(y, want):
    y = y.double().cpu().numpy()
    return np.linalg.norm(y - want, axis=0) / np.linalg.norm(want, axis=0)


@pytest.mark.parametrize("name,leaf,m,tol", [("sphere1280", 32, 3, 1e-6), ("ellipsoid1280", 16, 3, 1e-6),
                                             ("perturbed1280", 32, 4, 1e-8)])
def test_imported_oracle_h2_matches_oracle_products(lib, name, leaf, m, tol):
    v, t = synth.mesh_for_config(name)
    p = OParams(leaf_size=leaf, eta=2.0, box_gauss_m=m, aca_tol=tol, sauter_q=5)
    h2o = ogca.build_h2(v, t, p)
    h = lib.import_h2(h2o.tree, len(t), oracle_dump(h2o))
    st = h.stats()
    assert st["rank_sum"] == int(np.sum(h2o.bases.rank)) and st["nfar"] == len(h2o.far)
    x = synth.normal_rhs(len(t), 5, seed=3)
    want = oh2.matvec(h2o, x)
    want_t = oh2.matvec_t(h2o, x)
    for prec in ("f64", "f32", "bf16"):
        dt = torch.float64 if prec == "f64" else torch.float32
        xd = torch.from_numpy(x).to(dt).cuda()
        assert _rel(h.matvec(xd, prec), want).max() <= TOL[prec], prec
        assert _rel(h.matvec(xd, prec, transpose=True), want_t).max() <= TOL[prec], prec
        assert _rel(h.matvec_noalloc(xd, prec), want).max() <= TOL[prec], prec
    h.check()


def test_export_import_round_trip(lib, sphere1280, small_params):
    v, t = sphere1280
    tree = lib.tree_build(v, t, small_params.leaf_size)
    h = lib.build(v, t, tree, lib.Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5))
    d = h.export()
    h2 = lib.import_h2(tree, len(t), d)
    d2 = h2.export()
    for k in ("rank", "pivots", "far", "near", "V", "E", "S", "N"):
        assert np.array_equal(np.asarray(d[k]), np.asarray(d2[k])), k
    x = torch.from_numpy(synth.uniform_rhs(len(t), 3, seed=9)).cuda()
    a = h.matvec(x, "f64").cpu().numpy()
    assert _rel(h2.matvec(x, "f64"), a).max() <= 1e-13


def test_import_flags_drop_precision(lib):
    v, t = synth.mesh_for_config("sphere320")
    h2o = ogca.build_h2(v, t, OParams(leaf_size=16, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5))
    h = lib.import_h2(h2o.tree, len(t), oracle_dump(h2o), flags=lib.DROP_BF16 | lib.DROP_EXPORT)
    x = torch.from_numpy(synth.uniform_rhs(len(t), 2, seed=1)).float().cuda()
    with pytest.raises(lib.GCAError) as e:
        h.matvec(x, "bf16")
    assert e.value.status == lib.ERR_UNSUPPORTED
    assert _rel(h.matvec(x, "f32"), oh2.matvec(h2o, x.double().cpu().numpy())).max() <= TOL["f32"]
