"""Checkpoints of handles: a saved and reloaded handle exports the same
representation bit for bit, keeps the construction's counts, and its
products equal the saved handle's and the oracle's (Sect. 4 representation);
two-sided handles are refused; a damaged file is refused before any device
allocation."""

import numpy as np
import pytest

import synth
from oracle import gca as ogca, h2 as oh2
from oracle.params import Params as OParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRM = dict(leaf_size=16, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)


def rel_cols(a, b):
    a = np.asarray(a).reshape(len(a), -1)
    b = np.asarray(b).reshape(len(b), -1)
    return (np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)).max()


@pytest.fixture(scope="module")
def single_layer():
    import paper_1810_08429_b300 as gca
    v, t = synth.mesh_for_config("sphere320")
    tree = gca.tree_build(v, t, PRM["leaf_size"])
    h = gca.build(v, t, tree, gca.Params(**PRM))
    return gca, v, t, h


def test_round_trip_single_layer(single_layer, tmp_path):
    gca, v, t, h = single_layer
    path = tmp_path / "sphere320.gca"
    h.save(str(path))
    assert path.exists() and not (tmp_path / "sphere320.gca.tmp").exists()
    g = gca.load(str(path))
    a, b = h.export(), g.export()
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    sa, sb = h.stats(), g.stats()
    for key in ("n", "nclusters", "depth", "k", "nfar", "nnear", "max_rank", "rank_sum", "v_entries",
                "e_entries", "s_entries", "n_entries"):
        assert sa[key] == sb[key], key
    assert list(sa["n_singular"]) == list(sb["n_singular"])
    x = torch.from_numpy(synth.normal_rhs(len(t), 5, seed=3)).cuda()
    for transpose in (False, True):
        ya = h.matvec(x, "f64", transpose=transpose)
        yb = g.matvec(x, "f64", transpose=transpose)
        assert rel_cols(yb.cpu().numpy(), ya.cpu().numpy()) <= 1e-14
    for prec in ("f32", "bf16"):
        ya = h.matvec(x.float(), prec)
        yb = g.matvec(x.float(), prec)
        assert rel_cols(yb.double().cpu().numpy(), ya.double().cpu().numpy()) <= 1e-6
    # and against the oracle's own construction
    ref = ogca.build_h2(v, t, OParams(**PRM))
    want = oh2.matvec(ref, x.cpu().numpy())
    assert rel_cols(g.matvec(x, "f64").cpu().numpy(), want) <= 1e-10
    assert g.status() == 0


def test_load_with_dropped_precisions(single_layer, tmp_path):
    gca, v, t, h = single_layer
    path = tmp_path / "lean.gca"
    h.save(str(path))
    g = gca.load(str(path), flags=gca.DROP_F64 | gca.DROP_BF16)
    x = torch.from_numpy(synth.normal_rhs(len(t), 2, seed=4)).float().cuda()
    assert rel_cols(g.matvec(x, "f32").double().cpu().numpy(),
                    h.matvec(x, "f32").double().cpu().numpy()) <= 1e-6
    with pytest.raises(gca.GCAError) as e:
        g.matvec(x.double(), "f64")
    assert e.value.status == gca.ERR_UNSUPPORTED


def test_overwrite_and_damaged_files(single_layer, tmp_path):
    gca, v, t, h = single_layer
    path = tmp_path / "h.gca"
    path.write_bytes(b"old contents")
    h.save(str(path))  # replaces the file
    data = path.read_bytes()
    free0 = torch.cuda.mem_get_info()[0]
    for blob in (data[: len(data) // 2], data[:8] + bytes([data[8] ^ 1]) + data[9:]):
        bad = tmp_path / "bad.gca"
        bad.write_bytes(blob)
        with pytest.raises(gca.GCAError) as e:
            gca.load(str(bad))
        assert e.value.status == gca.ERR_IO
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    g = gca.load(str(path))
    assert np.array_equal(g.export(("S",))["S"], h.export(("S",))["S"])


def test_round_trip_nodal_basis(tmp_path):
    import paper_1810_08429_b300 as gca
    v, t = synth.mesh_for_config("sphere320")
    tv = gca.tree_build_points(v, 16)
    h = gca.build_p1(v, t, tv, gca.Params(**PRM))
    path = tmp_path / "p1.gca"
    h.save(str(path))
    g = gca.load(str(path))
    x = torch.from_numpy(synth.normal_rhs(len(v), 3, seed=5)).cuda()
    for transpose in (False, True):
        ya = h.matvec(x, "f64", transpose=transpose)
        yb = g.matvec(x, "f64", transpose=transpose)
        assert rel_cols(yb.cpu().numpy(), ya.cpu().numpy()) <= 1e-14
    assert g.stats()["k"] == h.stats()["k"]


def test_two_sided_handles_refused(tmp_path):
    import paper_1810_08429_b300 as gca
    v, t = synth.mesh_for_config("sphere320")
    tree = gca.tree_build(v, t, 16)
    h = gca.build_double_layer(v, t, tree, gca.Params(**PRM))
    with pytest.raises(gca.GCAError) as e:
        h.save(str(tmp_path / "dl.gca"))
    assert e.value.status == gca.ERR_UNSUPPORTED
    assert not (tmp_path / "dl.gca").exists() and not (tmp_path / "dl.gca.tmp").exists()
