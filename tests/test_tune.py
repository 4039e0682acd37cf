"""Tile-width autotuner: the table's file format (host only) and a tuned
batched product on the GPU."""
import os

import numpy as np
import pytest

import synth


@pytest.fixture
def gca():
    import paper_1810_08429_b300 as g
    g.tune_clear()
    yield g
    g.tune_clear()


def test_tune_table_roundtrip(gca, tmp_path):
    p = tmp_path / "tune.txt"
    p.write_text("dev_a|1|0|16|15 8\ndev_a|0|1|4|10 4\ndev_b|2|0|16|15 16\n")
    gca.tune_load(str(p))
    assert gca.tune_get("dev_a", "f32", False, 16, 40960) == 8    # log2(40960) = 15
    assert gca.tune_get("dev_a", "f64", True, 4, 1500) == 4       # log2(1500) = 10
    assert gca.tune_get("dev_b", "bf16", False, 16, 32768) == 16
    assert gca.tune_get("dev_a", "f32", False, 16, 70000) == 0    # another size class
    assert gca.tune_get("dev_a", "f32", True, 16, 40960) == 0     # another direction
    out = tmp_path / "out.txt"
    gca.tune_save(str(out))
    assert sorted(out.read_text().split("\n")[:-1]) == sorted(p.read_text().split("\n")[:-1])
    gca.tune_clear()
    assert gca.tune_get("dev_a", "f32", False, 16, 40960) == 0
    gca.tune_load(str(out))
    assert gca.tune_get("dev_a", "f32", False, 16, 40960) == 8


@pytest.mark.parametrize("bad", ["dev|1|0|16|15 3\n", "dev|1|0|16|15\n", "just words\n"])
def test_tune_load_rejects_malformed(gca, tmp_path, bad):
    p = tmp_path / "bad.txt"
    p.write_text("dev|1|0|8|12 8\n" + bad)
    with pytest.raises(gca.GCAError):
        gca.tune_load(str(p))
    assert gca.tune_get("dev", "f32", False, 8, 4096) == 0  # nothing merged


@pytest.mark.gpu
def test_tuned_batch_product(gca):
    torch = pytest.importorskip("torch")
    meshes = [synth.icosphere(3), synth.icosphere(3)]
    trees = [gca.tree_build(v, t, 32) for v, t in meshes]
    b = gca.build_batch(meshes, trees, gca.Params(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6))
    xs = [torch.from_numpy(synth.normal_rhs(len(t), 16, seed=i)).float().cuda() for i, (_, t) in enumerate(meshes)]
    ref = b.matvec(xs, "f32")
    w = b.tune(xs, "f32")
    assert w in (16, 8, 4)
    rows = sum(len(t) for _, t in meshes)
    dev = torch.cuda.get_device_name().replace(" ", "_").replace("|", "_")
    assert gca.tune_get(dev, "f32", False, 16, rows) == w
    got = b.matvec(xs, "f32")
    torch.cuda.synchronize()
    for a, c in zip(got, ref):
        assert float((a - c).norm() / c.norm()) <= 1e-6
    assert b.status() == 0
