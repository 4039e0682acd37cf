"""C-ABI checks that need no GPU: the library loads, exports every entry
point declared in include/gca.h, its structs have the layout the header
gives them, the cluster-tree helper matches the oracle bit for bit, and
invalid input is rejected before any device work."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import synth
import paper_1810_08429_b300 as gca
from oracle import cluster, p1

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gca.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gca_build", "h2_matvec", "h2_matvec_transpose", "gca_tree_build",
                     "gca_h2_stats", "gca_h2_export", "gca_free", "gca_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(gca.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "gca.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(gca_mesh),sizeof(gca_tree),sizeof(gca_params),sizeof(gca_stats),"
        "sizeof(gca_host_dump),offsetof(gca_stats,rank_sum),offsetof(gca_params,omega_margin));"
        "return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(gca._Mesh), ctypes.sizeof(gca._Tree), ctypes.sizeof(gca._Params),
            ctypes.sizeof(gca._Stats), ctypes.sizeof(gca._Dump), gca._Stats.rank_sum.offset,
            gca._Params.omega_margin.offset]
    assert got == want


@pytest.mark.parametrize("name,leaf", [("sphere80", 8), ("sphere1280", 32), ("perturbed1280", 32),
                                       ("sphere20480", 64), ("perturbed20480", 64),
                                       ("ellipsoid1280", 16)])
def test_tree_build_matches_oracle(name, leaf):
    v, t = synth.mesh_for_config(name)
    ours = gca.tree_build(v, t, leaf)
    ref = cluster.build_tree(v, t, leaf)
    for key in ("perm", "begin", "end", "child0", "child1", "level"):
        assert np.array_equal(ours[key], ref[key]), key


@pytest.mark.parametrize("name,leaf", [("sphere1280", 32), ("sphere20480", 64), ("ellipsoid1280", 16),
                                       ("perturbed20480", 64)])
def test_point_tree_matches_oracle(name, leaf):
    """The vertex tree of the nodal basis (gca_tree_build_points)."""
    v, t = synth.mesh_for_config(name)
    ours = gca.tree_build_points(v, leaf)
    ref = p1.build_tree_points(v, leaf)
    for key in ("perm", "begin", "end", "child0", "child1", "level"):
        assert np.array_equal(ours[key], ref[key]), key


def test_p1_input_rejected_on_host():
    """gca_build_p1: a vertex outside every triangle, a tree over the
    triangles instead of the vertices, and a non-finite point."""
    v, t = synth.icosphere(1)
    p = gca.Params(leaf_size=8)
    vx = np.vstack([v, [[2.0, 0.0, 0.0]]])
    tree = gca.tree_build_points(vx, 8)
    with pytest.raises(gca.GCAError, match="belongs to no triangle"):
        gca.build_p1(vx, t, tree, p)
    with pytest.raises(gca.GCAError):
        gca.build_p1(v, t, gca.tree_build(v, t, 8), p)
    vn = v.copy()
    vn[2, 1] = np.inf
    with pytest.raises(gca.GCAError):
        gca.tree_build_points(vn, 8)


def test_tree_build_degenerate_split():
    # all centroids share x and y: the median rule must kick in
    n = 40
    v = np.zeros((3 * n, 3))
    t = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    for i in range(n):
        v[3 * i] = [0.0, 0.0, 0.0]
        v[3 * i + 1] = [1.0, 0.0, 0.0]
        v[3 * i + 2] = [0.0, 1.0, float(i % 3)]
    ours = gca.tree_build(v, t, 4)
    ref = cluster.build_tree(v, t, 4)
    for key in ("perm", "begin", "end", "child0", "child1", "level"):
        assert np.array_equal(ours[key], ref[key]), key


def test_tree_build_single_leaf():
    v, t = synth.icosahedron()
    tr = gca.tree_build(v, t, 64)
    assert len(tr["begin"]) == 1 and tr["child0"][0] == -1


def _raw_build(v, t, tree, params):
    m, keep_m = gca._mesh(v, t)
    tr, keep_t = gca._tree(tree)
    p = params._c()
    h = ctypes.c_void_p(None)
    return gca.lib.gca_build(ctypes.byref(m), ctypes.byref(tr), ctypes.byref(p), None,
                             ctypes.byref(h)), h


def test_invalid_input_rejected_on_host():
    v, t = synth.icosphere(1)
    tree = gca.tree_build(v, t, 8)
    p = gca.Params(leaf_size=8)
    # bad vertex id
    bad = t.copy()
    bad[3, 1] = 10_000
    st, h = _raw_build(v, bad, tree, p)
    assert st == -1 and not h.value
    # NaN coordinate
    vn = v.copy()
    vn[5, 2] = np.nan
    st, h = _raw_build(vn, t, tree, p)
    assert st == -4 and not h.value
    # broken tree: children do not split the parent range
    tb = {k: a.copy() for k, a in tree.items()}
    tb["end"][tb["child0"][0]] -= 1
    st, h = _raw_build(v, t, tb, p)
    assert st == -1 and not h.value
    # unsupported parameter
    st, h = _raw_build(v, t, tree, gca.Params(leaf_size=8, box_gauss_m=7))
    assert st == -1 and not h.value
    st, h = _raw_build(v, t, tree, gca.Params(leaf_size=8, tri_rule=6))
    assert st == -1 and not h.value
    with pytest.raises(gca.GCAError):
        gca.tree_build(v, bad, 8)
    assert "vertex id" in gca.lib.gca_last_error().decode()


def test_import_rejects_inconsistent_representation_on_host():
    """gca_h2_import validates the tree, ranks, pivots and block lists before
    any device work (so this runs without a GPU)."""
    from oracle import gca as ogca
    from oracle.params import Params as OParams
    from oracle_dump import oracle_dump
    v, t = synth.mesh_for_config("sphere320")
    h2o = ogca.build_h2(v, t, OParams(leaf_size=16, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5))
    good = oracle_dump(h2o)
    tree = h2o.tree

    def status_of(rep):
        with pytest.raises(gca.GCAError) as e:
            gca.import_h2(tree, len(t), rep)
        return e.value.status, str(e.value)

    bad = dict(good, rank=good["rank"].copy())
    bad["rank"][0] = 3
    assert status_of(bad)[0] == gca.ERR_INVALID_ARG
    leaf = int(np.nonzero(tree["child0"] < 0)[0][0])
    bad = dict(good, rank=good["rank"].copy())
    bad["rank"][leaf] = tree["end"][leaf] - tree["begin"][leaf] + 1
    assert "rank of cluster" in status_of(bad)[1]
    bad = dict(good, near=good["near"].copy())
    bad["near"][0, 0] = 0  # the root is not a leaf
    assert "near-field block" in status_of(bad)[1]
    bad = dict(good, far=good["far"].copy())
    bad["far"][0, 1] = len(tree["begin"])
    assert "coupling block" in status_of(bad)[1]
    bad = dict(good, pivots=good["pivots"].copy())
    bad["pivots"][0] = len(t)
    assert "pivot" in status_of(bad)[1]
    bad = dict(good, S=good["S"].copy())
    bad["S"][0] = np.nan
    assert status_of(bad)[0] == gca.ERR_NUMERIC


def test_test_hooks_reject_unknown_names():
    with pytest.raises(gca.GCAError) as e:
        gca.test_hook("no_such_hook", 1)
    assert e.value.status == gca.ERR_INVALID_ARG
    for name in ("wait_cycles", "stall_chain", "fail_alloc", "device_skew"):
        gca.test_hook(name, 0)


class _CheckpointHeader(ctypes.Structure):
    """The header of a gca_h2_save file (after its 8-byte magic)."""
    _fields_ = [("n", ctypes.c_int32), ("nc", ctypes.c_int32), ("nfar", ctypes.c_int32),
                ("nnear", ctypes.c_int32), ("op", ctypes.c_int32), ("k", ctypes.c_int32),
                ("m", ctypes.c_int32), ("reserved", ctypes.c_int32), ("rank_sum", ctypes.c_int64),
                ("v_entries", ctypes.c_int64), ("e_entries", ctypes.c_int64), ("s_entries", ctypes.c_int64),
                ("n_entries", ctypes.c_int64), ("n_singular", ctypes.c_int64 * 4), ("params", gca._Params)]


def _fnv1a(data):
    h = 1469598103934665603
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_checkpoint_files_checked_on_host(tmp_path):
    """gca_h2_load reads the documented layout and checks magic, length and
    checksum before any device work: a file in that layout whose
    representation is inconsistent (root rank 3) reaches the import's
    validation (INVALID_ARG); the same file truncated, with a flipped byte or
    a wrong magic, and a missing file, give ERR_IO."""
    from oracle import gca as ogca
    from oracle.params import Params as OParams
    from oracle_dump import oracle_dump
    v, t = synth.mesh_for_config("sphere80")
    h2o = ogca.build_h2(v, t, OParams(leaf_size=16, eta=2.0, box_gauss_m=2, aca_tol=1e-4, sauter_q=3))
    d = oracle_dump(h2o)
    tr = h2o.tree
    d["rank"] = d["rank"].copy()
    d["rank"][0] = 3
    hd = _CheckpointHeader(n=len(t), nc=len(tr["begin"]), nfar=len(d["far"]), nnear=len(d["near"]), op=0,
                           k=0, m=0, rank_sum=len(d["pivots"]), v_entries=len(d["V"]), e_entries=len(d["E"]),
                           s_entries=len(d["S"]), n_entries=len(d["N"]))
    parts = [b"GCAH2CK1", bytes(hd)]
    for key in ("perm", "begin", "end", "child0", "child1", "level"):
        parts.append(np.asarray(tr[key], dtype=np.int32).tobytes())
    for key in ("rank", "pivots", "far", "near"):
        parts.append(np.asarray(d[key], dtype=np.int32).tobytes())
    for key in ("V", "E", "S", "N"):
        parts.append(np.asarray(d[key], dtype=np.float64).tobytes())
    body = b"".join(parts)
    data = body + _fnv1a(body).to_bytes(8, "little")

    def status_of(blob, name):
        p = tmp_path / name
        p.write_bytes(blob)
        with pytest.raises(gca.GCAError) as e:
            gca.load(str(p))
        return e.value.status, str(e.value)

    st, msg = status_of(data, "inconsistent.gca")
    assert st == gca.ERR_INVALID_ARG and "gca_h2_import" in msg and "rank" in msg, msg
    assert status_of(data[:-9], "truncated.gca")[0] == gca.ERR_IO
    flipped = bytearray(data)
    flipped[len(data) // 2] ^= 0x10
    st, msg = status_of(bytes(flipped), "flipped.gca")
    assert st == gca.ERR_IO and "checksum" in msg
    assert status_of(b"GCAH2CK0" + data[8:], "magic.gca")[0] == gca.ERR_IO
    with pytest.raises(gca.GCAError) as e:
        gca.load(str(tmp_path / "missing.gca"))
    assert e.value.status == gca.ERR_IO
