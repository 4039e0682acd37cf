"""Pins for the oracle's cluster tree and block tree (Sect. 2)."""

import numpy as np
import pytest

import synth
from oracle import cluster


@pytest.mark.parametrize("level,leaf", [(2, 16), (3, 32), (4, 64)])
def test_tree_is_partition_hierarchy(level, leaf):
    v, t = synth.icosphere(level)
    n = len(t)
    tr = cluster.build_tree(v, t, leaf)
    assert np.array_equal(np.sort(tr["perm"]), np.arange(n))
    assert tr["begin"][0] == 0 and tr["end"][0] == n and tr["level"][0] == 0
    cent = (v[t[:, 0]] + v[t[:, 1]] + v[t[:, 2]]) / 3.0
    for c in range(len(tr["begin"])):
        b, e = tr["begin"][c], tr["end"][c]
        c0, c1 = tr["child0"][c], tr["child1"][c]
        if c0 < 0:
            assert c1 < 0 and 0 < e - b <= leaf
            continue
        assert e - b > leaf
        assert c1 == c0 + 1 and c0 > c
        assert tr["begin"][c0] == b and tr["end"][c0] == tr["begin"][c1] and tr["end"][c1] == e
        assert tr["end"][c0] > b and tr["begin"][c1] < e
        assert tr["level"][c0] == tr["level"][c] + 1
        # the split rule: midpoint of the centroid box across its longest axis
        pc = cent[tr["perm"][b:e]]
        lo, hi = pc.min(axis=0), pc.max(axis=0)
        ax = int(np.argmax(hi - lo))
        mid = 0.5 * (lo[ax] + hi[ax])
        low = cent[tr["perm"][b:tr["end"][c0]], ax]
        high = cent[tr["perm"][tr["begin"][c1]:e], ax]
        if (pc[:, ax] < mid).all() or not (pc[:, ax] < mid).any():
            assert low.max() <= high.min()
        else:
            assert (low < mid).all() and (high >= mid).all()
    # breadth-first numbering: levels never decrease
    assert np.all(np.diff(tr["level"]) >= 0)


@pytest.mark.parametrize("level,leaf,eta", [(2, 16, 2.0), (3, 32, 2.0), (3, 16, 1.0)])
def test_block_tree_covers_every_entry_once(level, leaf, eta):
    v, t = synth.icosphere(level)
    n = len(t)
    tr = cluster.build_tree(v, t, leaf)
    lo, hi = cluster.cluster_boxes(v, t, tr)
    far, near = cluster.block_tree(tr, lo, hi, eta)
    cover = np.zeros((n, n), dtype=np.int64)
    diam = cluster.diameter(lo, hi)
    for (a, b) in far + near:
        ra = tr["perm"][tr["begin"][a]:tr["end"][a]]
        rb = tr["perm"][tr["begin"][b]:tr["end"][b]]
        cover[np.ix_(ra, rb)] += 1
    assert (cover == 1).all()
    for (a, b) in far:
        d = cluster.distance(lo[a], hi[a], lo[b], hi[b])
        assert max(diam[a], diam[b]) <= 2 * eta * d
    for (a, b) in near:
        assert cluster.is_leaf(tr, a) and cluster.is_leaf(tr, b)
    # the admissibility condition is symmetric, so is the block structure
    assert set(far) == {(b, a) for (a, b) in far}
    assert set(near) == {(b, a) for (a, b) in near}


def test_boxes_contain_supports():
    v, t = synth.icosphere(3)
    tr = cluster.build_tree(v, t, 32)
    lo, hi = cluster.cluster_boxes(v, t, tr)
    for c in range(len(tr["begin"])):
        pts = v[t[tr["perm"][tr["begin"][c]:tr["end"][c]]].ravel()]
        assert (pts >= lo[c]).all() and (pts <= hi[c]).all()
        # tight: every face of the box touches a vertex
        assert np.allclose(pts.min(axis=0), lo[c]) and np.allclose(pts.max(axis=0), hi[c])


def test_distance_and_diameter():
    lo1, hi1 = np.array([0.0, 0, 0]), np.array([1.0, 1, 1])
    lo2, hi2 = np.array([4.0, 5, 1]), np.array([5.0, 6, 2])
    assert cluster.distance(lo1, hi1, lo2, hi2) == 5.0
    assert cluster.distance(lo2, hi2, lo1, hi1) == 5.0
    assert cluster.distance(lo1, hi1, lo1 + 0.5, hi1 + 0.5) == 0.0
    assert abs(cluster.diameter(lo1, hi1) - np.sqrt(3.0)) < 1e-15
