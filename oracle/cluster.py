"""Cluster tree, bounding boxes and block tree (oracle).

Sect. 2: index subsets tau-hat of the triangles are described by
axis-parallel boxes tau containing the supports of their basis functions;
a block tau x sigma is admissible (approximated) if
    max{diam(tau), diam(sigma)} <= 2 eta dist(tau, sigma).
The paper does not say how the cluster tree is built; the reading used here
(identical in the C library's ``gca_tree_build``, which a test checks bit
for bit) is:

* recursive bisection of the set of triangles: the bounding box of the
  triangle centroids (a+b+c)/3 is split at its midpoint across its longest
  axis (ties: lowest axis); centroids < midpoint go low, the rest high,
  each side keeping its order.  If one side is empty the set is sorted
  stably by that coordinate and split at half its size (low half first).
  Sets of at most ``leaf_size`` triangles are leaves.
* clusters are numbered breadth first (root 0, children consecutive).
* the box of a cluster is the bounding box of the vertices of its
  triangles; diam is its diagonal, dist the Euclidean gap between boxes.

The block tree starts at (root, root): admissible pairs become coupling
blocks; inadmissible pairs of two leaves become near-field blocks; otherwise
the non-leaf side is split (both sides if both are non-leaves).

Pinned by tests: the tree is a partition hierarchy with leaves of at most
``leaf_size`` triangles, and the block tree covers every (i, j) exactly once
(brute force on small meshes).
"""

import numpy as np


def build_tree(vertices, triangles, leaf_size):
    v = np.asarray(vertices, dtype=np.float64)
    t = np.asarray(triangles, dtype=np.int64)
    cent = (v[t[:, 0]] + v[t[:, 1]] + v[t[:, 2]]) / 3.0
    return build_tree_from_centers(cent, leaf_size)


def build_tree_from_centers(cent, leaf_size):
    """The bisection above on given points (one per index)."""
    cent = np.asarray(cent, dtype=np.float64)
    n = cent.shape[0]
    perm = np.arange(n, dtype=np.int64)
    begin, end, child0, child1, level = [0], [n], [-1], [-1], [0]
    queue = [0]
    head = 0
    while head < len(queue):
        c = queue[head]
        head += 1
        b, e = begin[c], end[c]
        if e - b <= leaf_size:
            continue
        idx = perm[b:e]
        pc = cent[idx]
        lo = pc.min(axis=0)
        hi = pc.max(axis=0)
        ext = hi - lo
        axis = 0
        for d in (1, 2):
            if ext[d] > ext[axis]:
                axis = d
        mid = 0.5 * (lo[axis] + hi[axis])
        low = pc[:, axis] < mid
        if low.all() or not low.any():
            order = np.argsort(pc[:, axis], kind="stable")
            half = (e - b) // 2
            new = idx[order]
            nlow = half
        else:
            new = np.concatenate([idx[low], idx[~low]])
            nlow = int(low.sum())
        perm[b:e] = new
        for cb, ce in ((b, b + nlow), (b + nlow, e)):
            begin.append(cb)
            end.append(ce)
            child0.append(-1)
            child1.append(-1)
            level.append(level[c] + 1)
            queue.append(len(begin) - 1)
        child0[c] = len(begin) - 2
        child1[c] = len(begin) - 1
    return {
        "perm": perm,
        "begin": np.array(begin, dtype=np.int64),
        "end": np.array(end, dtype=np.int64),
        "child0": np.array(child0, dtype=np.int64),
        "child1": np.array(child1, dtype=np.int64),
        "level": np.array(level, dtype=np.int64),
    }


def parents(tree):
    par = np.full(len(tree["begin"]), -1, dtype=np.int64)
    for c in range(len(par)):
        for ch in (tree["child0"][c], tree["child1"][c]):
            if ch >= 0:
                par[ch] = c
    return par


def is_leaf(tree, c):
    return tree["child0"][c] < 0


def cluster_boxes(vertices, triangles, tree):
    """Bounding boxes of the supports (all vertices of the triangles)."""
    v = np.asarray(vertices, dtype=np.float64)
    t = np.asarray(triangles, dtype=np.int64)
    nc = len(tree["begin"])
    lo = np.empty((nc, 3))
    hi = np.empty((nc, 3))
    for c in range(nc):
        tri = tree["perm"][tree["begin"][c]:tree["end"][c]]
        pts = v[t[tri].ravel()]
        lo[c] = pts.min(axis=0)
        hi[c] = pts.max(axis=0)
    return lo, hi


def diameter(lo, hi):
    d = hi - lo
    return np.sqrt(d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2])


def distance(lo1, hi1, lo2, hi2):
    gap = np.maximum(0.0, np.maximum(lo2 - hi1, lo1 - hi2))
    return np.sqrt(gap[..., 0] * gap[..., 0] + gap[..., 1] * gap[..., 1]
                   + gap[..., 2] * gap[..., 2])


def admissible(diam_t, diam_s, dist, eta):
    return max(diam_t, diam_s) <= 2.0 * eta * dist


def block_tree(tree, lo, hi, eta):
    """Admissible (coupling) and inadmissible leaf (near-field) blocks.

    Returns two lists of (tau, sigma) cluster pairs in traversal order.
    """
    diam = diameter(lo, hi)
    far, near = [], []
    stack = [(0, 0)]
    while stack:
        t, s = stack.pop()
        dist = float(distance(lo[t], hi[t], lo[s], hi[s]))
        if admissible(float(diam[t]), float(diam[s]), dist, eta):
            far.append((t, s))
            continue
        lt, ls = is_leaf(tree, t), is_leaf(tree, s)
        if lt and ls:
            near.append((t, s))
        elif lt:
            for cs in (tree["child1"][s], tree["child0"][s]):
                stack.append((t, cs))
        elif ls:
            for ct in (tree["child1"][t], tree["child0"][t]):
                stack.append((ct, s))
        else:
            for ct in (tree["child1"][t], tree["child0"][t]):
                for cs in (tree["child1"][s], tree["child0"][s]):
                    stack.append((ct, cs))
    return far, near
