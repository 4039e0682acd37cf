"""The oracle's GCA-H^2 representation in the host layout of gca_host_dump
(include/gca.h), for gca_h2_import: the products then run on the oracle's
own bases, transfers, couplings and near field, with the GPU construction
bypassed."""

import numpy as np

from oracle import cluster


def oracle_dump(h2o):
    tree = h2o.tree
    nc = len(tree["begin"])
    rank = np.asarray(h2o.bases.rank, dtype=np.int32)
    pivots = [np.asarray(h2o.bases.pivots[c], dtype=np.int32) for c in range(nc)]
    parent = cluster.parents(tree)
    V = [h2o.bases.V[c].reshape(-1) for c in range(1, nc) if cluster.is_leaf(tree, c)]
    E = [h2o.bases.E[c].reshape(-1) for c in range(1, nc) if parent[c] > 0]
    far = np.asarray(h2o.far, dtype=np.int32).reshape(-1, 2)
    near = np.asarray(h2o.near, dtype=np.int32).reshape(-1, 2)
    S = [h2o.S[(int(t), int(s))].reshape(-1) for t, s in far]
    N = [h2o.N[(int(t), int(s))].reshape(-1) for t, s in near]
    cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0)
    return {"rank": rank, "pivots": cat(pivots).astype(np.int32), "far": far, "near": near,
            "V": cat(V), "E": cat(E), "S": cat(S), "N": cat(N)}
