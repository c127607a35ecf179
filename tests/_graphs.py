"""Brute-force graph helpers for tests (scipy's connected components)."""
import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components


def min_labels(V, edge_ids):
    """Component label = minimum vertex id, from the explicit edge set."""
    ids = np.asarray(edge_ids, dtype=np.int64)
    u, v = ids // V, ids % V
    m = coo_matrix((np.ones(len(ids)), (u, v)), shape=(V, V))
    _, comp = connected_components(m, directed=False)
    first = np.full(comp.max() + 1 if V else 0, V, dtype=np.int64)
    np.minimum.at(first, comp, np.arange(V))
    return first[comp].astype(np.uint32)


def check_forest(V, forest, edge_ids):
    """A spanning forest: ascending distinct ids, edges of G, acyclic, and
    |F| = V - #components."""
    f = np.asarray(forest, dtype=np.int64)
    assert np.all(np.diff(f) > 0), "forest ids must be strictly ascending"
    present = set(np.asarray(edge_ids, dtype=np.int64).tolist())
    assert all(x in present for x in f.tolist()), "forest edge not in G"
    parent = list(range(V))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for x in f.tolist():
        a, b = find(x // V), find(x % V)
        assert a != b, "forest has a cycle"
        parent[a] = b
    ncomp = len(set(min_labels(V, edge_ids).tolist()))
    assert len(f) == V - ncomp, "forest does not span every component"


def edge_ids(V, edges):
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    return np.minimum(e[:, 0], e[:, 1]) * V + np.maximum(e[:, 0], e[:, 1])
