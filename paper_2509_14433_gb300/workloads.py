"""Seeded synthetic input streams for sketch-based connectivity.

This module only draws inputs. It holds none of the method's arithmetic (no
hashing, no sketching, no recovery) and imports neither the CUDA binding nor
the oracle, so both sides can be fed the same streams.

Random numbers come from numpy's PCG64 generator (O'Neill, "PCG: A family of
simple fast space-efficient statistically good algorithms for random number
generation", 2014). Streams follow the stream model of App. A.1 (Problem 1):
an update inserts an absent edge or deletes a present one, u != v.

A stream is a list of steps:
    ("update", edges[n, 2] uint32, ops[n] int8 (+1 insert, -1 delete))
    ("query",  pairs[m, 2] uint32)
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def er_edges(V: int, p: float, seed: int, rows_per_chunk: int = 1024) -> np.ndarray:
    """All pairs u < v kept independently with probability p (Erdos-Renyi
    G(V, p)), in lexicographic order, as an [E, 2] uint32 array."""
    g = rng(seed)
    out = []
    cols = np.arange(V, dtype=np.int64)
    for a in range(0, V, rows_per_chunk):
        b = min(V, a + rows_per_chunk)
        keep = g.random((b - a, V), dtype=np.float32) < np.float32(p)
        keep &= cols[None, :] > np.arange(a, b, dtype=np.int64)[:, None]
        ru, v = np.nonzero(keep)
        out.append(np.stack([ru + a, v], axis=1).astype(np.uint32))
    return np.concatenate(out) if out else np.zeros((0, 2), np.uint32)


def uniform_pairs(V: int, m: int, g: np.random.Generator, distinct: bool = True) -> np.ndarray:
    """m uniform vertex pairs (u != v when ``distinct``), [m, 2] uint32."""
    u = g.integers(0, V, size=m, dtype=np.int64)
    if distinct:
        v = (u + g.integers(1, V, size=m, dtype=np.int64)) % V
    else:
        v = g.integers(0, V, size=m, dtype=np.int64)
    return np.stack([u, v], axis=1).astype(np.uint32)


def batches(edges: np.ndarray, ops: np.ndarray, size: int):
    for i in range(0, len(edges), size):
        yield ("update", edges[i:i + size], ops[i:i + size])


def toggle_stream(V: int, start_edges: np.ndarray, n_toggles: int, query_every: int,
                  query_size: int, seed: int, batch_cap: int = 1 << 20):
    """Insert ``start_edges`` (in batches of at most ``batch_cap``), then
    ``n_toggles`` uniform random pairs u < v, each inserted if absent and
    deleted if present, with a batch of ``query_size`` uniform Connected pairs
    after every ``query_every`` toggles."""
    g = rng(seed)
    steps = []
    ins = np.ones(len(start_edges), dtype=np.int8)
    steps.extend(batches(start_edges, ins, batch_cap))
    present = np.zeros(V * V, dtype=bool)
    present[start_edges[:, 0].astype(np.int64) * V + start_edges[:, 1]] = True
    done = 0
    while done < n_toggles:
        k = min(query_every, n_toggles - done)
        pr = uniform_pairs(V, k, g)
        a = np.minimum(pr[:, 0], pr[:, 1])
        b = np.maximum(pr[:, 0], pr[:, 1])
        idx = a.astype(np.int64) * V + b
        ops = np.empty(k, dtype=np.int8)
        for i in range(k):  # sequential: a pair may repeat inside the window
            ops[i] = -1 if present[idx[i]] else 1
            present[idx[i]] = not present[idx[i]]
        steps.append(("update", np.stack([a, b], axis=1).astype(np.uint32), ops))
        steps.append(("query", uniform_pairs(V, query_size, g, distinct=False)))
        done += k
    return steps


def plain_stream(V: int = 1024, p: float = 0.5, n_toggles: int = 200_000,
                 query_every: int = 10_000, query_size: int = 1000, seed: int = 1):
    """Toggle stream on an ER(p) start graph with periodic query batches."""
    start = er_edges(V, p, seed)
    return toggle_stream(V, start, n_toggles, query_every, query_size, seed + 1000)


def dense_stream(V: int = 16384, p: float = 0.5, batch: int = 1 << 20,
                 delete_frac: float = 0.1, seed: int = 1):
    """ER(p) edges inserted in a seeded random order in batches, then a
    uniform random ``delete_frac`` of them deleted in batches. Returns
    (edges_in_insert_order, n_deleted, delete_order) so a caller can stage
    the whole stream on the device: the deleted edges are
    edges[delete_order[:n_deleted]]."""
    e = er_edges(V, p, seed)
    g = rng(seed + 2000)
    e = e[g.permutation(len(e))]
    n_del = int(round(delete_frac * len(e)))
    order = g.permutation(len(e))[:n_del]
    return e, n_del, order


def final_edge_set(V: int, steps) -> np.ndarray:
    """Edge ids u*V+v present after applying every update step (toggle
    semantics), sorted ascending."""
    present = {}
    for st in steps:
        if st[0] != "update":
            continue
        e = st[1]
        idx = np.minimum(e[:, 0], e[:, 1]).astype(np.int64) * V + np.maximum(e[:, 0], e[:, 1])
        for x in idx.tolist():
            present[x] = not present.get(x, False)
    return np.array(sorted(k for k, v in present.items() if v), dtype=np.uint64)
