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


def standard_stream(V: int, p: float, seed: int):
    """The standard stream of a static ER(p) graph, as in the paper's
    experiments (§5, datasets): insert every edge, then delete every edge,
    each phase in its own seeded random order. Returns edges [2E, 2] uint32
    and ops [2E] int8."""
    e = er_edges(V, p, seed)
    g = rng(seed + 3000)
    ins, dels = e[g.permutation(len(e))], e[g.permutation(len(e))]
    ops = np.concatenate([np.ones(len(e), np.int8), -np.ones(len(e), np.int8)])
    return np.concatenate([ins, dels]), ops


def spanning_forest_edges(V: int, e: np.ndarray, g: np.random.Generator) -> np.ndarray:
    """One spanning forest of the graph (V, e): the minimum spanning forest
    under seeded random distinct weights, so that it is unrelated to edge
    ids. [F, 2] uint32 rows u < v, F = V - #components."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import minimum_spanning_tree
    if len(e) == 0:
        return np.zeros((0, 2), np.uint32)
    w = g.permutation(len(e)).astype(np.float64) + 1.0
    t = minimum_spanning_tree(sp.csr_matrix((w, (e[:, 0], e[:, 1])), shape=(V, V))).tocoo()
    f = np.stack([np.minimum(t.row, t.col), np.maximum(t.row, t.col)], 1).astype(np.uint32)
    return f[g.permutation(len(f))]


def fixed_forest_stream(V: int, p: float, seed: int, cycles: int = 1):
    """The fixed forest stream of a static ER(p) graph, as in the paper's
    experiments (§5 and App. C, datasets): insert the edges of one spanning
    forest, then ``cycles`` times insert every other edge and delete them
    all again, each pass in a fresh seeded random order. The forest is never
    deleted, so most updates are non-tree updates. Returns edges [n, 2]
    uint32, ops [n] int8 and the number of forest edges (the first ones)."""
    e = er_edges(V, p, seed)
    g = rng(seed + 4000)
    f = spanning_forest_edges(V, e, g)
    fid = np.sort(f[:, 0].astype(np.int64) * V + f[:, 1])
    eid = e[:, 0].astype(np.int64) * V + e[:, 1]
    pos = np.minimum(np.searchsorted(fid, eid), max(0, len(fid) - 1))
    rest = e[fid[pos] != eid] if len(fid) else e
    parts, ops = [f], [np.ones(len(f), np.int8)]
    for _ in range(cycles):
        parts += [rest[g.permutation(len(rest))], rest[g.permutation(len(rest))]]
        ops += [np.ones(len(rest), np.int8), -np.ones(len(rest), np.int8)]
    return np.concatenate(parts), np.concatenate(ops), len(f)


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


# ---- R-MAT stream with deletes and uneven batches (torch; any device) -------

def rmat_pairs(n: int, levels: int, probs, gen, device):
    """n R-MAT pairs over 2^levels vertices (Chakrabarti, Zhan, Faloutsos,
    SDM 2004): at each level pick quadrant a/b/c/d, i.e. (row bit, column bit)
    = (0,0)/(0,1)/(1,0)/(1,1), from one uniform draw r: the row bit is
    r >= a+b, the column bit is a <= r < a+b or r >= a+b+c. Returns int64
    tensors (u, v)."""
    import torch
    a, b, c, _ = probs
    r = torch.rand((levels, n), generator=gen, device=device)
    u = torch.zeros(n, dtype=torch.int64, device=device)
    v = torch.zeros(n, dtype=torch.int64, device=device)
    for lv in range(levels):
        rl = r[lv]
        u.mul_(2).add_(rl >= a + b)
        v.mul_(2).add_(((rl >= a) & (rl < a + b)) | (rl >= a + b + c))
    return u, v


class RmatStream:
    """Batches of a valid insert/delete stream on V = 2^levels vertices.

    Each batch has a size drawn log-uniformly in [batch_lo, batch_hi]; a
    fraction `del_frac` of it deletes edges inserted by earlier batches
    (positions drawn uniformly from the append-only list of inserted edges and
    kept if the edge is still present), the rest inserts R-MAT edges
    (self-loops and edges already present or repeated in the batch are
    redrawn, in up to 64 passes sized by the previous pass's acceptance,
    then replaced by uniform absent pairs; the count of those fallbacks is
    kept). Within a batch the deletes come first, so
    applying the batch in order keeps the stream valid. Presence is a V^2-bit
    bitmap (2 GiB at V = 2^17) on the same device."""

    def __init__(self, levels: int = 17, seed: int = 1, probs=(0.57, 0.19, 0.19, 0.05),
                 batch_lo: int = 1000, batch_hi: int = 4 << 20, del_frac: float = 0.2, device="cpu"):
        import torch
        self.torch = torch
        self.levels, self.V = levels, 1 << levels
        self.probs, self.lo, self.hi, self.del_frac = probs, batch_lo, batch_hi, del_frac
        self.device = torch.device(device)
        self.gen = torch.Generator(device=self.device).manual_seed(seed)
        nbits = self.V * self.V
        self.bitmap = torch.zeros((nbits + 63) // 64, dtype=torch.int64, device=self.device)
        self.pool = torch.zeros(1 << 20, dtype=torch.int64, device=self.device)  # inserted ids, append-only
        self.n_inserted = 0
        self.fallbacks = 0
        self.accept = 1.0  # acceptance of the last insert draw (sizes the next one)

    def _bits(self, ids):
        return (self.bitmap[ids >> 6] >> (ids & 63)) & 1

    def _flip(self, ids, sign):
        # distinct bits of absent (present) edges: adding (subtracting) each
        # power of two sets (clears) exactly that bit, wrap-around included
        one = self.torch.ones_like(ids)
        self.bitmap.index_add_(0, ids >> 6, sign * (one << (ids & 63)))

    def _unique_keep(self, ids):
        u, inv = self.torch.unique(ids, return_inverse=True)
        first = self.torch.full((u.numel(),), ids.numel(), dtype=self.torch.int64, device=self.device)
        first.scatter_reduce_(0, inv, self.torch.arange(ids.numel(), device=self.device), "amin")
        keep = self.torch.zeros(ids.numel(), dtype=self.torch.bool, device=self.device)
        keep[first] = True
        return keep

    def next_size(self) -> int:
        t = self.torch
        x = t.rand(1, generator=self.gen, device=self.device).item()
        return int(np.exp(np.log(self.lo) + x * (np.log(self.hi) - np.log(self.lo))))

    def _take(self, cand, want_bit, need, counted=False):
        """Up to `need` ids of `cand` whose presence bit is `want_bit`, first
        occurrences only, in draw order; their bits are flipped at once, so
        later draws of the same batch see them as taken. With `counted`, also
        the number of such ids before the cut to `need`."""
        cand = cand[self._bits(cand) == want_bit]
        cand = cand[self._unique_keep(cand)]
        m = cand.numel()
        cand = cand[:need]
        self._flip(cand, 1 if want_bit == 0 else -1)
        return (cand, m) if counted else cand

    def _deletes(self, k):
        t = self.torch
        if k == 0 or self.n_inserted == 0:
            return t.zeros(0, dtype=t.int64, device=self.device)
        pool = self.pool[:self.n_inserted]
        parts, have = [], 0
        for _ in range(64):
            need = k - have
            if need <= 0:
                break
            pos = t.randint(0, pool.numel(), (2 * need + 16,), generator=self.gen, device=self.device)
            got = self._take(pool[pos], 1, need)
            parts.append(got)
            have += got.numel()
        return t.cat(parts) if parts else t.zeros(0, dtype=t.int64, device=self.device)

    def _inserts(self, k):
        t = self.torch
        parts, have = [], 0
        accept = self.accept
        for _ in range(64):
            need = k - have
            if need <= 0:
                break
            # draw in proportion to the last pass's acceptance (at most 16x,
            # at most 2^23 pairs: the uniforms of all levels are held at once)
            draw = min(16 * need, 1 << 23, max(1024, int(1.1 * need / accept)))
            u, v = rmat_pairs(draw, self.levels, self.probs, self.gen, self.device)
            ok = u != v
            got, m = self._take(t.minimum(u, v)[ok] * self.V + t.maximum(u, v)[ok], 0, need, counted=True)
            accept = max(m / draw, 1.0 / 16)
            parts.append(got)
            have += got.numel()
        while have < k:  # uniform absent pairs
            need = k - have
            u = t.randint(0, self.V, (need,), generator=self.gen, device=self.device)
            v = t.randint(0, self.V, (need,), generator=self.gen, device=self.device)
            ok = u != v
            got = self._take(t.minimum(u, v)[ok] * self.V + t.maximum(u, v)[ok], 0, need)
            parts.append(got)
            have += got.numel()
            self.fallbacks += got.numel()
        self.accept = accept
        got = t.cat(parts) if parts else t.zeros(0, dtype=t.int64, device=self.device)
        need = self.n_inserted + got.numel()
        if need > self.pool.numel():
            cap = self.pool.numel()
            while cap < need:
                cap *= 2
            grown = t.zeros(cap, dtype=t.int64, device=self.device)
            grown[:self.n_inserted] = self.pool[:self.n_inserted]
            self.pool = grown
        self.pool[self.n_inserted:need] = got
        self.n_inserted = need
        return got

    def next_batch(self, size: int | None = None):
        """Returns (edges int32 [n, 2], ops int8 [n]) on the stream's device."""
        t = self.torch
        n = self.next_size() if size is None else size
        k_del = int(round(self.del_frac * n)) if self.n_inserted else 0
        dels = self._deletes(k_del)
        ins = self._inserts(n - dels.numel())
        ids = t.cat([dels, ins])
        edges = t.stack([ids // self.V, ids % self.V], 1).to(t.int32)
        ops = t.cat([t.full((dels.numel(),), -1, dtype=t.int8, device=self.device),
                     t.ones(ins.numel(), dtype=t.int8, device=self.device)])
        return edges, ops


# ---- many independent graphs with interleaved requests (serving) ----------

def _distinct_pairs(V: int, k: int, g: np.random.Generator, exclude: np.ndarray | None = None) -> np.ndarray:
    """k distinct uniform pair ids u*V+v (u<v), none in sorted `exclude`."""
    out = np.zeros(0, np.int64)
    while out.size < k:
        need = k - out.size
        u = g.integers(0, V, size=2 * need + 16)
        v = g.integers(0, V, size=2 * need + 16)
        ok = u != v
        ids = np.minimum(u, v)[ok] * V + np.maximum(u, v)[ok]
        if exclude is not None and exclude.size:
            ids = ids[~np.isin(ids, exclude)]
        out = np.unique(np.concatenate([out, ids]))
        if out.size > k:
            out = g.permutation(out)[:k]
    return g.permutation(out)


def serving_streams(n_graphs: int = 64, v_exp=(10.0, 15.0), p_range=(0.1, 0.9), upd_range=(1e5, 1e6),
                    batch_range=(1000, 1 << 20), rho: int = 100_000, q_size: int = 1000, seed: int = 1):
    """Per-graph request lists for the serving workload.

    Graph i has V = floor(2^U[v_exp]) vertices and an ER(p), p ~ U[p_range],
    insert/delete stream of U ~ log-uniform[upd_range] updates: first the
    edges of ER(p) in a random order (a prefix of that order is a uniform
    random set of distinct pairs; at most 70% of the updates), then uniform
    toggles (distinct within a batch: insert if absent, delete if present).
    Updates come in batches of log-uniform size in batch_range; after every
    `rho` updates of the graph a batch of q_size uniform Connected pairs
    follows. Returns [(V, seed_i, steps)] with steps as in toggle_stream and
    the number of updates of each graph."""
    g = rng(seed)
    out = []
    for i in range(n_graphs):
        V = int(2 ** g.uniform(*v_exp))
        p = g.uniform(*p_range)
        total = int(np.exp(g.uniform(np.log(upd_range[0]), np.log(upd_range[1]))))
        n_ins = int(min(round(p * V * (V - 1) / 2), 0.7 * total))
        present = _distinct_pairs(V, n_ins, g)
        steps, done, next_q = [], 0, rho
        pos = 0
        while done < total:
            b = int(np.exp(g.uniform(np.log(batch_range[0]), np.log(batch_range[1]))))
            b = min(b, total - done)
            if pos < n_ins:
                ids = present[pos:pos + b]
                pos += ids.size
                ops = np.ones(ids.size, np.int8)
            else:
                ids = _distinct_pairs(V, b, g)
                ops = np.ones(ids.size, np.int8)
                cur = np.sort(present[:pos]) if pos else np.zeros(0, np.int64)
                hit = np.isin(ids, cur)
                ops[hit] = -1
                keep = np.concatenate([cur[~np.isin(cur, ids[hit])], ids[~hit]])
                present = keep
                pos = keep.size
                n_ins = pos
            e = np.stack([ids // V, ids % V], 1).astype(np.uint32)
            steps.append(("update", e, ops))
            done += ids.size
            while done >= next_q:
                steps.append(("query", uniform_pairs(V, q_size, g, distinct=False)))
                next_q += rho
        out.append((V, 1000 + i, steps, done))
    return out


def round_robin(streams):
    """Arrival order: one step of each graph in turn, as (graph index, step)."""
    idx = [0] * len(streams)
    order = []
    live = True
    while live:
        live = False
        for i, st in enumerate(streams):
            steps = st[2]
            if idx[i] < len(steps):
                order.append((i, steps[idx[i]]))
                idx[i] += 1
                live = True
    return order


# ---- adversarial components: disjoint cliques joined and split by bridges ----

def clique_stream(V: int = 131072, k: int = 256, s: int = 512, n_batches: int = 8, batch: int = 65536,
                  seed: int = 7):
    """k disjoint s-cliques on seeded permuted vertex ids, joined by
    n_batches batches of `batch` distinct random bridge inserts between
    different cliques, then split again by n_batches shuffled batches
    deleting them; one 1k-pair Connected batch (500 pairs inside one clique,
    500 across two) is asked after every bridge batch.

    Returns (clique_edges [k*s*(s-1)/2, 2] uint32 in clique order,
    bridge batches [(edges [batch, 2] uint32, op +1/-1)], pairs [1000, 2]
    uint32, clique of every vertex [V] int64)."""
    g = rng(seed)
    perm = g.permutation(V).astype(np.uint32)
    iu, ju = np.triu_indices(s, 1)
    cl = np.concatenate([np.stack([perm[c * s + iu], perm[c * s + ju]], 1) for c in range(k)])
    comp = np.empty(V, np.int64)
    comp[perm] = np.repeat(np.arange(k), s)
    nb = n_batches * batch
    a = g.integers(0, V, 3 * nb)
    b = g.integers(0, V, 3 * nb)
    ok = comp[a] != comp[b]
    bid = np.unique(np.minimum(a, b)[ok] * V + np.maximum(a, b)[ok])
    bid = g.permutation(bid)[:nb]
    bridges = np.stack([bid // V, bid % V], 1).astype(np.uint32)
    dels = g.permutation(nb)
    order = [(bridges[i * batch:(i + 1) * batch], 1) for i in range(n_batches)]
    order += [(bridges[dels[i * batch:(i + 1) * batch]], -1) for i in range(n_batches)]
    cs = g.integers(0, k, 500)
    same = np.stack([perm[cs * s + g.integers(0, s, 500)], perm[cs * s + g.integers(0, s, 500)]], 1)
    c1 = g.integers(0, k, 500)
    c2 = (c1 + g.integers(1, k, 500)) % k
    diff = np.stack([perm[c1 * s + g.integers(0, s, 500)], perm[c2 * s + g.integers(0, s, 500)]], 1)
    pairs = np.ascontiguousarray(np.concatenate([same, diff])[g.permutation(1000)], np.uint32)
    return cl, order, pairs, comp


# ---- Kronecker-shaped dense graphs (the paper's K13..K17 shape) --------------

def kronecker_b(levels: int, density: float = 0.5) -> float:
    """Entry b of the rank-one initiator [[1, b], [b, b^2]] whose k-th
    Kronecker power has mean entry ((1 + b) / 2)^(2k) = density."""
    return 2.0 * density ** (1.0 / (2 * levels)) - 1.0


def kronecker_graph(levels: int, seed: int, device="cpu", density: float = 0.5, block_pairs: int = 1 << 27):
    """Stochastic Kronecker graph (Leskovec, Chakrabarti, Kleinberg,
    Faloutsos, Ghahramani, JMLR 2010) on V = 2^levels vertices with the
    initiator [[1, b], [b, b^2]] (b = kronecker_b(levels, density)): each
    pair u < v is an edge independently with probability
    b^(popcount(u) + popcount(v)), the product over the levels of the
    initiator entry picked by the two vertices' bits. The expected density
    is `density` (0.5: the density of the paper's Kronecker datasets), with
    degrees skewed towards vertices of few one-bits.

    Drawn on `device` (torch) in blocks of rows. Returns (edge ids u*V+v
    int64 ascending, parent int64 [V]): parent[v] = the smallest neighbour
    u < v of v, or v itself when it has none, so the edges (parent[v], v),
    v != parent[v], form a spanning forest of every component whose
    vertices other than its minimum have a smaller neighbour."""
    import torch
    V = 1 << levels
    b = kronecker_b(levels, density)
    dev = torch.device(device)
    gen = torch.Generator(device=dev).manual_seed(seed)
    pc = torch.zeros(V, dtype=torch.int64, device=dev)
    ar = torch.arange(V, device=dev)
    for lv in range(levels):
        pc += (ar >> lv) & 1
    w = torch.pow(torch.tensor(b, dtype=torch.float64, device=dev), pc.double()).float()
    rows = max(1, min(V, block_pairs // V))
    parts = []
    parent = ar.clone()
    for u0 in range(0, V, rows):
        u1 = min(V, u0 + rows)
        p = w[u0:u1, None] * w[None, :]
        keep = torch.rand((u1 - u0, V), generator=gen, device=dev) < p
        keep &= ar[None, :] > ar[u0:u1, None]
        ru, v = torch.nonzero(keep, as_tuple=True)
        u = ru + u0
        parts.append(u * V + v)
        parent.scatter_reduce_(0, v, u, "amin")
        del p, keep
    return torch.cat(parts), parent
