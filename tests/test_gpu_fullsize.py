"""Parity at the workloads' full sizes, in the launch configuration bench.py
uses (2^20-edge batches, tuned apply settings): outputs the oracle can
compute one by one (the sketch of a sampled vertex from its final neighbour
set) and properties that hold at any size (labels = connected components of
the final edge set, forest edges present, acyclic and spanning)."""
import numpy as np
import pytest

import oracle as O
from paper_2509_14433_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BATCH = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _graph(V, seed, max_batch=BATCH):
    from paper_2509_14433_gb300 import autotune as AT
    from paper_2509_14433_gb300 import cupc as C
    st, g = C.cupc_init(V, seed, (0, 0, 0, max_batch), None, None)
    C.check(st)
    AT.apply(g, V, BATCH)
    return g


def _apply(g, E, ops):
    from paper_2509_14433_gb300 import cupc as C
    e_d = torch.from_numpy(np.ascontiguousarray(E, np.uint32).reshape(-1)).cuda()
    o_d = torch.from_numpy(np.ascontiguousarray(ops, np.int8)).cuda()
    for i in range(0, len(ops), BATCH):
        C.check(C.cupc_update_batch(g, e_d[2 * i:], o_d[i:], min(BATCH, len(ops) - i), None))
    torch.cuda.synchronize()


def _sampled_rows(g, V, ws):
    """Layer rows of the sampled vertices, via a device copy of the sketches."""
    from paper_2509_14433_gb300 import cupc as C
    p = np.zeros(4, np.uint32)
    C.cupc_get_params(g, p)
    L, _, _, W = (int(x) for x in p)
    buf = torch.empty(L * V * W * 2, dtype=torch.int64, device="cuda")
    C.check(C.cupc_export_sketches(g, buf, buf.numel() * 8, None))
    rows = buf.view(L, V, W, 2)[:, torch.tensor(ws, device="cuda")].cpu().numpy().view(np.uint64)
    del buf
    torch.cuda.empty_cache()
    return rows  # [L, len(ws), W, 2]


def _check_forest(V, forest, present, labels):
    """forest ids ascending and present in G; acyclic; both endpoints share a
    label; |F| = V - #labels."""
    f = np.asarray(forest, np.int64)
    assert np.all(np.diff(f) > 0)
    assert np.all(present(f))
    parent = np.arange(V)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for x in f.tolist():
        a, b = find(x // V), find(x % V)
        assert a != b
        parent[a] = b
    u, v = f // V, f % V
    assert np.all(labels[u] == labels[v])
    assert len(f) == V - len(np.unique(labels))


def _labels_of(V, u, v):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    m = coo_matrix((np.ones(len(u), np.int8), (u, v)), shape=(V, V))
    _, comp = connected_components(m, directed=False)
    first = np.full(comp.max() + 1, V, np.int64)
    np.minimum.at(first, comp, np.arange(V))
    return first[comp].astype(np.uint32)


def test_dense_v16384_full_size():
    from paper_2509_14433_gb300 import cupc as C
    V, seed = 16384, 1
    E, n_del, order = WL.dense_stream(V=V, p=0.5, seed=1)
    D = E[order[:n_del]]
    g = _graph(V, seed)
    try:
        _apply(g, E, np.ones(len(E), np.int8))
        _apply(g, D, -np.ones(len(D), np.int8))
        forest = np.zeros(V, np.uint64)
        st, nf = C.cupc_spanning_forest(g, forest, V, None)
        assert st == 0
        lab = np.zeros(V, np.uint32)
        C.check(C.cupc_labels(g, lab, None))
        ids = np.setdiff1d(np.minimum(E[:, 0], E[:, 1]).astype(np.int64) * V + np.maximum(E[:, 0], E[:, 1]),
                           np.minimum(D[:, 0], D[:, 1]).astype(np.int64) * V + np.maximum(D[:, 0], D[:, 1]))
        u, v = ids // V, ids % V
        assert np.array_equal(lab, _labels_of(V, u, v))
        _check_forest(V, forest[:nf], lambda f: np.isin(f, ids), lab)
        ws = [0, 1, 777, 4095, 8191, 12345, 16382, 16383]
        rows = _sampled_rows(g, V, ws)
        for k, w in enumerate(ws):
            nb = np.concatenate([v[u == w], u[v == w]])
            assert np.array_equal(rows[:, k], O.vertex_sketch(V, seed, w, nb)), w
    finally:
        C.cupc_destroy(g)


def test_cliques_v131072_full_size():
    # 256 disjoint 512-cliques joined by 8 batches of 64k random bridges and
    # split again by 8 shuffled batches deleting them; a 1k-pair query batch
    # (half inside one clique, half across two) after every batch, checked
    # against the exact components
    from paper_2509_14433_gb300 import cupc as C
    V, k, s, seed = 131072, 256, 512, 7
    g_rng = WL.rng(seed)
    perm = g_rng.permutation(V).astype(np.uint32)
    iu, ju = np.triu_indices(s, 1)
    cl = np.concatenate([np.stack([perm[c * s + iu], perm[c * s + ju]], 1) for c in range(k)])
    comp = np.empty(V, np.int64)
    comp[perm] = np.repeat(np.arange(k), s)
    a = g_rng.integers(0, V, 600000)
    b = g_rng.integers(0, V, 600000)
    ok = comp[a] != comp[b]
    bid = np.unique(np.minimum(a, b)[ok] * V + np.maximum(a, b)[ok])[: 8 * 65536]
    bid = g_rng.permutation(bid)
    bridges = np.stack([bid // V, bid % V], 1).astype(np.uint32)
    g = _graph(V, seed)
    try:
        _apply(g, cl, np.ones(len(cl), np.int8))
        present = np.zeros(0, np.int64)
        order = [(bridges[i * 65536:(i + 1) * 65536], 1) for i in range(8)]
        dels = g_rng.permutation(len(bridges))
        order += [(bridges[dels[i * 65536:(i + 1) * 65536]], -1) for i in range(8)]
        for E, op in order:
            _apply(g, E, np.full(len(E), op, np.int8))
            ids = E[:, 0].astype(np.int64) * V + E[:, 1]
            present = np.union1d(present, ids) if op == 1 else np.setdiff1d(present, ids)
            # exact components: cliques joined by the present bridges
            parent = np.arange(k)

            def find(x):
                while parent[x] != x:
                    parent[x] = parent[parent[x]]
                    x = parent[x]
                return x

            for x, y in zip(comp[present // V].tolist(), comp[present % V].tolist()):
                rx, ry = find(x), find(y)
                if rx != ry:
                    parent[rx] = ry
            root = np.array([find(c) for c in range(k)])
            # 500 pairs inside one clique, 500 pairs across two cliques
            cs = g_rng.integers(0, k, 500)
            same = np.stack([perm[cs * s + g_rng.integers(0, s, 500)], perm[cs * s + g_rng.integers(0, s, 500)]], 1)
            c1 = g_rng.integers(0, k, 500)
            c2 = (c1 + g_rng.integers(1, k, 500)) % k
            diff = np.stack([perm[c1 * s + g_rng.integers(0, s, 500)], perm[c2 * s + g_rng.integers(0, s, 500)]], 1)
            pr = np.ascontiguousarray(np.concatenate([same, diff])[g_rng.permutation(1000)], np.uint32)
            out = torch.zeros(1000, dtype=torch.uint8, device="cuda")
            C.check(C.cupc_query(g, torch.from_numpy(pr.reshape(-1)).cuda(), 1000, out, None))
            want = root[comp[pr[:, 0]]] == root[comp[pr[:, 1]]]
            assert np.array_equal(out.cpu().numpy().astype(bool), want)
        assert C.cupc_sync(g, None) == 0
        lab = np.zeros(V, np.uint32)
        C.check(C.cupc_labels(g, lab, None))
        first = np.full(k, V, np.int64)
        np.minimum.at(first, comp, np.arange(V))
        assert np.array_equal(lab, first[comp].astype(np.uint32))
        forest = np.zeros(V, np.uint64)
        st, nf = C.cupc_spanning_forest(g, forest, V, None)
        assert st == 0
        cid = np.sort(np.minimum(cl[:, 0], cl[:, 1]).astype(np.int64) * V + np.maximum(cl[:, 0], cl[:, 1]))
        _check_forest(V, forest[:nf], lambda f: np.isin(f, cid), lab)
        ws = [int(perm[0]), int(perm[511]), int(perm[512 * 100 + 3]), int(perm[-1])]
        rows = _sampled_rows(g, V, ws)
        for j, w in enumerate(ws):
            nb = perm[comp[perm] == comp[w]]
            nb = nb[nb != w]
            assert np.array_equal(rows[:, j], O.vertex_sketch(V, seed, w, nb)), w
    finally:
        C.cupc_destroy(g)


def test_rmat_v131072_1e9_updates():
    # the batched workload at full size: 1e9 R-MAT updates with 20% deletes,
    # batch sizes log-uniform in [1k, 4M], applied as back-to-back batches
    from paper_2509_14433_gb300 import cupc as C
    V, seed = 1 << 17, 1
    s = WL.RmatStream(levels=17, seed=3, device="cuda")
    g = _graph(V, seed, max_batch=4 << 20)
    try:
        done = 0
        while done < 1_000_000_000:
            E, ops = s.next_batch()
            n = len(ops)
            C.check(C.cupc_update_batch(g, E.reshape(-1), ops, n, None))
            done += n
        torch.cuda.synchronize()
        assert C.cupc_sync(g, None) == 0
        forest = np.zeros(V, np.uint64)
        st, nf = C.cupc_spanning_forest(g, forest, V, None)
        assert st == 0
        lab = np.zeros(V, np.uint32)
        C.check(C.cupc_labels(g, lab, None))
        # components of the final edge set with plain torch ops (pointer
        # jumping with scatter-min), independent of the library
        words = s.bitmap
        ids_list = []
        for c0 in range(0, words.numel(), 1 << 20):
            w = words[c0:c0 + (1 << 20)]
            nz = torch.nonzero(w, as_tuple=True)[0]
            if nz.numel() == 0:
                continue
            bits = (w[nz].unsqueeze(1) >> torch.arange(64, device="cuda")) & 1
            r, b = torch.nonzero(bits, as_tuple=True)
            ids_list.append((nz[r] + c0) * 64 + b)
        ids = torch.cat(ids_list)
        u, v = ids // V, ids % V
        comp = torch.arange(V, device="cuda")
        for _ in range(200):
            m = torch.minimum(comp[u], comp[v])
            new = comp.clone()
            new.scatter_reduce_(0, u, m, "amin")
            new.scatter_reduce_(0, v, m, "amin")
            new = new[new]
            if torch.equal(new, comp):
                break
            comp = new
        assert np.array_equal(lab, comp.cpu().numpy().astype(np.uint32))
        ids_sorted, _ = torch.sort(ids)
        f = torch.from_numpy(forest[:nf].astype(np.int64)).cuda()
        pos = torch.searchsorted(ids_sorted, f).clamp(max=ids_sorted.numel() - 1)

        def present(x):
            return (ids_sorted[pos] == f).cpu().numpy()

        _check_forest(V, forest[:nf], present, lab)
        ws = [0, 1, 2, 1000, 65535, 131071]
        rows = _sampled_rows(g, V, ws)
        for j, w in enumerate(ws):
            nb = torch.cat([v[u == w], u[v == w]]).cpu().numpy()
            assert np.array_equal(rows[:, j], O.vertex_sketch(V, seed, w, nb)), w
    finally:
        C.cupc_destroy(g)
