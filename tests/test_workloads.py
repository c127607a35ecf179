"""The seeded input generators produce valid streams (Problem 1 asks that an
insert names an absent edge and a delete a present one): every batch is
replayed against a set of present edges, update by update."""
import numpy as np
import pytest

from paper_2509_14433_gb300 import workloads as WL


def _replay(batches, V):
    present = set()
    for E, ops in batches:
        for (u, v), o in zip(np.asarray(E).tolist(), np.asarray(ops).tolist()):
            assert 0 <= u < v < V
            i = u * V + v
            if o == 1:
                assert i not in present
                present.add(i)
            else:
                assert o == -1 and i in present
                present.remove(i)
    return present


def test_rmat_stream_is_valid_and_bitmap_tracks_it():
    s = WL.RmatStream(levels=9, seed=5, batch_lo=50, batch_hi=4000)
    batches = [tuple(x.numpy() for x in s.next_batch()) for _ in range(60)]
    sizes = [len(o) for _, o in batches]
    assert min(sizes) >= 50 and max(sizes) <= 4000
    # 20% of each batch after the first deletes, deletes first
    for _, o in batches[1:]:
        k = int(np.sum(o == -1))
        assert abs(k - 0.2 * len(o)) <= 1
        assert np.all(o[:k] == -1) and np.all(o[k:] == 1)
    present = _replay(batches, s.V)
    bits = np.unpackbits(s.bitmap.numpy().view(np.uint8), bitorder="little")
    assert set(np.nonzero(bits)[0].tolist()) == present


def test_toggle_and_dense_streams_are_valid():
    V = 300
    steps = WL.plain_stream(V=V, p=0.3, n_toggles=20000, query_every=5000, query_size=10, seed=2)
    ups = [(st[1], st[2]) for st in steps if st[0] == "update"]
    assert sum(st[0] == "query" for st in steps) == 4
    present = _replay(ups, V)
    assert present == set(int(x) for x in WL.final_edge_set(V, steps))
    Ed, n_del, order = WL.dense_stream(V=V, p=0.5, seed=3)
    assert abs(len(Ed) - 0.5 * V * (V - 1) / 2) < 5 * np.sqrt(V * V / 8)
    dels = Ed[order[:n_del]]
    assert n_del == round(0.1 * len(Ed))
    _replay([(Ed, np.ones(len(Ed), np.int8)), (dels, -np.ones(len(dels), np.int8))], V)


def _components(V, E):
    sp = pytest.importorskip("scipy.sparse")
    from scipy.sparse.csgraph import connected_components
    E = np.asarray(E, np.int64).reshape(-1, 2)
    A = sp.csr_matrix((np.ones(len(E)), (E[:, 0], E[:, 1])), shape=(V, V))
    return connected_components(A, directed=False)


def test_standard_stream_inserts_all_then_deletes_all():
    V = 120
    E, ops = WL.standard_stream(V, 0.1, 4)
    n = len(E) // 2
    assert np.all(ops[:n] == 1) and np.all(ops[n:] == -1)
    assert _replay([(E, ops)], V) == set()
    ins = set((E[:n, 0].astype(np.int64) * V + E[:n, 1]).tolist())
    assert ins == set((WL.er_edges(V, 0.1, 4)[:, 0].astype(np.int64) * V + WL.er_edges(V, 0.1, 4)[:, 1]).tolist())
    assert not np.array_equal(E[:n], E[n:])  # each phase has its own order


def test_fixed_forest_stream_keeps_a_spanning_forest():
    V, p = 150, 0.02  # sparse: several components and isolated vertices
    E, ops, nf = WL.fixed_forest_stream(V, p, 6, cycles=2)
    static = WL.er_edges(V, p, 6)
    ncomp, lab = _components(V, static)
    F = E[:nf]
    assert np.all(ops[:nf] == 1) and nf == V - ncomp
    # the forest spans the static graph's components (V - ncomp acyclic edges)
    ncf, labf = _components(V, F)
    assert ncf == ncomp and np.array_equal(lab[F[:, 0]], lab[F[:, 1]])
    for a in range(ncomp):  # same partition
        assert len(set(labf[lab == a].tolist())) == 1
    # then every other edge is inserted and deleted, twice; the forest stays
    rest = len(static) - nf
    assert len(E) == nf + 4 * rest
    present = _replay([(E, ops)], V)
    assert present == set((F[:, 0].astype(np.int64) * V + F[:, 1]).tolist())
    for k in range(4):
        seg = slice(nf + k * rest, nf + (k + 1) * rest)
        assert np.all(ops[seg] == (1 if k % 2 == 0 else -1))


def test_serving_streams_are_valid_per_graph():
    streams = WL.serving_streams(n_graphs=4, v_exp=(6.0, 8.0), upd_range=(3000, 9000),
                                 batch_range=(50, 800), rho=2000, q_size=10, seed=3)
    for V, _, steps, done in streams:
        ups = [(st[1], st[2]) for st in steps if st[0] == "update"]
        assert sum(len(o) for _, o in ups) == done
        _replay(ups, V)
        for st in steps:
            if st[0] == "query":
                assert st[1].shape == (10, 2) and int(st[1].max()) < V
        nq = sum(st[0] == "query" for st in steps)
        assert nq == done // 2000
    order = WL.round_robin(streams)
    assert len(order) == sum(len(s[2]) for s in streams)
    for i, s in enumerate(streams):  # each graph's steps arrive in its own order
        mine = [st for j, st in order if j == i]
        assert len(mine) == len(s[2]) and all(a is b for a, b in zip(mine, s[2]))
    assert [j for j, _ in order[:len(streams)]] == list(range(len(streams)))


def test_clique_stream_is_a_valid_stream_of_the_stated_shape():
    # small instance of the adversarial workload: cliques are complete and
    # disjoint, bridges join different cliques, are distinct and absent from
    # the cliques, every insert batch is deleted again in the second half
    V, k, s = 64 * 8, 8, 64
    cl, order, pairs, comp = WL.clique_stream(V=V, k=k, s=s, n_batches=2, batch=100, seed=3)
    assert len(cl) == k * s * (s - 1) // 2
    assert np.all(comp[cl[:, 0]] == comp[cl[:, 1]])
    assert np.bincount(comp, minlength=k).tolist() == [s] * k
    ids = np.minimum(cl[:, 0], cl[:, 1]).astype(np.int64) * V + np.maximum(cl[:, 0], cl[:, 1])
    assert len(np.unique(ids)) == len(ids)
    ins = np.concatenate([E for E, op in order if op == 1])
    dels = np.concatenate([E for E, op in order if op == -1])
    assert [op for _, op in order] == [1, 1, -1, -1]
    assert np.all(comp[ins[:, 0]] != comp[ins[:, 1]])
    bid = ins[:, 0].astype(np.int64) * V + ins[:, 1]
    assert len(np.unique(bid)) == len(bid) == 200
    assert np.all(ins[:, 0] < ins[:, 1])
    assert np.array_equal(np.sort(bid), np.sort(dels[:, 0].astype(np.int64) * V + dels[:, 1]))
    assert pairs.shape == (1000, 2)
    same = comp[pairs[:, 0]] == comp[pairs[:, 1]]
    assert same.sum() >= 500  # 500 drawn inside one clique (+ chance collisions of the rest: none, c1 != c2)
    assert same.sum() == 500
    a, b, c, d = WL.clique_stream(V=V, k=k, s=s, n_batches=2, batch=100, seed=3)
    assert np.array_equal(a, cl) and np.array_equal(c, pairs)


def test_kronecker_graph_density_skew_and_forest():
    # the initiator [[1, b], [b, b^2]] at density 0.5: mean entry
    # ((1 + b) / 2)^(2k) = 0.5; pair (u, v) is an edge with probability
    # b^(popcount u + popcount v); parent[v] is v's smallest neighbour
    import torch
    k = 9
    b = WL.kronecker_b(k)
    assert abs(((1 + b) / 2) ** (2 * k) - 0.5) < 1e-12
    V = 1 << k
    ids, parent = WL.kronecker_graph(k, 3)
    ids = ids.numpy()
    parent = parent.numpy()
    n_pairs = V * (V - 1) // 2
    p = np.array([[b ** (bin(u).count("1") + bin(v).count("1")) for v in range(V)] for u in range(V)])
    want = p[np.triu_indices(V, 1)].sum()
    sd = np.sqrt((p[np.triu_indices(V, 1)] * (1 - p[np.triu_indices(V, 1)])).sum())
    assert abs(len(ids) - want) < 5 * sd and abs(len(ids) / n_pairs - 0.5) < 0.02
    u, v = ids // V, ids % V
    assert np.all(u < v) and np.all(np.diff(ids) != 0)
    deg = np.bincount(np.concatenate([u, v]), minlength=V)
    assert deg[0] > deg[V - 1]  # fewer one-bits: more neighbours
    # parent: the smallest neighbour below v, else v itself
    for w in (1, 5, V // 2, V - 1):
        nb = np.concatenate([u[v == w]])
        assert parent[w] == (nb.min() if nb.size else w)
    assert torch.equal(WL.kronecker_graph(k, 3)[0], torch.from_numpy(ids))
