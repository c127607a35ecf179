"""Incremental labels (cupc_set_incremental): on a valid stream, every
Connected answer equals the oracle's (a full recovery from the sketches),
queries after insert-only batches skip the recovery, a deleted forest edge
brings it back, and the spanning forest is always a full recovery's."""
import numpy as np
import pytest

import oracle as O
from paper_2509_14433_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev(*a, **k):
    from tests._dev import Dev
    return Dev(*a, **k)


def _absent_pairs(V, k, present, g):
    out = []
    while len(out) < k:
        u, v = (int(x) for x in g.integers(0, V, 2))
        if u == v:
            continue
        a, b = min(u, v), max(u, v)
        if a * V + b not in present and (a, b) not in out:
            out.append((a, b))
    return np.array(out, np.uint32)


# V up to 4096 recovers in one thread-block cluster, larger V across the grid
@pytest.mark.parametrize("V,p", [(1500, 0.0008), (5000, 0.00024)])
def test_incremental_labels_match_full_recovery(V, p):
    from paper_2509_14433_gb300 import cupc as C
    from tests.test_gpu_parity import assert_same_recovery
    seed = 31
    g = WL.rng(seed)
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    assert C.cupc_set_incremental(dev.h, 1, None) == 0
    E0 = WL.er_edges(V, p, seed)  # sparse: many components to merge
    present = set(int(a) * V + int(b) for a, b in E0)
    assert dev.update(E0) == 0 and ref.update(E0) == O.OK
    queries = 0
    plan = ["ins"] * 12 + ["del"] * 4 + ["ins"] * 6 + ["mix"] * 3 + ["ins"] * 4
    for kind in plan:
        if kind in ("ins", "mix"):
            E = _absent_pairs(V, int(g.integers(1, 200)), present, g)
            ops = np.ones(len(E), np.int8)
            present.update(int(a) * V + int(b) for a, b in E)
        if kind in ("del", "mix"):
            ids = np.array(sorted(present), np.int64)
            pick = ids[g.choice(len(ids), min(len(ids), int(g.integers(1, 60))), replace=False)]
            D = np.stack([pick // V, pick % V], 1).astype(np.uint32)
            present.difference_update(int(x) for x in pick)
            if kind == "mix":  # deletes first: a valid order
                E, ops = np.concatenate([D, E]), np.concatenate([-np.ones(len(D), np.int8), ops])
            else:
                E, ops = D, -np.ones(len(D), np.int8)
        assert dev.update(E, ops) == 0 and ref.update(E, ops) == O.OK
        pairs = WL.uniform_pairs(V, 500, g, distinct=False)
        s1, a1 = dev.query(pairs)
        s2, a2 = ref.query(pairs)
        assert s1 == s2 == 0 and np.array_equal(a1, a2), kind
        queries += 1
    st = dev.stats()
    # the first query recovers; insert-only batches after it do not
    assert st["recoveries"] < queries - 10, st
    assert np.array_equal(dev.labels(), ref.labels())
    # the forest is a full recovery's, bit-exact with the oracle's
    assert_same_recovery(dev, ref)
    assert dev.stats()["recoveries"] == st["recoveries"] + 1


def test_incremental_off_by_default_and_switchable():
    from paper_2509_14433_gb300 import cupc as C
    V = 400
    dev, ref = _dev(V, 5), O.Graph(V, 5)
    E = WL.er_edges(V, 0.01, 5)
    assert dev.update(E) == 0 and ref.update(E) == O.OK
    p = WL.uniform_pairs(V, 200, WL.rng(5), distinct=False)
    present = set(int(a) * V + int(b) for a, b in E)
    e = np.array([next((0, v) for v in range(1, V) if v not in present)], np.uint32)  # an absent edge
    for on in (0, 1, 0):
        assert C.cupc_set_incremental(dev.h, on, None) == 0
        n0 = dev.stats()["recoveries"]
        for k in range(4):  # insert, delete, insert, delete: a valid stream
            s1, a1 = dev.query(p)
            assert np.array_equal(a1, ref.query(p)[1])
            op = np.array([1 if k % 2 == 0 else -1], np.int8)
            assert dev.update(e, op) == 0 and ref.update(e, op) == O.OK
        if not on:  # off: every query after an update recovers
            assert dev.stats()["recoveries"] == n0 + 4
    assert C.cupc_set_incremental(None, 1, None) == C.CUPC_EINVAL


@pytest.mark.parametrize("V,p,per_batch", [(600, 0.02, 120), (5000, 0.0024, 1000)])
def test_warm_start_after_forest_edge_deletes(V, p, per_batch):
    # delete-only batches: a deleted forest edge makes the next recovery
    # start from the fragments of the remaining forest (round 0 samples
    # fewer than V components); the graph falls apart over the batches and
    # every answer still equals the oracle's full recovery
    from paper_2509_14433_gb300 import cupc as C
    from tests.test_gpu_parity import assert_same_recovery
    seed = 41
    g = WL.rng(seed)
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    assert C.cupc_set_incremental(dev.h, 1, None) == 0
    E = WL.er_edges(V, p, seed)
    present = set(int(a) * V + int(b) for a, b in E)
    assert dev.update(E) == 0 and ref.update(E) == O.OK
    warm = 0
    for k in range(25):
        ids = np.array(sorted(present), np.int64)
        pick = ids[g.choice(len(ids), min(len(ids), per_batch), replace=False)]
        present.difference_update(int(x) for x in pick)
        D = np.stack([pick // V, pick % V], 1).astype(np.uint32)
        ops = -np.ones(len(D), np.int8)
        assert dev.update(D, ops) == 0 and ref.update(D, ops) == O.OK
        pairs = WL.uniform_pairs(V, 400, g, distinct=False)
        s1, a1 = dev.query(pairs)
        s2, a2 = ref.query(pairs)
        assert s1 == s2 == 0 and np.array_equal(a1, a2), k
        if dev.round_log()[0][0] < V:
            warm += 1
    assert warm > 0
    assert np.array_equal(dev.labels(), ref.labels())
    assert len(np.unique(ref.labels())) > 1  # the graph did fall apart
    assert_same_recovery(dev, ref)


def test_fixed_forest_stream_keeps_the_labels():
    # the forest goes in first (one recovery, then merges recorded as forest
    # edges), then every other edge is inserted and deleted in delete-only
    # batches: no delete hits the forest, so no further recovery runs, and
    # every answer equals the oracle's full recovery
    from paper_2509_14433_gb300 import cupc as C
    from tests.test_gpu_parity import assert_same_recovery
    V, seed = 700, 51
    E, ops, nf = WL.fixed_forest_stream(V, 0.05, seed, cycles=1)
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    assert C.cupc_set_incremental(dev.h, 1, None) == 0
    g = WL.rng(seed)
    cuts = [0, nf // 3, nf] + list(range(nf + 400, len(E), 400)) + [len(E)]
    for a, b in zip(cuts[:-1], cuts[1:]):
        assert dev.update(E[a:b], ops[a:b]) == 0 and ref.update(E[a:b], ops[a:b]) == O.OK
        pairs = WL.uniform_pairs(V, 300, g, distinct=False)
        s1, a1 = dev.query(pairs)
        s2, a2 = ref.query(pairs)
        assert s1 == s2 == 0 and np.array_equal(a1, a2), a
    assert dev.stats()["recoveries"] == 1
    assert np.array_equal(dev.labels(), ref.labels())
    assert_same_recovery(dev, ref)


@pytest.mark.parametrize("V,p", [(800, 0.002), (5000, 0.00032)])
def test_deleting_merge_edges_recovers_warm(V, p):
    # inserts that join components become forest edges; deleting them (and
    # recovered forest edges) in a delete-only batch splits the components
    # again: the next query starts from the remaining fragments
    from paper_2509_14433_gb300 import cupc as C
    seed = 61
    g = WL.rng(seed)
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    assert C.cupc_set_incremental(dev.h, 1, None) == 0
    E0 = WL.er_edges(V, p, seed)  # sparse: many components
    present = set(int(a) * V + int(b) for a, b in E0)
    assert dev.update(E0) == 0 and ref.update(E0) == O.OK
    pairs = WL.uniform_pairs(V, 500, g, distinct=False)
    assert np.array_equal(dev.query(pairs)[1], ref.query(pairs)[1])
    n0 = dev.stats()["recoveries"]
    for k in range(3):
        B = _absent_pairs(V, 150, present, g)
        present.update(int(a) * V + int(b) for a, b in B)
        assert dev.update(B) == 0 and ref.update(B) == O.OK  # insert-only: merges, no recovery
        assert np.array_equal(dev.query(pairs)[1], ref.query(pairs)[1])
        assert dev.stats()["recoveries"] == n0
        # delete-only: half of the bridges just added plus some old edges
        D = np.concatenate([B[: len(B) // 2], np.array([divmod(x, V) for x in
                                                       sorted(present)[:: max(1, len(present) // 40)]], np.uint32)])
        D = np.unique(D, axis=0)
        present.difference_update(int(a) * V + int(b) for a, b in D)
        o = -np.ones(len(D), np.int8)
        assert dev.update(D, o) == 0 and ref.update(D, o) == O.OK
        s1, a1 = dev.query(pairs)
        s2, a2 = ref.query(pairs)
        assert s1 == s2 == 0 and np.array_equal(a1, a2), k
        assert dev.stats()["recoveries"] == n0 + 1
        assert dev.round_log()[0][0] < V  # warm: round 0 starts from fragments
        n0 += 1
    assert np.array_equal(dev.labels(), ref.labels())


def test_batcher_updates_drop_incremental_labels():
    from paper_2509_14433_gb300 import cupc as C
    V, seed = 500, 71
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    assert C.cupc_set_incremental(dev.h, 1, None) == 0
    E0 = WL.er_edges(V, 0.002, seed)
    assert dev.update(E0) == 0 and ref.update(E0) == O.OK
    pairs = WL.uniform_pairs(V, 400, WL.rng(seed), distinct=False)
    assert np.array_equal(dev.query(pairs)[1], ref.query(pairs)[1])
    st, b = C.cupc_batcher_create(4, True)
    assert st == 0
    try:
        present = set(int(a) * V + int(x) for a, x in E0)
        B = _absent_pairs(V, 300, present, WL.rng(seed + 1))
        e = torch.from_numpy(np.ascontiguousarray(B).reshape(-1)).cuda()
        o = torch.ones(len(B), dtype=torch.int8, device="cuda")
        assert C.cupc_batcher_update(b, [dev.h], [e], [o], [len(B)]) == 0
        torch.cuda.synchronize()
        ref.update(B)
        assert np.array_equal(dev.query(pairs)[1], ref.query(pairs)[1])
        assert np.array_equal(dev.labels(), ref.labels())
    finally:
        C.cupc_batcher_destroy(b)


def test_mixed_batches_keep_the_labels_and_follow_the_order_inside_a_batch():
    # batches that both merge components and delete edges, in a valid order
    # inside the batch: deletes of present edges (forest edges among them),
    # inserts that merge, and inserts deleted again later in the same batch
    # (an edge that joined two components and is removed at once). Every
    # answer equals the oracle's full recovery; batches whose deletes miss
    # the kept forest need no recovery.
    from paper_2509_14433_gb300 import cupc as C
    V, seed = 800, 12
    g = WL.rng(seed)
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    assert C.cupc_set_incremental(dev.h, 1, None) == 0
    E0 = WL.er_edges(V, 0.0015, seed)
    present = set(int(a) * V + int(b) for a, b in E0)
    assert dev.update(E0) == 0 and ref.update(E0) == O.OK
    pairs = WL.uniform_pairs(V, 600, g, distinct=False)
    assert np.array_equal(dev.query(pairs)[1], ref.query(pairs)[1])
    rec0 = dev.stats()["recoveries"]
    for step in range(30):
        ids = np.array(sorted(present), np.int64)
        pick = ids[g.choice(len(ids), int(g.integers(1, 25)), replace=False)]
        D = np.stack([pick // V, pick % V], 1).astype(np.uint32)
        present.difference_update(int(x) for x in pick)
        I = _absent_pairs(V, int(g.integers(5, 80)), present, g)
        again = I[: int(g.integers(0, 4))]  # inserted, then deleted again in this batch
        present.update(int(a) * V + int(b) for a, b in I[len(again):])
        E = np.concatenate([D, I, again])
        ops = np.concatenate([-np.ones(len(D), np.int8), np.ones(len(I), np.int8), -np.ones(len(again), np.int8)])
        assert dev.update(E, ops) == 0 and ref.update(E, ops) == O.OK
        pairs = WL.uniform_pairs(V, 600, g, distinct=False)
        s1, a1 = dev.query(pairs)
        s2, a2 = ref.query(pairs)
        assert s1 == s2 == 0 and np.array_equal(a1, a2), step
        assert np.array_equal(dev.labels(), ref.labels()), step
    # at most one recovery per query (a warm one after a forest edge went)
    assert dev.stats()["recoveries"] - rec0 <= 30
    ids = np.array(sorted(present), np.int64)
    # a batch that merges and deletes only edges outside the kept forest:
    # no recovery at all
    st, forest = dev.forest()
    fset = set(int(x) for x in forest)
    nonf = np.array([x for x in ids.tolist() if x not in fset][:10], np.int64)
    rec1 = dev.stats()["recoveries"]
    I = _absent_pairs(V, 40, present, g)
    E = np.concatenate([np.stack([nonf // V, nonf % V], 1).astype(np.uint32), I])
    ops = np.concatenate([-np.ones(len(nonf), np.int8), np.ones(len(I), np.int8)])
    assert dev.update(E, ops) == 0 and ref.update(E, ops) == O.OK
    pairs = WL.uniform_pairs(V, 600, g, distinct=False)
    assert np.array_equal(dev.query(pairs)[1], ref.query(pairs)[1])
    assert dev.stats()["recoveries"] == rec1



# V up to 4096 recovers in one thread-block cluster, larger V across the grid
@pytest.mark.parametrize("V,k", [(600, 20), (5000, 100)])
def test_warm_start_samples_only_the_split_components(V, k):
    # k components, each a cycle with chords; deleting one forest edge splits
    # one component in two: the warm recovery samples those two fragments
    # only (every other component starts final, its cut being empty) and
    # finds the replacement edge; answers and labels equal the oracle's
    from paper_2509_14433_gb300 import cupc as C
    seed = 81
    g = WL.rng(seed)
    s = V // k
    edges = set()
    for c in range(k):
        base = c * s
        for i in range(s):
            a, b = base + i, base + (i + 1) % s
            edges.add((min(a, b), max(a, b)))
        for _ in range(s // 2):
            a, b = (base + int(x) for x in g.choice(s, 2, replace=False))
            edges.add((min(a, b), max(a, b)))
    E = np.array(sorted(edges), np.uint32)
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    assert C.cupc_set_incremental(dev.h, 1, None) == 0
    assert dev.update(E) == 0 and ref.update(E) == O.OK
    pairs = WL.uniform_pairs(V, 500, g, distinct=False)
    assert np.array_equal(dev.query(pairs)[1], ref.query(pairs)[1])
    st, F = dev.forest()
    assert st == 0 and len(F) == V - k
    e = next(int(x) for x in F if (int(x) // V) // s == 3)  # a forest edge of component 3
    D = np.array([[e // V, e % V]], np.uint32)
    o = -np.ones(1, np.int8)
    assert dev.update(D, o) == 0 and ref.update(D, o) == O.OK
    s1, a1 = dev.query(pairs)
    s2, a2 = ref.query(pairs)
    assert s1 == s2 == 0 and np.array_equal(a1, a2)
    assert dev.round_log()[0][0] == 2  # the two sides of the deleted edge, not all k components
    assert np.array_equal(dev.labels(), ref.labels())
    assert len(np.unique(dev.labels())) == k
