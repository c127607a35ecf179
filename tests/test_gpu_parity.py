"""CUDA path vs the CPU oracle, through the C-ABI, on the same seeded inputs.

All arithmetic is integer, so the bar is bit-exact: sketches (every bucket
word), per-round live counts and candidate sets, labels, forests and query
answers. Sizes span many work items and ragged tails; edge cases cover empty
and single-edge batches, a hub vertex split over several work items, repeated
toggles, chunked and host-staged batches, invalid batches and too few
rounds."""
import numpy as np
import pytest

import oracle as O
from paper_2509_14433_gb300 import workloads as WL
from tests._graphs import check_forest, min_labels

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


def assert_same_recovery(dev, ref):
    s_ref, f_ref = ref.spanning_forest()
    s_dev, f_dev = dev.forest()
    assert s_dev == s_ref
    assert np.array_equal(dev.labels(), ref.labels())
    assert np.array_equal(f_dev, f_ref)
    glog, olog = dev.round_log(), ref.round_log()
    assert len(glog) == len(olog)
    for (gl, gids), (ol, oids) in zip(glog, olog):
        assert gl == ol
        assert np.array_equal(gids, oids)
    gs, os_ = dev.stats(), ref.stats()
    assert (gs["rounds"], gs["fail"], gs["false_pos"], gs["complete"]) == \
        (os_["rounds"], os_["fail"], os_["false_pos"], os_["complete"])


# V up to 4096 recovers in one thread-block cluster, larger V across the grid
@pytest.mark.parametrize("V,p,seed", [(2, 1.0, 1), (5, 0.5, 2), (37, 0.2, 3), (256, 0.05, 4),
                                       (1000, 0.01, 5), (1024, 0.5, 6), (3001, 0.002, 7), (4096, 0.01, 8),
                                       (5000, 0.002, 9)])
def test_sketches_and_recovery_bit_exact(V, p, seed):
    steps = WL.toggle_stream(V, WL.er_edges(V, p, seed), 3 * V, max(1, V // 2), 64, seed=seed + 10,
                             batch_cap=max(1, V * 7))
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    for k, st in enumerate(steps):
        if st[0] == "update":
            assert dev.update(st[1], st[2]) == 0
            assert ref.update(st[1], st[2]) == O.OK
            if k < 3 or k == len(steps) - 2:
                assert np.array_equal(dev.export(), ref.export())
        else:
            s1, a1 = dev.query(st[1])
            s2, a2 = ref.query(st[1])
            assert s1 == 0 and np.array_equal(a1, a2)
    assert np.array_equal(dev.export(), ref.export())
    assert_same_recovery(dev, ref)
    assert dev.sync() == (0 if ref.stats()["complete"] else 3)


@pytest.mark.parametrize("V,p,seed", [(20000, 0.0001, 8), (40000, 0.00004, 9)])
def test_recovery_with_many_candidates_after_round_0(V, p, seed):
    # sparse graphs whose round 1 still has more than 1024 candidates: later
    # rounds hook across the grid as well as in one CTA (up to 1024)
    E = WL.er_edges(V, p, seed)
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    assert dev.update(E) == 0
    assert ref.update(E) == O.OK
    assert_same_recovery(dev, ref)
    ncand = [len(ids) for _, ids in ref.round_log()]
    assert ncand[1] > 1024 and min(ncand[2:]) <= 1024


def test_plain_stream_full_size():
    # V=1024: ER(0.5) start graph, 200k uniform toggles, 1k-pair Connected
    # batch every 10k updates; every answer and the final sketch bit-exact
    V, seed = 1024, 1
    steps = WL.plain_stream(V=V, seed=1)
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    nq = 0
    for st in steps:
        if st[0] == "update":
            assert dev.update(st[1], st[2]) == 0
            ref.update(st[1], st[2])
        else:
            s1, a1 = dev.query(st[1])
            s2, a2 = ref.query(st[1])
            assert s1 == 0 and s2 == O.OK and np.array_equal(a1, a2)
            nq += 1
    assert nq == 20
    assert np.array_equal(dev.export(), ref.export())
    assert_same_recovery(dev, ref)
    lab = min_labels(V, WL.final_edge_set(V, steps))
    assert np.array_equal(dev.labels(), lab)


def test_empty_and_single_edge_batches():
    V = 64
    dev, ref = _dev(V, 3), O.Graph(V, 3)
    assert dev.update(np.zeros((0, 2), np.uint32)) == 0
    st, f = dev.forest()
    assert st == 0 and f.size == 0
    assert np.array_equal(dev.labels(), np.arange(V, dtype=np.uint32))
    for e in ([5, 9], [9, 5], [0, 63], [62, 63]):
        assert dev.update([e]) == 0
        ref.update(np.array([e], np.uint32))
        assert np.array_equal(dev.export(), ref.export())
    assert_same_recovery(dev, ref)


def test_hub_vertex_split_over_work_items():
    # vertex 0 has V-1 records (> one work item): several CTAs fold its
    # buckets, deep rows and the deterministic bucket see many writers
    V = 5000
    E = np.stack([np.zeros(V - 1, np.uint32), np.arange(1, V, dtype=np.uint32)], 1)
    rng = np.random.default_rng(0)
    E = E[rng.permutation(len(E))]
    E[::3] = E[::3, ::-1]
    extra = WL.er_edges(V, 0.0005, 9)
    dev, ref = _dev(V, 11), O.Graph(V, 11)
    for batch in (E, extra):
        dev.update(batch)
        ref.update(batch)
    assert np.array_equal(dev.export(), ref.export())
    assert_same_recovery(dev, ref)


def test_repeated_toggles_cancel():
    V = 100
    e = np.array([[3, 7]] * 1001 + [[4, 8]] * 1000 + [[1, 2]], np.uint32)
    ops = np.where(np.arange(len(e)) % 2 == 0, 1, -1).astype(np.int8)
    dev, ref = _dev(V, 5), O.Graph(V, 5)
    dev.update(e, ops)
    ref.update(e, ops)
    x = dev.export()
    assert np.array_equal(x, ref.export())
    nz = np.nonzero(x.any(axis=(0, 2, 3)))[0].tolist()
    assert nz == [1, 2, 3, 7]


@pytest.mark.parametrize("host", [False, True])
def test_chunked_batches_and_host_buffers(host):
    V = 700
    params = (0, 0, 0, 1000)  # max_batch = 1000 edges per internal chunk
    E = WL.er_edges(V, 0.03, 12)
    ops = np.ones(len(E), np.int8)
    dev, ref = _dev(V, 8, params), O.Graph(V, 8)
    assert len(E) > 3 * 1000
    assert dev.update(E, ops, host=host) == 0
    ref.update(E, ops)
    assert np.array_equal(dev.export(), ref.export())
    pairs = WL.uniform_pairs(V, 2500, WL.rng(3), distinct=False)
    s1, a1 = dev.query(pairs, host=host)
    s2, a2 = ref.query(pairs)
    assert s1 == 0 and np.array_equal(a1, a2)
    assert_same_recovery(dev, ref)
    assert dev.stats()["chunks"] >= 7 if not host else True


def test_host_batches_in_a_row_alternate_staging():
    # host batches are copied on the graph's copy stream into two staging
    # buffers in turn; pinned and pageable buffers, a host query (which
    # stages on the caller's stream) and a mixed host/device batch between
    from paper_2509_14433_gb300 import cupc as C
    V = 3000
    dev, ref = _dev(V, 21, (0, 0, 0, 5000)), O.Graph(V, 21)
    g = WL.rng(21)
    keep = []
    for k in range(12):
        E = WL.uniform_pairs(V, 4000, g)
        if k % 2:
            e = torch.from_numpy(E.reshape(-1).copy()).pin_memory()
            o = torch.ones(len(E), dtype=torch.int8).pin_memory()
        else:
            e, o = E.reshape(-1).copy(), np.ones(len(E), np.int8)
        keep.append((e, o))
        assert C.cupc_update_batch(dev.h, e, o, len(E), None) == 0
        ref.update(E)
        if k == 5:
            pairs = WL.uniform_pairs(V, 300, g, distinct=False)
            s1, a1 = dev.query(pairs, host=True)
            s2, a2 = ref.query(pairs)
            assert s1 == 0 and np.array_equal(a1, a2)
        if k == 8:
            M = WL.uniform_pairs(V, 2000, g)
            ed = torch.from_numpy(M.reshape(-1).copy()).cuda()
            assert C.cupc_update_batch(dev.h, ed, np.ones(len(M), np.int8), len(M), None) == 0
            ref.update(M)
    torch.cuda.synchronize()
    assert np.array_equal(dev.export(), ref.export())
    assert_same_recovery(dev, ref)


@pytest.mark.parametrize("host", [False, True])
def test_invalid_batch_is_dropped_whole_and_sticky(host):
    V = 50
    params = (0, 0, 0, 4)
    dev, ref = _dev(V, 2, params), O.Graph(V, 2)
    good = np.array([[0, 1], [1, 2], [2, 3]], np.uint32)
    dev.update(good, host=host)
    ref.update(good)
    before = dev.export()
    bad_cases = [
        (np.array([[4, 5], [6, 7], [8, 9], [10, 11], [12, 13], [7, 7]], np.uint32), None),
        (np.array([[4, 5], [6, 50]], np.uint32), None),
        (np.array([[4, 5]], np.uint32), np.array([0], np.int8)),
    ]
    for e, o in bad_cases:
        dev.update(e, o, host=host)
        assert np.array_equal(dev.export(), before)
        # later batches are dropped while the error is pending
        dev.update(np.array([[20, 21]], np.uint32), host=host)
        assert np.array_equal(dev.export(), before)
        assert dev.sync() == 1
        assert dev.sync() == 0
    dev.update(np.array([[20, 21]], np.uint32), host=host)
    ref.update(np.array([[20, 21]], np.uint32))
    assert np.array_equal(dev.export(), ref.export())


@pytest.mark.parametrize("host", [False, True])
def test_large_invalid_batch_on_small_graph_is_dropped_whole(host):
    # a batch of 2^16 edges on V=1000 is counted through shared histograms
    # and validated in that same pass: one bad entry anywhere still drops
    # the whole batch, leaves no counts behind, and the next batch is exact
    V, n = 1000, 1 << 16
    dev, ref = _dev(V, 9), O.Graph(V, 9)
    E = WL.er_edges(V, 0.3, 9)
    E = E[WL.rng(9).permutation(len(E))]
    first, second = E[:n], E[n:2 * n]
    assert dev.update(first, host=host) == 0 and ref.update(first) == O.OK
    before = dev.export()
    for pos, fix in ((n - 1, "loop"), (n // 2, "op"), (0, "range"), (12345, "range_u")):
        e, o = second.copy(), np.ones(n, np.int8)
        if fix == "loop":
            e[pos, 1] = e[pos, 0]
        elif fix == "op":
            o[pos] = 0
        elif fix == "range":
            e[pos, 1] = V
        else:
            e[pos, 0] = 0xFFFFFFFF
        dev.update(e, o, host=host)
        if host:
            torch.cuda.synchronize()
        assert np.array_equal(dev.export(), before), fix
        assert dev.sync() == 1 and dev.sync() == 0
    assert dev.update(second, host=host) == 0 and ref.update(second) == O.OK
    assert dev.sync() == 0
    assert np.array_equal(dev.export(), ref.export())
    pairs = WL.uniform_pairs(V, 300, WL.rng(10), distinct=False)
    assert np.array_equal(dev.query(pairs)[1], ref.query(pairs)[1])


def test_query_pair_out_of_range():
    V = 30
    dev = _dev(V, 1)
    dev.update(np.array([[0, 1]], np.uint32))
    st, a = dev.query(np.array([[0, 1], [0, 30], [2, 3]], np.uint32))
    assert a.tolist() == [1, 0, 0]
    assert dev.sync() == 1
    # an invalid query does not drop updates
    dev.update(np.array([[2, 3]], np.uint32))
    st, a = dev.query(np.array([[2, 3]], np.uint32))
    assert a.tolist() == [1]
    assert dev.sync() == 0


def test_too_few_rounds_incomplete_matches_oracle():
    V = 64
    E = np.array([[i, i + 1] for i in range(V - 1)], np.uint32)
    params = (2, 0, 0, 0)
    dev, ref = _dev(V, 1, params), O.Graph(V, 1, L=2)
    dev.update(E)
    ref.update(E)
    assert np.array_equal(dev.export(), ref.export())
    assert_same_recovery(dev, ref)
    assert dev.sync() == 3  # CUPC_EINCOMPLETE


@pytest.mark.parametrize("L,Cc,D", [(4, 2, 5), (3, 1, 3), (9, 12, 20)])
def test_parameter_overrides(L, Cc, D):
    V = 300
    E = WL.er_edges(V, 0.02, L * 100 + Cc)
    dev, ref = _dev(V, 4, (L, Cc, D, 0)), O.Graph(V, 4, L=L, C=Cc, D=D)
    assert (dev.L, dev.C, dev.D) == (L, Cc, D)
    dev.update(E)
    ref.update(E)
    assert np.array_equal(dev.export(), ref.export())
    assert_same_recovery(dev, ref)


def test_many_components_cliques_and_bridges():
    # scaled-down adversarial shape: disjoint cliques joined then split by
    # bridges; a query batch after every batch
    k, s, V = 16, 24, 16 * 24
    perm = WL.rng(5).permutation(V).astype(np.uint32)
    cl = []
    for c in range(k):
        m = perm[c * s:(c + 1) * s]
        iu, ju = np.triu_indices(s, 1)
        cl.append(np.stack([m[iu], m[ju]], 1))
    cl = np.concatenate(cl)
    g = WL.rng(6)
    dev, ref = _dev(V, 9), O.Graph(V, 9)
    dev.update(cl)
    ref.update(cl)
    comp = np.repeat(np.arange(k), s)[np.argsort(perm)]
    bridges = []
    while len(bridges) < 40:
        u, v = g.integers(0, V, 2)
        if comp[u] != comp[v]:
            bridges.append((min(u, v), max(u, v)))
    bridges = np.unique(np.array(bridges, np.uint32), axis=0)
    batches = [(b, 1) for b in np.array_split(bridges, 4)] + [(b, -1) for b in np.array_split(bridges[::-1], 4)]
    for b, op in batches:
        ops = np.full(len(b), op, np.int8)
        dev.update(b, ops)
        ref.update(b, ops)
        pairs = WL.uniform_pairs(V, 300, g, distinct=False)
        s1, a1 = dev.query(pairs)
        s2, a2 = ref.query(pairs)
        assert np.array_equal(a1, a2)
        assert_same_recovery(dev, ref)
    assert np.array_equal(dev.labels(), min_labels(V, np.sort((cl[:, 0].astype(np.int64) * V + cl[:, 1]))))


def test_workspace_borrowed_from_torch():
    from paper_2509_14433_gb300 import cupc as C
    V = 500
    nbytes = C.cupc_workspace_bytes(V, None)
    ws = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = ws.data_ptr()
    off = (-base) % 256
    dev = _dev(V, 3, None, base + off)
    ref = O.Graph(V, 3)
    E = WL.er_edges(V, 0.01, 2)
    dev.update(E)
    ref.update(E)
    assert np.array_equal(dev.export(), ref.export())
    assert_same_recovery(dev, ref)
    dev.close()
    assert C.cupc_init(V, 3, None, base + off + 8, None)[0] == C.CUPC_EINVAL


def test_smaller_graph_does_not_shrink_an_earlier_graphs_launch():
    # the apply kernel's shared-memory limit is process-wide; a graph that
    # needs less must not lower it under one that needs more
    big = (20, 12, 0, 0)  # 20 layers x 16 lanes: > 48 KB of dynamic shared memory
    V = 400
    E = WL.er_edges(V, 0.02, 31)
    dev_big, ref = _dev(V, 7, big), O.Graph(V, 7, L=20, C=12)
    small = _dev(100, 1)
    small.update(np.array([[1, 2]], np.uint32))
    assert dev_big.update(E) == 0
    ref.update(E)
    assert dev_big.sync() == 0
    assert np.array_equal(dev_big.export(), ref.export())
    assert_same_recovery(dev_big, ref)


def test_bounded_device_wait_reports_timeout_and_context_survives():
    # one CTA never reaches the grid barrier: the others give up after the
    # limit, report CUPC_ETIMEOUT, and the context keeps working
    from paper_2509_14433_gb300 import cupc as C
    import time
    t = time.perf_counter()
    assert C.cupc_selftest_wait_timeout(8, 20000, 3) == C.CUPC_ETIMEOUT
    assert time.perf_counter() - t < 5.0
    assert C.cupc_selftest_wait_timeout(8, 20000, -1) == C.CUPC_OK
    V = 50
    dev, ref = _dev(V, 1), O.Graph(V, 1)
    E = WL.er_edges(V, 0.1, 2)
    dev.update(E)
    ref.update(E)
    assert np.array_equal(dev.export(), ref.export())
    assert C.cupc_selftest_wait_timeout(1, 100, -1) == C.CUPC_EINVAL


def test_kernels_are_built_for_sm_103a():
    # what the CUDA runtime loaded for this device: SASS for compute 10.3
    from paper_2509_14433_gb300 import cupc as C
    st, binary, ptx = C.cupc_build_info()
    assert st == C.CUPC_OK
    assert binary == 103, binary
    major, minor = torch.cuda.get_device_capability(0)
    assert (major, minor) == (10, 3)
