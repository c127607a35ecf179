"""Serving runtime (cupc_server): each graph's results are the same alone and
in a mix of graphs served concurrently (bit-identical answers and sketches,
answers equal to the oracle's), admission waits for memory, and an invalid
batch is reported on its own ticket only."""
import numpy as np
import pytest

import oracle as O
from paper_2509_14433_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAXB = 1 << 15


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _serve(streams, which, mem_bytes, query_streams=3):
    """Submit the steps of graphs `which` round-robin; wait for everything.
    Returns {graph: (answers list, sketch export)}."""
    from paper_2509_14433_gb300 import cupc as C
    st, srv = C.cupc_server_create(mem_bytes, 16, MAXB, query_streams)
    assert st == 0
    try:
        ids, outs, tickets = {}, {i: [] for i in which}, []
        for i in which:
            V, seed, _, _ = streams[i]
            st, ids[i] = C.cupc_server_open(srv, V, seed)
            assert st == 0
        order = WL.round_robin([streams[i] if i in which else (0, 0, [], 0) for i in range(len(streams))])
        keep = []
        for i, stp in order:
            if stp[0] == "update":
                e = np.ascontiguousarray(stp[1], np.uint32)
                o = np.ascontiguousarray(stp[2], np.int8)
                keep.append((e, o))
                st, t = C.cupc_server_update(srv, ids[i], e, o, len(o))
            else:
                p = np.ascontiguousarray(stp[1], np.uint32)
                out = np.full(len(p), 7, np.uint8)
                keep.append((p, out))
                outs[i].append(out)
                st, t = C.cupc_server_query(srv, ids[i], p, len(p), out)
            assert st == 0
            tickets.append(t)
        for t in tickets:
            st, lat = C.cupc_server_wait(srv, t, 120000)
            assert st == 0 and lat > 0
        res = {}
        for i in which:
            V = streams[i][0]
            L, Cc, D, W = O.params(V)
            ex = np.zeros((L, V, W, 2), np.uint64)
            assert C.cupc_server_export(srv, ids[i], ex, ex.nbytes) == 0
            res[i] = (outs[i], ex)
        stats = np.zeros(8, np.uint64)
        C.cupc_server_stats(srv, stats)
        return res, stats
    finally:
        C.cupc_server_destroy(srv)


def test_each_graph_is_the_same_alone_and_in_the_mix():
    streams = WL.serving_streams(n_graphs=6, v_exp=(8, 11), upd_range=(2e4, 8e4), batch_range=(200, 20000),
                                 rho=15000, q_size=300, seed=11)
    mem = 4 << 30
    mixed, stats = _serve(streams, list(range(6)), mem)
    assert stats[2] <= stats[3]  # one launch sequence serves one or more update requests
    for i in (0, 3):
        alone, _ = _serve(streams, [i], mem)
        a_out, a_ex = alone[i]
        m_out, m_ex = mixed[i]
        assert len(a_out) == len(m_out) > 0
        for x, y in zip(a_out, m_out):
            assert np.array_equal(x, y)
        assert np.array_equal(a_ex, m_ex)
        # and both equal the oracle on the same stream
        V, seed, steps, _ = streams[i]
        ref = O.Graph(V, seed)
        k = 0
        for stp in steps:
            if stp[0] == "update":
                ref.update(stp[1], stp[2])
            else:
                s, ans = ref.query(stp[1])
                assert np.array_equal(ans, m_out[k])
                k += 1
        assert np.array_equal(ref.export(), m_ex)


def test_admission_waits_for_memory():
    from paper_2509_14433_gb300 import cupc as C
    V = 2000
    one = C.cupc_workspace_bytes(V, (0, 0, 0, MAXB))
    st, srv = C.cupc_server_create(int(2.5 * one), 8, MAXB, 2)
    assert st == 0
    try:
        g = WL.rng(3)
        ids = [C.cupc_server_open(srv, V, 50 + k)[1] for k in range(5)]
        tickets, outs = [], []
        for k, gid in enumerate(ids):
            E = WL.uniform_pairs(V, 3000, g)
            tickets.append(C.cupc_server_update(srv, gid, E, np.ones(len(E), np.int8), len(E))[1])
            p = WL.uniform_pairs(V, 100, g, distinct=False)
            out = np.zeros(100, np.uint8)
            outs.append((E, p, out))
            tickets.append(C.cupc_server_query(srv, gid, p, 100, out)[1])
            tickets.append(C.cupc_server_close(srv, gid)[1])
        for t in tickets:
            assert C.cupc_server_wait(srv, t, 120000)[0] == 0
        stats = np.zeros(8, np.uint64)
        C.cupc_server_stats(srv, stats)
        assert stats[4] == 5 and stats[5] > 0 and stats[6] == 0
        for k, (E, p, out) in enumerate(outs):
            ref = O.Graph(V, 50 + k)
            ref.update(E)
            assert np.array_equal(ref.query(p)[1], out)
    finally:
        C.cupc_server_destroy(srv)


def test_invalid_batch_reported_on_its_ticket_only():
    from paper_2509_14433_gb300 import cupc as C
    st, srv = C.cupc_server_create(1 << 30, 4, MAXB, 2)
    try:
        a = C.cupc_server_open(srv, 100, 1)[1]
        b = C.cupc_server_open(srv, 100, 2)[1]
        good = np.array([[1, 2], [3, 4]], np.uint32)
        bad = np.array([[5, 5]], np.uint32)
        t1 = C.cupc_server_update(srv, a, good, np.ones(2, np.int8), 2)[1]
        t2 = C.cupc_server_update(srv, b, bad, np.ones(1, np.int8), 1)[1]
        assert C.cupc_server_wait(srv, t1)[0] == 0
        assert C.cupc_server_wait(srv, t2)[0] == C.CUPC_EINVAL
        # the error was reported; the next batch of b applies
        t3 = C.cupc_server_update(srv, b, good, np.ones(2, np.int8), 2)[1]
        out = np.zeros(2, np.uint8)
        t4 = C.cupc_server_query(srv, b, np.array([[1, 2], [1, 3]], np.uint32), 2, out)[1]
        assert C.cupc_server_wait(srv, t3)[0] == 0
        assert C.cupc_server_wait(srv, t4)[0] == 0
        assert out.tolist() == [1, 0]
        assert C.cupc_server_update(srv, 999, good, np.ones(2, np.int8), 2)[0] == C.CUPC_EINVAL
    finally:
        C.cupc_server_destroy(srv)
