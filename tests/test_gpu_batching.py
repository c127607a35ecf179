"""Batching paths vs the oracle, bit-exact: uneven batches of one graph
coalesced (cupc_update_batches) and one batch per graph for many graphs of
different shapes in one launch sequence (cupc_batcher, with and without
CUDA-graph replay)."""
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


def test_uneven_batches_coalesced_match_oracle():
    from paper_2509_14433_gb300 import cupc as C
    V = 2000
    s = WL.RmatStream(levels=11, seed=4, batch_lo=10, batch_hi=30000, device="cpu")
    batches = [s.next_batch() for _ in range(25)]
    E = np.concatenate([b[0].numpy() for b in batches]).astype(np.uint32)
    ops = np.concatenate([b[1].numpy() for b in batches]).astype(np.int8)
    offs = np.cumsum([0] + [len(b[1]) for b in batches]).astype(np.uint64)
    dev = _dev(s.V, 3, (0, 0, 0, 4096))  # small chunks: coalesced groups span several
    ref = O.Graph(s.V, 3)
    e_d = torch.from_numpy(E.reshape(-1)).cuda()
    o_d = torch.from_numpy(ops).cuda()
    assert C.cupc_update_batches(dev.h, e_d, o_d, offs, len(batches)) == 0
    for b in batches:
        ref.update(b[0].numpy().astype(np.uint32), b[1].numpy())
    assert np.array_equal(dev.export(), ref.export())
    # an invalid entry anywhere drops the whole group
    before = dev.export()
    ops2 = ops.copy()
    ops2[len(ops2) // 2] = 0
    assert C.cupc_update_batches(dev.h, e_d, torch.from_numpy(ops2).cuda(), offs, len(batches)) == 0
    assert dev.sync() == 1
    assert np.array_equal(dev.export(), before)


@pytest.mark.parametrize("use_graph", [True, False])
def test_batcher_many_graphs_match_oracle(use_graph):
    from paper_2509_14433_gb300 import cupc as C
    # (500, rows 40) takes the wide-depth (D > 32) path of the apply kernel
    shapes = [(1500, None), (500, (0, 5, 40, 0)), (300, (5, 12, 0, 0)), (2, None), (4096, None), (999, (0, 3, 7, 0))]
    devs, refs = [], []
    for i, (V, prm) in enumerate(shapes):
        devs.append(_dev(V, 100 + i, prm))
        if prm is None:
            refs.append(O.Graph(V, 100 + i))
        else:
            refs.append(O.Graph(V, 100 + i, L=prm[0], C=prm[1], D=prm[2]))
    st, b = C.cupc_batcher_create(16, use_graph)
    assert st == 0
    try:
        g = WL.rng(9)
        for step in range(3):
            edges, ops, ns, keep = [], [], [], []
            for i, (V, _) in enumerate(shapes):
                m = int(g.integers(0, 3000)) if step != 1 or i != 3 else 0
                E = WL.uniform_pairs(V, m, g) if m else np.zeros((0, 2), np.uint32)
                o = np.where(g.random(m) < 0.5, 1, -1).astype(np.int8)
                if step == 2 and i == 4 and m:
                    o[m // 3] = 3  # invalid op: only this graph's batch is dropped
                keep.append((E, o))
                edges.append(torch.from_numpy(np.ascontiguousarray(E).reshape(-1)).cuda() if m else 0)
                ops.append(torch.from_numpy(o).cuda() if m else 0)
                ns.append(m)
            assert C.cupc_batcher_update(b, [d.h for d in devs], edges, ops, ns) == 0
            torch.cuda.synchronize()
            for i, (E, o) in enumerate(keep):
                if len(o):
                    refs[i].update(E, o)
            for i, (d, r) in enumerate(zip(devs, refs)):
                assert np.array_equal(d.export(), r.export()), (step, i)
            if step == 2:
                assert devs[4].sync() == 1
                assert refs[4].sync() == 1
        for d, r in zip(devs, refs):
            s_ref, f_ref = r.spanning_forest()
            s_dev, f_dev = d.forest()
            assert s_dev == s_ref and np.array_equal(f_dev, f_ref)
    finally:
        C.cupc_batcher_destroy(b)


def test_batcher_rejects_bad_calls():
    from paper_2509_14433_gb300 import cupc as C
    a, b2 = _dev(100, 1, (0, 0, 0, 64)), _dev(100, 2)
    st, b = C.cupc_batcher_create(2, True)
    try:
        e = torch.zeros(2 * 100, dtype=torch.int32, device="cuda")
        o = torch.ones(100, dtype=torch.int8, device="cuda")
        assert C.cupc_batcher_update(b, [a.h, a.h], [e, e], [o, o], [1, 1]) == C.CUPC_EINVAL  # same graph twice
        assert C.cupc_batcher_update(b, [a.h], [e], [o], [100]) == C.CUPC_EINVAL  # above max_batch
        assert C.cupc_batcher_update(b, [a.h, b2.h, a.h], [e] * 3, [o] * 3, [1] * 3) == C.CUPC_EINVAL  # k > max
        h = np.zeros(4, np.uint32)
        assert C.cupc_batcher_update(b, [b2.h], [h], [np.ones(2, np.int8)], [2]) == C.CUPC_EINVAL  # host memory
    finally:
        C.cupc_batcher_destroy(b)


def test_every_tuning_gives_identical_sketches():
    # the apply kernel's tunables change speed only, never the result
    from paper_2509_14433_gb300 import autotune as AT
    from paper_2509_14433_gb300 import cupc as C
    V = 3000
    E = WL.er_edges(V, 0.01, 5)
    ref = O.Graph(V, 8)
    ref.update(E)
    want = ref.export()
    for setting in [(64, 8, 0), (128, 16, 2), (512, 12, 0), (256, 1, 4), (512, 16, 1)]:
        dev = _dev(V, 8)
        assert C.cupc_set_tuning(dev.h, *setting) == 0
        out = np.zeros(4, np.uint32)
        C.cupc_get_tuning(dev.h, out)
        assert tuple(int(x) for x in out[:3]) == setting
        assert dev.update(E) == 0
        assert np.array_equal(dev.export(), want), setting
    # per-bucket settings: batches of 1k, 5k and 20k edges each take their
    # own bucket's setting (5, 6, 7); the default serves the rest
    dev = _dev(V, 8)
    for b, setting in ((5, (64, 4, 1)), (6, (512, 16, 0)), (7, (128, 12, 3))):
        assert C.cupc_set_tuning_bucket(dev.h, b, *setting) == 0
    assert C.cupc_set_tuning_bucket(dev.h, 8, 0, 0, 0) == 0  # cleared: the default
    i = 0
    for n in (1000, 5000, 20000, 3, 1 << 12):
        assert dev.update(E[i:i + n]) == 0
        i += n
    assert dev.update(E[i:]) == 0
    assert np.array_equal(dev.export(), want)
    assert C.cupc_set_tuning_bucket(dev.h, 4, 64, 8, 0) == C.CUPC_EINVAL
    assert C.cupc_set_tuning_bucket(dev.h, 16, 64, 8, 0) == C.CUPC_EINVAL
    assert C.cupc_set_tuning_bucket(dev.h, 6, 32, 8, 0) == C.CUPC_EINVAL
    assert C.cupc_set_tuning(dev.h, 32, 12, 0) == C.CUPC_EINVAL  # records per item below 64
    assert C.cupc_set_tuning(dev.h, 512, 17, 0) == C.CUPC_EINVAL  # more than 16 shared rows
    # both write-backs of single-item vertices, forced per bucket, and the automatic choice
    for mode in (C.CUPC_WRITEBACK_LOAD_STORE, C.CUPC_WRITEBACK_ATOMIC, C.CUPC_WRITEBACK_AUTO):
        dev = _dev(V, 8)
        for b in range(5, 16):
            assert C.cupc_set_writeback_bucket(dev.h, b, mode) == 0
        i = 0
        for n in (1000, 5000, 20000, 3):
            assert dev.update(E[i:i + n]) == 0
            i += n
        assert dev.update(E[i:]) == 0
        assert np.array_equal(dev.export(), want), mode
    assert C.cupc_set_writeback_bucket(dev.h, 4, C.CUPC_WRITEBACK_ATOMIC) == C.CUPC_EINVAL
    assert C.cupc_set_writeback_bucket(dev.h, 10, 3) == C.CUPC_EINVAL
    assert AT.bucket_of(1000) == 5 and AT.bucket_of(4096) == 6 and AT.bucket_of(1 << 20) == 10


def test_autotuner_writes_a_table_and_applies_it(tmp_path):
    from paper_2509_14433_gb300 import autotune as AT
    from paper_2509_14433_gb300 import cupc as C
    path = str(tmp_path / "t.json")
    ent = AT.tune(2048, sizes=[4096, 65536], reps=1, path=path, verbose=False)
    assert set(ent) == {"6", "8"}
    table = AT.load(path)
    dev = _dev(2048, 1)
    assert AT.apply(dev.h, 2048, 65536, table)
    out = np.zeros(4, np.uint32)
    C.cupc_get_tuning(dev.h, out)
    assert list(int(x) for x in out[:3]) == ent["8"]["setting"]
    # R-MAT batches (the skewed-degree workload) fill the same table
    ent2 = AT.tune(2048, sizes=[4096], reps=1, path=path, verbose=False, batches="rmat")
    assert ent2["6"]["batches"] == "rmat" and ent2["8"]["batches"] == "uniform"
    assert ent2["6"]["writeback"] in (C.CUPC_WRITEBACK_LOAD_STORE, C.CUPC_WRITEBACK_ATOMIC)
    assert AT.apply_buckets(dev.h, 2048, AT.load(path)) == 2
