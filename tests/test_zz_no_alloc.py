"""The allocation-free update entry point.

cupc_update_sketch_static serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or their path must not pay an
allocation's synchronisation): the caller owns the sketch buffer and the
library's scratch is a fixed static device array. Two calls in a row must
leave the caller's buffer bit-identical to what cupc_update_batch +
cupc_export_sketches produce for the same batches, and to the oracle's
sketches (the bar for this integer path is exact equality). This file is
collected last on purpose."""
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


def _static(sketch, V, seed, E, ops, status):
    from paper_2509_14433_gb300 import cupc as C
    e_d = torch.from_numpy(np.ascontiguousarray(E, np.uint32).reshape(-1)).cuda()
    o_d = torch.from_numpy(np.ascontiguousarray(ops, np.int8)).cuda()
    st = C.cupc_update_sketch_static(sketch, V, seed, e_d, o_d, len(ops), status, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return st


def test_static_scratch_update_matches_regular_update_and_oracle_twice():
    from paper_2509_14433_gb300 import cupc as C
    from tests._dev import Dev

    V, seed = 3000, 17
    dev = Dev(V, seed)
    ref = O.Graph(V, seed)
    sketch = torch.zeros(dev.L * V * dev.W * 2, dtype=torch.int64, device="cuda")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    g = WL.rng(5)
    batches = [WL.er_edges(V, 0.003, 41), WL.uniform_pairs(V, 20000, g)]
    for k, E in enumerate(batches):
        ops = np.where(np.arange(len(E)) % 3 == 0, -1, 1).astype(np.int8)
        assert len(E) <= C.CUPC_STATIC_MAX_EDGES
        assert dev.update(E, ops) == 0
        assert ref.update(E, ops) == O.OK
        assert _static(sketch, V, seed, E, ops, status) == C.CUPC_OK
        assert int(status.item()) == 0
        want = dev.export()
        got = sketch.cpu().numpy().view(np.uint64).reshape(want.shape)
        assert np.array_equal(got, want), f"call {k} differs from cupc_update_batch"
        assert np.array_equal(got, ref.export()), f"call {k} differs from the oracle"
    ref.close()
    dev.close()


def test_static_scratch_widest_graph_matches_the_oracle():
    # V = CUPC_STATIC_MAX_V: the launch shape the set-up sized for the widest
    # graph; one batch dense enough for the shared-histogram grouping, one
    # sparse (direct path); sampled vertices against the oracle's one-vertex
    # sketch and every word against cupc_update_batch
    from paper_2509_14433_gb300 import cupc as C
    from tests._dev import Dev

    V, seed = C.CUPC_STATIC_MAX_V, 23
    dev = Dev(V, seed)
    sketch = torch.zeros(dev.L * V * dev.W * 2, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rng = WL.rng(9)
    E1 = WL.uniform_pairs(V, C.CUPC_STATIC_MAX_EDGES, rng)
    ids = np.unique(np.minimum(E1[:, 0], E1[:, 1]).astype(np.int64) * V + np.maximum(E1[:, 0], E1[:, 1]))
    E1 = np.stack([ids // V, ids % V], 1).astype(np.uint32)
    hub = np.stack([np.zeros(3000, np.int64), np.arange(1, 3001)], 1).astype(np.uint32)  # a vertex of 3000 records
    hub = hub[~np.isin(hub[:, 1].astype(np.int64), ids[ids // V == 0] % V)]
    E = np.concatenate([E1[: C.CUPC_STATIC_MAX_EDGES - len(hub)], hub])
    for part in (E[:100], E[100:]):
        ops = np.ones(len(part), np.int8)
        assert dev.update(part, ops) == 0
        assert _static(sketch, V, seed, part, ops, status) == C.CUPC_OK
        assert int(status.item()) == 0
    want = dev.export()
    got = sketch.cpu().numpy().view(np.uint64).reshape(want.shape)
    assert np.array_equal(got, want)
    for w in (0, 1, int(E[5, 0]), V - 1):
        nb = np.concatenate([E[E[:, 0] == w, 1], E[E[:, 1] == w, 0]])
        assert np.array_equal(got[:, w], O.vertex_sketch(V, seed, w, nb)), w
    dev.close()


def test_static_scratch_drops_an_invalid_batch_and_recovers():
    # one out-of-range edge: status 1, the caller's sketch unchanged; the
    # next valid call applies as usual (the scratch keeps no stale error)
    from paper_2509_14433_gb300 import cupc as C

    V, seed = 500, 3
    L, _, _, W = O.params(V)
    sketch = torch.zeros(L * V * W * 2, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    E = WL.uniform_pairs(V, 2000, WL.rng(4))
    ops = np.ones(len(E), np.int8)
    assert _static(sketch, V, seed, E, ops, status) == C.CUPC_OK
    before = sketch.clone()
    bad = E.copy()
    bad[777, 1] = V
    assert _static(sketch, V, seed, bad, ops, status) == C.CUPC_OK
    assert int(status.item()) == 1
    assert torch.equal(sketch, before)
    assert _static(sketch, V, seed, E[:10], ops[:10], status) == C.CUPC_OK
    assert int(status.item()) == 0
    ref = O.Graph(V, seed)
    ref.update(E, ops)
    ref.update(E[:10], ops[:10])
    assert np.array_equal(sketch.cpu().numpy().view(np.uint64).reshape(L, V, W, 2), ref.export())
    ref.close()


def test_static_scratch_refuses_host_and_misaligned_pointers():
    from paper_2509_14433_gb300 import cupc as C

    V = 100
    L, _, _, W = O.params(V)
    sketch = torch.zeros(L * V * W * 2 + 2, dtype=torch.int64, device="cuda")
    e_h = np.ascontiguousarray(WL.uniform_pairs(V, 10, WL.rng(1)).reshape(-1))
    o_h = np.ones(10, np.int8)
    e_d = torch.from_numpy(e_h).cuda()
    o_d = torch.from_numpy(o_h).cuda()
    assert C.cupc_update_sketch_static(sketch, V, 1, e_h, o_d, 10) == C.CUPC_EINVAL
    assert C.cupc_update_sketch_static(sketch, V, 1, e_d, o_h, 10) == C.CUPC_EINVAL
    host_sketch = np.zeros(L * V * W * 2, np.uint64)
    assert C.cupc_update_sketch_static(host_sketch, V, 1, e_d, o_d, 10) == C.CUPC_EINVAL
    assert C.cupc_update_sketch_static(sketch.data_ptr() + 8, V, 1, e_d, o_d, 10) == C.CUPC_EINVAL
    torch.cuda.synchronize()
    assert not sketch.any()  # nothing ran


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    from paper_2509_14433_gb300 import cupc as C

    big_v = C.CUPC_STATIC_MAX_V + 1
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    e = torch.zeros(2 * (C.CUPC_STATIC_MAX_EDGES + 1), dtype=torch.int32, device="cuda")
    o = torch.ones(C.CUPC_STATIC_MAX_EDGES + 1, dtype=torch.int8, device="cuda")
    assert C.cupc_update_sketch_static(dummy, big_v, 1, e, o, 1) == C.CUPC_EINVAL
    assert C.cupc_update_sketch_static(dummy, 100, 1, e, o, C.CUPC_STATIC_MAX_EDGES + 1) == C.CUPC_EINVAL
    assert C.cupc_update_sketch_static(dummy, 1, 1, e, o, 1) == C.CUPC_EINVAL
