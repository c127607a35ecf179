"""The allocation-free update entry point against the regular one.

cupc_update_sketch_static serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or their path must not pay an
allocation's synchronisation): the caller owns the sketch buffer and the
library's scratch is a fixed static device array. Two calls in a row must
leave the caller's buffer bit-identical to what cupc_update_batch +
cupc_export_sketches produce for the same batches (the tests' bar for this
integer path is exact equality). This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2509_14433_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_static_scratch_update_matches_regular_update_twice():
    from paper_2509_14433_gb300 import cupc as C
    from tests._dev import Dev

    V, seed = 3000, 17
    dev = Dev(V, seed)
    sketch = torch.zeros(dev.L * V * dev.W * 2, dtype=torch.int64, device="cuda")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    g = WL.rng(5)
    batches = [WL.er_edges(V, 0.003, 41), WL.uniform_pairs(V, 20000, g)]
    for k, E in enumerate(batches):
        ops = np.where(np.arange(len(E)) % 3 == 0, -1, 1).astype(np.int8)
        assert len(E) <= C.CUPC_STATIC_MAX_EDGES
        assert dev.update(E, ops) == 0
        e_d = torch.from_numpy(np.ascontiguousarray(E, np.uint32).reshape(-1)).cuda()
        o_d = torch.from_numpy(ops).cuda()
        st = C.cupc_update_sketch_static(sketch, V, seed, e_d, o_d, len(E), status, torch.cuda.current_stream())
        assert st == C.CUPC_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        ref = dev.export()
        got = sketch.cpu().numpy().view(np.uint64).reshape(ref.shape)
        assert np.array_equal(got, ref), f"call {k} differs from cupc_update_batch"


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    from paper_2509_14433_gb300 import cupc as C

    big_v = C.CUPC_STATIC_MAX_V + 1
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    e = torch.zeros(2 * (C.CUPC_STATIC_MAX_EDGES + 1), dtype=torch.int32, device="cuda")
    o = torch.ones(C.CUPC_STATIC_MAX_EDGES + 1, dtype=torch.int8, device="cuda")
    assert C.cupc_update_sketch_static(dummy, big_v, 1, e, o, 1) == C.CUPC_EINVAL
    assert C.cupc_update_sketch_static(dummy, 100, 1, e, o, C.CUPC_STATIC_MAX_EDGES + 1) == C.CUPC_EINVAL
    assert C.cupc_update_sketch_static(dummy, 1, 1, e, o, 1) == C.CUPC_EINVAL
