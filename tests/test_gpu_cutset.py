"""The parallel cutset (§3.1, Lemma 3.1) against the oracle.

After random sequences of links, cuts and graph updates (with refreshes of
the updated vertices), the sketch the cutset keeps for every tree of its
forest equals the oracle's sum of the tree members' vertex sketches
(orc_sketch_sum, every layer and word), and its query equals the oracle's
sample of that sum. Invalid operations stop a batch where they occur."""
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


class Forest:
    """The forest by adjacency sets (test-side bookkeeping)."""

    def __init__(self, V):
        self.adj = [set() for _ in range(V)]

    def tree(self, w):
        seen, todo = {w}, [w]
        while todo:
            x = todo.pop()
            for y in self.adj[x]:
                if y not in seen:
                    seen.add(y)
                    todo.append(y)
        return sorted(seen)

    def edges(self):
        return [(u, v) for u in range(len(self.adj)) for v in self.adj[u] if u < v]


def _check_trees(C, cs, ref, forest, V, L, W, rng, n_check=12):
    roots = rng.choice(V, size=n_check, replace=False)
    for w in roots.tolist():
        members = forest.tree(w)
        got = np.zeros((L, W, 2), np.uint64)
        assert C.cupc_cutset_tree_sketch(cs, w, got) == C.CUPC_OK
        for r in range(L):
            want = ref.sketch_sum(members, r)
            assert np.array_equal(got[r], want), (w, r, len(members))
        for r in (0, L - 1):
            st, res, edge = C.cupc_cutset_query(cs, w, r)
            assert st == C.CUPC_OK
            assert (res, edge if res == O.GOOD else 0) == ref.sample(got[r], r), (w, r)
            if res == O.GOOD:  # the sampled edge leaves the tree
                u, v = divmod(edge, V)
                assert (u in members) != (v in members)
        for x in members[:3]:
            assert C.cupc_cutset_connected(cs, w, x) == (C.CUPC_OK, True)


def test_cutset_tree_sketches_equal_the_oracle_after_links_cuts_and_updates():
    from paper_2509_14433_gb300 import cupc as C
    from tests._dev import Dev

    V, seed = 300, 5
    rng = np.random.default_rng(3)
    dev = Dev(V, seed)
    ref = O.Graph(V, seed)
    E = WL.uniform_pairs(V, 1500, WL.rng(4))
    assert dev.update(E) == 0 and ref.update(E) == O.OK
    st, cs = C.cupc_cutset_create(dev.h)
    assert st == C.CUPC_OK
    forest = Forest(V)
    try:
        _check_trees(C, cs, ref, forest, V, dev.L, dev.W, rng)
        for batch in range(8):
            ops = []
            for _ in range(60):
                fe = forest.edges()
                if fe and rng.random() < 0.35:
                    u, v = fe[rng.integers(len(fe))]
                    forest.adj[u].discard(v)
                    forest.adj[v].discard(u)
                    ops += [C.CUPC_CUTSET_CUT, v, u]
                else:
                    u, v = (int(x) for x in rng.choice(V, size=2, replace=False))
                    if v in forest.tree(u):
                        continue
                    forest.adj[u].add(v)
                    forest.adj[v].add(u)
                    ops += [C.CUPC_CUTSET_LINK, u, v]
            st, applied = C.cupc_cutset_apply(cs, np.array(ops, np.uint32))
            assert (st, applied) == (C.CUPC_OK, len(ops) // 3)
            # the graph changes: refresh the vertices whose sketches did
            upd = WL.uniform_pairs(V, 40, WL.rng(100 + batch))
            assert dev.update(upd) == 0 and ref.update(upd) == O.OK
            touched = np.unique(upd.reshape(-1))
            ref_ops = np.stack([np.full(len(touched), C.CUPC_CUTSET_REFRESH), touched, touched], 1)
            st, applied = C.cupc_cutset_apply(cs, np.ascontiguousarray(ref_ops, np.uint32).reshape(-1))
            assert (st, applied) == (C.CUPC_OK, len(touched))
            _check_trees(C, cs, ref, forest, V, dev.L, dev.W, rng)
        s = np.zeros(4, np.uint64)
        C.check(C.cupc_cutset_stats(cs, s))
        assert s[2] > 0 and s[3] > 0 and s[1] >= 17
    finally:
        C.cupc_cutset_destroy(cs)
        dev.close()
        ref.close()


def test_cutset_spanning_tree_sketch_samples_zero_and_invalid_ops_stop_a_batch():
    # a spanning tree of a connected graph: the tree's sketch is the sum of
    # all vertex sketches, zero by linearity (no edge leaves it); linking two
    # vertices of one tree or cutting a non-forest edge stops the batch
    from paper_2509_14433_gb300 import cupc as C
    from tests._dev import Dev

    V, seed = 64, 9
    dev = Dev(V, seed)
    E = np.array([[i, i + 1] for i in range(V - 1)] + [[0, 40], [5, 63]], np.uint32)
    assert dev.update(E) == 0
    st, cs = C.cupc_cutset_create(dev.h)
    assert st == C.CUPC_OK
    try:
        ops = np.array([[C.CUPC_CUTSET_LINK, i, i + 1] for i in range(V - 1)], np.uint32).reshape(-1)
        assert C.cupc_cutset_apply(cs, ops) == (C.CUPC_OK, V - 1)
        got = np.zeros((dev.L, dev.W, 2), np.uint64)
        assert C.cupc_cutset_tree_sketch(cs, 17, got) == C.CUPC_OK
        assert not got.any()
        assert C.cupc_cutset_query(cs, 3, 0)[1] == O.ZERO
        # cut the path in the middle: each half's cut is {31-32, 0-40, 5-63}
        assert C.cupc_cutset_apply(cs, np.array([C.CUPC_CUTSET_CUT, 32, 31], np.uint32)) == (C.CUPC_OK, 1)
        ref = O.Graph(V, seed)
        ref.update(E)
        half = list(range(32))
        assert C.cupc_cutset_tree_sketch(cs, 0, got) == C.CUPC_OK
        for r in range(dev.L):
            assert np.array_equal(got[r], ref.sketch_sum(half, r))
        st, res, edge = C.cupc_cutset_query(cs, 0, 0)
        assert res == O.GOOD and edge in (31 * V + 32, 0 * V + 40, 5 * V + 63)
        bad = np.array([C.CUPC_CUTSET_LINK, 0, 63, C.CUPC_CUTSET_LINK, 1, 2, C.CUPC_CUTSET_LINK, 10, 50],
                       np.uint32)
        assert C.cupc_cutset_apply(cs, bad) == (C.CUPC_EINVAL, 1)  # 1-2 is already in one tree
        assert C.cupc_cutset_connected(cs, 0, 63) == (C.CUPC_OK, True)
        assert C.cupc_cutset_connected(cs, 10, 50) == (C.CUPC_OK, True)  # joined by 0-63 before the stop
        assert C.cupc_cutset_apply(cs, np.array([C.CUPC_CUTSET_CUT, 3, 9], np.uint32)) == (C.CUPC_EINVAL, 0)
        assert C.cupc_cutset_apply(cs, np.array([C.CUPC_CUTSET_LINK, 0, V], np.uint32)) == (C.CUPC_EINVAL, 0)
        ref.close()
    finally:
        C.cupc_cutset_destroy(cs)
        dev.close()
