"""Parity at the workloads' full sizes, in the launch configuration bench.py
uses (tuned apply settings per batch size).

dense V=16384 and cliques V=131072: every sketch word, the labels, the
forest, the round log and counters of every recovery and every query answer
are compared, as SHA-256 digests, with the oracle's digests of the same
whole streams (tests/golden/fullsize_*.json, written by
tests/golden/make_fullsize_digests.py, which calls only the oracle).

batched R-MAT V=2^17: the first 2^21 updates of the stream (the generator's
first batches), applied as back-to-back batches, are run through the oracle
here and compared the same way; the whole 1e9-update stream is checked by
properties that hold at any size (labels = connected components of the final
edge set, forest edges present, acyclic and spanning) and by the oracle's
sketch of sampled vertices from their final neighbour sets."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2509_14433_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
BATCH = 1 << 20
SEED = 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def round_log_digest(log) -> str:
    h = hashlib.sha256()
    for live, ids in log:
        h.update(np.array([live, len(ids)], np.uint64).tobytes())
        h.update(np.ascontiguousarray(np.sort(ids), np.uint64).tobytes())
    return h.hexdigest()


def _dev(V, max_batch=BATCH):
    from paper_2509_14433_gb300 import autotune as AT
    from tests._dev import Dev
    d = Dev(V, SEED, (0, 0, 0, max_batch))
    AT.apply_buckets(d.h, V)
    return d


def _apply(d, E, op, chunk=BATCH):
    from paper_2509_14433_gb300 import cupc as C
    e_d = torch.from_numpy(np.ascontiguousarray(E, np.uint32).reshape(-1)).cuda()
    o_d = torch.full((len(E),), op, dtype=torch.int8, device="cuda")
    for i in range(0, len(E), chunk):
        C.check(C.cupc_update_batch(d.h, e_d[2 * i:], o_d[i:], min(chunk, len(E) - i), None))
    torch.cuda.synchronize()


def _recovery(d, status, answers):
    st = d.stats()
    return {"status": int(status), "rounds": st["rounds"], "fail": st["fail"], "false_pos": st["false_pos"],
            "complete": bool(st["complete"]), "round_log": round_log_digest(d.round_log()),
            "answers": sha(np.asarray(answers, np.uint8)), "connected": int(np.count_nonzero(answers))}


def _final(d):
    s, forest = d.forest()
    return {"forest_status": int(s), "forest_edges": int(len(forest)), "forest": sha(forest.astype(np.uint64)),
            "labels": sha(d.labels()), "sketches": sha(d.export())}


def _golden(name):
    return json.load(open(os.path.join(GOLD, f"fullsize_{name}.json")))


def _same(got, want, keys):
    for k in keys:
        assert got[k] == want[k], (k, got[k], want[k])


QKEYS = ("status", "rounds", "fail", "false_pos", "complete", "round_log", "answers", "connected")
FKEYS = ("forest_status", "forest_edges", "forest", "labels", "sketches")


def test_dense_v16384_full_size_equals_the_oracle():
    want = _golden("dense_v16384")
    V = 16384
    E, n_del, order = WL.dense_stream(V=V, p=0.5, batch=BATCH, delete_frac=0.1, seed=SEED)
    D = E[order[:n_del]]
    assert want["updates"] == len(E) + len(D)
    d = _dev(V)
    try:
        _apply(d, E, 1)
        _apply(d, D, -1)
        pairs = WL.uniform_pairs(V, 1000, WL.rng(77), distinct=False)
        s, ans = d.query(pairs)
        _same(_recovery(d, s, ans), want["queries"][0], QKEYS)
        _same(_final(d), want, FKEYS)
    finally:
        d.close()


def test_cliques_v131072_full_size_equals_the_oracle():
    want = _golden("cliques_v131072")
    V = 131072
    cl, order, pairs, _ = WL.clique_stream(V=V, seed=7)
    d = _dev(V)
    try:
        _apply(d, cl, 1)
        assert len(want["queries"]) == len(order)
        for (E, op), wq in zip(order, want["queries"]):
            _apply(d, E, op)
            s, ans = d.query(pairs)
            _same(_recovery(d, s, ans), wq, QKEYS)
        _same(_final(d), want, FKEYS)
    finally:
        d.close()


def _rmat_batches(n_updates):
    s = WL.RmatStream(levels=17, seed=3, device="cuda")
    E, O_, offs = [], [], [0]
    while offs[-1] < n_updates:
        e, o = s.next_batch()
        E.append(e)
        O_.append(o)
        offs.append(offs[-1] + len(o))
    return s, torch.cat(E).contiguous(), torch.cat(O_).contiguous(), np.array(offs, np.uint64)


def test_rmat_v131072_prefix_equals_the_oracle():
    # the first batches of the batched workload (at least 2^21 updates),
    # applied back to back as bench.py applies the whole stream
    from paper_2509_14433_gb300 import cupc as C
    V = 1 << 17
    _, E, O_, offs = _rmat_batches(1 << 21)
    n = int(offs[-1])
    d = _dev(V, max_batch=4 << 20)
    ref = O.Graph(V, SEED)
    try:
        C.check(C.cupc_update_batches(d.h, E.reshape(-1), O_, offs, len(offs) - 1, None))
        torch.cuda.synchronize()
        E_h = E.cpu().numpy().astype(np.uint32)
        O_h = O_.cpu().numpy()
        assert ref.update(E_h, O_h) == O.OK
        pairs = WL.uniform_pairs(V, 1000, WL.rng(77), distinct=False)
        s, ans = d.query(pairs)
        rs, rans = ref.query(pairs)
        assert (s, rs) == (0, 0)
        assert np.array_equal(ans, rans)
        sd, sr = d.stats(), ref.stats()
        assert [sd[k] for k in ("rounds", "fail", "false_pos", "complete")] == \
            [sr[k] for k in ("rounds", "fail", "false_pos", "complete")]
        assert round_log_digest(d.round_log()) == round_log_digest(ref.round_log())
        sf, forest = d.forest()
        rsf, rforest = ref.spanning_forest()
        assert np.array_equal(forest, rforest)
        assert np.array_equal(d.labels(), ref.labels())
        assert sha(d.export()) == sha(ref.export()), f"sketch words differ after {n} updates"
    finally:
        d.close()
        ref.close()


def _labels_of(V, u, v):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    m = coo_matrix((np.ones(len(u), np.int8), (u, v)), shape=(V, V))
    _, comp = connected_components(m, directed=False)
    first = np.full(comp.max() + 1, V, np.int64)
    np.minimum.at(first, comp, np.arange(V))
    return first[comp].astype(np.uint32)


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


def test_rmat_v131072_1e9_updates():
    # the batched workload at full size: 1e9 R-MAT updates with 20% deletes,
    # batch sizes log-uniform in [1k, 4M], applied as back-to-back batches
    from paper_2509_14433_gb300 import cupc as C
    V = 1 << 17
    s = WL.RmatStream(levels=17, seed=3, device="cuda")
    d = _dev(V, max_batch=4 << 20)
    g = d.h
    try:
        done = 0
        while done < 1_000_000_000:
            E, ops = s.next_batch()
            n = len(ops)
            C.check(C.cupc_update_batch(g, E.reshape(-1), ops, n, None))
            done += n
        torch.cuda.synchronize()
        assert C.cupc_sync(g, None) == 0
        st, forest = d.forest()
        assert st == 0
        lab = d.labels()
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
        f = torch.from_numpy(forest.astype(np.int64)).cuda()
        pos = torch.searchsorted(ids_sorted, f).clamp(max=ids_sorted.numel() - 1)

        def present(x):
            return (ids_sorted[pos] == f).cpu().numpy()

        _check_forest(V, forest, present, lab)
        ws = [0, 1, 2, 1000, 65535, 131071]
        p = np.zeros(4, np.uint32)
        C.cupc_get_params(g, p)
        L, _, _, W = (int(x) for x in p)
        buf = torch.empty(L * V * W * 2, dtype=torch.int64, device="cuda")
        C.check(C.cupc_export_sketches(g, buf, buf.numel() * 8, None))
        rows = buf.view(L, V, W, 2)[:, torch.tensor(ws, device="cuda")].cpu().numpy().view(np.uint64)
        del buf
        for j, w in enumerate(ws):
            nb = torch.cat([v[u == w], u[v == w]]).cpu().numpy()
            assert np.array_equal(rows[:, j], O.vertex_sketch(V, SEED, w, nb)), w
    finally:
        d.close()
