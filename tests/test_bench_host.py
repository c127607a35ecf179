"""Host-side figures of bench.py's roofline line (CPU): the algorithmic
bytes of an update batch (expected distinct buckets touched) against a
dense sweep of the touched vertices' whole sketches."""
import numpy as np

import bench


def test_expected_touched_buckets_closed_forms():
    L, C, D = 3, 7, 10
    # one record per vertex: every layer touches the deterministic bucket
    # and exactly one row per column
    counts = np.array([1, 0, 1, 1])
    assert abs(bench.expected_touched_buckets(counts, L, C, D) - 3 * L * (1 + C)) < 1e-9
    # no records: nothing touched
    assert bench.expected_touched_buckets(np.zeros(5, np.int64), L, C, D) == 0.0
    # very many records: every row of every column
    big = np.array([10 ** 7])
    assert abs(bench.expected_touched_buckets(big, L, C, D) - L * (1 + C * D)) < 1e-6


def test_expected_touched_buckets_matches_simulation():
    # draw depths with P(d) = 2^-(d+1), the last row taking the tail, and
    # count distinct rows per column
    g = np.random.default_rng(3)
    L, C, D, n = 1, 200, 12, 9
    d = np.minimum(g.geometric(0.5, size=(C, n)) - 1, D - 1)
    distinct = np.mean([len(np.unique(row)) for row in d])
    exp = bench.expected_touched_buckets(np.array([n]), L, C, D)
    assert abs((1 + C * distinct) - exp) / exp < 0.03


def test_dense_sweep_bytes():
    L, W = 16, 197
    counts = np.zeros(100, np.int64)
    counts[[3, 50, 99]] = [1, 5, 1000]
    assert bench.dense_sweep_bytes(counts, L, W) == 3 * 2 * L * W * 16
    # the dense V=16384 batch touches every vertex: 3.7x its distinct buckets
    V = 16384
    c = np.full(V, 128)
    ratio = bench.dense_sweep_bytes(c, 16, 197) / (32 * bench.expected_touched_buckets(c, 16, 7, 28))
    assert 3.5 < ratio < 4.0


def test_shuffled_parts_is_a_permutation_in_strided_parts(monkeypatch):
    # streams longer than the device sort's limit are permuted in strided
    # parts; every element appears exactly once, and each part spans the
    # whole id range (small limits stand in for 2^31 - 1 and 2^30)
    torch = __import__("pytest").importorskip("torch")
    monkeypatch.setattr(bench, "PERM_ONE", 100)
    monkeypatch.setattr(bench, "PERM_CHUNK", 64)
    x = torch.arange(1000, dtype=torch.int64) * 7
    gen = torch.Generator().manual_seed(5)
    parts = list(bench.shuffled_parts(x, gen))
    assert len(parts) == 16  # ceil(1000 / 64)
    y = torch.cat(parts)
    assert sorted(y.tolist()) == sorted(x.tolist())
    for p in parts:
        assert p.min().item() < 7 * 100 and p.max().item() > 7 * 900
    # at or below the limit: one uniform permutation
    gen = torch.Generator().manual_seed(5)
    one = list(bench.shuffled_parts(x[:100], gen))
    assert len(one) == 1 and sorted(one[0].tolist()) == sorted(x[:100].tolist())
