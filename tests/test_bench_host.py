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
