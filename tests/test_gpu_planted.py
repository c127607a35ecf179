"""Recovery on planted sketch contents (cupc_import_sketches) against the
oracle on the same words: the branches a real stream only reaches through a
2^-64 checksum collision. A checksum-valid sample whose edge crosses no cut
is counted as a false positive and not hooked; a ZERO component that absorbs
another is sampled again. Status, labels, forest, round logs and counters
must be identical."""
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


def _sketch_of(V, seed, E):
    g = O.Graph(V, seed)
    assert g.update(np.asarray(E, np.uint32).reshape(-1, 2)) == O.OK
    sk = g.export()
    g.close()
    return sk


def _both(V, seed, sk):
    from paper_2509_14433_gb300 import cupc as C
    from tests.test_gpu_parity import assert_same_recovery
    dev, ref = _dev(V, seed), O.Graph(V, seed)
    a = np.ascontiguousarray(sk, np.uint64)
    assert C.cupc_import_sketches(dev.h, a, a.nbytes, None) == 0
    ref.import_(a)
    assert np.array_equal(dev.export(), ref.export())
    assert_same_recovery(dev, ref)
    return dev, ref


def test_false_positive_sample_is_not_hooked():
    V, seed = 8, 3
    one = _sketch_of(V, seed, [[4, 5]])
    sk = np.zeros_like(one)
    sk[0, 2] = one[0, 4]
    dev, ref = _both(V, seed, sk)
    assert dev.stats()["false_pos"] == 1


def test_zero_component_that_absorbs_another_is_sampled_again():
    V, seed = 8, 5
    sk = _sketch_of(V, seed, [[0, 1]])
    sk[:, 0] = 0
    dev, ref = _both(V, seed, sk)
    assert not dev.stats()["complete"] and dev.stats()["false_pos"] == ref.L - 1


@pytest.mark.parametrize("V,p,seed", [(300, 0.01, 11), (2000, 0.002, 12)])
def test_random_planted_words(V, p, seed):
    # a real graph's sketches, then some vertices' layer words overwritten
    # by other vertices' (checksum-valid samples that may cross no cut, in
    # any round) and some by random words (checksum failures)
    g = WL.rng(seed)
    sk = _sketch_of(V, seed, WL.er_edges(V, p, seed))
    L = sk.shape[0]
    for _ in range(V // 10):
        r, w, x = int(g.integers(0, L)), int(g.integers(0, V)), int(g.integers(0, V))
        sk[r, w] = sk[r, x]
    for _ in range(V // 20):
        r, w = int(g.integers(0, L)), int(g.integers(0, V))
        sk[r, w, int(g.integers(0, sk.shape[2]))] = g.integers(0, 2**63, size=2, dtype=np.uint64)
    _both(V, seed, sk)
