"""Pins for the oracle's Hamming matching: brute force on bit vectors, the
paper's similarity identity S = h(x)^T h(y) = K - 2*Hamming for +-1 codes
(Sec. III-A), hand-built ties, empty and single-entry train sets, and the
strictness of the ratio test."""
import numpy as np
import pytest

import oracle


def _unpack(d, K):
    return np.unpackbits(np.ascontiguousarray(d).view(np.uint8), axis=1, bitorder="little")[:, :K]


@pytest.mark.parametrize("K", [256, 512])
def test_bruteforce_top2(K):
    rng = np.random.default_rng(K)
    q = rng.integers(0, 2 ** 32, size=(40, K // 32), dtype=np.uint64).astype(np.uint32)
    t = rng.integers(0, 2 ** 32, size=(70, K // 32), dtype=np.uint64).astype(np.uint32)
    t[5] = t[9]  # duplicate entries make ties
    q[3] = t[9]
    idx, d1, d2, acc = oracle.match(q, t, K)
    bq, bt = _unpack(q, K).astype(np.int64), _unpack(t, K).astype(np.int64)
    D = (bq[:, None, :] != bt[None, :, :]).sum(axis=2)
    for i in range(q.shape[0]):
        order = np.lexsort((np.arange(t.shape[0]), D[i]))
        assert idx[i] == order[0]
        assert d1[i] == D[i, order[0]]
        assert d2[i] == D[i, order[1]]
        assert acc[i] == (5 * d1[i] < 4 * d2[i])
    assert idx[3] == 5 and d1[3] == 0 and d2[3] == 0 and acc[3] == 0


def test_similarity_identity():
    """S(x,y) = h(x)^T h(y) with h in {-1,+1}^K equals K - 2 * Hamming."""
    K = 256
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2 ** 32, size=(30, K // 32), dtype=np.uint64).astype(np.uint32)
    pa = _unpack(a, K).astype(np.int64) * 2 - 1
    for i in range(30):
        for j in range(30):
            assert K - 2 * oracle.hamming(a[i], a[j]) == int(pa[i] @ pa[j])


def test_empty_and_single_train_sets():
    K = 256
    q = np.arange(16, dtype=np.uint32).reshape(2, 8)
    idx, d1, d2, acc = oracle.match(q, np.zeros((0, 8), np.uint32), K)
    assert list(idx) == [-1, -1] and list(d1) == [K + 1] * 2 and list(d2) == [K + 1] * 2
    assert list(acc) == [0, 0]
    t = np.zeros((1, 8), np.uint32)
    idx, d1, d2, acc = oracle.match(q, t, K)
    assert list(idx) == [0, 0] and list(d2) == [K + 1] * 2
    assert d1[0] == sum(bin(v).count("1") for v in range(8))


def test_ratio_test_is_strict():
    K = 256
    q = np.zeros((1, 8), np.uint32)
    t = np.zeros((2, 8), np.uint32)
    t[0, 0] = 0b1111          # d1 = 4
    t[1, 0] = 0b11111         # d2 = 5 -> 4/5 = 0.8 exactly: rejected
    assert oracle.match(q, t, K)[3][0] == 0
    t[0, 0] = 0b111           # d1 = 3 -> 0.6: accepted
    assert oracle.match(q, t, K)[3][0] == 1
    assert oracle.match(q, t, K, 1, 1)[3][0] == 1


# ---------------------------------------------------------------------------
# mutual nearest neighbours (Sec. V, Hamming MNN matching)

def _rand(rng, n, K):
    return rng.integers(0, 2 ** 32, size=(n, K // 32), dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("K", [256, 512])
def test_mnn_bruteforce(K):
    """Against numpy argmin (first minimum = lowest index) over the unpacked
    distance matrix, in both directions."""
    rng = np.random.default_rng(K + 7)
    t = _rand(rng, 60, K)
    q = _rand(rng, 45, K)
    q[:20] = t[rng.integers(0, 60, size=20)]
    bits = np.unpackbits(q[:20].view(np.uint8), axis=1, bitorder="little")
    bits[:, :K // 16] ^= 1  # near copies, not exact ones
    q[:20] = np.packbits(bits, axis=1, bitorder="little").view(np.uint32)
    t[7] = t[3]  # a duplicated train entry
    D = (_unpack(q, K)[:, None, :] != _unpack(t, K)[None, :, :]).sum(axis=2)
    fwd = D.argmin(axis=1)
    back = D.argmin(axis=0)
    want = np.where(back[fwd] == np.arange(q.shape[0]), fwd, -1)
    got = oracle.match_mnn(q, t, K)
    assert np.array_equal(got, want)
    assert (got >= 0).sum() >= 15


def test_mnn_is_a_symmetric_partial_matching():
    K = 256
    rng = np.random.default_rng(11)
    t = _rand(rng, 80, K)
    q = np.concatenate([t[rng.permutation(80)[:50]], _rand(rng, 30, K)])
    a = oracle.match_mnn(q, t, K)
    b = oracle.match_mnn(t, q, K)
    pairs_a = {(i, int(j)) for i, j in enumerate(a) if j >= 0}
    pairs_b = {(int(i), j) for j, i in enumerate(b) if i >= 0}
    assert pairs_a == pairs_b
    partners = [j for j in a if j >= 0]
    assert len(partners) == len(set(partners))  # no train entry used twice
    idx, _, _, _ = oracle.match(q, t, K)
    assert np.all((a == -1) | (a == idx))  # a mutual partner is the nearest entry


def test_mnn_identical_sets_and_duplicates():
    K = 256
    rng = np.random.default_rng(5)
    base = _rand(rng, 40, K)
    assert np.array_equal(oracle.match_mnn(base, base, K), np.arange(40))
    # every train entry twice: only the first copy (lowest index) can be mutual
    t = np.concatenate([base, base])
    assert np.array_equal(oracle.match_mnn(base, t, K), np.arange(40))
    # two equal queries: the lower query index wins the train entry's tie
    q = np.concatenate([base[:1], base[:1]])
    assert list(oracle.match_mnn(q, base, K)) == [0, -1]


def test_mnn_empty_sets():
    K = 512
    rng = np.random.default_rng(2)
    q = _rand(rng, 5, K)
    assert np.array_equal(oracle.match_mnn(q, np.zeros((0, K // 32), np.uint32), K), [-1] * 5)
    assert oracle.match_mnn(np.zeros((0, K // 32), np.uint32), q, K).shape == (0,)
