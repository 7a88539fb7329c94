"""Pins for the oracle's feature-selection round (Algorithm 1 with Algorithm 2's
threshold search on the 0.1 grid): the threshold and loss against a brute
force that evaluates the per-step triplet loss at every threshold directly,
a hand-computed case, the equality of the loss at both ends of the grid, and
the tie rules (lowest threshold, first candidate)."""
import numpy as np
import pytest

import oracle

QMIN, QMAX = -2551, 2550


def _box(p, cx, cy, s):
    """Sum of the s x s box with top-left (cx - s//2, cy - s//2), zero outside."""
    pad = np.zeros((32 + 64, 32 + 64), dtype=np.int64)
    pad[32:64, 32:64] = p
    x0, y0 = cx - s // 2 + 32, cy - s // 2 + 32
    return int(pad[y0:y0 + s, x0:x0 + s].sum())


def _key(p, c):
    d = _box(p, c[0], c[1], c[4]) - _box(p, c[2], c[3], c[4])
    return -((-10 * d) // (c[4] * c[4]))  # ceil(10 d / s^2) in integers


def _brute(P, c, sap, san, tau):
    """L(q) for every q of the grid from the definition; first minimum."""
    n = P.shape[1]
    keys = np.array([[_key(P[m, i], c) for i in range(n)] for m in range(3)])
    q = np.arange(QMIN, QMAX + 1)[:, None]
    h = np.where(keys[:, None, :] <= q[None], 1, -1)  # [3, Q, n]
    term = tau - sap[None] - h[0] * h[1] + san[None] + h[0] * h[2]
    L = np.maximum(term, 0).sum(axis=1)
    j = int(np.argmin(L))
    return int(q[j, 0]), int(L[j]), L


def _problem(seed, n):
    rng = np.random.default_rng(seed)
    P = rng.integers(0, 256, size=(3, n, 32, 32)).astype(np.uint8)
    P[1] = np.clip(P[0].astype(int) + rng.integers(-20, 21, size=(n, 32, 32)), 0, 255)
    sap = rng.integers(-10, 11, size=n).astype(np.int32)
    san = rng.integers(-10, 11, size=n).astype(np.int32)
    return P, sap, san


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_find_threshold_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    P, sap, san = _problem(seed, 9)
    for _ in range(6):
        s = int(rng.integers(1, 12))
        c = [int(v) for v in rng.integers(0, 32, size=4)] + [s]
        bq, bl, L = _brute(P, c, sap, san, 12)
        q, loss = oracle.find_threshold(P, c, sap, san, 12)
        assert (q, loss) == (bq, bl)
        assert L[0] == L[-1]  # all -1 and all +1 give the same products
        for m in range(3):
            for i in range(P.shape[1]):
                assert oracle.select_key(P[m, i], c) == _key(P[m, i], c)


def test_hand_computed_negative_darker_box():
    """Anchor and positive flat (f = 0), negative with box 1 darker by 5 per
    pixel (f = -5, key -50): thresholds in [-50, -1] give h(n) = +1 while
    h(a) = h(p) = -1, lowering the term by 2."""
    n = 1
    P = np.full((3, n, 32, 32), 100, dtype=np.uint8)
    c = [8, 8, 24, 24, 5]
    P[2, 0, 6:11, 6:11] = 95  # box 1 of the negative (centre (8, 8), side 5)
    sap = np.array([3], np.int32)
    san = np.array([1], np.int32)
    tau = 10
    base = max(tau - 3 - 1 + 1 + 1, 0)
    q, loss = oracle.find_threshold(P, c, sap, san, tau)
    assert oracle.select_key(P[2, 0], c) == -50
    assert (q, loss) == (-50, base - 2)


def test_flat_patches_keep_the_lowest_threshold():
    P = np.full((3, 4, 32, 32), 77, dtype=np.uint8)
    sap = np.zeros(4, np.int32)
    san = np.zeros(4, np.int32)
    q, loss = oracle.find_threshold(P, [5, 5, 20, 20, 3], sap, san, 4)
    assert (q, loss) == (QMIN, 4 * 4)  # every key is 0: no threshold changes a product


def test_select_feature_first_minimum():
    P, sap, san = _problem(7, 12)
    rng = np.random.default_rng(8)
    C = np.concatenate([rng.integers(0, 32, size=(6, 4)), rng.integers(1, 9, size=(6, 1))], axis=1)
    C = np.concatenate([C, C[::-1]]).astype(np.int32)  # each candidate twice
    tq, loss, best = oracle.select_feature(P, C, sap, san, 12)
    for j in range(C.shape[0]):
        assert (tq[j], loss[j]) == oracle.find_threshold(P, C[j], sap, san, 12)
    assert loss[best] == loss.min() and best == int(np.argmin(loss))
    assert best < 6  # the first copy wins
