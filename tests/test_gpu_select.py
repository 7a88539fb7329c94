"""GPU parity of one round of BAD feature selection (Algorithm 1 with
Algorithm 2 on the 0.1 threshold grid) against the oracle: thresholds,
losses and the chosen candidate are integers and must be identical."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _problem(seed, n, J, smax=12):
    rng = np.random.default_rng(seed)
    P = rng.integers(0, 256, size=(3, n, 32, 32)).astype(np.uint8)
    P[1] = np.clip(P[0].astype(int) + rng.integers(-25, 26, size=(n, 32, 32)), 0, 255)
    sap = rng.integers(-40, 41, size=n).astype(np.int32)
    san = rng.integers(-40, 41, size=n).astype(np.int32)
    centres = rng.integers(-3, 35, size=(J, 4)).astype(np.int32)  # some boxes leave the patch
    sides = rng.integers(1, smax + 1, size=J).astype(np.int32)
    return P, sap, san, centres, sides


def _run(ctx, P, sap, san, tau, centres, sides):
    import torch
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    tq, loss, best = ctx.select_feature(d(P), d(sap), d(san), tau, centres, sides)
    return tq.cpu().numpy(), loss.cpu().numpy(), int(best.cpu().numpy()[0])


@pytest.mark.parametrize("n,J,tau", [(1, 1, 5), (37, 17, 20), (700, 64, 48), (1000, 3, -3)])
def test_select_exact(gpu_ctx, n, J, tau):
    P, sap, san, centres, sides = _problem(n + J, n, J)
    tq, loss, best = _run(gpu_ctx, P, sap, san, tau, centres, sides)
    cands = np.concatenate([centres, sides[:, None]], axis=1)
    rq, rl, rb = oracle.select_feature(P, cands, sap, san, tau)
    assert np.array_equal(tq, rq)
    assert np.array_equal(loss, rl)
    assert best == rb


@pytest.mark.parametrize("smax", [16, 17, 32])
def test_select_exact_large_boxes(gpu_ctx, smax):
    """Sides up to 16 take the 16-bit summed-area tables (box sums below
    2^16), larger ones the 32-bit tables; bright patches push side-16 sums to
    their largest value, 256 x 255."""
    n, J = 260, 48
    P, sap, san, centres, sides = _problem(smax, n, J, smax=smax)
    P[:, :40] = 255
    sides[:4] = smax
    tq, loss, best = _run(gpu_ctx, P, sap, san, 24, centres, sides)
    cands = np.concatenate([centres, sides[:, None]], axis=1)
    rq, rl, rb = oracle.select_feature(P, cands, sap, san, 24)
    assert np.array_equal(tq, rq)
    assert np.array_equal(loss, rl)
    assert best == rb


def test_select_ties_and_flat_patches(gpu_ctx):
    """Flat patches: every key is 0, the lowest threshold wins; duplicated
    candidates: the first copy is chosen."""
    n, J = 50, 6
    P = np.full((3, n, 32, 32), 90, dtype=np.uint8)
    sap = np.zeros(n, np.int32)
    san = np.zeros(n, np.int32)
    rng = np.random.default_rng(4)
    centres = np.tile(rng.integers(0, 32, size=(1, 4)), (J, 1)).astype(np.int32)
    sides = np.full(J, 5, np.int32)
    tq, loss, best = _run(gpu_ctx, P, sap, san, 8, centres, sides)
    assert np.all(tq == oracle.SELECT_QMIN) and np.all(loss == 8 * n) and best == 0


def test_select_full_size_sampled(gpu_ctx):
    """65536 triplets x 1000 candidates (the bench's round): a sample of the
    candidates against the oracle, and the chosen one is the minimum."""
    n, J = 65536, 1000
    P, sap, san, centres, sides = _problem(11, n, J, smax=15)
    tq, loss, best = _run(gpu_ctx, P, sap, san, 64, centres, sides)
    assert loss[best] == loss.min() and best == int(np.argmin(loss))
    rng = np.random.default_rng(12)
    for j in rng.choice(J, size=4, replace=False):
        c = np.concatenate([centres[j], sides[j:j + 1]])
        assert (tq[j], loss[j]) == oracle.find_threshold(P, c, sap, san, 64)


def test_select_rejects_bad_candidates(gpu_ctx):
    import torch
    import paper_2108_08380_gb300 as bd
    P, sap, san, centres, sides = _problem(1, 10, 3)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bad_sides = sides.copy()
    bad_sides[1] = 0
    with pytest.raises(bd.BindescError):
        gpu_ctx.select_feature(d(P), d(sap), d(san), 5, centres, bad_sides)
    bad_c = centres.copy()
    bad_c[2, 0] = 1 << 16
    with pytest.raises(bd.BindescError):
        gpu_ctx.select_feature(d(P), d(sap), d(san), 5, bad_c, sides)
