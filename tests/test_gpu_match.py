"""GPU parity of brute-force Hamming matching with fused top-2 and ratio test
against the CPU oracle: bit-exact index, distances and verdict (Sec. IV-C).
Every case runs through both the POPC kernel (bd_match) and the tensor-core
kernel (bd_match_tc, +-1 codes in FP8, S = K - 2 Hamming)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _rand_desc(rng, n, K):
    return rng.integers(0, 2 ** 32, size=(n, K // 32), dtype=np.uint64).astype(np.uint32)


def _noisy(rng, d, K, flips):
    """Copies of descriptors with `flips` random bits flipped each."""
    out = d.copy()
    bits = np.unpackbits(out.view(np.uint8), axis=1, bitorder="little")
    for i in range(bits.shape[0]):
        bits[i, rng.choice(K, size=flips, replace=False)] ^= 1
    return np.packbits(bits, axis=1, bitorder="little").view(np.uint32)


@pytest.fixture(params=[False, True], ids=["popc", "tensor"])
def tc(request):
    return request.param


def _check(ctx, q, t, K, rnum=4, rden=5, rows=None, tc=False):
    import paper_2108_08380_gb300 as bd
    m = ctx.match(_dev(q), _dev(t), K, rnum, rden, tensor_cores=tc)
    idx, d1, d2, acc = bd.unpack_matches(m)
    if rows is None:
        rows = np.arange(q.shape[0])
    ri, r1, r2, ra = oracle.match(q[rows], t, K, rnum, rden)
    assert np.array_equal(idx[rows], ri)
    assert np.array_equal(d1[rows], r1)
    assert np.array_equal(d2[rows], r2)
    assert np.array_equal(acc[rows], ra)
    return idx, d1, d2, acc


@pytest.mark.parametrize("K,nq,nt", [(256, 1000, 1000), (512, 1000, 1000), (256, 333, 777),
                                     (512, 129, 4099), (256, 5000, 3), (256, 1, 1), (512, 7, 0),
                                     (256, 300, 1), (512, 2, 2)])
def test_match_random_exact(gpu_ctx, K, nq, nt, tc):
    rng = np.random.default_rng(K + 31 * nq + nt)
    t = _rand_desc(rng, nt, K)
    q = _rand_desc(rng, nq, K)
    if nt:
        pick = rng.integers(0, nt, size=nq)
        q[: nq // 2] = _noisy(rng, t[pick[: nq // 2]], K, K // 8)
    _check(gpu_ctx, q, t, K, tc=tc)


def test_match_ties_lowest_index(gpu_ctx, tc):
    K = 256
    rng = np.random.default_rng(3)
    base = _rand_desc(rng, 50, K)
    t = np.concatenate([base, base, base[::-1]])  # every entry three times
    q = _noisy(rng, base, K, 3)
    idx, d1, d2, acc = _check(gpu_ctx, q, t, K, tc=tc)
    assert np.all(d1 == d2) and not acc.any()
    assert np.all(idx < 50)


def test_match_bad_descriptors_of_noisy_pair(gpu_ctx, tc):
    """Plain workload: BAD-256 of image A against image B = A + N(0,5)."""
    wl = synth.plain_workload(1000)
    qa, _ = oracle.bad_describe(wl.img_a, wl.kps_a, wl.bad)
    tb, _ = oracle.bad_describe(wl.img_b, wl.kps_b, wl.bad)
    idx, d1, d2, acc = _check(gpu_ctx, qa, tb, 256, tc=tc)
    assert (idx == np.arange(1000)).mean() > 0.5  # most keypoints find themselves


@pytest.mark.parametrize("K", [256, 512])
def test_match_full_size_sampled(gpu_ctx, K, tc):
    """20000 x 20000 in the launch configuration of the large workload; a
    seeded sample of 400 queries checked against the oracle."""
    rng = np.random.default_rng(K)
    n = 20000
    t = _rand_desc(rng, n, K)
    perm = rng.permutation(n)
    q = _noisy(rng, t[perm], K, K // 10)
    rows = np.sort(rng.choice(n, size=400, replace=False))
    idx, d1, d2, acc = _check(gpu_ctx, q, t, K, rows=rows, tc=tc)
    assert np.array_equal(idx[rows], perm[rows])


def test_match_rejects_bad_arguments(gpu_ctx):
    import paper_2108_08380_gb300 as bd
    rng = np.random.default_rng(0)
    q = _dev(_rand_desc(rng, 4, 256))
    with pytest.raises(bd.BindescError):
        gpu_ctx.match(q, q, 300)
    with pytest.raises(bd.BindescError):
        gpu_ctx.match(q, q, 256, 6, 5)


@pytest.mark.parametrize("K", [256, 512])
def test_tensor_core_and_popc_agree_on_full_size(gpu_ctx, K):
    """All 20000 queries: the two kernels return identical records."""
    import torch
    rng = np.random.default_rng(K + 1)
    n = 20000
    t = _rand_desc(rng, n, K)
    q = _noisy(rng, t[rng.permutation(n)], K, K // 6)
    a = gpu_ctx.match(_dev(q), _dev(t), K).cpu().numpy()
    b = gpu_ctx.match(_dev(q), _dev(t), K, tensor_cores=True).cpu().numpy()
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# mutual nearest neighbours (bd_match_mnn, Sec. V)

@pytest.mark.parametrize("K,nq,nt", [(256, 1000, 1000), (512, 333, 777), (256, 129, 4099),
                                     (512, 5000, 3), (256, 1, 1), (256, 7, 0), (512, 300, 1)])
def test_mnn_exact(gpu_ctx, K, nq, nt, tc):
    import paper_2108_08380_gb300 as bd
    rng = np.random.default_rng(K + 17 * nq + nt)
    t = _rand_desc(rng, nt, K)
    q = _rand_desc(rng, nq, K)
    if nt:
        q[: nq // 2] = _noisy(rng, t[rng.integers(0, nt, size=nq // 2)], K, K // 8)
    out, mnn = gpu_ctx.match_mnn(_dev(q), _dev(t), K, tensor_cores=tc)
    idx, d1, d2, acc = bd.unpack_matches(out)
    ri, r1, r2, ra = oracle.match(q, t, K)
    assert np.array_equal(idx, ri) and np.array_equal(d1, r1) and np.array_equal(d2, r2)
    assert np.array_equal(acc, ra)
    assert np.array_equal(mnn.cpu().numpy(), oracle.match_mnn(q, t, K))


def test_mnn_duplicates_and_equal_queries(gpu_ctx, tc):
    K = 256
    rng = np.random.default_rng(9)
    base = _rand_desc(rng, 64, K)
    t = np.concatenate([base, base])                  # each entry twice
    q = np.concatenate([base[:10], base[:10], base])  # equal queries compete for one entry
    _, mnn = gpu_ctx.match_mnn(_dev(q), _dev(t), K, tensor_cores=tc)
    want = oracle.match_mnn(q, t, K)
    assert np.array_equal(mnn.cpu().numpy(), want)
    assert np.array_equal(want[:10], np.arange(10)) and np.all(want[10:20] == -1)


@pytest.mark.parametrize("K", [256, 512])
def test_mnn_full_size_sampled(gpu_ctx, K, tc):
    """20000 x 20000: for a seeded sample of queries the oracle gives the
    nearest train entry j, then the nearest query of t[j] over all queries."""
    rng = np.random.default_rng(K + 3)
    n = 20000
    t = _rand_desc(rng, n, K)
    q = _noisy(rng, t[rng.permutation(n)], K, K // 5)
    q[rng.choice(n, size=n // 4, replace=False)] = _rand_desc(rng, n // 4, K)  # unmatched queries
    _, mnn = gpu_ctx.match_mnn(_dev(q), _dev(t), K, tensor_cores=tc)
    mnn = mnn.cpu().numpy()
    rows = np.sort(rng.choice(n, size=150, replace=False))
    fwd, _, _, _ = oracle.match(q[rows], t, K)
    back, _, _, _ = oracle.match(t[fwd], q, K)
    want = np.where(back == rows, fwd, -1)
    assert np.array_equal(mnn[rows], want)
    partners = mnn[mnn >= 0]
    assert len(partners) == len(np.unique(partners))  # a partial one-to-one matching


# ---------------------------------------------------------------------------
# several matchings in one launch (bd_match_batch)

def test_match_batch_mixed_jobs(gpu_ctx):
    """Jobs of both widths, ragged sizes, an empty train set and an empty
    query set: every job equals the oracle and the single-job call."""
    import paper_2108_08380_gb300 as bd
    rng = np.random.default_rng(77)
    shapes = [(256, 1000, 1000), (512, 333, 777), (256, 129, 0), (512, 0, 50), (256, 5000, 3),
              (512, 1, 1), (256, 300, 4099)]
    jobs, host = [], []
    for K, nq, nt in shapes:
        t = _rand_desc(rng, nt, K)
        q = _rand_desc(rng, nq, K)
        if nt and nq:
            q[: nq // 2] = _noisy(rng, t[rng.integers(0, nt, size=nq // 2)], K, K // 8)
        jobs.append((_dev(q), _dev(t), K))
        host.append((q, t, K))
    outs = gpu_ctx.match_batch(jobs)
    for (q, t, K), out, (dq, dt, _) in zip(host, outs, jobs):
        if q.shape[0] == 0:
            continue
        idx, d1, d2, acc = bd.unpack_matches(out)
        ri, r1, r2, ra = oracle.match(q, t, K)
        assert np.array_equal(idx, ri) and np.array_equal(d1, r1)
        assert np.array_equal(d2, r2) and np.array_equal(acc, ra)
        single = gpu_ctx.match(dq, dt, K)
        assert np.array_equal(single.cpu().numpy(), out.cpu().numpy())


def test_match_batch_refuses_bad_jobs(gpu_ctx):
    import paper_2108_08380_gb300 as bd
    rng = np.random.default_rng(1)
    q = _dev(_rand_desc(rng, 4, 256))
    with pytest.raises(bd.BindescError):
        gpu_ctx.match_batch([(q, q, 256)] * 9)          # more than BD_MATCH_MAX_JOBS
    with pytest.raises(bd.BindescError):
        gpu_ctx.match_batch([(q, q, 256), (q, q, 300)])  # second job invalid
    assert gpu_ctx.match_batch([]) == []
