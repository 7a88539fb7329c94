"""GPU parity of the differentiable training step (relaxed BAD and HashSIFT,
triplet ranking loss with hard-negative mining and anchor swap, hand-written
backward) against the FP64 oracle, whose gradient is pinned to central finite
differences (test_oracle_train.py).  Gradients must agree within 1e-4 relative
(norm of the difference over the norm of the oracle's gradient)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _setup(n, seed=11, kh=256):
    import torch
    import paper_2108_08380_gb300 as bd
    rng = np.random.default_rng(seed)
    P = synth.triplet_workload(seed, n=n).patches
    bad = synth.make_bad_params(256, rng)
    theta = rng.uniform(-15, 15, size=256).astype(np.float32)
    hs = synth.make_hashsift_params(kh, rng)
    return P, bad, theta, hs, rng


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def _unpack(bits, K):
    return np.unpackbits(np.ascontiguousarray(bits).view(np.uint8), axis=1, bitorder="little")[:, :K]


@pytest.mark.parametrize("kh", [256, 512])
def test_forward_backward_match_oracle(gpu_ctx, kh):
    import torch
    import paper_2108_08380_gb300 as bd
    n = 384
    P, bad, theta, hs, rng = _setup(n, kh=kh)
    T = 0.1
    ref = oracle.train_step(P, bad, theta.astype(np.float64), hs, T=T, w_bad=1.0, w_hs=0.5,
                            want_r=True)
    bh = gpu_ctx.bad_params(bad)
    step = bd.TrainStep(gpu_ctx, bh, kh, n, temperature=T)
    dP_ = torch.from_numpy(np.ascontiguousarray(P)).cuda()
    dth = torch.from_numpy(theta).cuda()
    dW = torch.from_numpy(hs.W).cuda()
    dbias = torch.from_numpy(hs.b).cuda()
    # mining from the GPU's own hard codes: BAD codes are decided in FP64 on both
    # sides; HashSIFT codes may differ where |m| is at rounding level
    loss, mining = step.forward(dP_, dth, dW, dbias)
    mining = mining.cpu().numpy()
    assert np.array_equal(mining[:2], ref["mining"][:2])
    assert (mining[2:] == ref["mining"][2:]).mean() > 0.97
    # with the oracle's mining: losses and all gradients
    fm = torch.from_numpy(np.ascontiguousarray(ref["mining"])).cuda()
    loss, _ = step.forward(dP_, dth, dW, dbias, fixed_mining=fm)
    loss = loss.cpu().numpy()
    assert abs(loss[0] - ref["loss"][0]) <= 1e-4 * abs(ref["loss"][0])
    assert abs(loss[1] - ref["loss"][1]) <= 1e-4 * abs(ref["loss"][1])
    g = torch.tensor([1.0, 0.5], dtype=torch.float32, device="cuda")
    dP, dtheta, dWg, db = step.backward(dP_, dW, g)
    assert _rel(dtheta.cpu().numpy(), ref["dtheta"]) < 1e-4
    assert _rel(dWg.cpu().numpy(), ref["dW"]) < 1e-4
    assert _rel(db.cpu().numpy(), ref["db"]) < 1e-4
    assert _rel(dP.cpu().numpy(), ref["dpatches"]) < 1e-4
    assert gpu_ctx.sync_status() == 0


def test_autograd_function_and_mining_sizes(gpu_ctx):
    """The torch.autograd.Function: its mining equals the oracle's on this
    batch (both sides decide the BAD codes exactly; the HashSIFT margins here
    clear the FP32 error), and with the oracle's mining passed in, every
    gradient is compared with the FP64 oracle's, unconditionally."""
    import torch
    import paper_2108_08380_gb300 as bd
    n = 200
    P, bad, theta, hs, rng = _setup(n, seed=12)
    ref = oracle.train_step(P, bad, theta.astype(np.float64), hs, T=0.1)
    bh = gpu_ctx.bad_params(bad)
    step = bd.TrainStep(gpu_ctx, bh, 256, n)
    _, mining = step.forward(torch.from_numpy(np.ascontiguousarray(P)).cuda(),
                             torch.from_numpy(theta).cuda(), torch.from_numpy(hs.W).cuda(),
                             torch.from_numpy(hs.b).cuda())
    assert np.array_equal(mining.cpu().numpy(), ref["mining"])
    fm = torch.from_numpy(np.ascontiguousarray(ref["mining"])).cuda()
    for fixed in (None, fm):
        patches = torch.from_numpy(np.ascontiguousarray(P)).cuda().requires_grad_(True)
        th = torch.from_numpy(theta).cuda().requires_grad_(True)
        W = torch.from_numpy(hs.W).cuda().requires_grad_(True)
        b = torch.from_numpy(hs.b).cuda().requires_grad_(True)
        loss = bd.triplet_loss(step, patches, th, W, b, fixed_mining=fixed)
        loss.sum().backward()
        assert _rel(loss.detach().cpu().numpy(), ref["loss"]) < 1e-4
        assert _rel(th.grad.cpu().numpy(), ref["dtheta"]) < 1e-4
        assert _rel(W.grad.cpu().numpy(), ref["dW"]) < 1e-4
        assert _rel(b.grad.cpu().numpy(), ref["db"]) < 1e-4
        assert _rel(patches.grad.cpu().numpy(), ref["dpatches"]) < 1e-4
    assert gpu_ctx.sync_status() == 0


def test_single_triplet_and_identical_patches(gpu_ctx):
    import torch
    import paper_2108_08380_gb300 as bd
    P, bad, theta, hs, rng = _setup(1, seed=13)
    bh = gpu_ctx.bad_params(bad)
    step = bd.TrainStep(gpu_ctx, bh, 256, 1, tau_bad=7.5, tau_hs=3.25)
    same = np.broadcast_to(P[0, 0], P.shape).copy()
    loss, mining = step.forward(torch.from_numpy(same).cuda(), torch.from_numpy(theta).cuda(),
                                torch.from_numpy(hs.W).cuda(), torch.from_numpy(hs.b).cuda())
    loss = loss.cpu().numpy()
    assert abs(loss[0] - 7.5) < 1e-4 and abs(loss[1] - 3.25) < 1e-4
    assert mining.cpu().numpy()[0, 0] == 0


def _mining_sample_checks(m, n, sel, codes, Kb, Kh, eps=1e-4):
    """The GPU's mining of the sampled anchors against a brute force over the
    oracle's hard codes of all n negatives.  BAD codes are exact on both
    sides: the nearest negative and the swap must be equal.  HashSIFT codes
    can differ where |margin| is at rounding level: a code that differs in d
    bits moves a similarity by at most 2 d, so the GPU's pick must be the
    oracle's best up to the bits whose oracle margin is below eps."""
    neg_b, neg_h, ap_b, ap_h, neg_amb, ap_amb = codes
    for t, i in enumerate(sel):
        a, p = ap_b[2 * t], ap_b[2 * t + 1]
        score = np.maximum(a @ neg_b.T, p @ neg_b.T)
        score[i] = -10 ** 9
        assert m[0, i] == int(np.argmax(score))
        g = m[0, i]
        assert m[1, i] == (0 if a @ neg_b[g] >= p @ neg_b[g] else 1)
        a, p = ap_h[2 * t], ap_h[2 * t + 1]
        score = np.maximum(a @ neg_h.T, p @ neg_h.T)
        score[i] = -10 ** 9
        g, best = m[2, i], int(np.argmax(score))
        slack = 2 * (2 * (ap_amb[2 * t] + ap_amb[2 * t + 1]) + neg_amb[g] + neg_amb[best])
        assert score[best] - score[g] <= slack, (i, score[best], score[g], slack)


def test_full_size_65536_triplets_match_oracle(gpu_ctx):
    """The training workload at its full size and in the configuration the
    benchmark times (65536 triplets of the seeded training generator,
    BAD-256 + HashSIFT-256 relaxed at T = 0.1): the GPU's mining is checked
    on a seeded sample of anchors against a brute force over the oracle's
    codes of all 65536 negatives, then passed as fixed mining to both the GPU
    step and the FP64 oracle, whose loss and gradients (dtheta, dW, db over
    all 196608 patches, dpatches whole and on a sample of patches) must agree
    within 1e-4 norm-relative."""
    import torch
    import paper_2108_08380_gb300 as bd
    n = 65536
    rng = np.random.default_rng(1003)
    P = synth.triplet_workload(1003, n=n).patches
    bad = synth.make_bad_params(256, rng)
    theta = rng.uniform(-20, 20, size=256).astype(np.float32)
    hs = synth.make_hashsift_params(256, rng)
    dP_ = torch.from_numpy(P).cuda()
    th, W, b = (torch.from_numpy(x).cuda() for x in (theta, hs.W, hs.b))
    step = bd.TrainStep(gpu_ctx, gpu_ctx.bad_params(bad), 256, n, temperature=0.1)
    _, mining = step.forward(dP_, th, W, b)
    m = mining.cpu().numpy()
    assert m[0].min() >= 0 and m[0].max() < n and m[2].min() >= 0 and m[2].max() < n
    assert (m[0] != np.arange(n)).all() and (m[2] != np.arange(n)).all()
    assert set(np.unique(m[1])) <= {0, 1} and set(np.unique(m[3])) <= {0, 1}

    # mining of a seeded sample of anchors against the oracle's codes
    sel = np.random.default_rng(7).choice(n, size=8, replace=False)
    rows = [P[2]] + [np.stack([P[0, i], P[1, i]]) for i in sel]
    stack = np.concatenate(rows)
    pad = (-stack.shape[0]) % 3
    stack = np.concatenate([stack, np.zeros((pad, 32, 32), np.float32)])
    bb, bhs, _, mh = oracle.train_codes(stack.reshape(3, -1, 32, 32), bad,
                                        theta.astype(np.float64), hs)
    pm = lambda w, K: _unpack(w, K).astype(np.int64) * 2 - 1
    amb = (np.abs(mh) < 1e-4).sum(axis=1)
    codes = (pm(bb[:n], 256), pm(bhs[:n], 256), pm(bb[n:n + 16], 256), pm(bhs[n:n + 16], 256),
             amb[:n], amb[n:n + 16])
    _mining_sample_checks(m, n, sel, codes, 256, 256)
    assert amb[:n].sum() < 1e-3 * n * 256

    # the same mining on both sides: losses and gradients
    wts = (1.0, 0.5)
    loss, _ = step.forward(dP_, th, W, b, fixed_mining=mining)
    dP, dth, dWg, db = step.backward(dP_, W, torch.tensor(wts, dtype=torch.float32, device="cuda"))
    assert gpu_ctx.sync_status() == 0
    ref = oracle.train_step(P, bad, theta.astype(np.float64), hs, T=0.1, w_bad=wts[0], w_hs=wts[1],
                            fixed_mining=m)
    loss = loss.cpu().numpy()
    assert abs(loss[0] - ref["loss"][0]) <= 1e-4 * abs(ref["loss"][0])
    assert abs(loss[1] - ref["loss"][1]) <= 1e-4 * abs(ref["loss"][1])
    assert _rel(dth.cpu().numpy(), ref["dtheta"]) < 1e-4
    assert _rel(dWg.cpu().numpy(), ref["dW"]) < 1e-4
    assert _rel(db.cpu().numpy(), ref["db"]) < 1e-4
    dP = dP.cpu().numpy()
    assert np.isfinite(dP).all()
    assert _rel(dP, ref["dpatches"]) < 1e-4
    # a seeded sample of 384 patches, each against the tensor's scale
    flat, rflat = dP.reshape(3 * n, 1024), ref["dpatches"].reshape(3 * n, 1024)
    rows = np.random.default_rng(8).choice(3 * n, size=384, replace=False)
    scale = np.abs(rflat).max()
    assert np.abs(flat[rows] - rflat[rows]).max() <= 1e-4 * scale
    assert _rel(flat[rows], rflat[rows]) < 1e-4
