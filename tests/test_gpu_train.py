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
    import torch
    import paper_2108_08380_gb300 as bd
    n = 200
    P, bad, theta, hs, rng = _setup(n, seed=12)
    ref = oracle.train_step(P, bad, theta.astype(np.float64), hs, T=0.1)
    bh = gpu_ctx.bad_params(bad)
    step = bd.TrainStep(gpu_ctx, bh, 256, n)
    patches = torch.from_numpy(np.ascontiguousarray(P)).cuda().requires_grad_(True)
    th = torch.from_numpy(theta).cuda().requires_grad_(True)
    W = torch.from_numpy(hs.W).cuda().requires_grad_(True)
    b = torch.from_numpy(hs.b).cuda().requires_grad_(True)
    loss = bd.triplet_loss(step, patches, th, W, b)
    loss.sum().backward()
    _, mining = step.forward(patches.detach(), th.detach(), W.detach(), b.detach())
    if np.array_equal(mining.cpu().numpy(), ref["mining"]):
        assert _rel(th.grad.cpu().numpy(), ref["dtheta"]) < 1e-4
        assert _rel(W.grad.cpu().numpy(), ref["dW"]) < 1e-4
        assert _rel(patches.grad.cpu().numpy(), ref["dpatches"]) < 1e-4
    assert torch.isfinite(patches.grad).all()


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


def test_full_batch_65536_runs(gpu_ctx):
    """The training workload's size, 65536 triplets: finite loss and gradients,
    valid mining, and the BAD mining of a seeded sample of anchors equal to a
    brute force over the oracle's hard codes of all 65536 negatives."""
    import torch
    import paper_2108_08380_gb300 as bd
    n = 65536
    rng = np.random.default_rng(5)
    P = torch.rand((3, n, 32, 32), device="cuda", generator=torch.Generator("cuda").manual_seed(1)) * 255
    bad = synth.make_bad_params(256, rng)
    theta = torch.from_numpy(rng.uniform(-15, 15, size=256).astype(np.float32)).cuda()
    hs = synth.make_hashsift_params(256, rng)
    W, b = torch.from_numpy(hs.W).cuda(), torch.from_numpy(hs.b).cuda()
    step = bd.TrainStep(gpu_ctx, gpu_ctx.bad_params(bad), 256, n)
    loss, mining = step.forward(P, theta, W, b)
    dP, dth, dW, db = step.backward(P, W, torch.ones(2, device="cuda"))
    assert torch.isfinite(loss).all() and torch.isfinite(dP).all() and torch.isfinite(dW).all()
    m = mining.cpu().numpy()
    assert m[0].min() >= 0 and m[0].max() < n and set(np.unique(m[1])) <= {0, 1}
    assert (m[0] != np.arange(n)).all()
    # a seeded sample of anchors: the oracle mines them over all negatives
    Pn = P.cpu().numpy()
    sel = rng.choice(n, size=8, replace=False)
    negs, _, _, _ = oracle.train_codes(np.stack([Pn[2]] * 3), bad, theta.cpu().numpy().astype(np.float64), hs)
    neg_bits = _unpack(negs[:n], 256).astype(np.int64) * 2 - 1
    for i in sel:
        ai, _, _, _ = oracle.train_codes(np.stack([Pn[0, i:i + 1], Pn[1, i:i + 1], Pn[2, i:i + 1]]), bad,
                                         theta.cpu().numpy().astype(np.float64), hs)
        ua = _unpack(ai[:2], 256).astype(np.int64) * 2 - 1
        score = np.maximum(ua[0] @ neg_bits.T, ua[1] @ neg_bits.T)
        score[i] = -10 ** 9
        assert m[0, i] == int(np.argmax(score))
