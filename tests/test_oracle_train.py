"""Pins for the oracle's training step (Sec. III-A Eq. 1, Sec. III-B Eq. 3 with
relaxed tanh responses, hard-negative mining and anchor swap): the analytic
gradient against central finite differences in FP64 (away from kinks), the
mining against brute force over unpacked hard codes, the BAD features against
direct slice sums, and closed forms of the loss."""
import math

import numpy as np
import pytest

import oracle
import synth


def _problem(n=5, Kb=64, Kh=64, seed=3, jitter=True):
    """Small triplet problem.  The jitter removes exactly flat regions, where
    the gradient magnitude |grad P| and the L2 normalisation of a zero
    histogram are not differentiable (one-sided slopes differ there)."""
    rng = np.random.default_rng(seed)
    P = synth.triplet_workload(seed, n=n).patches.astype(np.float64)
    if jitter:
        P += rng.uniform(-0.5, 0.5, size=P.shape)
    bad = synth.make_bad_params(Kb, rng)
    theta = rng.uniform(-15, 15, size=Kb)
    hs = synth.make_hashsift_params(Kh, rng)
    hs.W = hs.W.astype(np.float64)
    hs.b = hs.b.astype(np.float64)
    return P, bad, theta, hs


def _loss(P, bad, theta, hs, mining, T, wb, wh):
    out = oracle.train_step(P, bad, theta, hs, T=T, fixed_mining=mining, want_grads=False)
    return wb * out["loss"][0] + wh * out["loss"][1]


def _fd_check(get, set_, analytic, idx, f, scale):
    """Central differences at two steps; coordinates whose two estimates
    disagree sit on a kink and are skipped."""
    checked = 0
    for i in idx:
        x0 = get(i)
        h = 2e-6 * max(1.0, abs(x0))
        est = []
        for hh in (h, h / 2):
            set_(i, x0 + hh)
            lp = f()
            set_(i, x0 - hh)
            lm = f()
            set_(i, x0)
            est.append((lp - lm) / (2 * hh))
        if abs(est[0] - est[1]) > 2e-6 * (scale + abs(est[1])):
            continue
        assert abs(analytic[i] - est[1]) <= 1e-5 * (scale + abs(est[1])), (i, analytic[i], est[1])
        checked += 1
    return checked


@pytest.mark.parametrize("T", [0.1, 1.0])
def test_gradients_match_finite_differences(T):
    P, bad, theta, hs = _problem()
    wb, wh = 1.0, 0.7
    base = oracle.train_step(P, bad, theta, hs, T=T, w_bad=wb, w_hs=wh)
    mining = base["mining"]
    f = lambda: _loss(P, bad, theta, hs, mining, T, wb, wh)
    rng = np.random.default_rng(1)

    g = base["dtheta"]
    n_ok = _fd_check(lambda i: theta[i], lambda i, v: theta.__setitem__(i, v), g,
                     range(len(theta)), f, np.abs(g).max())
    assert n_ok > 40

    g = base["db"]
    n_ok = _fd_check(lambda i: hs.b[i], lambda i, v: hs.b.__setitem__(i, v), g, range(len(hs.b)), f,
                     np.abs(g).max())
    assert n_ok > 40

    g = base["dW"].ravel()
    Wf = hs.W.reshape(-1)
    idx = rng.choice(Wf.size, size=60, replace=False)
    n_ok = _fd_check(lambda i: Wf[i], lambda i, v: Wf.__setitem__(i, v), g, idx, f, np.abs(g).max())
    assert n_ok > 40

    g = base["dpatches"].ravel()
    Pf = P.reshape(-1)
    idx = np.concatenate([rng.choice(Pf.size, size=60, replace=False), np.argsort(-np.abs(g))[:20]])
    n_ok = _fd_check(lambda i: Pf[i], lambda i, v: Pf.__setitem__(i, v), g, idx, f, np.abs(g).max())
    assert n_ok > 45


def _unpack(b, K):
    return np.unpackbits(b.view(np.uint8), axis=1, bitorder="little")[:, :K].astype(np.int64)


def test_mining_and_anchor_swap_bruteforce():
    n = 23
    P, bad, theta, hs = _problem(n=n, Kb=256, Kh=256, seed=9)
    out = oracle.train_step(P, bad, theta, hs, want_grads=False)
    bb, bh, _, _ = oracle.train_codes(P, bad, theta, hs)
    for bits, K, row in ((bb, 256, 0), (bh, 256, 2)):
        u = _unpack(bits, K) * 2 - 1  # +-1 codes
        a, p, ng = u[:n], u[n:2 * n], u[2 * n:]
        Sa, Sp = a @ ng.T, p @ ng.T   # S = h(x)^T h(y)
        score = np.maximum(Sa, Sp)
        np.fill_diagonal(score, np.iinfo(np.int64).min)
        nstar = np.argmax(score, axis=1)  # first maximum = lowest index
        assert np.array_equal(out["mining"][row], nstar)
        xsel = (Sa[np.arange(n), nstar] < Sp[np.arange(n), nstar]).astype(np.int32)
        assert np.array_equal(out["mining"][row + 1], xsel)


def test_anchor_swap_picks_the_positive():
    P, bad, theta, hs = _problem(n=2, Kb=64, Kh=64, seed=4)
    P = P.copy()
    P[1, 0] = P[2, 1]          # p_0 identical to n_1, the only candidate for i = 0
    out = oracle.train_step(P, bad, theta, hs, want_grads=False)
    assert out["mining"][0, 0] == 1 and out["mining"][2, 0] == 1
    assert out["mining"][1, 0] == 1 and out["mining"][3, 0] == 1


def test_identical_triplets_give_n_tau():
    P, bad, theta, hs = _problem(n=4, seed=5)
    same = np.broadcast_to(P[0, 0], P.shape).copy()
    out = oracle.train_step(same, bad, theta, hs, tau_bad=7.5, tau_hs=3.25, want_grads=True)
    assert math.isclose(out["loss"][0], 4 * 7.5, rel_tol=1e-12)
    assert math.isclose(out["loss"][1], 4 * 3.25, rel_tol=1e-12)


def test_loss_is_piecewise_linear_in_tau():
    P, bad, theta, hs = _problem(n=8, seed=6)
    o1 = oracle.train_step(P, bad, theta, hs, tau_bad=32.0, tau_hs=32.0, want_grads=False, want_r=True)
    o2 = oracle.train_step(P, bad, theta, hs, tau_bad=32.5, tau_hs=32.5, fixed_mining=o1["mining"],
                           want_grads=False, want_r=True)
    n = 8
    for d, key, row in ((0, "r_bad", 0), (1, "r_hs", 2)):
        r = o1[key]
        nst, xs = o1["mining"][row], o1["mining"][row + 1]
        terms = []
        for i in range(n):
            x = r[n + i] if xs[i] else r[i]
            terms.append(32.0 - r[i] @ r[n + i] + x @ r[2 * n + nst[i]])
        active = sum(t > 0 for t in terms)
        inactive_near = sum(-0.5 < t <= 0 for t in terms)
        assert inactive_near == 0
        assert math.isclose(o2["loss"][d] - o1["loss"][d], 0.5 * active, rel_tol=1e-9, abs_tol=1e-9)


def test_bad_patch_features_and_relaxed_sign():
    P, bad, theta, hs = _problem(n=3, Kb=64, seed=7)
    bb, _, fb, _ = oracle.train_codes(P, bad, theta, hs)
    flat = P.reshape(-1, 32, 32)
    pad = np.zeros((flat.shape[0], 32 + 64, 32 + 64))
    pad[:, 32:64, 32:64] = flat
    for k in range(64):
        s = int(bad.sides[k])
        (x1, y1), (x2, y2) = bad.centres[k].astype(int)
        b1 = pad[:, 32 + y1 - s // 2:32 + y1 - s // 2 + s, 32 + x1 - s // 2:32 + x1 - s // 2 + s].sum(axis=(1, 2))
        b2 = pad[:, 32 + y2 - s // 2:32 + y2 - s // 2 + s, 32 + x2 - s // 2:32 + x2 - s // 2 + s].sum(axis=(1, 2))
        assert np.allclose(fb[:, k], (b1 - b2) / s ** 2, atol=1e-9)
    assert np.array_equal(_unpack(bb, 64).astype(bool), fb <= theta[None, :])
    out = oracle.train_step(P, bad, theta, hs, T=0.01, want_grads=False, want_r=True)
    far = np.abs(fb - theta[None, :]) > 5
    assert np.array_equal((out["r_bad"] > 0)[far], (fb <= theta[None, :])[far])
