"""Pins for the oracle's HashSIFT path (Sec. III-B): the bilinear patch warp,
the 4x4x8 gradient-orientation histogram and the sign of the learned
projection, checked against exact samples, closed-form ramps, an exact
quarter-turn equivariance, and a library matrix product."""
import math

import numpy as np
import pytest

import oracle
import synth


def _kp(x, y, scale=1.0, angle=0.0):
    return np.array([[x, y, scale, angle]], np.float32)


# --------------------------------------------------------------------------
# patch warp
# --------------------------------------------------------------------------

def test_patch_integer_translation_is_exact():
    rng = np.random.default_rng(0)
    img = synth.make_image(100, 90, rng)
    x0, y0 = 31, 22
    P = oracle.hs_patches(img, _kp(x0 + 15.5, y0 + 15.5))[0]
    assert np.array_equal(P, img[y0:y0 + 32, x0:x0 + 32].astype(np.float64))


def test_patch_bilinear_weights():
    rng = np.random.default_rng(1)
    img = synth.make_image(100, 90, rng)
    x0, y0 = 20, 30
    P = oracle.hs_patches(img, _kp(x0 + 15.5 + 0.25, y0 + 15.5 + 0.5))[0]
    I = img.astype(np.float64)
    ref = 0.5 * (0.75 * I[y0:y0 + 32, x0:x0 + 32] + 0.25 * I[y0:y0 + 32, x0 + 1:x0 + 33]) \
        + 0.5 * (0.75 * I[y0 + 1:y0 + 33, x0:x0 + 32] + 0.25 * I[y0 + 1:y0 + 33, x0 + 1:x0 + 33])
    assert np.allclose(P, ref, atol=1e-9)


def test_patch_quarter_turn_and_scale():
    rng = np.random.default_rng(2)
    img = synth.make_image(200, 200, rng)
    X, Y = 90, 100
    # angle pi/2, y down: sample (X+0.5 - (i-15.5), Y+0.5 + (j-15.5))
    P = oracle.hs_patches(img, _kp(X + 0.5, Y + 0.5, 1.0, math.pi / 2))[0]
    ii, jj = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    ref = img[Y + jj - 15, X + 16 - ii].astype(np.float64)
    assert np.allclose(P, ref, atol=1e-3)  # float32 pi/2 leaves cos ~ -4e-8
    # scale 2 at angle 0: samples every second pixel
    P2 = oracle.hs_patches(img, _kp(X + 31.0, Y + 31.0, 2.0, 0.0))[0]
    assert np.array_equal(P2, img[Y:Y + 64:2, X:X + 64:2].astype(np.float64))


def test_patch_clamps_to_edge():
    img = np.zeros((40, 40), np.uint8)
    img[:, 0] = 100
    img[0, :] = 50
    P = oracle.hs_patches(img, _kp(-100.0, 20.0))[0]
    assert np.all(P == 100)
    P = oracle.hs_patches(img, _kp(20.0, -100.0))[0]
    assert np.all(P[:, :] >= 50) and np.all(P <= 100)


def test_constant_image_constant_patch():
    img = np.full((64, 64), 77, np.uint8)
    P = oracle.hs_patches(img, _kp(30.3, 31.7, 1.3, 0.7))[0]
    assert np.allclose(P, 77.0, atol=1e-12)


# --------------------------------------------------------------------------
# histogram
# --------------------------------------------------------------------------

def _gauss():
    ii, jj = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    return np.exp(-((ii - 15.5) ** 2 + (jj - 15.5) ** 2) / (2 * 16.0 ** 2))


def _cells(weights_per_pixel):
    """Sum a 32x32 per-pixel array into the 4x4 cells (row-major cell index)."""
    return weights_per_pixel.reshape(4, 8, 4, 8).sum(axis=(1, 3)).reshape(16)


def test_zero_gradient_gives_zero_histogram():
    H, nrm = oracle.hs_hist_raw(np.full((32, 32), 12.5))
    assert nrm == 0.0 and np.all(H == 0)
    assert np.all(oracle.hs_hist(np.full((1, 32, 32), 3.0)) == 0)


@pytest.mark.parametrize("direction,bin_", [("+x", 0), ("+y", 2), ("-x", 4), ("-y", 6)])
def test_linear_ramps_vote_into_one_bin(direction, bin_):
    a = 3.0
    ii, jj = np.meshgrid(np.arange(32, dtype=float), np.arange(32, dtype=float), indexing="ij")
    along = {"+x": jj, "-x": -jj, "+y": ii, "-y": -ii}[direction]
    P = a * along
    # central differences: magnitude a inside, a/2 on the replicated edge
    m = np.full((32, 32), a)
    if direction in ("+x", "-x"):
        m[:, 0] = m[:, 31] = a / 2
    else:
        m[0, :] = m[31, :] = a / 2
    expect = np.zeros((16, 8))
    expect[:, bin_] = _cells(_gauss() * m)
    H, nrm = oracle.hs_hist_raw(P)
    assert np.allclose(H.reshape(16, 8), expect, rtol=1e-12, atol=1e-12)
    h = oracle.hs_hist(P[None])[0]
    assert np.allclose(h, expect.ravel() / np.linalg.norm(expect), atol=1e-14)


def test_soft_vote_splits_between_neighbouring_bins():
    """Gradient at 3*pi/8 (t = 1.5) votes half into bin 1 and half into bin 2."""
    phi = 3 * math.pi / 8
    ii, jj = np.meshgrid(np.arange(32, dtype=float), np.arange(32, dtype=float), indexing="ij")
    P = 2.0 * (math.cos(phi) * jj + math.sin(phi) * ii)
    H, _ = oracle.hs_hist_raw(P)
    H = H.reshape(16, 8)
    # interior pixels vote 50/50; cells with edge pixels lean on the edge direction
    inner = H[5]  # cell (1,1): no edge pixels
    assert np.allclose(inner[[0, 3, 4, 5, 6, 7]], 0, atol=1e-12)
    assert abs(inner[1] - inner[2]) < 1e-10 * inner[1]
    total = (_gauss()[8:16, 8:16] * 2.0).sum()
    assert abs(inner[1] + inner[2] - total) < 1e-10 * total


def test_quarter_turn_equivariance():
    """Turning the patch a quarter turn rotates every gradient by pi/2: the
    histogram is the cell permutation (r, c) -> (c, 3 - r) with bins shifted by 2."""
    rng = np.random.default_rng(3)
    img = synth.make_image(64, 64, rng).astype(np.float64)
    P = img[10:42, 20:52]
    Pr = np.rot90(P, -1)  # Pr[i][j] = P[31 - j][i]
    H, _ = oracle.hs_hist_raw(P)
    Hr, _ = oracle.hs_hist_raw(np.ascontiguousarray(Pr))
    H = H.reshape(4, 4, 8)
    Hr = Hr.reshape(4, 4, 8)
    for ci in range(4):
        for cj in range(4):
            assert np.allclose(Hr[ci, cj], np.roll(H[3 - cj, ci], 2), rtol=1e-11, atol=1e-9)


def test_histogram_is_unit_norm_and_nonnegative():
    rng = np.random.default_rng(4)
    img = synth.make_image(160, 120, rng)
    kps = synth.make_keypoints(50, 160, 120, rng, angle_bins=None)
    h = oracle.hs_hist(oracle.hs_patches(img, kps))
    assert np.all(h >= 0)
    assert np.allclose(np.linalg.norm(h, axis=1), 1.0, atol=1e-12)


def test_histogram_scale_invariance_of_intensity():
    """h is invariant to intensity gain and offset (L2 normalisation, differences)."""
    rng = np.random.default_rng(5)
    P = rng.uniform(0, 255, size=(32, 32))
    h1 = oracle.hs_hist(P[None])[0]
    h2 = oracle.hs_hist((3.5 * P + 40.0)[None])[0]
    assert np.allclose(h1, h2, atol=1e-12)


# --------------------------------------------------------------------------
# projection and sign
# --------------------------------------------------------------------------

def test_projection_matches_library_product():
    rng = np.random.default_rng(6)
    hs = synth.make_hashsift_params(256, rng)
    h = rng.uniform(0, 1, size=(20, 128))
    h /= np.linalg.norm(h, axis=1, keepdims=True)
    m, bits = oracle.hs_project(h, hs.W, hs.b)
    ref = h @ hs.W.astype(np.float64) + hs.b.astype(np.float64)
    assert np.allclose(m, ref, atol=1e-12)
    ub = np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little").astype(bool)
    assert np.array_equal(ub, ref > 0)


def test_zero_histogram_bits_are_offset_signs_and_zero_margin_is_bit0():
    rng = np.random.default_rng(7)
    hs = synth.make_hashsift_params(256, rng)
    hs.b[:8] = 0.0
    m, bits = oracle.hs_project(np.zeros((1, 128)), hs.W, hs.b)
    ub = np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little").astype(bool)[0]
    assert np.array_equal(ub, hs.b > 0)
    assert not ub[:8].any()


def test_identity_like_projection():
    """W = I (first 128 columns), b = -0.05: bit i = [h_i > 0.05]."""
    W = np.zeros((128, 256), np.float32)
    W[np.arange(128), np.arange(128)] = 1.0
    b = np.full(256, -0.05, np.float32)
    rng = np.random.default_rng(8)
    h = rng.uniform(0, 0.2, size=(5, 128))
    _, bits = oracle.hs_project(h, W, b)
    ub = np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little").astype(bool)
    assert np.array_equal(ub[:, :128], h > np.float64(np.float32(0.05)))
    assert not ub[:, 128:].any()


def test_describe_consistent_with_stages():
    rng = np.random.default_rng(9)
    img = synth.make_image(120, 100, rng)
    kps = synth.make_keypoints(12, 120, 100, rng, angle_bins=None)
    hs = synth.make_hashsift_params(512, rng)
    out = oracle.hs_describe(img, kps, hs, want_patches=True)
    P = oracle.hs_patches(img, kps)
    assert np.array_equal(out["patches"], P)
    h = oracle.hs_hist(P)
    assert np.array_equal(out["hist"], h)
    m, bits = oracle.hs_project(h, hs.W, hs.b)
    assert np.array_equal(out["bits"], bits)


# ---------------------------------------------------------------------------
# SIFT variants before hashing (trilinear binning, 0.2 clip, RootSIFT)

def _ramp(a=3.0):
    j = np.arange(32, dtype=np.float64)
    return np.tile(a * j, (32, 1))


def test_variant_none_is_the_base_histogram():
    rng = np.random.default_rng(3)
    P = rng.uniform(0, 255, size=(4, 32, 32))
    assert np.allclose(oracle.hs_hist_variant(P, 0), oracle.hs_hist(P), atol=1e-15)


def test_trilinear_ramp_is_separable_and_symmetric():
    """Horizontal ramp: every vote in bin 0 with weight g_i g_j m_j, so the
    4x4 cell matrix of bin 0 has rank one and the grid's mirror symmetries."""
    h = oracle.hs_hist_variant(_ramp(), oracle.HS_TRILINEAR)[0].reshape(4, 4, 8)
    assert np.allclose(h[:, :, 1:], 0.0)
    M = h[:, :, 0]
    assert np.linalg.matrix_rank(M, tol=1e-12) == 1
    assert np.allclose(M, M[::-1, :]) and np.allclose(M, M[:, ::-1])
    base = oracle.hs_hist(_ramp())[0].reshape(4, 4, 8)[:, :, 0]
    assert not np.allclose(M / M.sum(), base / base.sum())  # the binning did change


def test_trilinear_vertical_edge_weights():
    """A step between columns 4 and 5 has gradient (of equal magnitude) at
    columns 4 and 5 only; with cell centres at 3.5 and 11.5 cell column 1 over
    cell column 0 is (w1(4) g4 + w1(5) g5) / (w0(4) g4 + w0(5) g5), w the
    linear column weights and g the Gaussian column factors; cell columns 2
    and 3 get nothing."""
    P = np.zeros((32, 32))
    P[:, 5:] = 200.0
    h = oracle.hs_hist_variant(P, oracle.HS_TRILINEAR)[0].reshape(4, 4, 8)
    col = h[:, :, 0].sum(axis=0)
    assert np.allclose(col[2:], 0.0)
    g = lambda j: np.exp(-((j - 15.5) ** 2) / 512.0)
    w = lambda j, c: max(0.0, 1.0 - abs(j - (8 * c + 3.5)) / 8.0)
    ratio = (w(4, 1) * g(4) + w(5, 1) * g(5)) / (w(4, 0) * g(4) + w(5, 0) * g(5))
    assert np.isclose(col[1] / col[0], ratio, rtol=1e-12)


def test_clip_keeps_order_and_scales_the_small_entries():
    rng = np.random.default_rng(5)
    P = rng.uniform(0, 255, size=(3, 32, 32))
    P[0] = _ramp()
    base = oracle.hs_hist(P)
    clip = oracle.hs_hist_variant(P, oracle.HS_CLIP)
    for b, c in zip(base, clip):
        assert np.isclose(np.linalg.norm(c), 1.0)
        small = (b > 0) & (b < 0.2)
        big = b >= 0.2
        if small.any():
            s = c[small] / b[small]
            assert np.allclose(s, s[0]) and s[0] >= 1.0 - 1e-12  # one common factor
        if big.any():
            assert np.allclose(c[big], c[big][0])  # clipped entries become equal
            assert c[big][0] >= c[small].max() - 1e-12 if small.any() else True


def test_rootsift_is_the_hellinger_kernel():
    """RootSIFT(x) . RootSIFT(y) = sum_i sqrt(x_i y_i) of the L1-normalised
    histograms (the Hellinger kernel), and RootSIFT has unit L2 norm."""
    rng = np.random.default_rng(6)
    P = rng.uniform(0, 255, size=(5, 32, 32))
    base = oracle.hs_hist(P)
    r = oracle.hs_hist_variant(P, oracle.HS_ROOT)
    l1 = base / base.sum(axis=1, keepdims=True)
    for a in range(5):
        assert np.isclose(np.linalg.norm(r[a]), 1.0)
        for b in range(5):
            assert np.isclose(r[a] @ r[b], np.sqrt(l1[a] * l1[b]).sum(), rtol=1e-12)


def test_variants_of_a_flat_patch_stay_zero():
    P = np.full((32, 32), 42.0)
    for f in range(8):
        assert np.all(oracle.hs_hist_variant(P, f) == 0.0)
