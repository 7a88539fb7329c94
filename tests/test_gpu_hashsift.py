"""GPU parity of HashSIFT (Sec. III-B) against the CPU oracle.

Tolerances, from the FP32 arithmetic of the kernels:
  - patch warp: the FP32 sample position is off by at most ~1e-5 * scale px
    (sincosf and two fmaf roundings on offsets below 23*scale), and a bilinear
    sample moves at most 255 per px along each axis, plus three FP32 lerps:
    |dP| <= 2 * 255 * 1e-5 * scale + 1e-4;
  - histogram of the same FP32 patch: 1e-5 absolute on the unit-norm vector
    (the orientation weight w1 is off by ~2e-6 at most, times sqrt(8) at worst);
  - bits: equal wherever the oracle's margin clears the margin error that the
    measured histogram error can cause, sqrt(128) * max|dh| * ||W_k||_2, plus
    the FP32 dot-product rounding; the BF16 + rescue path equals the FP32 path
    bit for bit with the sound band."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bits(words, K):
    return np.unpackbits(np.ascontiguousarray(words).view(np.uint8), axis=1,
                         bitorder="little")[:, :K].astype(bool)


@pytest.fixture(scope="module")
def plain():
    return synth.plain_workload(1001)


def test_patch_warp_within_fp32_bound(gpu_ctx, plain):
    rng = np.random.default_rng(2)
    kps = plain.kps_a.copy()
    kps[:, 3] = rng.uniform(-7, 7, size=kps.shape[0]).astype(np.float32)
    kps[:, 2] = rng.uniform(0.5, 2.5, size=kps.shape[0]).astype(np.float32)
    kps[:10, 0] = rng.uniform(-30, 5, size=10)  # clamp-to-edge region
    hp = gpu_ctx.hs_params(plain.hs, precision=0)
    P = gpu_ctx.hashsift_warp(hp, _dev(plain.img_a), _dev(kps)).cpu().numpy().astype(np.float64)
    ref = oracle.hs_patches(plain.img_a, kps)
    tol = 2 * 255 * 1e-5 * kps[:, 2].astype(np.float64) + 1e-4
    err = np.abs(P - ref).reshape(len(kps), -1).max(axis=1)
    assert np.all(err <= tol), (err.max(), np.argmax(err / tol))


def test_histogram_same_patch_1e5(gpu_ctx, plain):
    hp = gpu_ctx.hs_params(plain.hs, precision=0)
    P = gpu_ctx.hashsift_warp(hp, _dev(plain.img_a), _dev(plain.kps_a))
    h = gpu_ctx.hashsift_hist(P).cpu().numpy().astype(np.float64)
    ref = oracle.hs_hist(P.cpu().numpy().astype(np.float64))
    err = np.abs(h - ref).max()
    assert err <= 1e-5, err


def test_histogram_of_oracle_patches_1e5_and_error_split(gpu_ctx, plain):
    """The plain workload's patches as the oracle warps them (FP64, rounded
    to FP32) through the GPU histogram: within 1e-5 of the oracle's histogram
    of the same patches.  End to end from the image, the only other source of
    error is the patch warp's FP32 sample positions: the end-to-end error is
    bounded by the histogram error plus the oracle's own change between the
    GPU's warped patches and its FP64 ones (triangle inequality), and that
    change is what makes the end-to-end figure larger than 1e-5."""
    import torch
    Po = oracle.hs_patches(plain.img_a, plain.kps_a).astype(np.float32)
    h = gpu_ctx.hashsift_hist(torch.from_numpy(Po).cuda()).cpu().numpy().astype(np.float64)
    ref_same = oracle.hs_hist(Po.astype(np.float64))
    assert np.abs(h - ref_same).max() <= 1e-5
    hp = gpu_ctx.hs_params(plain.hs, precision=0)
    Pg = gpu_ctx.hashsift_warp(hp, _dev(plain.img_a), _dev(plain.kps_a))
    hist = torch.empty((plain.kps_a.shape[0], 128), dtype=torch.float32, device="cuda")
    gpu_ctx.hashsift_describe(hp, _dev(plain.img_a), _dev(plain.kps_a), hist_out=hist)
    e2e = np.abs(hist.cpu().numpy().astype(np.float64) - oracle.hs_describe(
        plain.img_a, plain.kps_a, plain.hs)["hist"]).max(axis=1)
    hist_err = np.abs(gpu_ctx.hashsift_hist(Pg).cpu().numpy().astype(np.float64)
                      - oracle.hs_hist(Pg.cpu().numpy().astype(np.float64))).max(axis=1)
    warp_err = np.abs(oracle.hs_hist(Pg.cpu().numpy().astype(np.float64))
                      - oracle.hs_hist(oracle.hs_patches(plain.img_a, plain.kps_a))).max(axis=1)
    assert hist_err.max() <= 1e-5
    assert np.all(e2e <= hist_err + warp_err + 1e-6)
    assert e2e.max() <= 2e-4


def test_histogram_special_patches(gpu_ctx):
    import torch
    ii, jj = np.meshgrid(np.arange(32.0), np.arange(32.0), indexing="ij")
    P = np.stack([np.zeros((32, 32)), np.full((32, 32), 7.0), 3 * jj, 3 * ii, -3 * jj,
                  2 * (math.cos(3 * math.pi / 8) * jj + math.sin(3 * math.pi / 8) * ii)]).astype(np.float32)
    h = gpu_ctx.hashsift_hist(torch.from_numpy(P).cuda()).cpu().numpy()
    ref = oracle.hs_hist(P.astype(np.float64))
    assert np.abs(h - ref).max() <= 1e-5
    assert np.all(h[:2] == 0)


def _margins_tol(h_gpu, h_or, W):
    wn = np.linalg.norm(W.astype(np.float64), axis=0)
    err = np.abs(h_gpu - h_or).max(axis=1)
    return (math.sqrt(128) * err[:, None] + 2.0 ** -20) * wn[None, :] + 1e-6


@pytest.mark.parametrize("K", [256, 512])
def test_describe_fp32_bits_exact_outside_error_band(gpu_ctx, K):
    import torch
    wl = synth.plain_workload(1002, hs_bits=K)
    hp = gpu_ctx.hs_params(wl.hs, precision=0)
    hist = torch.empty((1000, 128), dtype=torch.float32, device="cuda")
    bits = gpu_ctx.hashsift_describe(hp, _dev(wl.img_a), _dev(wl.kps_a), hist_out=hist)
    got = _bits(bits.cpu().numpy(), K)
    ref = oracle.hs_describe(wl.img_a, wl.kps_a, wl.hs)
    h = hist.cpu().numpy().astype(np.float64)
    herr = np.abs(h - ref["hist"]).max()
    assert herr <= 2e-4, herr
    tol = _margins_tol(h, ref["hist"], wl.hs.W)
    sure = np.abs(ref["margins"]) >= tol
    refb = ref["margins"] > 0
    assert np.array_equal(got[sure], refb[sure])
    assert (~sure).mean() < 1e-3


@pytest.mark.parametrize("K", [256, 512])
def test_bf16_rescue_equals_fp32_path(gpu_ctx, K):
    wl = synth.plain_workload(1003, hs_bits=K)
    h32 = gpu_ctx.hs_params(wl.hs, precision=0)
    h16 = gpu_ctx.hs_params(wl.hs, precision=1)
    img, kps = _dev(wl.img_a), _dev(wl.kps_a)
    a = gpu_ctx.hashsift_describe(h32, img, kps).cpu().numpy()
    gpu_ctx.rescued_count(reset=True)
    b = gpu_ctx.hashsift_describe(h16, img, kps).cpu().numpy()
    rescued = gpu_ctx.rescued_count(reset=True)
    assert np.array_equal(a, b)
    assert rescued < 0.01 * a.size * 32
    assert gpu_ctx.sync_status() == 0
    # a wide band sends a third of the bits through the FP32 re-check: same bits
    hw = gpu_ctx.hs_params(wl.hs, precision=1, band=0.05)
    c = gpu_ctx.hashsift_describe(hw, img, kps).cpu().numpy()
    rescued = gpu_ctx.rescued_count(reset=True)
    assert np.array_equal(a, c)
    assert rescued > 0.05 * a.size * 32


def test_projection_of_oracle_histograms(gpu_ctx):
    """a6 alone: the oracle's histograms (rounded to FP32) through both GPU
    projections give the oracle's bits wherever |m| clears the FP32 rounding."""
    import torch
    rng = np.random.default_rng(9)
    hs = synth.make_hashsift_params(512, rng)
    img = synth.make_image(300, 200, rng)
    kps = synth.make_keypoints(777, 300, 200, rng, angle_bins=None)
    ref = oracle.hs_describe(img, kps, hs)
    h32 = ref["hist"].astype(np.float32)
    m64, _ = oracle.hs_project(h32.astype(np.float64), hs.W, hs.b)
    refb = m64 > 0
    sure = np.abs(m64) > 1e-5
    for prec in (0, 1):
        hp = gpu_ctx.hs_params(hs, precision=prec)
        got = _bits(gpu_ctx.hashsift_project(hp, torch.from_numpy(h32).cuda()).cpu().numpy(), 512)
        assert np.array_equal(got[sure], refb[sure]), prec


def test_zero_rows_project_to_the_bias_without_rescue(gpu_ctx):
    """A histogram row of zeros (a patch without gradients) projects to exactly
    b_k on both paths (every product is zero): its bits are b_k > 0, and none
    of them is re-checked in FP32, even where |b_k| lies inside the band."""
    import torch
    rng = np.random.default_rng(21)
    hs = synth.make_hashsift_params(512, rng)
    b = hs.b.copy()
    b[:8] = np.array([1e-7, -1e-7, 3e-6, -3e-6, 0.0, -0.0, 5e-5, -5e-5], np.float32)
    hs = synth.HashSiftParams(hs.W, b, hs.spacing)
    n = 300  # two full 128-row tiles and a ragged tail
    h = rng.random((n, 128)).astype(np.float32)
    h /= np.linalg.norm(h, axis=1, keepdims=True)
    zero = rng.random(n) < 0.5
    h[zero] = 0.0
    want = b > 0
    hp32 = gpu_ctx.hs_params(hs, precision=0)
    hp16 = gpu_ctx.hs_params(hs, precision=1)
    a = _bits(gpu_ctx.hashsift_project(hp32, torch.from_numpy(h).cuda()).cpu().numpy(), 512)
    c = _bits(gpu_ctx.hashsift_project(hp16, torch.from_numpy(h).cuda()).cpu().numpy(), 512)
    assert np.array_equal(a, c)
    assert (a[zero] == want).all()
    z = torch.zeros((n, 128), dtype=torch.float32, device="cuda")
    gpu_ctx.rescued_count(reset=True)
    cz = _bits(gpu_ctx.hashsift_project(hp16, z).cpu().numpy(), 512)
    assert gpu_ctx.rescued_count(reset=True) == 0
    assert (cz == want).all()
    assert gpu_ctx.sync_status() == 0


def test_fixed_band_1e3_reports_disagreements(gpu_ctx):
    """The batched workload's fixed 1e-3 band: with the split BF16 product the
    margin error is below 2^-13 ||W_k|| < 1e-3, so any bit it gets wrong (none
    expected) must lie inside the sound per-bit bound."""
    wl = synth.plain_workload(1004, hs_bits=512)
    img, kps = _dev(wl.img_a), _dev(wl.kps_a)
    ref = gpu_ctx.hashsift_describe(gpu_ctx.hs_params(wl.hs, precision=0), img, kps).cpu().numpy()
    got = gpu_ctx.hashsift_describe(gpu_ctx.hs_params(wl.hs, precision=1, band=1e-3), img, kps).cpu().numpy()
    bad = _bits(ref, 512) != _bits(got, 512)
    orc = oracle.hs_describe(wl.img_a, wl.kps_a, wl.hs)
    wn = np.linalg.norm(wl.hs.W.astype(np.float64), axis=0)
    bound = 2 ** -13 * wn + 2e-4 * wn
    assert np.all(np.abs(orc["margins"][bad]) < np.broadcast_to(bound, bad.shape)[bad])
    if np.all(2 ** -13 * wn < 1e-3):
        assert not bad.any()


def test_invalid_keypoints_zero_bits_and_hist(gpu_ctx, plain):
    import torch
    import paper_2108_08380_gb300 as bd
    kps = plain.kps_a[:200].copy()
    kps[5, 2] = -1.0
    kps[77, 0] = np.nan
    for prec in (0, 1):
        hp = gpu_ctx.hs_params(plain.hs, precision=prec)
        hist = torch.full((200, 128), 5.0, dtype=torch.float32, device="cuda")
        bits = gpu_ctx.hashsift_describe(hp, _dev(plain.img_a), _dev(kps), hist_out=hist).cpu().numpy()
        assert gpu_ctx.sync_status() & bd.BD_FLAG_INVALID_KEYPOINT
        assert np.all(bits[[5, 77]] == 0)
        assert np.all(hist.cpu().numpy()[[5, 77]] == 0)
        assert np.any(bits[6] != 0)


@pytest.mark.parametrize("n", [1, 127, 129, 4097])
def test_ragged_counts(gpu_ctx, n):
    rng = np.random.default_rng(n)
    img = synth.make_image(200, 160, rng)
    kps = synth.make_keypoints(n, 200, 160, rng, angle_bins=None)
    hs = synth.make_hashsift_params(256, rng)
    a = gpu_ctx.hashsift_describe(gpu_ctx.hs_params(hs, precision=0), _dev(img), _dev(kps)).cpu().numpy()
    b = gpu_ctx.hashsift_describe(gpu_ctx.hs_params(hs, precision=1), _dev(img), _dev(kps)).cpu().numpy()
    assert np.array_equal(a, b)
    sel = rng.choice(n, size=min(n, 64), replace=False)
    ref = oracle.hs_describe(img, kps[sel], hs)
    agree = (_bits(a[sel], 256) == (ref["margins"] > 0)) | (np.abs(ref["margins"]) < 1e-3)
    assert agree.all()


# ---------------------------------------------------------------------------
# SIFT variants before hashing (bd_hs_params_set_variant)

_VARIANTS = [0, 2, 4, 6, 1, 7]


@pytest.mark.parametrize("flags", _VARIANTS)
@pytest.mark.parametrize("n", [1000, 5000])
def test_variant_histograms_and_bits(gpu_ctx, plain, flags, n):
    """Histograms within 1e-5 of the oracle's variant on the GPU's own patches
    (the patch warp is pinned separately) and bits exact outside the error
    band; 1000 keypoints run the cooperative kernel, 5000 the warp kernel
    (trilinear always the warp kernel).  RootSIFT is compared squared: its
    square is the L1-normalised histogram, while the square root turns an
    absolute error e of a near-zero entry into up to sqrt(e)."""
    import paper_2108_08380_gb300 as bd
    rng = np.random.default_rng(n + flags)
    kps = synth.make_keypoints(n, 640, 480, rng, border=32.0, scales=(1.0,), angle_bins=None)
    kps[:5, 0] = rng.uniform(-10, 8, size=5)  # some footprints leave the image
    hp = gpu_ctx.hs_params(plain.hs, precision=bd.BD_HS_FP32)
    hp.set_variant(flags)
    import torch
    hist = torch.empty((n, 128), dtype=torch.float32, device="cuda")
    bits = gpu_ctx.hashsift_describe(hp, _dev(plain.img_a), _dev(kps), hist_out=hist).cpu().numpy()
    h = hist.cpu().numpy().astype(np.float64)
    P = gpu_ctx.hashsift_warp(hp, _dev(plain.img_a), _dev(kps)).cpu().numpy().astype(np.float64)
    ref = oracle.hs_hist_variant(P, flags)
    if flags & bd.BD_HS_VARIANT_ROOT:
        assert np.abs(h * h - ref * ref).max() <= 1e-5
    else:
        assert np.abs(h - ref).max() <= 1e-5
    margins, rbits = oracle.hs_project(ref, plain.hs.W, plain.hs.b)
    tol = _margins_tol(h, ref, plain.hs.W)
    sure = np.abs(margins) > tol
    got = _bits(bits, plain.hs.nbits)
    want = _bits(rbits, plain.hs.nbits)
    assert np.array_equal(got[sure], want[sure])


def test_variant_batch_matches_per_image_and_refuses_trilinear(gpu_ctx, plain):
    import paper_2108_08380_gb300 as bd
    import torch
    hp = gpu_ctx.hs_params(plain.hs, precision=bd.BD_HS_BF16_RESCUE)
    hp.set_variant(bd.BD_HS_VARIANT_CLIP | bd.BD_HS_VARIANT_ROOT)
    img = _dev(plain.img_a)
    kps = _dev(plain.kps_a)
    n = plain.kps_a.shape[0]
    flags = bd.BD_HS_VARIANT_CLIP | bd.BD_HS_VARIANT_ROOT
    P = gpu_ctx.hashsift_warp(hp, img, kps).cpu().numpy().astype(np.float64)
    ref = oracle.hs_hist_variant(P, flags)
    margins, _ = oracle.hs_project(ref, plain.hs.W, plain.hs.b)
    sure = np.abs(margins) > _margins_tol(ref + 1e-5, ref, plain.hs.W)  # 1e-5 histogram error
    want = margins > 0
    one = gpu_ctx.hashsift_describe(hp, img, kps).cpu().numpy()
    assert np.array_equal(_bits(one, plain.hs.nbits)[sure], want[sure])
    plan = gpu_ctx.batch(None, hp, [img], [0, n])
    out = torch.empty((n, plain.hs.nbits // 32), dtype=torch.int32, device="cuda")
    for mode in (1, 4):
        plan.set_config(8, 4, 0, mode)
        plan.describe([img], kps, None, out)
        assert np.array_equal(_bits(out.cpu().numpy(), plain.hs.nbits)[sure], want[sure])
    plan.close()
    hp.set_variant(bd.BD_HS_VARIANT_TRILINEAR)
    with pytest.raises(bd.BindescError):
        gpu_ctx.batch(None, hp, [img], [0, n])
    with pytest.raises(bd.BindescError):
        hp.set_variant(8)
