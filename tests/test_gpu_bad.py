"""GPU parity of the integral image and BAD descriptors against the CPU oracle:
bit-exact (Sec. III-A; integer arithmetic on both sides)."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("h,w", [(1, 1), (1, 300), (300, 1), (33, 129), (127, 255), (480, 640),
                                 (1080, 1920), (31, 4000)])
def test_integral_bit_exact(gpu_ctx, h, w):
    rng = np.random.default_rng(h * 7919 + w)
    img = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
    ii = gpu_ctx.integral(_dev(img))
    assert np.array_equal(_u32(ii), oracle.integral(img))


def test_integral_largest_image_and_pitch(gpu_ctx):
    import torch
    h, w = 4095, 4096  # 255*w*h just below 2^32
    img = np.full((h, w), 255, np.uint8)
    ii = gpu_ctx.integral(_dev(img))
    got = _u32(ii)
    assert int(got[-1, -1]) == 255 * w * h
    rows = np.random.default_rng(0).integers(0, h + 1, size=50)
    ref = oracle.integral(img)
    assert np.array_equal(got[rows], ref[rows])
    # pitched source: a column window of a wider image
    rng = np.random.default_rng(1)
    big = rng.integers(0, 256, size=(200, 333)).astype(np.uint8)
    tb = _dev(big)
    view = tb[:, 17:17 + 250]
    out = torch.empty((201, 251), dtype=torch.int32, device="cuda")
    import paper_2108_08380_gb300 as bd
    import ctypes
    st = bd.lib().bd_integral(gpu_ctx.handle, ctypes.c_void_p(view.data_ptr()), 250, 200, 333,
                              ctypes.c_void_p(out.data_ptr()), 251)
    assert st == 0
    assert np.array_equal(_u32(out), oracle.integral(big[:, 17:267]))


def test_offset_table_matches_oracle_geometry(gpu_ctx):
    rng = np.random.default_rng(5)
    p = synth.make_bad_params(512, rng, level_scales=tuple(synth.pyramid_scales(5)))
    hp = gpu_ctx.bad_params(p)
    off, sides = hp.table()
    for l, sg in enumerate(p.level_scales):
        for b in range(32):
            o, s = oracle.bad_geometry(p.centres, p.sides, float(sg), 2 * math.pi * b / 32)
            assert np.array_equal(off[l, b], o), (l, b)
            assert np.array_equal(sides[l], s)


def _check_bad(ctx, img, kps, p):
    hp = ctx.bad_params(p)
    got = _u32(ctx.bad_describe(hp, _dev(img), _dev(kps)))
    ref, nbad = oracle.bad_describe(img, kps, p)
    flags = ctx.sync_status()
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:10]
    return flags, nbad


def test_bad256_plain_workload_bit_exact(gpu_ctx):
    wl = synth.plain_workload(1000)
    for img in (wl.img_a, wl.img_b):
        flags, nbad = _check_bad(gpu_ctx, img, wl.kps_a, wl.bad)
        assert flags == 0 and nbad == 0


def test_bad512_pyramid_continuous_angles(gpu_ctx):
    rng = np.random.default_rng(77)
    img = synth.make_image(1001, 777, rng)
    levels = synth.pyramid_scales(5)
    kps = synth.make_keypoints(2053, 1001, 777, rng, border=0.0,
                               scales=tuple(float(s) for s in levels), angle_bins=None)
    kps[:, 2] *= rng.uniform(0.85, 1.15, size=kps.shape[0]).astype(np.float32)  # off-level scales
    p = synth.make_bad_params(512, rng, level_scales=tuple(levels))
    flags, nbad = _check_bad(gpu_ctx, img, kps, p)
    assert flags == 0


def test_bad_fixed_point_thresholds_and_borders(gpu_ctx):
    rng = np.random.default_rng(78)
    img = synth.make_image(64, 48, rng)
    kps = np.concatenate([
        synth.make_keypoints(300, 64, 48, rng, border=-40.0, angle_bins=None),  # around and outside
        np.array([[0, 0, 1, 0], [63, 47, 1, 3.0], [-1000, 5, 1, 0], [31.5, 23.5, 1, -7.0]], np.float32)])
    p = synth.make_bad_params(256, rng, thr_den=10, thr_range=(-30, 30), side_range=(1, 32),
                              level_scales=(1.0, 1.5))
    _check_bad(gpu_ctx, img, kps, p)


def test_bad_invalid_keypoints_zero_and_flagged(gpu_ctx):
    import paper_2108_08380_gb300 as bd
    rng = np.random.default_rng(79)
    img = synth.make_image(128, 128, rng)
    kps = synth.make_keypoints(64, 128, 128, rng)
    kps[3, 0] = np.nan
    kps[10, 2] = 0.0
    kps[20, 3] = np.inf
    kps[30, 1] = 3e6
    p = synth.make_bad_params(256, rng)
    flags, nbad = _check_bad(gpu_ctx, img, kps, p)
    assert nbad == 4
    assert flags & bd.BD_FLAG_INVALID_KEYPOINT
    assert gpu_ctx.sync_status() == 0


def test_bad_empty_and_single(gpu_ctx):
    import torch
    rng = np.random.default_rng(80)
    img = synth.make_image(50, 40, rng)
    p = synth.make_bad_params(256, rng)
    hp = gpu_ctx.bad_params(p)
    out = gpu_ctx.bad_describe(hp, _dev(img), torch.empty((0, 4), dtype=torch.float32, device="cuda"))
    assert out.shape == (0, 8)
    _check_bad(gpu_ctx, img, np.array([[25, 20, 1, 1]], np.float32), p)


def test_bad_large_image_sampled(gpu_ctx):
    """1920x1080, 8000 keypoints on a 5-level pyramid, BAD-512, in the launch
    configuration of the large workloads: every GPU descriptor computed, a
    seeded sample of 600 checked against the oracle."""
    rng = np.random.default_rng(81)
    img = synth.make_image(1920, 1080, rng)
    levels = synth.pyramid_scales(5)
    kps = synth.make_keypoints(8000, 1920, 1080, rng, border=57,
                               scales=tuple(float(s) for s in levels), angle_bins=None)
    p = synth.make_bad_params(512, rng, level_scales=tuple(levels))
    hp = gpu_ctx.bad_params(p)
    got = _u32(gpu_ctx.bad_describe(hp, _dev(img), _dev(kps)))
    sel = np.sort(rng.choice(8000, size=600, replace=False))
    ref, _ = oracle.bad_describe(img, kps[sel], p)
    assert np.array_equal(got[sel], ref)
    # every descriptor is a plausible BAD code: about half the bits set on average
    frac = np.unpackbits(got.view(np.uint8)).mean()
    assert 0.2 < frac < 0.8
