"""Pins for the oracle's integral image, box sums, keypoint quantisation and BAD
descriptor (Sec. III-A of the paper), each checked against something other
than the oracle itself: brute-force sums, closed forms on constant and delta
images, the ORB special case (Sec. IV-A: ORB = BAD with 5x5 boxes and zero
threshold), and invariants (threshold sign flips, exact 90-degree rotation)."""
import math

import numpy as np
import pytest

import oracle
import synth


# --------------------------------------------------------------------------
# integral image
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_integral_matches_bruteforce(seed):
    rng = np.random.default_rng(seed)
    h, w = rng.integers(1, 10, size=2)
    img = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
    ii = oracle.integral(img)
    assert ii.shape == (h + 1, w + 1)
    for y in range(h + 1):
        for x in range(w + 1):
            assert int(ii[y, x]) == int(img[:y, :x].astype(np.int64).sum())


def test_integral_constant_closed_form():
    c = 37
    img = np.full((23, 31), c, np.uint8)
    ii = oracle.integral(img).astype(np.int64)
    yy, xx = np.meshgrid(np.arange(24), np.arange(32), indexing="ij")
    assert np.array_equal(ii, c * xx * yy)


def test_integral_largest_sum_fits_uint32():
    img = np.full((2160, 3840), 255, np.uint8)
    ii = oracle.integral(img)
    assert int(ii[-1, -1]) == 255 * 2160 * 3840


def test_box_sum_zero_padding_bruteforce():
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, size=(9, 11)).astype(np.uint8)
    pad = np.zeros((9 + 40, 11 + 40), np.int64)
    pad[20:29, 20:31] = img
    for _ in range(200):
        x0, y0 = rng.integers(-15, 15, size=2)
        s = int(rng.integers(1, 12))
        ref = pad[y0 + 20:y0 + 20 + s, x0 + 20:x0 + 20 + s].sum()
        assert oracle.box_sum(img, x0, y0, s) == ref


# --------------------------------------------------------------------------
# keypoint quantisation
# --------------------------------------------------------------------------

def test_round_coord():
    assert oracle.round_coord(2.5) == 3
    assert oracle.round_coord(2.4999) == 2
    assert oracle.round_coord(-0.5) == 0
    assert oracle.round_coord(-0.51) == -1
    assert oracle.round_coord(100.0) == 100


def test_angle_bin_centres_and_wrap():
    for b in range(32):
        a = np.float32(2 * math.pi * b / 32)
        assert oracle.angle_bin(float(a)) == b
        assert oracle.angle_bin(float(np.float32(a - 2 * math.pi))) == b
    # half a bin below / above the boundary between bins 3 and 4
    edge = 3.5 * 2 * math.pi / 32
    assert oracle.angle_bin(edge - 1e-4) == 3
    assert oracle.angle_bin(edge + 1e-4) == 4
    # the last half bin wraps to bin 0
    assert oracle.angle_bin(2 * math.pi - 1e-3) == 0


def test_scale_level_midpoints():
    ls = synth.pyramid_scales(5)
    for l, s in enumerate(ls):
        assert oracle.scale_level(float(s), ls) == l
    assert oracle.scale_level(0.01, ls) == 0
    assert oracle.scale_level(100.0, ls) == 4
    mid = math.sqrt(float(ls[1]) * float(ls[2]))
    assert oracle.scale_level(mid * (1 - 1e-6), ls) == 1
    assert oracle.scale_level(mid * (1 + 1e-6), ls) == 2


# --------------------------------------------------------------------------
# box geometry
# --------------------------------------------------------------------------

def test_geometry_axis_aligned():
    rng = np.random.default_rng(3)
    p = synth.make_bad_params(64, rng)
    off, sp = oracle.bad_geometry(p.centres, p.sides, 1.0, 0.0)
    d = p.centres.astype(np.int32) - 16
    assert np.array_equal(off, d)
    assert np.array_equal(sp, p.sides.astype(np.int32))
    # quarter turn, y axis down: (dx, dy) -> (-dy, dx)
    off90, _ = oracle.bad_geometry(p.centres, p.sides, 1.0, math.pi / 2)
    assert np.array_equal(off90[..., 0], -d[..., 1])
    assert np.array_equal(off90[..., 1], d[..., 0])
    # exact pyramid scale 2: offsets and sides double
    off2, sp2 = oracle.bad_geometry(p.centres, p.sides, 2.0, 0.0)
    assert np.array_equal(off2, 2 * d)
    assert np.array_equal(sp2, 2 * p.sides.astype(np.int32))


# --------------------------------------------------------------------------
# BAD descriptor
# --------------------------------------------------------------------------

def _bits(desc, K):
    return np.unpackbits(desc.view(np.uint8), bitorder="little")[:K].astype(bool)


def _kp(x, y, scale=1.0, angle=0.0):
    return np.array([[x, y, scale, angle]], np.float32)


def test_constant_image_gives_threshold_sign():
    rng = np.random.default_rng(11)
    p = synth.make_bad_params(256, rng)
    img = np.full((200, 200), 91, np.uint8)
    d, bad = oracle.bad_describe(img, _kp(100, 100, 1.0, 1.3), p)
    assert bad == 0
    assert np.array_equal(_bits(d[0], 256), p.thr_num >= 0)


def test_delta_image_pins_box_placement():
    """One bright pixel: box 1 holds it iff |p - c1| is inside [-s//2, s - s//2)."""
    rng = np.random.default_rng(5)
    K = 256
    p = synth.make_bad_params(K, rng, thr_range=(0, 0))
    for trial in range(20):
        img = np.zeros((120, 120), np.uint8)
        px, py = rng.integers(40, 80, size=2)
        img[py, px] = 255
        kx, ky = 60, 60
        b = int(rng.integers(0, 4)) * 8  # axis-aligned bins: exact offsets
        d, _ = oracle.bad_describe(img, _kp(kx, ky, 1.0, 2 * math.pi * b / 32), p)
        got = _bits(d[0], K)
        for k in range(K):
            s = int(p.sides[k])
            inside = []
            for j in range(2):
                dx, dy = int(p.centres[k, j, 0]) - 16, int(p.centres[k, j, 1]) - 16
                for _ in range(b // 8):  # quarter turns, y down: (dx,dy)->(-dy,dx)
                    dx, dy = -dy, dx
                cx, cy = kx + dx, ky + dy
                x0, y0 = cx - s // 2, cy - s // 2
                inside.append(x0 <= px < x0 + s and y0 <= py < y0 + s)
            # f = (255*[in1] - 255*[in2]) / s^2 <= 0
            assert got[k] == (not (inside[0] and not inside[1])), (trial, k)


def _box5(img):
    """5x5 box sums centred on every pixel (zero padding), brute force."""
    h, w = img.shape
    pad = np.zeros((h + 4, w + 4), np.int64)
    pad[2:-2, 2:-2] = img
    out = np.zeros((h, w), np.int64)
    for dy in range(5):
        for dx in range(5):
            out += pad[dy:dy + h, dx:dx + w]
    return out


def test_orb_special_case():
    """Sec. IV-A: ORB's test on a 5x5 box-filtered image = BAD with s=5, theta=0."""
    rng = np.random.default_rng(2)
    img = synth.make_image(96, 80, rng)
    K = 256
    p = synth.make_bad_params(K, rng, side_range=(5, 5), thr_range=(0, 0))
    box = _box5(img)
    kps = synth.make_keypoints(40, 96, 80, rng, border=20, angle_bins=1)
    d, _ = oracle.bad_describe(img, kps, p)
    for i in range(kps.shape[0]):
        kx, ky = int(math.floor(kps[i, 0] + 0.5)), int(math.floor(kps[i, 1] + 0.5))
        u = p.centres.astype(np.int64) - 16
        v1 = box[ky + u[:, 0, 1], kx + u[:, 0, 0]]
        v2 = box[ky + u[:, 1, 1], kx + u[:, 1, 0]]
        assert np.array_equal(_bits(d[i], K), v1 <= v2)


def test_swapping_boxes_and_negating_threshold_flips_exactly_those_bits():
    rng = np.random.default_rng(9)
    img = synth.make_image(160, 120, rng)
    K = 256
    p = synth.make_bad_params(K, rng)
    q = synth.BadParams(p.centres[:, ::-1, :].copy(), p.sides, (-p.thr_num).astype(np.int32),
                        p.thr_den, p.level_scales, p.n_angle_bins)
    kps = synth.make_keypoints(30, 160, 120, rng, border=34)
    d1, _ = oracle.bad_describe(img, kps, p)
    d2, _ = oracle.bad_describe(img, kps, q)
    for i in range(kps.shape[0]):
        kx = oracle.round_coord(float(kps[i, 0]))
        ky = oracle.round_coord(float(kps[i, 1]))
        b = oracle.angle_bin(float(kps[i, 3]))
        off, sp = oracle.bad_geometry(p.centres, p.sides, 1.0, 2 * math.pi * b / 32)
        for k in range(K):
            s = int(sp[k])
            sums = [oracle.box_sum(img, kx + off[k, j, 0] - s // 2, ky + off[k, j, 1] - s // 2, s)
                    for j in range(2)]
            on_threshold = (sums[0] - sums[1]) == int(p.thr_num[k]) * s * s
            a, bq = _bits(d1[i], K)[k], _bits(d2[i], K)[k]
            if on_threshold:
                assert a and bq
            else:
                assert a != bq


def test_extreme_thresholds_force_bits():
    rng = np.random.default_rng(4)
    img = synth.make_image(100, 100, rng)
    kps = synth.make_keypoints(10, 100, 100, rng, border=34)
    p = synth.make_bad_params(256, rng)
    hi = synth.BadParams(p.centres, p.sides, np.full(256, 255, np.int32), 1, p.level_scales)
    lo = synth.BadParams(p.centres, p.sides, np.full(256, -256, np.int32), 1, p.level_scales)
    assert np.all(oracle.bad_describe(img, kps, hi)[0] == 0xFFFFFFFF)
    assert np.all(oracle.bad_describe(img, kps, lo)[0] == 0)


def test_fixed_point_threshold_matches_rational_compare():
    """theta = num/den: the bit is f <= num/den with f a rational box-mean difference."""
    rng = np.random.default_rng(14)
    img = synth.make_image(90, 90, rng)
    K = 64
    p = synth.make_bad_params(K, rng, thr_den=10, thr_range=(-3, 3))
    kps = synth.make_keypoints(8, 90, 90, rng, border=34, angle_bins=1)
    d, _ = oracle.bad_describe(img, kps, p)
    from fractions import Fraction
    for i in range(8):
        kx, ky = oracle.round_coord(float(kps[i, 0])), oracle.round_coord(float(kps[i, 1]))
        for k in range(K):
            s = int(p.sides[k])
            u = p.centres[k].astype(int) - 16
            s1 = int(img[ky + u[0, 1] - s // 2: ky + u[0, 1] - s // 2 + s,
                         kx + u[0, 0] - s // 2: kx + u[0, 0] - s // 2 + s].astype(np.int64).sum())
            s2 = int(img[ky + u[1, 1] - s // 2: ky + u[1, 1] - s // 2 + s,
                         kx + u[1, 0] - s // 2: kx + u[1, 0] - s // 2 + s].astype(np.int64).sum())
            f = Fraction(s1 - s2, s * s)
            assert _bits(d[i], K)[k] == (f <= Fraction(int(p.thr_num[k]), 10))


def test_quarter_turn_rotation_invariance():
    """Rotating the image a quarter turn about the keypoint and adding 8 angle
    bins gives the same descriptor, for odd box sides."""
    rng = np.random.default_rng(21)
    N = 161
    img = synth.make_image(N, N, rng)
    K = 256
    p = synth.make_bad_params(K, rng)
    p.sides[:] = 2 * (p.sides // 2) + 1
    c = (N - 1) / 2
    rot = np.ascontiguousarray(np.rot90(img, -1))  # rot[y][x] = img[N-1-x][y]
    for b in range(32):
        d0, _ = oracle.bad_describe(img, _kp(c, c, 1.0, 2 * math.pi * b / 32), p)
        d1, _ = oracle.bad_describe(rot, _kp(c, c, 1.0, 2 * math.pi * ((b + 8) % 32) / 32), p)
        assert np.array_equal(d0, d1), b


def test_pyramid_level_two_doubles_geometry():
    """At an exact level scale of 2 each box doubles its offset and side."""
    rng = np.random.default_rng(8)
    K = 128
    p = synth.make_bad_params(K, rng, level_scales=(1.0, 2.0))
    img = synth.make_image(200, 200, rng)
    d, _ = oracle.bad_describe(img, _kp(100, 100, 2.0, 0.0), p)
    u = p.centres.astype(np.int64) - 16
    for k in range(K):
        s = 2 * int(p.sides[k])
        sums = []
        for j in range(2):
            cx, cy = 100 + 2 * u[k, j, 0], 100 + 2 * u[k, j, 1]
            sums.append(int(img[cy - s // 2:cy - s // 2 + s, cx - s // 2:cx - s // 2 + s].astype(np.int64).sum()))
        assert _bits(d[0], K)[k] == (sums[0] - sums[1] <= int(p.thr_num[k]) * s * s)


def test_invalid_keypoints_give_zero_descriptors():
    rng = np.random.default_rng(1)
    img = synth.make_image(64, 64, rng)
    p = synth.make_bad_params(256, rng, thr_range=(10, 20))
    kps = np.array([[32, 32, 1, 0], [np.nan, 32, 1, 0], [32, 32, 0, 0], [32, 32, -1, 0],
                    [32, 32, 1, np.inf], [2e6, 3, 1, 0], [32, 32, 2000, 0]], np.float32)
    d, bad = oracle.bad_describe(img, kps, p)
    assert bad == 6
    assert np.all(d[1:] == 0)
    assert np.any(d[0] != 0)


def test_keypoint_outside_image_uses_zero_padding():
    img = np.full((50, 50), 200, np.uint8)
    rng = np.random.default_rng(6)
    p = synth.make_bad_params(256, rng)
    d, bad = oracle.bad_describe(img, _kp(-500, -500), p)
    assert bad == 0
    assert np.array_equal(_bits(d[0], 256), p.thr_num >= 0)
