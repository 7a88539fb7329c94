"""Seeded synthetic inputs for the BAD / HashSIFT descriptor path.

This module only draws inputs: images, keypoints, descriptor parameters,
image pairs and training triplets.  It holds none of the descriptor
arithmetic, so both the CPU oracle's tests and the CUDA path's tests and
benchmark can take their inputs from here without sharing any of the method.

Every generator takes a ``numpy.random.Generator`` (``np.random.default_rng``)
so a workload is fixed by its seed.  The shapes and value distributions stand
in for the paper's workloads (Sec. IV-F: Oxford images about 800 px wide with
at most 2000 keypoints; Sec. III: 32x32 patches); no dataset is read.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------
# images
# --------------------------------------------------------------------------


def _gauss_taps(sigma: float, radius: int) -> np.ndarray:
    x = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-(x * x) / (2.0 * sigma * sigma))
    return k / k.sum()


def _blur_reflect(a: np.ndarray, sigma: float = 2.0, radius: int = 6) -> np.ndarray:
    """Separable Gaussian blur with mirror padding (input generation only)."""
    k = _gauss_taps(sigma, radius)
    p = np.pad(a, ((0, 0), (radius, radius)), mode="reflect")
    out = np.zeros_like(a, dtype=np.float64)
    for t in range(2 * radius + 1):
        out += k[t] * p[:, t:t + a.shape[1]]
    p = np.pad(out, ((radius, radius), (0, 0)), mode="reflect")
    out2 = np.zeros_like(out)
    for t in range(2 * radius + 1):
        out2 += k[t] * p[t:t + a.shape[0], :]
    return out2


def make_image(w: int, h: int, rng: np.random.Generator, n_rects: int = 20) -> np.ndarray:
    """uint8 [h, w]: white noise blurred with sigma=2, then filled rectangles."""
    noise = rng.integers(0, 256, size=(h, w)).astype(np.float64)
    img = np.clip(np.rint(_blur_reflect(noise)), 0, 255).astype(np.uint8)
    for _ in range(n_rects):
        x0, x1 = np.sort(rng.integers(0, w, size=2))
        y0, y1 = np.sort(rng.integers(0, h, size=2))
        img[y0:y1 + 1, x0:x1 + 1] = np.uint8(rng.integers(0, 256))
    return img


def add_noise(img: np.ndarray, rng: np.random.Generator, sigma: float = 5.0) -> np.ndarray:
    """img + N(0, sigma^2), rounded half-to-even and clipped to uint8."""
    n = rng.normal(0.0, sigma, size=img.shape)
    return np.clip(np.rint(img.astype(np.float64) + n), 0, 255).astype(np.uint8)


def random_homography(rng: np.random.Generator, w: int, h: int, rot_deg: float = 15.0,
                      scale=(0.9, 1.1), persp: float = 1e-5, shift: float = 50.0) -> np.ndarray:
    """3x3 homography about the image centre: rotation, scale, small perspective, shift."""
    a = math.radians(rng.uniform(-rot_deg, rot_deg))
    s = rng.uniform(*scale)
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    T0 = np.array([[1, 0, -cx], [0, 1, -cy], [0, 0, 1]], dtype=np.float64)
    R = np.array([[s * math.cos(a), -s * math.sin(a), 0],
                  [s * math.sin(a), s * math.cos(a), 0], [0, 0, 1]], dtype=np.float64)
    P = np.array([[1, 0, 0], [0, 1, 0],
                  [rng.uniform(-persp, persp), rng.uniform(-persp, persp), 1]], dtype=np.float64)
    T1 = np.array([[1, 0, cx + rng.uniform(-shift, shift)],
                   [0, 1, cy + rng.uniform(-shift, shift)], [0, 0, 1]], dtype=np.float64)
    return T1 @ P @ R @ T0


def warp_image(img: np.ndarray, H: np.ndarray, out_w: int, out_h: int,
               chunk_rows: int = 256) -> np.ndarray:
    """out(p) = bilinear img(H^-1 p), zero outside (float64 result)."""
    Hi = np.linalg.inv(H)
    h, w = img.shape
    src = img.astype(np.float64)
    out = np.zeros((out_h, out_w), dtype=np.float64)
    xs = np.arange(out_w, dtype=np.float64)
    for r0 in range(0, out_h, chunk_rows):
        r1 = min(out_h, r0 + chunk_rows)
        yy, xx = np.meshgrid(np.arange(r0, r1, dtype=np.float64), xs, indexing="ij")
        den = Hi[2, 0] * xx + Hi[2, 1] * yy + Hi[2, 2]
        sx = (Hi[0, 0] * xx + Hi[0, 1] * yy + Hi[0, 2]) / den
        sy = (Hi[1, 0] * xx + Hi[1, 1] * yy + Hi[1, 2]) / den
        x0 = np.floor(sx)
        y0 = np.floor(sy)
        fx = sx - x0
        fy = sy - y0
        x0 = x0.astype(np.int64)
        y0 = y0.astype(np.int64)
        acc = np.zeros_like(sx)
        for dy, wy in ((0, 1.0 - fy), (1, fy)):
            for dx, wx in ((0, 1.0 - fx), (1, fx)):
                xi = x0 + dx
                yi = y0 + dy
                ok = (xi >= 0) & (xi < w) & (yi >= 0) & (yi < h)
                v = np.where(ok, src[np.clip(yi, 0, h - 1), np.clip(xi, 0, w - 1)], 0.0)
                acc += wy * wx * v
        out[r0:r1] = acc
    return out


# --------------------------------------------------------------------------
# keypoints (x, y, scale, angle) float32, pixel centres at integers
# --------------------------------------------------------------------------


def make_keypoints(n: int, w: int, h: int, rng: np.random.Generator, border: float = 32.0,
                   scales=(1.0,), angle_bins: int | None = 32) -> np.ndarray:
    """float32 [n, 4]; x, y uniform inside the border; scale drawn from ``scales``;
    angle = 2*pi*U{0..angle_bins-1}/angle_bins, or U[0, 2*pi) if angle_bins is None."""
    kp = np.empty((n, 4), dtype=np.float32)
    kp[:, 0] = rng.uniform(border, w - border, size=n)
    kp[:, 1] = rng.uniform(border, h - border, size=n)
    kp[:, 2] = np.asarray(scales, dtype=np.float32)[rng.integers(0, len(scales), size=n)]
    if angle_bins is None:
        kp[:, 3] = rng.uniform(0.0, 2.0 * math.pi, size=n)
    else:
        kp[:, 3] = (2.0 * math.pi / angle_bins) * rng.integers(0, angle_bins, size=n)
    return kp


# --------------------------------------------------------------------------
# descriptor parameters (stand-ins for the learned ones)
# --------------------------------------------------------------------------


@dataclass
class BadParams:
    """K box pairs: centres [K,2,2] uint8 (box, (x,y)) in the 32x32 patch frame,
    sides [K] uint8, thresholds thr_num[K]/thr_den, plus the scale pyramid."""
    centres: np.ndarray
    sides: np.ndarray
    thr_num: np.ndarray
    thr_den: int
    level_scales: np.ndarray
    n_angle_bins: int = 32

    @property
    def nbits(self) -> int:
        return int(self.sides.shape[0])


def make_bad_params(nbits: int, rng: np.random.Generator, side_range=(1, 7), thr_range=(-20, 20),
                    level_scales=(1.0,), n_angle_bins: int = 32, thr_den: int = 1) -> BadParams:
    centres = rng.integers(0, 32, size=(nbits, 2, 2)).astype(np.uint8)
    sides = rng.integers(side_range[0], side_range[1] + 1, size=nbits).astype(np.uint8)
    thr = rng.integers(thr_range[0] * thr_den, thr_range[1] * thr_den + 1, size=nbits).astype(np.int32)
    return BadParams(centres, sides, thr, int(thr_den),
                     np.asarray(level_scales, dtype=np.float32), n_angle_bins)


def pyramid_scales(levels: int = 5, factor: float = 1.2) -> np.ndarray:
    return np.asarray([factor ** l for l in range(levels)], dtype=np.float32)


@dataclass
class HashSiftParams:
    """Projection W [128, K] float32 and offset b [K] float32 (B = [W^T | b])."""
    W: np.ndarray
    b: np.ndarray
    spacing: float = 1.0

    @property
    def nbits(self) -> int:
        return int(self.W.shape[1])


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """float32 values rounded to the nearest bfloat16 (ties to even), as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def make_hashsift_params(nbits: int, rng: np.random.Generator, spacing: float = 1.0,
                         bf16: bool = False) -> HashSiftParams:
    """W ~ N(0, 1/128) (rounded to bfloat16 values if bf16); zero-mean offset
    b_k = -(1/sqrt(128)) * sum_i W_ik, which centres the projection of a flat
    unit-norm histogram."""
    W = rng.normal(0.0, 1.0 / math.sqrt(128.0), size=(128, nbits)).astype(np.float32)
    if bf16:
        W = round_to_bf16(W)
    b = (-(W.astype(np.float64).sum(axis=0)) / math.sqrt(128.0)).astype(np.float32)
    return HashSiftParams(W, b, float(spacing))


# --------------------------------------------------------------------------
# whole workloads
# --------------------------------------------------------------------------


@dataclass
class ImagePairWorkload:
    """Two images (B = A + N(0,5) noise) and shared keypoints."""
    img_a: np.ndarray
    img_b: np.ndarray
    kps_a: np.ndarray
    kps_b: np.ndarray
    bad: BadParams
    hs: HashSiftParams


def plain_workload(seed: int = 1000, w: int = 640, h: int = 480, n_kp: int = 1000,
                   bad_bits: int = 256, hs_bits: int = 256) -> ImagePairWorkload:
    """One 640x480 image, its noisy copy, 1000 keypoints (scale 1, 32 angle bins)."""
    rng = np.random.default_rng(seed)
    a = make_image(w, h, rng)
    b = add_noise(a, rng, 5.0)
    kps = make_keypoints(n_kp, w, h, rng, border=32.0, scales=(1.0,), angle_bins=32)
    bad = make_bad_params(bad_bits, rng)
    hs = make_hashsift_params(hs_bits, rng)
    return ImagePairWorkload(a, b, kps, kps.copy(), bad, hs)


def large_pair_workload(seed: int = 1004, w: int = 3840, h: int = 2160, n_kp: int = 20000,
                        bad_bits: int = 256, hs_bits: int = 512, border: float = 32.0) -> ImagePairWorkload:
    """Image A, B = A under a random homography plus N(0,5); A's keypoints are
    projected into B and kept if inside the border, the rest drawn at random."""
    rng = np.random.default_rng(seed)
    a = make_image(w, h, rng)
    H = random_homography(rng, w, h)
    b = np.clip(np.rint(warp_image(a, H, w, h) + rng.normal(0.0, 5.0, size=(h, w))), 0, 255).astype(np.uint8)
    kps_a = make_keypoints(n_kp, w, h, rng, border=border, scales=(1.0,), angle_bins=None)
    pts = np.concatenate([kps_a[:, :2].astype(np.float64), np.ones((n_kp, 1))], axis=1) @ H.T
    pts = pts[:, :2] / pts[:, 2:3]
    inside = (pts[:, 0] >= border) & (pts[:, 0] < w - border) & (pts[:, 1] >= border) & (pts[:, 1] < h - border)
    kps_b = make_keypoints(n_kp, w, h, rng, border=border, scales=(1.0,), angle_bins=None)
    kps_b[inside, 0] = pts[inside, 0]
    kps_b[inside, 1] = pts[inside, 1]
    kps_b[inside, 3] = kps_a[inside, 3]
    bad = make_bad_params(bad_bits, rng)
    hs = make_hashsift_params(hs_bits, rng)
    return ImagePairWorkload(a, b, kps_a, kps_b, bad, hs)


@dataclass
class BatchWorkload:
    images: list
    kps: np.ndarray          # float32 [total, 4], image-major
    kp_offsets: np.ndarray   # int32 [n_img + 1]
    bad: BadParams
    hs: HashSiftParams


def batch_workload(seed: int = 1002, n_img: int = 64, total_kp: int = 200_000,
                   bad_bits: int = 512, hs_bits: int = 512, size_range=((480, 1920), (360, 1080)),
                   kp_range=(500, 8000), levels: int = 5) -> BatchWorkload:
    """64 images of seeded sizes, log-uniform keypoint counts rescaled to the
    total, scales on a 5-level 1.2 pyramid, continuous angles."""
    rng = np.random.default_rng(seed)
    ws = rng.integers(size_range[0][0], size_range[0][1] + 1, size=n_img)
    hs_ = rng.integers(size_range[1][0], size_range[1][1] + 1, size=n_img)
    raw = np.exp(rng.uniform(math.log(kp_range[0]), math.log(kp_range[1]), size=n_img))
    counts = np.floor(raw * (total_kp / raw.sum())).astype(np.int64)
    counts[: total_kp - int(counts.sum())] += 1
    scales = pyramid_scales(levels)
    border = math.ceil(16 * math.sqrt(2) * float(scales[-1]) + 4 * float(scales[-1])) + 1
    images, kps = [], []
    for i in range(n_img):
        images.append(make_image(int(ws[i]), int(hs_[i]), rng))
        kps.append(make_keypoints(int(counts[i]), int(ws[i]), int(hs_[i]), rng, border=border,
                                  scales=tuple(float(s) for s in scales), angle_bins=None))
    offs = np.zeros(n_img + 1, dtype=np.int32)
    offs[1:] = np.cumsum(counts)
    bad = make_bad_params(bad_bits, rng, level_scales=tuple(float(s) for s in scales))
    hs = make_hashsift_params(hs_bits, rng, bf16=True)
    return BatchWorkload(images, np.concatenate(kps, axis=0), offs, bad, hs)


@dataclass
class TripletWorkload:
    """Anchor, positive, negative 32x32 float32 patches: [3, N, 32, 32]."""
    patches: np.ndarray


def _sample_patches(img: np.ndarray, cx, cy, A) -> np.ndarray:
    """m 32x32 bilinear crops: p(i,j) = img(c + A @ (j-15.5, i-15.5)), edge-clamped.
    cx, cy: [m]; A: [m, 2, 2]."""
    h, w = img.shape
    jj, ii = np.meshgrid(np.arange(32) - 15.5, np.arange(32) - 15.5)
    sx = cx[:, None, None] + A[:, 0, 0, None, None] * jj + A[:, 0, 1, None, None] * ii
    sy = cy[:, None, None] + A[:, 1, 0, None, None] * jj + A[:, 1, 1, None, None] * ii
    x0 = np.floor(sx)
    y0 = np.floor(sy)
    fx = sx - x0
    fy = sy - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    src = img.astype(np.float32)

    def at(yy, xx):
        return src[np.clip(yy, 0, h - 1), np.clip(xx, 0, w - 1)]
    return ((1 - fy) * ((1 - fx) * at(y0, x0) + fx * at(y0, x0 + 1))
            + fy * ((1 - fx) * at(y0 + 1, x0) + fx * at(y0 + 1, x0 + 1)))


def triplet_workload(seed: int = 1003, n: int = 65536, n_images: int = 4,
                     w: int = 640, h: int = 480, chunk: int = 4096) -> "TripletWorkload":
    """Positive = anchor region under rotation U(+-15 deg), scale U[0.9, 1.1],
    plus N(0, 5) noise; negatives = random patches elsewhere.  The random
    draws are taken chunk by chunk in a fixed order; the patch sampling of
    each chunk (numpy, which releases the GIL) runs on a thread pool, so the
    result does not depend on the thread count."""
    import concurrent.futures as cf
    import os
    rng = np.random.default_rng(seed)
    imgs = [make_image(w, h, rng) for _ in range(n_images)]
    out = np.empty((3, n, 32, 32), dtype=np.float32)
    eye = np.eye(2)

    def fill(c0, m, src, cx, cy, A, noise, src2, nx, ny):
        I = np.broadcast_to(eye, (m, 2, 2))
        for im in range(n_images):
            sel = np.nonzero(src == im)[0]
            if len(sel):
                out[0, c0 + sel] = _sample_patches(imgs[im], cx[sel], cy[sel], I[sel])
                out[1, c0 + sel] = _sample_patches(imgs[im], cx[sel], cy[sel], A[sel]) + noise[sel]
            sel2 = np.nonzero(src2 == im)[0]
            if len(sel2):
                out[2, c0 + sel2] = _sample_patches(imgs[im], nx[sel2], ny[sel2], I[sel2])

    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        pending = []
        for c0 in range(0, n, chunk):
            m = min(chunk, n - c0)
            src = rng.integers(0, n_images, size=m)
            cx = rng.uniform(40, w - 40, size=m)
            cy = rng.uniform(40, h - 40, size=m)
            a = np.radians(rng.uniform(-15, 15, size=m))
            s = rng.uniform(0.9, 1.1, size=m)
            A = np.empty((m, 2, 2))
            A[:, 0, 0] = s * np.cos(a)
            A[:, 0, 1] = -s * np.sin(a)
            A[:, 1, 0] = s * np.sin(a)
            A[:, 1, 1] = s * np.cos(a)
            noise = rng.normal(0.0, 5.0, size=(m, 32, 32))
            src2 = rng.integers(0, n_images, size=m)
            nx = rng.uniform(40, w - 40, size=m)
            ny = rng.uniform(40, h - 40, size=m)
            pending.append(ex.submit(fill, c0, m, src, cx, cy, A, noise, src2, nx, ny))
            if len(pending) >= 2 * workers:
                pending.pop(0).result()
        for f in pending:
            f.result()
    return TripletWorkload(out)


class SelectWorkload:
    """Inputs of one feature-selection round: uint8 triplet patches, the
    similarities of the bits chosen before, candidate box pairs."""

    def __init__(self, patches, sim_ap, sim_an, tau, centres, sides):
        self.patches = patches
        self.sim_ap = sim_ap
        self.sim_an = sim_an
        self.tau = tau
        self.centres = centres
        self.sides = sides


def select_workload(seed: int = 1005, n: int = 65536, J: int = 1000, prev_bits: int = 128,
                    max_side: int = 15) -> SelectWorkload:
    """n triplets of uint8 32x32 patches (the training generator, rounded),
    similarities of `prev_bits` earlier bits drawn as 2 Binomial(prev_bits, p) -
    prev_bits with p = 0.8 for matching and 0.5 for non-matching pairs, margin
    tau = prev_bits / 2, and J candidates: centres U{0..31}^2, sides U{1..max_side}."""
    rng = np.random.default_rng(seed)
    tw = triplet_workload(seed, n=n)
    patches = np.clip(np.rint(tw.patches), 0, 255).astype(np.uint8)
    sim_ap = (2 * rng.binomial(prev_bits, 0.8, size=n) - prev_bits).astype(np.int32)
    sim_an = (2 * rng.binomial(prev_bits, 0.5, size=n) - prev_bits).astype(np.int32)
    centres = rng.integers(0, 32, size=(J, 4)).astype(np.int32)
    sides = rng.integers(1, max_side + 1, size=J).astype(np.int32)
    return SelectWorkload(patches, sim_ap, sim_an, prev_bits // 2, centres, sides)
