"""CPU oracle for BAD / HashSIFT extraction and Hamming matching.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product library never loads
it, and it shares no code with the CUDA path.  The arithmetic lives in plain C
(``bd_oracle.c``, integers and double precision, single-threaded); this module
compiles it with gcc on first use and marshals numpy arrays into it.

Every function follows a definition of the paper (Suarez et al., RA-L 2021):
Sec. III-A for the integral image, the box features and the BAD stumps,
Sec. III-B for the HashSIFT histogram and hash, Sec. IV-C for nearest
neighbour matching, Eq. 1 / Eq. 3 for the triplet ranking loss of the
training step (``bd_oracle_train.c``), the feature-selection round
(``bd_oracle_select.c``); the readings taken where the paper is
silent are listed at the top of the two C files.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "bd_oracle.c"), os.path.join(_HERE, "bd_oracle_train.c"),
        os.path.join(_HERE, "bd_oracle_select.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, no OpenMP, no intrinsics)."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    stale = force or not os.path.exists(_LIB_PATH) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB_PATH) for s in srcs)
    if stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, *srcs, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _u8p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _f32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            L.or_box_sum.restype = ctypes.c_int64
            L.or_bad_describe.restype = ctypes.c_int
            L.or_hs_describe.restype = ctypes.c_int
            L.or_hs_hist_raw.restype = ctypes.c_double
            L.or_hamming.restype = ctypes.c_int
            L.or_angle_bin.argtypes = [ctypes.c_float, ctypes.c_int]
            L.or_round_coord.argtypes = [ctypes.c_float]
            L.or_scale_level.argtypes = [ctypes.c_float, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
            L.or_bad_geometry.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint8),
                                          ctypes.POINTER(ctypes.c_uint8), ctypes.c_double,
                                          ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]
        return _lib


def _img(img):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    return img, w, h


# ---------------------------------------------------------------------------
# integral image and box sums (Sec. III-A)
# ---------------------------------------------------------------------------

def integral(img) -> np.ndarray:
    """uint32 [(h+1), (w+1)] summed-area table with a zero first row and column."""
    img, w, h = _img(img)
    ii = np.empty((h + 1, w + 1), dtype=np.uint32)
    lib().or_integral(_u8p(img), w, h, w, _u32p(ii))
    return ii


def box_sum(img, x0: int, y0: int, side: int) -> int:
    img, w, h = _img(img)
    return int(lib().or_box_sum(_u8p(img), w, h, w, int(x0), int(y0), int(side)))


# ---------------------------------------------------------------------------
# keypoint quantisation and BAD (Sec. III-A)
# ---------------------------------------------------------------------------

def round_coord(v: float) -> int:
    return int(lib().or_round_coord(ctypes.c_float(v)))


def angle_bin(angle: float, nbins: int = 32) -> int:
    return int(lib().or_angle_bin(ctypes.c_float(angle), int(nbins)))


def scale_level(scale: float, level_scales) -> int:
    ls = np.ascontiguousarray(level_scales, dtype=np.float32)
    return int(lib().or_scale_level(ctypes.c_float(scale), _f32p(ls), len(ls)))


def bad_geometry(centres, sides, sigma: float, theta: float):
    """(offsets [K,2,2] int (box, (dx,dy)), sides [K] int) at one scale and angle."""
    centres = np.ascontiguousarray(centres, dtype=np.uint8)
    sides = np.ascontiguousarray(sides, dtype=np.uint8)
    K = sides.shape[0]
    off = np.empty((K, 2, 2), dtype=np.int32)
    sp = np.empty(K, dtype=np.int32)
    lib().or_bad_geometry(K, _u8p(centres), _u8p(sides), float(sigma), float(theta),
                          off.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          sp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return off, sp


def bad_describe(img, kps, params):
    """uint32 [n, K/32] BAD descriptors, and the number of invalid keypoints."""
    img, w, h = _img(img)
    kps = np.ascontiguousarray(kps, dtype=np.float32).reshape(-1, 4)
    n = kps.shape[0]
    K = params.nbits
    out = np.zeros((n, K // 32), dtype=np.uint32)
    c = np.ascontiguousarray(params.centres, dtype=np.uint8)
    s = np.ascontiguousarray(params.sides, dtype=np.uint8)
    t = np.ascontiguousarray(params.thr_num, dtype=np.int32)
    ls = np.ascontiguousarray(params.level_scales, dtype=np.float32)
    bad = lib().or_bad_describe(_u8p(img), w, h, w, _f32p(kps), n, K, _u8p(c), _u8p(s), _i32p(t),
                                int(params.thr_den), int(params.n_angle_bins), _f32p(ls), len(ls),
                                _u32p(out))
    return out, int(bad)


# ---------------------------------------------------------------------------
# HashSIFT (Sec. III-B)
# ---------------------------------------------------------------------------

def hs_patches(img, kps, spacing: float = 1.0) -> np.ndarray:
    """float64 [n, 32, 32] bilinear patches (zeros for invalid keypoints)."""
    img, w, h = _img(img)
    kps = np.ascontiguousarray(kps, dtype=np.float32).reshape(-1, 4)
    n = kps.shape[0]
    P = np.zeros((n, 32, 32), dtype=np.float64)
    tmp = np.empty(1024, dtype=np.float64)
    L = lib()
    for i in range(n):
        if not L.or_kp_valid(_f32p(kps[i])):
            continue
        L.or_hs_patch(_u8p(img), w, h, w, _f32p(kps[i]), ctypes.c_double(spacing), _f64p(tmp))
        P[i] = tmp.reshape(32, 32)
    return P


def hs_hist(patches) -> np.ndarray:
    """float64 [n, 128] L2-normalised gradient-orientation histograms."""
    P = np.ascontiguousarray(patches, dtype=np.float64).reshape(-1, 1024)
    n = P.shape[0]
    H = np.empty((n, 128), dtype=np.float64)
    lib().or_hs_hist(_f64p(P), n, _f64p(H))
    return H


HS_TRILINEAR, HS_CLIP, HS_ROOT = 1, 2, 4


def hs_hist_variant(patches, flags: int) -> np.ndarray:
    """float64 [n, 128] histograms with the SIFT variants in `flags`
    (HS_TRILINEAR, HS_CLIP, HS_ROOT), unit L2 norm."""
    P = np.ascontiguousarray(patches, dtype=np.float64).reshape(-1, 1024)
    H = np.empty((P.shape[0], 128), dtype=np.float64)
    for i in range(P.shape[0]):
        lib().or_hs_hist_variant(_f64p(P[i]), int(flags), _f64p(H[i]))
    return H


def hs_hist_raw(patch):
    """(unnormalised histogram [128], its L2 norm) of one 32x32 patch."""
    P = np.ascontiguousarray(patch, dtype=np.float64).reshape(1024)
    H = np.empty(128, dtype=np.float64)
    nrm = lib().or_hs_hist_raw(_f64p(P), _f64p(H))
    return H, float(nrm)


def hs_project(hist, W, b):
    """(margins [n, K] float64, bits [n, K/32] uint32) of D = sgn(W^T h + b)."""
    hist = np.ascontiguousarray(hist, dtype=np.float64).reshape(-1, 128)
    W = np.ascontiguousarray(W, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    n = hist.shape[0]
    K = W.shape[1]
    m = np.empty((n, K), dtype=np.float64)
    bits = np.empty((n, K // 32), dtype=np.uint32)
    lib().or_hs_project(_f64p(hist), n, _f32p(W), _f32p(b), K, _f64p(m), _u32p(bits))
    return m, bits


def hs_describe(img, kps, params, want_patches: bool = False):
    """dict(bits, hist, margins[, patches], invalid) for n keypoints."""
    img, w, h = _img(img)
    kps = np.ascontiguousarray(kps, dtype=np.float32).reshape(-1, 4)
    n = kps.shape[0]
    W = np.ascontiguousarray(params.W, dtype=np.float32)
    b = np.ascontiguousarray(params.b, dtype=np.float32)
    K = W.shape[1]
    bits = np.empty((n, K // 32), dtype=np.uint32)
    hist = np.empty((n, 128), dtype=np.float64)
    marg = np.empty((n, K), dtype=np.float64)
    pat = np.empty((n, 1024), dtype=np.float64) if want_patches else None
    L = lib()
    inv = L.or_hs_describe(_u8p(img), ctypes.c_int(w), ctypes.c_int(h), ctypes.c_int(w), _f32p(kps),
                           ctypes.c_int(n), ctypes.c_double(params.spacing), _f32p(W), _f32p(b),
                           ctypes.c_int(K), _u32p(bits), _f64p(hist), _f64p(marg),
                           _f64p(pat) if pat is not None else ctypes.POINTER(ctypes.c_double)())
    out = dict(bits=bits, hist=hist, margins=marg, invalid=int(inv))
    if pat is not None:
        out["patches"] = pat.reshape(n, 32, 32)
    return out


# ---------------------------------------------------------------------------
# Hamming matching (Sec. III-A similarity, Sec. IV-C nearest neighbour)
# ---------------------------------------------------------------------------

def hamming(a, b) -> int:
    a = np.ascontiguousarray(a, dtype=np.uint32).ravel()
    b = np.ascontiguousarray(b, dtype=np.uint32).ravel()
    return int(lib().or_hamming(_u32p(a), _u32p(b), a.shape[0]))


def match(q, t, nbits: int, ratio_num: int = 4, ratio_den: int = 5):
    """(idx int32, d1 int32, d2 int32, accept uint8) per query."""
    q = np.ascontiguousarray(q, dtype=np.uint32).reshape(-1, nbits // 32)
    t = np.ascontiguousarray(t, dtype=np.uint32).reshape(-1, nbits // 32)
    nq, nt = q.shape[0], t.shape[0]
    idx = np.empty(nq, dtype=np.int32)
    d1 = np.empty(nq, dtype=np.int32)
    d2 = np.empty(nq, dtype=np.int32)
    acc = np.empty(nq, dtype=np.uint8)
    lib().or_match(_u32p(q), nq, _u32p(t), nt, nbits, ratio_num, ratio_den, _i32p(idx), _i32p(d1),
                   _i32p(d2), _u8p(acc))
    return idx, d1, d2, acc


def match_mnn(q, t, nbits: int):
    """Mutual nearest neighbours: int32 [nq], the partner in t or -1 (Sec. V,
    Hamming MNN matching; ties to the lowest index on both sides)."""
    q = np.ascontiguousarray(q, dtype=np.uint32).reshape(-1, nbits // 32)
    t = np.ascontiguousarray(t, dtype=np.uint32).reshape(-1, nbits // 32)
    out = np.empty(q.shape[0], dtype=np.int32)
    lib().or_match_mnn(_u32p(q), q.shape[0], _u32p(t), t.shape[0], nbits, _i32p(out))
    return out


# ---------------------------------------------------------------------------
# training step (Sec. III-A Eq. 1, Sec. III-B Eq. 3; relaxed tanh responses)
# ---------------------------------------------------------------------------

def train_step(patches, bad, theta, hs, T=0.1, tau_bad=None, tau_hs=None, w_bad=1.0, w_hs=1.0,
               fixed_mining=None, want_grads=True, want_r=False):
    """One FP64 training step on [3, n, 32, 32] patches (anchors, positives,
    negatives).  bad: BadParams (box geometry; its level 0 is the patch frame),
    theta: float thresholds [Kb]; hs: HashSiftParams (W, b).  Returns a dict
    with loss [2] (BAD, HashSIFT), mining [4, n] (nstar_bad, xsel_bad,
    nstar_hs, xsel_hs) and, if asked, the gradients of w_bad*L_bad + w_hs*L_hs
    and the relaxed responses."""
    P = np.ascontiguousarray(patches, dtype=np.float64).reshape(-1, 1024)
    rows = P.shape[0]
    n = rows // 3
    Kb, Kh = bad.nbits, hs.nbits
    tau_bad = Kb / 2.0 if tau_bad is None else tau_bad
    tau_hs = Kh / 2.0 if tau_hs is None else tau_hs
    c = np.ascontiguousarray(bad.centres, dtype=np.uint8)
    s = np.ascontiguousarray(bad.sides, dtype=np.uint8)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    W = np.ascontiguousarray(hs.W, dtype=np.float64)
    b = np.ascontiguousarray(hs.b, dtype=np.float64)
    loss = np.zeros(2)
    mining = np.zeros((4, n), dtype=np.int32)
    fm = None if fixed_mining is None else np.ascontiguousarray(fixed_mining, dtype=np.int32)
    out = dict(loss=loss, mining=mining)
    dth = dW = db = dP = rb = rh = None
    if want_grads:
        dth = np.zeros(Kb)
        dW = np.zeros((128, Kh))
        db = np.zeros(Kh)
        dP = np.zeros((rows, 1024))
    if want_r:
        rb = np.zeros((rows, Kb))
        rh = np.zeros((rows, Kh))
    null = ctypes.POINTER(ctypes.c_double)()
    lib().or_train_step(_f64p(P), ctypes.c_int(n), ctypes.c_int(Kb), _u8p(c), _u8p(s), _f64p(th),
                        ctypes.c_int(Kh), _f64p(W), _f64p(b), ctypes.c_double(T),
                        ctypes.c_double(tau_bad), ctypes.c_double(tau_hs), ctypes.c_double(w_bad),
                        ctypes.c_double(w_hs), _i32p(fm) if fm is not None else ctypes.POINTER(ctypes.c_int32)(),
                        _f64p(loss), _i32p(mining),
                        _f64p(dth) if dth is not None else null, _f64p(dW) if dW is not None else null,
                        _f64p(db) if db is not None else null, _f64p(dP) if dP is not None else null,
                        _f64p(rb) if rb is not None else null, _f64p(rh) if rh is not None else null)
    if want_grads:
        out.update(dtheta=dth, dW=dW, db=db, dpatches=dP.reshape(3, n, 32, 32))
    if want_r:
        out.update(r_bad=rb, r_hs=rh)
    return out


def train_codes(patches, bad, theta, hs):
    """Hard codes of all 3n patches: (bits_bad, bits_hs, f_bad, m_hs)."""
    P = np.ascontiguousarray(patches, dtype=np.float64).reshape(-1, 1024)
    rows = P.shape[0]
    n = rows // 3
    Kb, Kh = bad.nbits, hs.nbits
    bb = np.zeros((rows, Kb // 32), dtype=np.uint32)
    bh = np.zeros((rows, Kh // 32), dtype=np.uint32)
    fb = np.zeros((rows, Kb))
    mh = np.zeros((rows, Kh))
    c = np.ascontiguousarray(bad.centres, dtype=np.uint8)
    s = np.ascontiguousarray(bad.sides, dtype=np.uint8)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    W = np.ascontiguousarray(hs.W, dtype=np.float64)
    b = np.ascontiguousarray(hs.b, dtype=np.float64)
    lib().or_train_codes(_f64p(P), ctypes.c_int(n), ctypes.c_int(Kb), _u8p(c), _u8p(s), _f64p(th),
                         ctypes.c_int(Kh), _f64p(W), _f64p(b), _u32p(bb), _u32p(bh), _f64p(fb), _f64p(mh))
    return bb, bh, fb, mh


# ---------------------------------------------------------------------------
# feature selection (Algorithms 1 and 2, integer-sorted thresholds)
# ---------------------------------------------------------------------------

SELECT_QMIN = -2551


def select_key(patch, cand) -> int:
    """ceil(10 (sum1 - sum2) / s^2) of one uint8 32x32 patch; cand = (x1, y1, x2, y2, s)."""
    p = np.ascontiguousarray(patch, dtype=np.uint8).reshape(32, 32)
    c = np.ascontiguousarray(cand, dtype=np.int32)
    return int(lib().or_select_key(_u8p(p), _i32p(c)))


def find_threshold(patches, cand, sap, san, tau: int):
    """Algorithm 2 for one candidate: (theta numerator q, loss); patches [3, n, 32, 32] uint8."""
    P = np.ascontiguousarray(patches, dtype=np.uint8).reshape(3, -1, 32, 32)
    n = P.shape[1]
    c = np.ascontiguousarray(cand, dtype=np.int32)
    a = np.ascontiguousarray(sap, dtype=np.int32)
    b = np.ascontiguousarray(san, dtype=np.int32)
    q = ctypes.c_int32(0)
    loss = ctypes.c_int64(0)
    lib().or_find_threshold(_u8p(P), n, _i32p(c), _i32p(a), _i32p(b), int(tau), ctypes.byref(q),
                            ctypes.byref(loss))
    return int(q.value), int(loss.value)


def select_feature(patches, cands, sap, san, tau: int):
    """Algorithm 1, one round: (theta_q [J], loss [J], best index)."""
    P = np.ascontiguousarray(patches, dtype=np.uint8).reshape(3, -1, 32, 32)
    n = P.shape[1]
    C = np.ascontiguousarray(cands, dtype=np.int32).reshape(-1, 5)
    J = C.shape[0]
    a = np.ascontiguousarray(sap, dtype=np.int32)
    b = np.ascontiguousarray(san, dtype=np.int32)
    tq = np.empty(J, dtype=np.int32)
    loss = np.empty(J, dtype=np.int64)
    best = ctypes.c_int32(-1)
    lib().or_select_feature(_u8p(P), n, _i32p(C), J, _i32p(a), _i32p(b), int(tau), _i32p(tq),
                            loss.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(best))
    return tq, loss, int(best.value)
