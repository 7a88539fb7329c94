"""Error bound of the orientation polynomial the HashSIFT kernels use for the
first-octant angle u = (4/pi) atan(r), r in [0, 1] (the histogram's soft
orientation vote, Sec. III-B): the coefficients are parsed from the CUDA
source and evaluated here in double precision and in FP32 with fused
multiply-adds, against numpy's arctan.  The histogram tolerance (1e-5 on the
unit vector) needs the vote weight to be exact to about 1e-6."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2108_08380_gb300", "csrc",
                   "hashsift_dev.cuh")


def _coefficients():
    text = open(SRC).read()
    body = text[text.index("orient_bin(float gx"):]
    body = body[:body.index("const float u")]
    first = re.search(r"float p = (-?[0-9.e+-]+)f;", body).group(1)
    rest = re.findall(r"p = fmaf\(p, z, (-?[0-9.e+-]+)f\);", body)
    return [float(first)] + [float(c) for c in rest]


def test_polynomial_error_double_and_fp32():
    c = _coefficients()
    assert len(c) == 8
    r = np.linspace(0.0, 1.0, 2_000_001)[:-1]  # r = 1 is returned as exactly 1
    ref = 4.0 / np.pi * np.arctan(r)
    p = np.zeros_like(r)
    for ci in c:
        p = p * r * r + ci
    assert np.abs(p * r - ref).max() <= 1.05e-7
    # FP32: r and z = r*r rounded to float, each fmaf rounded once
    r32 = r.astype(np.float32)
    z32 = (r32 * r32).astype(np.float32)
    p32 = np.full_like(r32, np.float32(c[0]))
    for ci in c[1:]:
        p32 = (p32.astype(np.float64) * z32.astype(np.float64) + float(np.float32(ci))).astype(np.float32)
    u32 = (p32 * r32).astype(np.float32).astype(np.float64)
    err32 = np.abs(u32 - 4.0 / np.pi * np.arctan(r32.astype(np.float64))).max()
    assert err32 <= 2.2e-7
    # monotone on the grid (bin weights never step backwards)
    assert np.all(np.diff(u32[::1000]) >= 0)
