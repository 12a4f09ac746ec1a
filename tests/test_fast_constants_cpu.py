"""Host checks of the constants the fast path's bin-coordinate estimate relies
on (no GPU): the atan polynomial in ivc_fast.cuh, evaluated in FP32 Horner
form exactly as the kernel does, stays within the error budget that the
0.03-bin ambiguity band assumes."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2003_02633_gb300", "csrc", "ivc_fast.cuh")


def _atan_coeffs():
    src = open(SRC).read()
    body = src[src.index("float2 atan01("):]
    body = body[:body.index("return mul2(p, q);")]
    return [float(x) for x in re.findall(r"bc\((-?[0-9.e-]+)f\)", body)]


def test_atan_polynomial_error_budget():
    c = np.array(_atan_coeffs(), dtype=np.float32)
    assert len(c) == 8
    q = np.linspace(0.0, 1.0, 400001).astype(np.float32)
    q2 = (q * q).astype(np.float32)
    p = np.full_like(q, c[0])
    for k in c[1:]:
        p = (p * q2 + k).astype(np.float32)
    r = (p * q).astype(np.float32).astype(np.float64)
    err = np.abs(r - np.arctan(q.astype(np.float64))).max()
    # 2e-7 rad is below 0.01 bin for both angle grids of <0,7,22>-17-18
    assert err < 2e-7
    bins_theta = err * ((1 << 18) - 1) / (2 * np.pi)
    bins_phi = err * ((1 << 17) - 1) / np.pi
    assert max(bins_theta, bins_phi) < 0.01


def test_estimate_flag_band_covers_budget():
    src = open(SRC).read()
    eps = float(re.search(r"kEps = ([0-9.]+)f", src).group(1))
    # polynomial (0.006) + quotient after one Newton step (< 0.0001) + FP32
    # rounding of g, N/4 - g, N/2 - u (0.002 + 0.002 + 0.004) bins
    assert eps >= 0.006 + 0.0001 + 0.008
