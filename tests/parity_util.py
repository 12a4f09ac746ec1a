"""Helpers for GPU-vs-oracle parity: format conversion and the near-boundary
rule for word mismatches.

Words must match the oracle bit for bit, except words whose pre-quantisation
vector lies within FP32 rounding of a quantisation boundary; those are counted
and may make up at most 1e-6 of the words (at least one is always allowed).
A mismatch is near a boundary when the GPU word is the oracle's word of some
FP32 vector within one ulp per component of the oracle's pre-quantisation
vector (for compress that vector is the input itself).
"""
import math

import numpy as np

from oracle import oracle as O
from paper_2003_02633_gb300 import ivc

FORMATS = {
    "primary": dict(),
    "L1617": dict(exp_bits=8, man_bits=23, phi_bits=16, theta_bits=17, exp_bias=127),
    "L1717": dict(exp_bits=7, man_bits=23, phi_bits=17, theta_bits=17, exp_bias=80),
    "base": dict(sign_bits=1, exp_bits=8, man_bits=23, phi_bits=16, theta_bits=16, exp_bias=127),
    "fracsplit": dict(map=2, nphi_max_p1=185363),
    "fracsplit_pow2": dict(map=2, nphi_max_p1=1 << 17),
    "tanh": dict(map=1, gamma=0.5),
    "tiny": dict(exp_bits=3, man_bits=4, phi_bits=4, theta_bits=5, exp_bias=3),
    "ftz_inf": dict(underflow_mode=1, overflow_mode=1),
}


def formats(name):
    kw = FORMATS[name]
    return O.Format(**kw), ivc.make_format(**kw)


def allowed_mismatches(n):
    return max(1, int(math.floor(1e-6 * n)))


def near_boundary(fo, pre, w_gpu):
    """True if w_gpu is the oracle word of an FP32 vector within one ulp per
    component of `pre` (checks the vector, its 6 one-ulp neighbours and the
    26 diagonal ones)."""
    pre = np.asarray(pre, np.float32)
    cands = [pre]
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                u = pre.copy()
                for k, d in enumerate((dx, dy, dz)):
                    if d:
                        u[k] = np.nextafter(u[k], np.float32(np.inf * d))
                cands.append(u)
    with np.errstate(invalid="ignore", over="ignore"):
        words = O.compress(fo, np.stack(cands))
    return int(w_gpu) in set(int(x) for x in words)


def check_words(fo, pre, w_gpu, w_orc, what=""):
    """Assert parity of words; returns the number of (near-boundary) mismatches."""
    w_gpu = np.asarray(w_gpu).view(np.uint64).reshape(-1)
    w_orc = np.asarray(w_orc, np.uint64).reshape(-1)
    bad = np.flatnonzero(w_gpu != w_orc)
    n = w_orc.shape[0]
    assert len(bad) <= allowed_mismatches(n), \
        f"{what}: {len(bad)} mismatches of {n} (first {bad[:5]}, " \
        f"gpu {[hex(int(w_gpu[i])) for i in bad[:3]]}, oracle {[hex(int(w_orc[i])) for i in bad[:3]]})"
    for i in bad:
        assert near_boundary(fo, pre[i], w_gpu[i]), \
            f"{what}: mismatch at {i} not near a boundary: pre={pre[i]!r} " \
            f"gpu={int(w_gpu[i]):#x} oracle={int(w_orc[i]):#x}"
    return len(bad)


def ulp_diff(a, b):
    """Distance in ulps between FP32 arrays (ordered-integer metric; +0 == -0)."""
    a = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
    b = np.asarray(b, np.float32).view(np.int32).astype(np.int64)
    a = np.where(a < 0, np.int64(-2 ** 31) - a, a)
    b = np.where(b < 0, np.int64(-2 ** 31) - b, b)
    return np.abs(a - b)


def check_decoded(got, want, what=""):
    """Decoded FP32 values within 1 ulp of the oracle's (NaN where it is NaN).
    Returns the fraction that is bit-identical."""
    got = np.asarray(got, np.float32)
    want = np.asarray(want, np.float32)
    nan_w = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan_w), what
    g, w = got[~nan_w], want[~nan_w]
    inf_w = np.isinf(w)
    assert np.array_equal(g[inf_w], w[inf_w]), what
    d = ulp_diff(g[~inf_w], w[~inf_w])
    assert d.max(initial=0) <= 1, f"{what}: max ulp diff {d.max()}"
    return float(np.mean(d == 0)) if d.size else 1.0
