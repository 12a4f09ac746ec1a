"""Host checks of the exact-decision arithmetic the CUDA codec falls back to
near rounding boundaries (paper_2003_02633_gb300/csrc/ivc_exact.cuh, compiled
as plain C++ by tests/exact_harness.cpp), against exact rational arithmetic
and 200-bit mpmath:

* pi / (2D) to 64 bits, truncated;
* cos / sin of the grid angles pi m / D within 2^-55 relative, with the
  values the method can hit exactly (0, 1, 1/2) flagged exact and exact;
* the RN32 norm of three FP32 components, exact, including exact ties at a
  rounding midpoint (Pythagorean quadruples), from any candidate within one
  ulp;
* rounding away from zero to FP32 (normal, subnormal, carry into the next
  binade), the product and sum of two 64-bit values (truncation and exact
  flags), and |h + l| of a float-float value.
"""
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS_SRC = os.path.join(ROOT, "tests", "exact_harness.cpp")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++") or shutil.which("c++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("exact") / "harness")
    subprocess.run([gxx, "-std=c++17", "-O2", "-w", "-o", exe, HARNESS_SRC], check=True)

    def run(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                           check=True)
        return [ln.split() for ln in r.stdout.strip().split("\n")]
    return run


def sf(m, e):
    return Fraction(int(m)) * Fraction(2) ** int(e)


def f32_bits(v):
    return int(np.float32(v).view(np.uint32))


def bits_f32(b):
    return float(np.uint32(b).view(np.float32))


def test_pi_over(harness):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 300
    dens = [2, 3, 2 * 262143, 4 * 131071, 2 * 185363, 4 * 185362, 2 * 131071, 4 * 65535, 14, 62]
    out = harness([f"P {d}" for d in dens])
    for d, (m, e) in zip(dens, out):
        m, e = int(m), int(e)
        assert m >> 63 == 1
        exact = mp.pi / d
        v = mp.mpf(m) * mp.mpf(2) ** e
        assert v <= exact < v + mp.mpf(2) ** e      # truncated to 64 bits


def _grid_cases():
    rng = np.random.default_rng(3)
    cases = []
    for D in (262143, 2 * 131071, 185363, 2 * 185362, 131071, 2 * 65535, 31, 2 * 15, 12, 6):
        ms = list(rng.integers(-D, D + 1, 60))
        ms += [0, D, -D, 1, -1, D - 1, D // 2, -(D // 2), D // 3, D // 4, D // 6, 2 * D // 3]
        cases += [(int(m), D) for m in ms]
    return cases


def test_sincospi_grid(harness):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    cases = _grid_cases()
    out = harness([f"S {m} {D}" for m, D in cases])
    for (m, D), r in zip(cases, out):
        cm, ce, cx, sm, se, sx, cn, sn = (int(t) for t in r)
        ang = mp.pi * m / D
        for mag, e, ex, neg, ref in ((cm, ce, cx, cn, mp.cos(ang)), (sm, se, sx, sn, mp.sin(ang))):
            val = sf(mag, e)
            got = -val if neg else val
            rat = None
            # exactly rational values of the grid: 0, +-1/2, +-1 (Niven)
            for q in (Fraction(0), Fraction(1, 2), Fraction(-1, 2), Fraction(1), Fraction(-1)):
                if abs(ref - mp.mpf(q.numerator) / q.denominator) < mp.mpf(2) ** -150:
                    rat = q
            if rat is not None:
                assert ex == 1 and got == rat, (m, D, got, rat)
            else:
                assert ex == 0, (m, D)
                err = abs(mp.mpf(got.numerator) / got.denominator - ref)
                assert err <= abs(ref) * mp.mpf(2) ** -55, (m, D, float(err / abs(ref)))


def _rn32_sqrt(S):
    """RN32 (ties to even) of sqrt(S) for a positive Fraction S in [1, 16)."""
    # value in [1, 4): FP32 grid 2^-23 on [1,2), 2^-22 on [2,4)
    for e in (0, 1):
        lo, hi = Fraction(2) ** e, Fraction(2) ** (e + 1)
        if lo * lo <= S < hi * hi:
            ulp = Fraction(2) ** (e - 23)
            break
    # k = floor(sqrt(S) / ulp) exactly
    k = math.isqrt(int(S / (ulp * ulp)))
    while Fraction(k + 1) ** 2 * ulp * ulp <= S:
        k += 1
    while Fraction(k) ** 2 * ulp * ulp > S:
        k -= 1
    mid = (Fraction(k) + Fraction(1, 2)) * ulp
    if S > mid * mid or (S == mid * mid and k % 2 == 1):
        k += 1
    return float(k * ulp)


def _quadruples(target, count, rng):
    """(a, b, c) with a^2 + b^2 + c^2 = target^2, all below 2^24, from the
    four-square parametrisation."""
    out = []
    t2 = target
    tries = 0
    while len(out) < count and tries < 200000:
        tries += 1
        m = int(rng.integers(0, math.isqrt(t2) + 1))
        rest = t2 - m * m
        n = int(rng.integers(0, math.isqrt(rest) + 1))
        rest -= n * n
        p = int(rng.integers(0, math.isqrt(rest) + 1))
        rest -= p * p
        q = math.isqrt(rest)
        if q * q != rest:
            continue
        a, b, c = abs(m * m + n * n - p * p - q * q), abs(2 * (m * q + n * p)), abs(2 * (n * q - m * p))
        if max(a, b, c) < (1 << 24) and a * a + b * b + c * c == target * target:
            out.append((a, b, c))
    return out


def test_norm_rn(harness):
    rng = np.random.default_rng(11)
    vecs = []
    # random scaled vectors: largest magnitude in [1, 2), the others spread in exponent
    for _ in range(400):
        a = rng.uniform(1.0, 2.0)
        b = a * 2.0 ** rng.uniform(-40, 0)
        c = b * 2.0 ** rng.uniform(-40, 0)
        v = np.float32([a, b, c])
        rng.shuffle(v)
        v *= np.float32(rng.choice([-1.0, 1.0], 3))
        vecs.append(v)
    # exact ties: a^2 + b^2 + c^2 = d^2 with d = 2^24 + 1 (a 25-bit odd integer:
    # an FP32 rounding midpoint once scaled), scaled so that the largest is in [1, 2)
    for d in ((1 << 24) + 1, (1 << 24) + 3, (1 << 25) - 1):
        for a, b, c in _quadruples(d, 6, rng):
            top = max(a, b, c)
            sc = 2.0 ** -(top.bit_length() - 1)
            v = np.float32([a * sc, b * sc, c * sc])
            vecs.append(v)
            for k in range(3):      # one ulp off in each component: no longer a tie
                w = v.copy()
                w[k] = np.nextafter(w[k], np.float32(np.inf))
                if np.max(np.abs(w)) < 2.0:
                    vecs.append(w)
    vecs.append(np.float32([1.0, 0.0, 0.0]))
    vecs.append(np.float32([1.5, 2.0 ** -30, 2.0 ** -60]))
    lines, want = [], []
    for v in vecs:
        S = sum(Fraction(float(x)) ** 2 for x in v)
        r = _rn32_sqrt(S)
        want.append(r)
        for cand in (r, float(np.nextafter(np.float32(r), np.float32(0))),
                     float(np.nextafter(np.float32(r), np.float32(8)))):
            if cand < 1.0:
                continue
            lines.append("N %d %d %d %d" % (f32_bits(v[0]), f32_bits(v[1]), f32_bits(v[2]),
                                            f32_bits(cand)))
    out = harness(lines)
    i = 0
    ties = 0
    for v, r in zip(vecs, want):
        for cand in (r, float(np.nextafter(np.float32(r), np.float32(0))),
                     float(np.nextafter(np.float32(r), np.float32(8)))):
            if cand < 1.0:
                continue
            got = bits_f32(int(out[i][0]))
            assert got == r, (v, cand, got, r)
            i += 1
        S = sum(Fraction(float(x)) ** 2 for x in v)
        k = Fraction(r)
        ties += int(any(S == ((k + s * Fraction(2) ** -24 * (1 if r < 2 else 2)) ** 2)
                        for s in (-1, 1)))
    assert ties >= 3      # the tie cases were really ties


def _ra32_ref(val):
    """Round a positive Fraction away from zero to FP32."""
    f = np.float32(float(val))
    while Fraction(float(f)) < val:
        f = np.nextafter(f, np.float32(np.inf))
    while True:
        g = np.nextafter(f, np.float32(0))
        if Fraction(float(g)) >= val:
            f = g
        else:
            break
    return float(f)


def test_ra32(harness):
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(300):
        m = int(rng.integers(1 << 62, 1 << 63)) * 2 + int(rng.integers(0, 2))
        e = int(rng.integers(-200, -70))       # values around 2^-137 .. 2^-7: normal and subnormal
        cases.append((m, e, 1))
    for e in (-100, -150, -170, -190, -200):
        cases.append(((1 << 63), e, 1))                           # exact powers of two
        cases.append(((1 << 64) - 1, e, 1))                       # carries into the next binade
        cases.append((((1 << 24) - 1) << 40, e, 1))               # exactly representable
    out = harness(["R %d %d %d" % c for c in cases])
    for (m, e, x), r in zip(cases, out):
        got = bits_f32(int(r[0]))
        assert got == _ra32_ref(sf(m, e)), (m, e, got)
    # an inexact value is rounded up even when its bits end on the grid
    inexact = harness(["R %d %d 0" % ((((1 << 24) - 1) << 40), -100)])
    assert bits_f32(int(inexact[0][0])) > float(sf(((1 << 24) - 1) << 40, -100))


def test_mul_add(harness):
    rng = np.random.default_rng(9)
    lines, cases = [], []
    for _ in range(300):
        a = (int(rng.integers(1 << 62, 1 << 63)) << 1) | int(rng.integers(0, 2))
        b = (int(rng.integers(1 << 62, 1 << 63)) << 1) | int(rng.integers(0, 2))
        if rng.random() < 0.3:      # short mantissas: exact products and sums
            a = (a >> 40) << 40
            b = (b >> 40) << 40
        ea, eb = int(rng.integers(-100, 0)), int(rng.integers(-100, 0))
        cases.append((a, ea, b, eb))
        lines.append(f"M {a} {ea} 1 {b} {eb} 1")
        lines.append(f"A {a} {ea} 1 {b} {eb} 1")
    out = harness(lines)
    for k, (a, ea, b, eb) in enumerate(cases):
        for r, exact in ((out[2 * k], sf(a, ea) * sf(b, eb)), (out[2 * k + 1], sf(a, ea) + sf(b, eb))):
            m, e, x = int(r[0]), int(r[1]), int(r[2])
            assert m >> 63 == 1
            v = sf(m, e)
            assert v <= exact < v + sf(1, e)          # truncated
            assert (x == 1) == (v == exact)


def test_from_float_float(harness):
    rng = np.random.default_rng(13)
    lines, cases = [], []
    for _ in range(300):
        h = np.float32(rng.uniform(-1, 1))
        l = np.float32(float(h) * 2.0 ** -24 * rng.uniform(-0.5, 0.5))
        cases.append((h, l))
        lines.append("F %d %d" % (f32_bits(h), f32_bits(l)))
    cases.append((np.float32(0.0), np.float32(0.0)))
    lines.append("F 0 0")
    out = harness(lines)
    for (h, l), r in zip(cases, out):
        m, e, x, neg = (int(t) for t in r)
        exact = Fraction(float(h)) + Fraction(float(l))
        v = sf(m, e) if m else Fraction(0)
        assert (-v if neg else v) == exact and x == 1, (h, l)
