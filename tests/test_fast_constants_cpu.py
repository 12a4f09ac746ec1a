"""Host checks of the constants the fast path's bin-coordinate estimate relies
on (no GPU): atan_ratio2 in ivc_fast.cuh, emulated in FP32 with the kernel's
operation order, stays within the error budget that the ambiguity band kEps
assumes (exact side tests run for every fraction within kEps of 1/2)."""
import os
import re

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2003_02633_gb300", "csrc", "ivc_fast.cuh")
F32 = np.float32


def _body(name, end):
    src = open(SRC).read()
    body = src[src.index(name):]
    return body[:body.index(end)]


def _r_coeffs():
    body = _body("void atan_ratio2(", "const float2 sv")
    return [float(x) for x in re.findall(r"bc\((-?[0-9.e-]+)f\)", body)
            if x not in ("1.0", "-0.5")]


def _fma(a, b, c):
    # FP32 products are exact in FP64; the sum is rounded (FP64 then FP32)
    return (a.astype(np.float64) * b + c).astype(F32)


def _atan_ratio(mn, mx):
    """The kernel's steps: approximate reciprocal, float-float quotient,
    q + q^3 R(q^2) with the ql term at slope 1 - q^2/2."""
    m = np.maximum(mx, F32(1e-30))
    # rcp.approx: within an ulp of 1/m; perturbed by up to one ulp either way
    r = (F32(1.0) / m).astype(F32)
    r = np.where(np.arange(r.size) % 3 == 0, np.nextafter(r, F32(np.inf)),
                 np.where(np.arange(r.size) % 3 == 1, np.nextafter(r, F32(0)), r)).astype(F32)
    qh = (mn * r).astype(F32)
    ql = (_fma(-m, qh, mn) * r).astype(F32)
    q2 = (qh * qh).astype(F32)
    c = _r_coeffs()
    R = np.full_like(q2, F32(c[0]))
    for k in c[1:]:
        R = _fma(R, q2, np.full_like(q2, F32(k)))
    sv = ((qh * q2).astype(F32) * R).astype(F32)
    bl = _fma(ql, _fma(q2, np.full_like(q2, F32(-0.5)), np.ones_like(q2)), sv)
    return qh, bl


def _max_err_rad():
    rng = np.random.default_rng(7)
    mx = rng.uniform(0.5, 4.0, 400000).astype(F32)
    mn = (mx * rng.uniform(0.0, 1.0, mx.size)).astype(F32)
    mn = np.minimum(mn, mx)
    # the whole ratio range, with q = 1 and q -> 0 included
    mn[:4] = [mx[0], 0.0, mx[2] * F32(1e-6), mx[3] * F32(0.999999)]
    bh, bl = _atan_ratio(mn, mx)
    exact = np.arctan(mn.astype(np.float64) / mx.astype(np.float64))
    return float(np.abs(bh.astype(np.float64) + bl - exact).max())


def test_r_coefficients_present():
    c = _r_coeffs()
    assert len(c) == 8
    # leading term of atan(q) = q - q^3/3 + ...: R(0) = -1/3
    assert abs(c[-1] + 1.0 / 3.0) < 1e-4


def test_atan_ratio_error():
    assert _max_err_rad() < 5e-8


def test_estimate_flag_band_covers_budget():
    src = open(SRC).read()
    eps = float(re.search(r"kEps = ([0-9.]+)f", src).group(1))
    err = _max_err_rad()
    n_theta, n_phi = (1 << 18) - 1, (1 << 17) - 1
    poly = err * max(n_theta / (2 * np.pi), n_phi / np.pi)
    # rho = sqrt(x^2 + y^2) after one Newton step on the double-float sum:
    # the final FMA's rounding, half an ulp, relative error <= 2^-24 (the
    # Newton residual is quadratic in rsqrt's 2^-22 and negligible);
    # d beta = (rho |z| / (rho^2 + z^2)) d rho / rho <= d rho / (2 rho)
    rho = 2.0 ** -24 / 2 * n_phi / np.pi
    # bin_coord2: C (double-float) times beta rounded once in the tail terms
    tail = 2e-4
    budget = poly + rho + tail
    assert budget < 0.0045
    assert eps >= budget + 0.0005


def test_bin_scale_constants():
    """Each fast layout's bin scales N / (2 pi) (theta) and M / pi (phi) are
    stored as float-float pairs: head = RN32 of the value, tail = RN32 of the
    remainder."""
    from mpmath import mp, mpf, pi
    mp.prec = 200
    src = open(SRC).read()
    geos = {"GeoPrimary": (262143, 131071), "GeoSplit": (185363, 185362),
            "GeoL1717": (131071, 131071), "GeoL1617": (131071, 65535)}
    for g, (N, M) in geos.items():
        body = src[src.index("struct %s {" % g):]
        body = body[:body.index("};")]
        vals = dict(re.findall(r"(C[TP][HL]) = (-?0x[0-9a-fA-Fp.+-]+)f", body))
        assert set(vals) == {"CTH", "CTL", "CPH", "CPL"}, g
        for (h, l), v in (((vals["CTH"], vals["CTL"]), mpf(N) / (2 * pi)),
                          ((vals["CPH"], vals["CPL"]), mpf(M) / pi)):
            hf, lf = float.fromhex(h), float.fromhex(l)
            assert hf == float(np.float32(float(v))), (g, h)
            assert lf == float(np.float32(float(v - mpf(hf)))), (g, l)


@pytest.mark.parametrize("gamma", [0.05, 0.5, 1.0])
def test_tanh_node_interpolation(gamma):
    """The tanh map's fast encoder interpolates the bin coordinate t(a) =
    n_max (tanh(gamma w(a)) + c) / (2c) quadratically from the nearest node
    j pi / 1024 (w = a / pi for |theta|, 2 a / pi - 1 for phi): within 1e-4
    bin of t everywhere, for the largest grids and gamma up to 1; and its
    slope is at most gamma / tanh(gamma) times the uniform map's, the factor
    the estimate's error band kEpsTanh allows for."""
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 80
    rng = np.random.default_rng(17)
    c = float(mp.tanh(gamma))
    for nmax, theta, amax in ((262143, True, np.pi), (131071, False, np.pi / 2)):
        s = nmax / (2 * c)
        dw = 1 / np.pi if theta else 2 / np.pi

        def t(a):
            w = a / mp.pi if theta else 2 * a / mp.pi - 1
            return s * (mp.tanh(gamma * w) + c)

        worst = 0.0
        for a in rng.uniform(0, amax, 300):
            j = round(a * 1024 / np.pi)
            aj = j * np.pi / 1024
            w = aj / np.pi if theta else 2 * aj / np.pi - 1
            th = np.tanh(gamma * w)
            sech2 = 1 - th * th
            d1 = s * gamma * dw * sech2
            d2 = s * gamma ** 2 * dw ** 2 * (-2 * sech2 * th) / 2
            d = a - aj
            est = t(mp.mpf(aj)) + d1 * d + d2 * d * d
            worst = max(worst, float(abs(est - t(mp.mpf(a)))))
        assert worst < 1e-4, (nmax, gamma, worst)
        # slope against the uniform map's n_max / (2 pi) (theta) or n_max / pi (phi)
        uni = nmax / (2 * np.pi) if theta else nmax / np.pi
        assert s * gamma * dw / uni <= gamma / c + 1e-12
    assert gamma / c <= 1.32
    src = open(SRC).read()
    eps = float(re.search(r"kEpsTanh = ([0-9.]+)f", src).group(1))
    assert eps >= 1.32 * 0.0045
