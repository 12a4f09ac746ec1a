"""Python face of the oracle for inline 3-vector compression.

TEST INFRASTRUCTURE ONLY: the oracle is a plain, slow CPU implementation of
what the compressed-vector hot path computes (Trojak & Witherden, arXiv
2003.02633, Sec. 2-3 and Sec. 5), written in C (``ivc_oracle.c``) and reached
here through ctypes.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this module.  It imports nothing from the CUDA package,
and the CUDA package never imports it.

Every function takes NumPy arrays on the host:
  * vectors are float32 arrays of shape (n, 3) (array-of-structures),
  * packed words are uint64 arrays of shape (n,).

Parity status of each function is recorded in the module docstrings of the
pin tests (``tests/test_oracle_pins.py``; ``tests/test_oracle_fdiv.py`` for the
flux divergence of Algorithm 1); every function here is pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, astuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ivc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libivc_oracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle with the host gcc into ``oracle/_build``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-Wall", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


@dataclass(frozen=True)
class Format:
    """Bit layout <s,e,m>-p-t plus the angle map (Fig. comp_regimes, Sec. 2.4-2.5).

    map: 0 uniform (Eq. a_disc), 1 tanh companding (Sec. 2.5),
         2 fractional split (Eq. q_split, ``nphi_max_p1`` = n_phi_max + 1).
    """
    sign_bits: int = 0
    exp_bits: int = 7
    man_bits: int = 22
    phi_bits: int = 17
    theta_bits: int = 18
    exp_bias: int = 80
    map: int = 0
    underflow_mode: int = 0
    overflow_mode: int = 0
    gamma: float = 0.5
    nphi_max_p1: int = 0


PRIMARY = Format()                                              # <0,7,22>-17-18
L1617 = Format(0, 8, 23, 16, 17, 127)                           # <0,8,23>-16-17
L1717 = Format(0, 7, 23, 17, 17, 80)                            # <0,7,23>-17-17
BASE = Format(1, 8, 23, 16, 16, 127)                            # <1,8,23>-16-16
TANH = Format(map=1, gamma=0.5)
FRACSPLIT = Format(map=2, nphi_max_p1=185363)


class _CFormat(ctypes.Structure):
    _fields_ = [("sign_bits", ctypes.c_int32), ("exp_bits", ctypes.c_int32),
                ("man_bits", ctypes.c_int32), ("phi_bits", ctypes.c_int32),
                ("theta_bits", ctypes.c_int32), ("exp_bias", ctypes.c_int32),
                ("map", ctypes.c_int32), ("underflow_mode", ctypes.c_int32),
                ("overflow_mode", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("nphi_max_p1", ctypes.c_int64)]


class _CCounts(ctypes.Structure):
    _fields_ = [("n_overflow", ctypes.c_int64), ("n_underflow", ctypes.c_int64),
                ("n_nonfinite", ctypes.c_int64), ("n_quad_angle", ctypes.c_int64),
                ("n_quad_decode", ctypes.c_int64)]


class _CStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("mean", "sd", "max", "mean_rel", "max_rel", "max_ang", "rms_ang",
                 "max_mag_rel", "rms_mag_rel")] + [("n", ctypes.c_int64)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(os.environ.get("IVC_ORACLE_LIB") or build())
        P = ctypes.POINTER
        f, c, st = P(_CFormat), P(_CCounts), P(_CStats)
        vp, i64, flt = ctypes.c_void_p, ctypes.c_int64, ctypes.c_float
        lib.ivco_encode.restype = ctypes.c_uint64
        lib.ivco_encode.argtypes = [f, flt, flt, flt, c]
        lib.ivco_compress.argtypes = [f, vp, i64, vp, c]
        lib.ivco_decompress.argtypes = [f, vp, i64, vp, c]
        lib.ivco_add.argtypes = [f, vp, vp, vp, i64, c]
        lib.ivco_axpy.argtypes = [f, flt, vp, vp, i64, c]
        lib.ivco_update.argtypes = [f, flt, vp, vp, vp, vp, vp, i64, c]
        lib.ivco_decode_exact.argtypes = [f, ctypes.c_uint64, vp]
        lib.ivco_fields.argtypes = [f, ctypes.c_uint64, vp]
        lib.ivco_nmax.argtypes = [f, vp]
        lib.ivco_bin_coords.argtypes = [f, flt, flt, flt, vp]
        lib.ivco_error_stats.argtypes = [vp, vp, i64, st]
        _lib = lib
    return _lib


def _cf(fmt: Format) -> _CFormat:
    d = dict(zip([n for n, _ in _CFormat._fields_ if n != "pad_"], ()))
    del d
    return _CFormat(fmt.sign_bits, fmt.exp_bits, fmt.man_bits, fmt.phi_bits,
                    fmt.theta_bits, fmt.exp_bias, fmt.map, fmt.underflow_mode,
                    fmt.overflow_mode, 0, float(fmt.gamma), int(fmt.nphi_max_p1))


def _vec(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        a = a.reshape(-1, 3)
    return a


def _words(w) -> np.ndarray:
    return np.ascontiguousarray(w, dtype=np.uint64).reshape(-1)


def _counts(c: _CCounts) -> dict:
    return {k: int(getattr(c, k)) for k, _ in _CCounts._fields_}


def nmax(fmt: Format) -> tuple[int, int]:
    """(n_theta_max, n_phi_max) of a format."""
    out = np.zeros(2, np.int64)
    _L().ivco_nmax(ctypes.byref(_cf(fmt)), out.ctypes.data)
    return int(out[0]), int(out[1])


def encode1(fmt: Format, x: float, y: float, z: float) -> int:
    return int(_L().ivco_encode(ctypes.byref(_cf(fmt)), x, y, z, None))


def compress(fmt: Format, xyz, return_counts: bool = False):
    """FP32 (n,3) -> uint64 (n,) words (Sec. 2-3)."""
    v = _vec(xyz)
    w = np.zeros(v.shape[0], np.uint64)
    c = _CCounts()
    _L().ivco_compress(ctypes.byref(_cf(fmt)), v.ctypes.data, v.shape[0], w.ctypes.data,
                       ctypes.byref(c))
    return (w, _counts(c)) if return_counts else w


def decompress(fmt: Format, w, return_counts: bool = False):
    """uint64 (n,) words -> FP32 (n,3), each component rounded away from zero."""
    ww = _words(w)
    out = np.zeros((ww.shape[0], 3), np.float32)
    c = _CCounts()
    _L().ivco_decompress(ctypes.byref(_cf(fmt)), ww.ctypes.data, ww.shape[0], out.ctypes.data,
                         ctypes.byref(c))
    return (out, _counts(c)) if return_counts else out


def decode_exact(fmt: Format, w) -> np.ndarray:
    """uint64 words -> unrounded decoded vectors, as FP64 (n,3)."""
    ww = _words(w)
    out = np.zeros((ww.shape[0], 3), np.float64)
    lib, cf = _L(), _cf(fmt)
    for i, x in enumerate(ww):
        lib.ivco_decode_exact(ctypes.byref(cf), int(x), out[i].ctypes.data)
    return out


def fields(fmt: Format, w) -> np.ndarray:
    """uint64 words -> int64 (n,4): exponent field, mantissa field, n_theta, n_phi."""
    ww = _words(w)
    out = np.zeros((ww.shape[0], 4), np.int64)
    lib, cf = _L(), _cf(fmt)
    for i, x in enumerate(ww):
        lib.ivco_fields(ctypes.byref(cf), int(x), out[i].ctypes.data)
    return out


def bin_coords(fmt: Format, xyz) -> np.ndarray:
    """Pre-rounding bin coordinates (t_theta, t_phi) of each vector, (n,2) FP64."""
    v = _vec(xyz)
    out = np.zeros((v.shape[0], 2), np.float64)
    lib, cf = _L(), _cf(fmt)
    for i in range(v.shape[0]):
        lib.ivco_bin_coords(ctypes.byref(cf), float(v[i, 0]), float(v[i, 1]), float(v[i, 2]),
                            out[i].ctypes.data)
    return out


def add(fmt: Format, a, b) -> np.ndarray:
    """c = compress(decompress(a) + decompress(b)) (Sec. 5)."""
    aa, bb = _words(a), _words(b)
    c = np.zeros_like(aa)
    _L().ivco_add(ctypes.byref(_cf(fmt)), aa.ctypes.data, bb.ctypes.data, c.ctypes.data,
                  aa.shape[0], None)
    return c


def axpy(fmt: Format, alpha: float, x, y) -> np.ndarray:
    """returns compress(fmaf(alpha, decompress(x), decompress(y)))."""
    xx = _words(x)
    yy = _words(y).copy()
    _L().ivco_axpy(ctypes.byref(_cf(fmt)), float(alpha), xx.ctypes.data, yy.ctypes.data,
                   xx.shape[0], None)
    return yy


def update(fmt: Format, dt: float, v, f, rho=None, want_m: bool = False):
    """(v_out, m_out): v_out = compress(fmaf(dt, f^, v^)), m_out = compress(rho * v_new)."""
    vv, ff = _words(v), _words(f)
    n = vv.shape[0]
    vo = np.zeros_like(vv)
    mo = np.zeros_like(vv) if want_m else None
    r = np.ascontiguousarray(rho, dtype=np.float32) if rho is not None else None
    _L().ivco_update(ctypes.byref(_cf(fmt)), float(dt), vv.ctypes.data, ff.ctypes.data,
                     r.ctypes.data if r is not None else None, vo.ctypes.data,
                     mo.ctypes.data if mo is not None else None, n, None)
    return vo, mo


def error_stats(x, xh) -> dict:
    """Eq. (stat) error statistics of stored vectors xh against FP32 inputs x (FP64)."""
    a, b = _vec(x), _vec(xh)
    s = _CStats()
    _L().ivco_error_stats(a.ctypes.data, b.ctypes.data, a.shape[0], ctypes.byref(s))
    return {k: (int(getattr(s, k)) if k == "n" else float(getattr(s, k)))
            for k, _ in _CStats._fields_}


def flux_divergence(fmt: Format, w, D, ns: int, nvars: int) -> np.ndarray:
    """Algorithm 1 (Sec. 4; Table fr_nse, step 10): divergence of a compressed flux.

    ``w`` holds one word per flux row, (point j, row p, element e) at
    ``w[j, p, e]`` (shape (ns, nvars, ne), or flat in that order); each row is
    the 3-vector (F_x, F_y, F_z) of one equation at one solution point.
    ``D`` is the (3 ns, ns) operator, ``D[c * ns + j, k]`` the derivative along
    axis c of the basis function of point j at point k, given as FP32.

    The steps follow the algorithm: for every element and solution point j,
    decompress the point's rows to X (nvars x 3); for every point k, take
    d = (D[j, k], D[j + ns, k], D[j + 2 ns, k]) and accumulate X d into the
    divergence at (k, element).  Accumulation in FP64 (the loop over elements
    is the array axis).  Returns float64 of shape (ns, nvars, ne)."""
    ww = np.asarray(w, dtype=np.uint64).reshape(ns, nvars, -1)
    ne = ww.shape[2]
    X = decompress(fmt, ww.reshape(-1)).reshape(ns, nvars, ne, 3).astype(np.float64)
    DD = np.asarray(D, dtype=np.float32).astype(np.float64).reshape(3 * ns, ns)
    div = np.zeros((ns, nvars, ne), dtype=np.float64)
    for j in range(ns):
        Xj = X[j]
        for k in range(ns):
            d = np.array([DD[j, k], DD[j + ns, k], DD[j + 2 * ns, k]])
            div[k] += Xj @ d
    return div
