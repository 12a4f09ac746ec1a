"""ctypes binding of the C ABI in ``include/ivc.h`` (library ``_build/libivc.so``).

Argument marshalling only: every entry point of the C ABI is exposed under
its own name with the same arguments (pointers as Python ints, stream as a
``cudaStream_t`` integer handle).  Small tensor helpers (``compress``,
``decompress``, ``add`` ...) take torch CUDA tensors, pass their device
pointers and the current stream, and raise ``IvcError`` on a non-OK status.
There is no fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

IVC_OK, IVC_ERR_ARG, IVC_ERR_FORMAT, IVC_ERR_ALIGN, IVC_ERR_CUDA = 0, 1, 2, 3, 4
IVC_ERR_TIMEOUT, IVC_ERR_NOMEM, IVC_ERR_UNSUPPORTED = 5, 6, 7
IVC_AOS, IVC_SOA = 0, 1
IVC_MAP_UNIFORM, IVC_MAP_TANH, IVC_MAP_FRACSPLIT = 0, 1, 2
IVC_F16, IVC_BF16 = 0, 1
IVC_OP_ADD, IVC_OP_AXPY = 0, 1
IVC_STATS_LEN = 11


class IvcError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_string(status)} ({status})")
        self.status = status


class ivc_format(ctypes.Structure):
    _fields_ = [("sign_bits", ctypes.c_int32), ("exp_bits", ctypes.c_int32),
                ("man_bits", ctypes.c_int32), ("phi_bits", ctypes.c_int32),
                ("theta_bits", ctypes.c_int32), ("exp_bias", ctypes.c_int32),
                ("map", ctypes.c_int32), ("underflow_mode", ctypes.c_int32),
                ("overflow_mode", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("nphi_max_p1", ctypes.c_int64)]


class ivc_counts(ctypes.Structure):
    _fields_ = [("n_overflow", ctypes.c_ulonglong), ("n_underflow", ctypes.c_ulonglong),
                ("n_nonfinite", ctypes.c_ulonglong)]


class ivc_field(ctypes.Structure):
    _fields_ = [("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("alpha", ctypes.c_float), ("reserved", ctypes.c_float)]


class ivc_launch_config(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("vec_per_thread", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


class ivc_fr_basis(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("dm", ctypes.c_float * 16),
                ("lm", ctypes.c_float * 4), ("lp", ctypes.c_float * 4),
                ("gl", ctypes.c_float * 4), ("gr", ctypes.c_float * 4)]


class ivc_fr_gas(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_float), ("mu", ctypes.c_float), ("prandtl", ctypes.c_float)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_F = ctypes.c_float
_I = ctypes.c_int
_FMT = ctypes.POINTER(ivc_format)
_BAS = ctypes.POINTER(ivc_fr_basis)
_GAS = ctypes.POINTER(ivc_fr_gas)
_DIMS = ctypes.POINTER(ctypes.c_int)
_SIGS = {
    "ivc_format_default": [_FMT],
    "ivc_format_validate": [_FMT],
    "ivc_release_tables": [],
    "ivc_compress": [_FMT, _P, _I, _I64, _I64, _P, _P, _P],
    "ivc_decompress": [_FMT, _P, _I64, _P, _I, _I64, _P],
    "ivc_compress_exact": [_FMT, _P, _I64, _P, _P, _P],
    "ivc_decompress_exact": [_FMT, _P, _I64, _P, _P],
    "ivc_add": [_FMT, _P, _P, _P, _I64, _P],
    "ivc_add_cfg": [_FMT, _P, _P, _P, _I64, ctypes.POINTER(ivc_launch_config), _P],
    "ivc_axpy": [_FMT, _F, _P, _P, _I64, _P],
    "ivc_pointwise_update": [_FMT, _F, _P, _P, _P, _P, _P, _I64, _P],
    "ivc_f32_add": [_I, _P, _P, _P, _I64, _I64, _P],
    "ivc_f32_axpy": [_I, _F, _P, _P, _I64, _I64, _P],
    "ivc_half_add": [_I, _P, _P, _P, _I64, _P],
    "ivc_half_axpy": [_I, _F, _P, _P, _I64, _P],
    "ivc_half_from_f32": [_I, _P, _P, _I64, _P],
    "ivc_half_to_f32": [_I, _P, _P, _I64, _P],
    "ivc_error_stats": [_P, _P, _I64, _P, _P],
    "ivc_plan_batched": [_FMT, _I, ctypes.POINTER(ivc_field), _I, _P,
                         ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ivc_launch_config), _P,
                         ctypes.POINTER(ctypes.c_void_p)],
    "ivc_launch_plan": [_P, _P],
    "ivc_launch_plan_direct": [_P, _P],
    "ivc_plan_status": [_P, _P],
    "ivc_plan_destroy": [_P],
    "ivc_set_flux_divergence_wait_limit": [ctypes.c_longlong],
    "ivc_tune": [_FMT, _I, _P, _P, _P, _I64, _P, ctypes.POINTER(ivc_launch_config)],
    "ivc_tune_batched": [_FMT, _I, _P, _I, _P, ctypes.c_size_t, _P,
                         ctypes.POINTER(ivc_launch_config)],
    "ivc_add_noalloc": [_FMT, _P, _P, _P, _I64, _P],
    "ivc_flux_divergence": [_FMT, _P, _I64, _I, _I, _I64, _P, _P, _I64, _P],
    "ivc_flux_divergence_simt": [_FMT, _P, _I64, _I, _I, _I64, _P, _P, _I64, _P],
    "ivc_f32_flux_divergence": [_P, _I64, _I, _I, _I64, _P, _P, _I64, _P],
    "ivc_f32_flux_divergence_simt": [_P, _I64, _I, _I, _I64, _P, _P, _I64, _P],
    "ivc_add_host": [_FMT, _P, _P, _P, _I64, _P, ctypes.c_size_t, _P],
    "ivc_flux_divergence_check": [],
    "ivc_gather_decompress": [_FMT, _P, _I64, _P, _I64, _P, _P],
    "ivc_f32_gather": [_I, _P, _I64, _I64, _P, _I64, _P, _P],
    "ivc_fr_gradient": [_FMT, _BAS, _P, _I64, _I64, _I, _P, _P],
    "ivc_f32_fr_gradient": [_BAS, _P, _I64, _I64, _I, _P, _P],
    "ivc_fr_correct_gradient": [_FMT, _BAS, _P, _P, _I64, _I64, _I, _P, _P],
    "ivc_f32_fr_correct_gradient": [_BAS, _P, _P, _I64, _I64, _I, _P, _P],
    "ivc_fr_interp_rows": [_FMT, _BAS, _P, _I64, _I64, _I, _P, _P],
    "ivc_f32_fr_interp_rows": [_BAS, _P, _I64, _I64, _I, _P, _P],
    "ivc_fr_common_viscous_flux": [_FMT, _I, _GAS, _DIMS, _P, _P, _P, _P, _P, _P, _I64, _P, _P],
    "ivc_f32_fr_common_viscous_flux": [_I, _GAS, _DIMS, _P, _P, _P, _P, _P, _P, _I64, _P, _P],
    "ivc_fr_flux": [_FMT, _I, _GAS, _P, _P, _P, _P, _I64, _I64, _P, _P],
    "ivc_f32_fr_flux": [_I, _GAS, _P, _P, _P, _P, _I64, _I64, _P, _P],
    "ivc_fr_flux_correction": [_FMT, _BAS, _P, _P, _I64, _I64, _I, _P, _P],
    "ivc_f32_fr_flux_correction": [_BAS, _P, _P, _I64, _I64, _I, _P, _P],
}
EXPORTS = sorted(list(_SIGS) + ["ivc_status_string", "ivc_version"])

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libivc.so (building it with nvcc when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libivc.so not built ({_build.LIB}); run paper_2003_02633_gb300.build")
    lib = ctypes.CDLL(_build.LIB)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.ivc_status_string.argtypes = [ctypes.c_int]
    lib.ivc_status_string.restype = ctypes.c_char_p
    lib.ivc_version.argtypes = []
    lib.ivc_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def status_string(s: int) -> str:
    return load().ivc_status_string(int(s)).decode()


def _chk(s: int, where: str) -> None:
    if s != IVC_OK:
        raise IvcError(s, where)


def make_format(sign_bits=0, exp_bits=7, man_bits=22, phi_bits=17, theta_bits=18, exp_bias=80,
                map=IVC_MAP_UNIFORM, underflow_mode=0, overflow_mode=0, gamma=0.5,
                nphi_max_p1=0) -> ivc_format:
    """An ivc_format; the defaults are the primary layout <0,7,22>-17-18."""
    return ivc_format(sign_bits, exp_bits, man_bits, phi_bits, theta_bits, exp_bias, map,
                      underflow_mode, overflow_mode, 0, float(gamma), int(nphi_max_p1))


def default_format() -> ivc_format:
    f = ivc_format()
    _chk(load().ivc_format_default(ctypes.byref(f)), "ivc_format_default")
    return f


# ----------------------------------------------------------- tensor helpers

def _stream(stream=None) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _ptr(t) -> int:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def compress(fmt, xyz, out=None, counts=None, stream=None):
    """(n,3) float32 CUDA tensor (AoS) -> (n,) int64 tensor of packed words."""
    import torch
    n = xyz.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=xyz.device)
    _chk(load().ivc_compress(ctypes.byref(fmt), _ptr(xyz), IVC_AOS, 0, n, _ptr(out),
                             _ptr(counts), _stream(stream)), "ivc_compress")
    return out


def compress_soa(fmt, xyz_rows, ld, n, out, stream=None):
    """SoA input: xyz_rows a float32 CUDA tensor holding rows x, y, z at stride ld."""
    _chk(load().ivc_compress(ctypes.byref(fmt), _ptr(xyz_rows), IVC_SOA, ld, n, _ptr(out),
                             None, _stream(stream)), "ivc_compress")
    return out


def decompress(fmt, w, out=None, stream=None):
    """(n,) int64 word tensor -> (n,3) float32 tensor (AoS)."""
    import torch
    n = w.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=w.device)
    _chk(load().ivc_decompress(ctypes.byref(fmt), _ptr(w), n, _ptr(out), IVC_AOS, 0,
                               _stream(stream)), "ivc_decompress")
    return out


def compress_exact(fmt, xyz, out=None, counts=None, stream=None):
    """ivc_compress_exact: every rounding decision by the exact integer path
    (AoS FP32 input of shape (n, 3))."""
    import torch
    n = xyz.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=xyz.device)
    cp = _ptr(counts) if counts is not None else None
    _chk(load().ivc_compress_exact(ctypes.byref(fmt), _ptr(xyz), n, _ptr(out), cp,
                                   _stream(stream)), "ivc_compress_exact")
    return out


def decompress_exact(fmt, w, out=None, stream=None):
    """ivc_decompress_exact: every decoded component by the exact integer path."""
    import torch
    n = w.shape[0]
    if out is None:
        out = torch.empty(n, 3, dtype=torch.float32, device=w.device)
    _chk(load().ivc_decompress_exact(ctypes.byref(fmt), _ptr(w), n, _ptr(out), _stream(stream)),
         "ivc_decompress_exact")
    return out


def add(fmt, a, b, out=None, cfg=None, stream=None):
    import torch
    if out is None:
        out = torch.empty_like(a)
    c = ctypes.byref(cfg) if cfg is not None else None
    _chk(load().ivc_add_cfg(ctypes.byref(fmt), _ptr(a), _ptr(b), _ptr(out), a.shape[0], c,
                            _stream(stream)), "ivc_add")
    return out


def flux_divergence(fmt, F, D, ne=None, out=None, stream=None, simt=False):
    """Algorithm 1: divergence of a compressed flux.  F: int64 words of shape
    (ns, nvars, ld) (element index fastest; the first ``ne`` elements are
    used, default all); D: float32 (3 ns, ns).  Returns float32
    (ns, nvars, ld_out) with ld_out = out.shape[2] (default ld).  ``simt``
    selects the CUDA-core kernel instead of the tensor-core one."""
    import torch
    ns, nv, ld = F.shape
    ne = ld if ne is None else int(ne)
    if out is None:
        out = torch.empty((ns, nv, ld), dtype=torch.float32, device=F.device)
    name = "ivc_flux_divergence_simt" if simt else "ivc_flux_divergence"
    _chk(getattr(load(), name)(ctypes.byref(fmt), _ptr(F), ld, ns, nv, ne, _ptr(D), _ptr(out),
                               out.shape[2], _stream(stream)), name)
    return out


def flux_divergence_check():
    """Raises IvcError if a flux-divergence launch ended early on a bounded
    wait since the last check (synchronises the device)."""
    _chk(load().ivc_flux_divergence_check(), "ivc_flux_divergence_check")


def f32_flux_divergence(F, D, ne=None, out=None, stream=None, simt=False):
    """Algorithm 1 on an uncompressed flux: F float32 of shape (3, ns, nvars, ld)
    (component c of row (j, p) of element e at F[c, j, p, e])."""
    import torch
    _, ns, nv, ld = F.shape
    ne = ld if ne is None else int(ne)
    if out is None:
        out = torch.empty((ns, nv, ld), dtype=torch.float32, device=F.device)
    name = "ivc_f32_flux_divergence_simt" if simt else "ivc_f32_flux_divergence"
    _chk(getattr(load(), name)(_ptr(F), ld, ns, nv, ne, _ptr(D), _ptr(out), out.shape[2],
                               _stream(stream)), name)
    return out


# ------------------------------------------- flux reconstruction, steps 5-11
# Every wrapper takes ``fmt``: an ivc_format for compressed rows (int64 word
# tensors of shape (npts, nrows, ld)), or None for the FP32 baseline (float32
# tensors of shape (3, npts, nrows, ld)).  Scalars are float32 (npts, nv, ld).
# ``ne`` (default ld) elements are processed.


def fr_basis(b: dict) -> ivc_fr_basis:
    """The C struct of a one-dimensional basis given as a dict with ``order``
    and the arrays ``dm`` (q x q, dm[i, a] = l_a'(xi_i)), ``lm``, ``lp``, ``gl``,
    ``gr`` (rounded to FP32)."""
    q = int(b["order"]) + 1
    out = ivc_fr_basis()
    out.order = int(b["order"])
    dm = [float(v) for row in b["dm"] for v in row]
    for i in range(q * q):
        out.dm[i] = dm[i]
    for name in ("lm", "lp", "gl", "gr"):
        arr = getattr(out, name)
        for i in range(q):
            arr[i] = float(b[name][i])
    return out


def fr_gas(gamma: float = 1.4, mu: float = 1.0 / 1600.0, prandtl: float = 0.72) -> ivc_fr_gas:
    return ivc_fr_gas(gamma, mu, prandtl)


def _rows_like(fmt, npts, nrows, ld, device):
    import torch
    if fmt is None:
        return torch.empty((3, npts, nrows, ld), dtype=torch.float32, device=device)
    return torch.empty((npts, nrows, ld), dtype=torch.int64, device=device)


def _fr(name, fmt, *args):
    lib = load()
    if fmt is None:
        _chk(getattr(lib, "ivc_f32_" + name)(*args), "ivc_f32_" + name)
    else:
        _chk(getattr(lib, "ivc_" + name)(ctypes.byref(fmt), *args), "ivc_" + name)


def fr_gradient(fmt, basis, w, ne=None, out=None, stream=None):
    """Step 5: gradient rows of the scalars w (ns, nv, ld) at the solution points."""
    ns, nv, ld = w.shape
    ne = ld if ne is None else int(ne)
    if out is None:
        out = _rows_like(fmt, ns, nv, ld, w.device)
    _fr("fr_gradient", fmt, ctypes.byref(basis), _ptr(w), ne, ld, nv, _ptr(out), _stream(stream))
    return out


def fr_correct_gradient(fmt, basis, grad, dw, ne=None, out=None, stream=None):
    """Step 6: gradient rows plus the lifted jumps dw (nf, nv, ld); out may be grad."""
    nf, nv, ld = dw.shape
    ns = grad.shape[-3]
    ne = ld if ne is None else int(ne)
    if out is None:
        out = _rows_like(fmt, ns, nv, ld, grad.device)
    _fr("fr_correct_gradient", fmt, ctypes.byref(basis), _ptr(grad), _ptr(dw), ne, ld, nv,
        _ptr(out), _stream(stream))
    return out


def fr_interp_rows(fmt, basis, rows, ne=None, out=None, stream=None):
    """Step 7: rows (ns, nv, ld) interpolated to the flux points (nf, nv, ld)."""
    ns, nv, ld = rows.shape[-3:]
    q = round(ns ** (1.0 / 3.0))
    ne = ld if ne is None else int(ne)
    if out is None:
        out = _rows_like(fmt, 6 * q * q, nv, ld, rows.device)
    _fr("fr_interp_rows", fmt, ctypes.byref(basis), _ptr(rows), ne, ld, nv, _ptr(out),
        _stream(stream))
    return out


def fr_common_viscous_flux(fmt, order, gas, dims, grad_f, nrm, S_f, detJ_f, q_f, nFinv,
                           out=None, stream=None):
    """Step 8: n.(F_inv - F_vis^I) (nf, 5, ld) on the periodic dims mesh."""
    import torch
    nf, _, ld = q_f.shape
    if out is None:
        out = torch.empty((nf, 5, ld), dtype=torch.float32, device=q_f.device)
    d = (ctypes.c_int * 3)(*[int(x) for x in dims])
    _fr("fr_common_viscous_flux", fmt, int(order), ctypes.byref(gas), d, _ptr(grad_f), _ptr(nrm),
        _ptr(S_f), _ptr(detJ_f), _ptr(q_f), _ptr(nFinv), ld, _ptr(out), _stream(stream))
    return out


def fr_flux(fmt, order, gas, q_s, grad, S_s, detJ_s, ne=None, out=None, stream=None):
    """Step 9: reference flux rows S (F_inv - F_vis) (ns, 5, ld)."""
    ns, _, ld = q_s.shape
    ne = ld if ne is None else int(ne)
    if out is None:
        out = _rows_like(fmt, ns, 5, ld, q_s.device)
    _fr("fr_flux", fmt, int(order), ctypes.byref(gas), _ptr(q_s), _ptr(grad), _ptr(S_s),
        _ptr(detJ_s), ne, ld, _ptr(out), _stream(stream))
    return out


def fr_flux_correction(fmt, basis, F, nF, ne=None, out=None, stream=None):
    """Step 11: nF (nf, nv, ld) minus the interior normal flux of rows F."""
    import torch
    nf, nv, ld = nF.shape
    ne = ld if ne is None else int(ne)
    if out is None:
        out = torch.empty((nf, nv, ld), dtype=torch.float32, device=nF.device)
    _fr("fr_flux_correction", fmt, ctypes.byref(basis), _ptr(F), _ptr(nF), ne, ld, nv,
        _ptr(out), _stream(stream))
    return out


def add_host(fmt, a, b, out, workspace=None, stream=None):
    """ivc_add_host: c = a + b for int64 word tensors in host memory.  Pinned
    tensors are read and written by the kernel directly; pageable ones stream
    through the device tensor ``workspace`` (any dtype, 16-byte aligned) in
    chunks.  Asynchronous on ``stream``: synchronise before reading ``out``."""
    for t in (a, b, out):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("add_host expects contiguous host tensors")
    ws_ptr = _ptr(workspace) if workspace is not None else None
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _chk(load().ivc_add_host(ctypes.byref(fmt), a.data_ptr(), b.data_ptr(), out.data_ptr(),
                             a.shape[0], ws_ptr, ws_bytes, _stream(stream)), "ivc_add_host")
    return out


def gather_decompress(fmt, w, idx, out=None, stream=None):
    """xyz[i] = decompress(w[idx[i]]): w (nw,) int64 words, idx (n,) int64 CUDA
    tensors; returns (n, 3) float32 (NaN rows for out-of-range indices)."""
    import torch
    n = idx.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=idx.device)
    _chk(load().ivc_gather_decompress(ctypes.byref(fmt), _ptr(w), w.shape[0], _ptr(idx), n,
                                      _ptr(out), _stream(stream)), "ivc_gather_decompress")
    return out


def f32_gather(src, idx, out=None, layout=IVC_AOS, ld=0, nsrc=None, stream=None):
    """out[i] = src vector idx[i]: AoS src (nsrc, 3) or SoA rows at stride ld."""
    import torch
    n = idx.shape[0]
    nsrc = (src.shape[0] if layout == IVC_AOS else ld) if nsrc is None else nsrc
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=idx.device)
    _chk(load().ivc_f32_gather(layout, _ptr(src), ld, nsrc, _ptr(idx), n, _ptr(out),
                               _stream(stream)), "ivc_f32_gather")
    return out


def add_noalloc(fmt, a, b, out, stream=None):
    """ivc_add_noalloc: the compressed add with its tables in the library's fixed
    device array (no device allocation); `out` must be given."""
    _chk(load().ivc_add_noalloc(ctypes.byref(fmt), _ptr(a), _ptr(b), _ptr(out), a.shape[0],
                                _stream(stream)), "ivc_add_noalloc")
    return out


def axpy(fmt, alpha, x, y, stream=None):
    """In place: y <- compress(alpha * x^ + y^)."""
    _chk(load().ivc_axpy(ctypes.byref(fmt), float(alpha), _ptr(x), _ptr(y), x.shape[0],
                         _stream(stream)), "ivc_axpy")
    return y


def pointwise_update(fmt, dt, v, f, rho=None, v_out=None, m_out=None, stream=None):
    import torch
    if v_out is None:
        v_out = torch.empty_like(v)
    _chk(load().ivc_pointwise_update(ctypes.byref(fmt), float(dt), _ptr(v), _ptr(f), _ptr(rho),
                                     _ptr(v_out), _ptr(m_out), v.shape[0], _stream(stream)),
         "ivc_pointwise_update")
    return v_out, m_out


def f32_add(a, b, out=None, layout=IVC_AOS, ld=0, n=None, stream=None):
    import torch
    if out is None:
        out = torch.empty_like(a)
    n = a.shape[0] if n is None else n
    _chk(load().ivc_f32_add(layout, _ptr(a), _ptr(b), _ptr(out), ld, n, _stream(stream)),
         "ivc_f32_add")
    return out


def f32_axpy(alpha, x, y, layout=IVC_AOS, ld=0, n=None, stream=None):
    n = x.shape[0] if n is None else n
    _chk(load().ivc_f32_axpy(layout, float(alpha), _ptr(x), _ptr(y), ld, n, _stream(stream)),
         "ivc_f32_axpy")
    return y


def half_from_f32(kind, xyz, out=None, stream=None):
    import torch
    n = xyz.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=torch.int16, device=xyz.device)
    _chk(load().ivc_half_from_f32(kind, _ptr(xyz), _ptr(out), n, _stream(stream)),
         "ivc_half_from_f32")
    return out


def half_to_f32(kind, h, out=None, stream=None):
    import torch
    n = h.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=h.device)
    _chk(load().ivc_half_to_f32(kind, _ptr(h), _ptr(out), n, _stream(stream)), "ivc_half_to_f32")
    return out


def half_add(kind, a, b, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty_like(a)
    _chk(load().ivc_half_add(kind, _ptr(a), _ptr(b), _ptr(out), a.shape[0], _stream(stream)),
         "ivc_half_add")
    return out


def half_axpy(kind, alpha, x, y, stream=None):
    _chk(load().ivc_half_axpy(kind, float(alpha), _ptr(x), _ptr(y), x.shape[0], _stream(stream)),
         "ivc_half_axpy")
    return y


def error_stats(x, xh, out=None, stream=None):
    """FP64 error statistics of xh against x; returns the accumulated 11 doubles."""
    import torch
    if out is None:
        out = torch.zeros(IVC_STATS_LEN, dtype=torch.float64, device=x.device)
    _chk(load().ivc_error_stats(_ptr(x), _ptr(xh), x.shape[0], _ptr(out), _stream(stream)),
         "ivc_error_stats")
    return out


def stats_dict(acc) -> dict:
    """Named statistics from the accumulated ivc_error_stats output."""
    v = [float(x) for x in acc.tolist()]
    n = max(v[0], 1.0)
    mean = v[1] / n
    var = max(0.0, (v[2] - v[1] * v[1] / n) / max(n - 1, 1.0))
    return {"n": int(v[0]), "mean": mean, "sd": var ** 0.5, "max": v[3], "mean_rel": v[4] / n,
            "max_rel": v[5], "rms_ang": (v[6] / n) ** 0.5, "max_ang": v[7],
            "rms_mag_rel": (v[8] / n) ** 0.5, "max_mag_rel": v[9], "n_nonfinite_out": int(v[10])}


class BatchedPlan:
    """ivc_plan_batched over a list of (a, b, c, alpha) tensor fields."""

    def __init__(self, fmt, op, fields, cfg=None, stream=None):
        import torch
        L = load()
        arr = (ivc_field * len(fields))()
        for i, (a, b, c, alpha) in enumerate(fields):
            arr[i] = ivc_field(_ptr(a), _ptr(b) if b is not None else None, _ptr(c), a.shape[0],
                               float(alpha), 0.0)
        self._keep = (fields, arr)
        ws = ctypes.c_size_t(0)
        c = ctypes.byref(cfg) if cfg is not None else None
        _chk(L.ivc_plan_batched(ctypes.byref(fmt), op, arr, len(fields), None, ctypes.byref(ws),
                                c, _stream(stream), None), "ivc_plan_batched(size)")
        dev = fields[0][0].device
        self.workspace = torch.empty(ws.value + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.plan = ctypes.c_void_p()
        _chk(L.ivc_plan_batched(ctypes.byref(fmt), op, arr, len(fields), aligned,
                                ctypes.byref(ws), c, _stream(stream), ctypes.byref(self.plan)),
             "ivc_plan_batched")

    def launch(self, stream=None, graph=True):
        fn = load().ivc_launch_plan if graph else load().ivc_launch_plan_direct
        _chk(fn(self.plan, _stream(stream)), "ivc_launch_plan")

    def status(self, stream=None) -> int:
        return load().ivc_plan_status(self.plan, _stream(stream))

    def close(self):
        if self.plan:
            load().ivc_plan_destroy(self.plan)
            self.plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_batched(fmt, op, fields, stream=None) -> ivc_launch_config:
    """ivc_tune_batched over a list of (a, b, c, alpha) tensor fields."""
    import torch
    L = load()
    arr = (ivc_field * len(fields))()
    for i, (a, b, c, alpha) in enumerate(fields):
        arr[i] = ivc_field(_ptr(a), _ptr(b) if b is not None else None, _ptr(c), a.shape[0],
                           float(alpha), 0.0)
    ws = ctypes.c_size_t(0)
    _chk(L.ivc_plan_batched(ctypes.byref(fmt), op, arr, len(fields), None, ctypes.byref(ws),
                            None, _stream(stream), None), "ivc_plan_batched(size)")
    buf = torch.empty(ws.value + 256, dtype=torch.uint8, device=fields[0][0].device)
    base = (buf.data_ptr() + 255) // 256 * 256
    best = ivc_launch_config()
    _chk(L.ivc_tune_batched(ctypes.byref(fmt), op, arr, len(fields), base, ws.value,
                            _stream(stream), ctypes.byref(best)), "ivc_tune_batched")
    return best


def tune(fmt, op, a, b, c, stream=None) -> ivc_launch_config:
    best = ivc_launch_config()
    _chk(load().ivc_tune(ctypes.byref(fmt), op, _ptr(a), _ptr(b), _ptr(c), a.shape[0],
                         _stream(stream), ctypes.byref(best)), "ivc_tune")
    return best


_MAX_FIELDS = (3, 5, 7, 9)


def merge_stats(parts):
    """Combine accumulated ivc_error_stats arrays (one per shard or rank):
    sums add, maxima take the maximum.  Accepts sequences of 11 numbers."""
    out = [0.0] * IVC_STATS_LEN
    for p in parts:
        v = [float(x) for x in p]
        for k in range(IVC_STATS_LEN):
            out[k] = max(out[k], v[k]) if k in _MAX_FIELDS else out[k] + v[k]
    return out
