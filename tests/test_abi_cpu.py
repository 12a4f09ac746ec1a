"""C-ABI library: it builds, loads and exports every symbol include/ivc.h
declares; host-only entry points (format set-up, validation, status text) and
argument checks that return before any device work run here without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2003_02633_gb300 import ivc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ivc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ivc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return ivc.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(ivc.EXPORTS) == names


def test_version_and_status_strings(lib):
    assert b"sm_103a" in lib.ivc_version()
    assert ivc.status_string(ivc.IVC_OK) == "ok"
    assert "format" in ivc.status_string(ivc.IVC_ERR_FORMAT)
    assert ivc.status_string(99) == "unknown status"


def test_default_format_is_primary_layout(lib):
    f = ivc.default_format()
    assert (f.sign_bits, f.exp_bits, f.man_bits, f.phi_bits, f.theta_bits, f.exp_bias) == \
        (0, 7, 22, 17, 18, 80)
    assert lib.ivc_format_validate(ctypes.byref(f)) == ivc.IVC_OK


@pytest.mark.parametrize("kw", [
    dict(exp_bits=9), dict(man_bits=24), dict(theta_bits=20), dict(phi_bits=40),
    dict(sign_bits=2), dict(exp_bias=300), dict(map=7), dict(map=1, gamma=0.0),
    dict(map=2, nphi_max_p1=1), dict(underflow_mode=2),
])
def test_invalid_formats_rejected(lib, kw):
    f = ivc.make_format(**kw)
    assert lib.ivc_format_validate(ctypes.byref(f)) == ivc.IVC_ERR_FORMAT


@pytest.mark.parametrize("kw", [
    dict(), dict(exp_bits=8, man_bits=23, phi_bits=16, theta_bits=17, exp_bias=127),
    dict(exp_bits=7, man_bits=23, phi_bits=17, theta_bits=17, exp_bias=80),
    dict(sign_bits=1, exp_bits=8, man_bits=23, phi_bits=16, theta_bits=16, exp_bias=127),
    dict(map=2, nphi_max_p1=185363), dict(map=1, gamma=0.5),
    dict(exp_bits=3, man_bits=4, phi_bits=4, theta_bits=5, exp_bias=3),
])
def test_paper_formats_accepted(lib, kw):
    f = ivc.make_format(**kw)
    assert lib.ivc_format_validate(ctypes.byref(f)) == ivc.IVC_OK


def test_argument_errors_before_device_work(lib):
    f = ivc.default_format()
    bad = ivc.make_format(exp_bits=9)
    assert lib.ivc_compress(ctypes.byref(f), None, 0, 0, -1, None, None, None) == ivc.IVC_ERR_ARG
    assert lib.ivc_compress(ctypes.byref(f), None, 5, 0, 1, None, None, None) == ivc.IVC_ERR_ARG
    assert lib.ivc_compress(ctypes.byref(bad), None, 0, 0, 1, None, None, None) == \
        ivc.IVC_ERR_FORMAT
    assert lib.ivc_add(ctypes.byref(f), None, None, None, -3, None) == ivc.IVC_ERR_ARG
    assert lib.ivc_f32_add(0, None, None, None, 0, -1, None) == ivc.IVC_ERR_ARG
    assert lib.ivc_f32_add(1, None, None, None, 2, 5, None) == ivc.IVC_ERR_ARG  # ld < n
    assert lib.ivc_half_add(9, None, None, None, 1, None) == ivc.IVC_ERR_ARG
    assert lib.ivc_error_stats(None, None, -1, None, None) == ivc.IVC_ERR_ARG
    # flux divergence: sizes out of range, ld < ne, NULL pointers, empty call
    fd = lib.ivc_flux_divergence
    assert fd(ctypes.byref(f), None, 0, 0, 5, 1, None, None, 1, None) == ivc.IVC_ERR_ARG
    assert fd(ctypes.byref(f), None, 0, 65, 5, 1, None, None, 1, None) == ivc.IVC_ERR_ARG
    assert fd(ctypes.byref(f), None, 0, 64, 6, 1, None, None, 1, None) == ivc.IVC_ERR_ARG
    assert fd(ctypes.byref(f), None, 0, 64, 5, 2, None, None, 2, None) == ivc.IVC_ERR_ARG
    assert fd(ctypes.byref(f), None, 0, 64, 5, 0, None, None, 0, None) == ivc.IVC_OK
    assert fd(ctypes.byref(bad), None, 0, 64, 5, 0, None, None, 0, None) == ivc.IVC_ERR_FORMAT
    gd = lib.ivc_gather_decompress
    assert gd(ctypes.byref(f), None, 0, None, -1, None, None) == ivc.IVC_ERR_ARG
    assert gd(ctypes.byref(f), None, -1, None, 1, None, None) == ivc.IVC_ERR_ARG
    assert gd(ctypes.byref(f), None, 0, None, 0, None, None) == ivc.IVC_OK
    assert gd(ctypes.byref(f), None, 4, None, 1, None, None) == ivc.IVC_ERR_ARG
    assert gd(ctypes.byref(bad), None, 0, None, 1, None, None) == ivc.IVC_ERR_FORMAT
    fg = lib.ivc_f32_gather
    assert fg(0, None, 0, 0, None, -1, None, None) == ivc.IVC_ERR_ARG
    assert fg(1, None, 2, 4, None, 1, None, None) == ivc.IVC_ERR_ARG   # SoA ld < nsrc
    assert fg(0, None, 0, 0, None, 0, None, None) == ivc.IVC_OK
    ah = lib.ivc_add_host
    assert ah(ctypes.byref(f), None, None, None, -1, None, 0, None) == ivc.IVC_ERR_ARG
    assert ah(ctypes.byref(f), None, None, None, 0, None, 0, None) == ivc.IVC_OK
    assert ah(ctypes.byref(f), None, None, None, 4, None, 0, None) == ivc.IVC_ERR_ARG
    assert ah(ctypes.byref(bad), None, None, None, 4, None, 0, None) == ivc.IVC_ERR_FORMAT
    buf = (ctypes.c_uint64 * 16)()
    p16 = (ctypes.addressof(buf) + 15) & ~15   # a 16-byte aligned workspace of 64 bytes
    assert ah(ctypes.byref(f), buf, buf, buf, 4, p16, 64, None) == ivc.IVC_ERR_NOMEM
    f32fd = lib.ivc_f32_flux_divergence
    assert f32fd(None, 4, 64, 5, 4, None, None, 4, None) == ivc.IVC_ERR_ARG
    assert f32fd(None, 0, 64, 5, -1, None, None, 0, None) == ivc.IVC_ERR_ARG
    assert f32fd(None, 0, 64, 5, 0, None, None, 0, None) == ivc.IVC_OK
    ws = ctypes.c_size_t(0)
    assert lib.ivc_plan_batched(ctypes.byref(f), 0, None, 0, None, ctypes.byref(ws), None, None,
                                None) == ivc.IVC_ERR_ARG
    assert lib.ivc_plan_batched(ctypes.byref(f), 0, None, 4, None, ctypes.byref(ws), None, None,
                                None) == ivc.IVC_OK
    assert ws.value >= 4 * 48
    assert lib.ivc_launch_plan(None, None) == ivc.IVC_ERR_ARG
    assert lib.ivc_plan_destroy(None) == ivc.IVC_ERR_ARG


def test_fr_argument_errors_before_device_work(lib):
    from paper_2003_02633_gb300 import synth
    f = ivc.default_format()
    bad = ivc.make_format(exp_bits=9)
    B = ivc.fr_basis(synth.fr_basis(3))
    B0 = ivc.fr_basis(synth.fr_basis(3))
    B0.order = 4                                   # degree outside 1..3
    gas = ivc.fr_gas()
    ref = ctypes.byref
    g = lib.ivc_fr_gradient
    assert g(ref(f), ref(B), None, 0, 0, 5, None, None) == ivc.IVC_OK      # empty
    assert g(ref(f), ref(B), None, -1, 0, 5, None, None) == ivc.IVC_ERR_ARG
    assert g(ref(f), ref(B), None, 4, 2, 5, None, None) == ivc.IVC_ERR_ARG  # ld < ne
    assert g(ref(f), ref(B), None, 4, 4, 6, None, None) == ivc.IVC_ERR_ARG  # nvars
    assert g(ref(f), ref(B0), None, 0, 0, 5, None, None) == ivc.IVC_ERR_ARG
    assert g(ref(f), None, None, 0, 0, 5, None, None) == ivc.IVC_ERR_ARG
    assert g(ref(bad), ref(B), None, 4, 4, 5, None, None) == ivc.IVC_ERR_FORMAT
    assert g(ref(f), ref(B), None, 4, 4, 5, None, None) == ivc.IVC_ERR_ARG  # NULL w
    buf = (ctypes.c_uint64 * 8)()
    a8 = ctypes.addressof(buf)
    assert g(ref(f), ref(B), a8, 4, 4, 5, a8 + 4, None) == ivc.IVC_ERR_ALIGN
    assert lib.ivc_f32_fr_gradient(ref(B), None, 4, 4, 5, None, None) == ivc.IVC_ERR_ARG
    cg = lib.ivc_fr_correct_gradient
    assert cg(ref(f), ref(B), a8, None, 4, 4, 5, a8, None) == ivc.IVC_ERR_ARG
    assert cg(ref(f), ref(B), a8 + 4, a8, 4, 4, 5, a8, None) == ivc.IVC_ERR_ALIGN
    ir = lib.ivc_fr_interp_rows
    assert ir(ref(f), ref(B), None, 0, 0, 1, None, None) == ivc.IVC_OK
    assert ir(ref(f), ref(B), a8, 4, 4, 0, a8, None) == ivc.IVC_ERR_ARG
    dims = (ctypes.c_int * 3)(2, 2, 2)
    zero = (ctypes.c_int * 3)(2, 0, 2)
    cv = lib.ivc_fr_common_viscous_flux
    assert cv(ref(f), 3, ref(gas), zero, a8, a8, a8, a8, a8, a8, 8, a8, None) == ivc.IVC_ERR_ARG
    assert cv(ref(f), 3, ref(gas), dims, a8, a8, a8, a8, a8, a8, 4, a8, None) == ivc.IVC_ERR_ARG
    assert cv(ref(f), 0, ref(gas), dims, a8, a8, a8, a8, a8, a8, 8, a8, None) == ivc.IVC_ERR_ARG
    assert cv(ref(f), 3, None, dims, a8, a8, a8, a8, a8, a8, 8, a8, None) == ivc.IVC_ERR_ARG
    assert cv(ref(f), 3, ref(gas), dims, a8, None, a8, a8, a8, a8, 8, a8, None) == \
        ivc.IVC_ERR_ARG
    fl = lib.ivc_fr_flux
    assert fl(ref(f), 3, ref(gas), None, None, None, None, 0, 0, None, None) == ivc.IVC_OK
    assert fl(ref(f), 3, ref(gas), a8, a8, a8, None, 4, 4, a8, None) == ivc.IVC_ERR_ARG
    assert fl(ref(f), 3, ref(gas), a8, a8 + 4, a8, a8, 4, 4, a8, None) == ivc.IVC_ERR_ALIGN
    fc = lib.ivc_fr_flux_correction
    assert fc(ref(bad), ref(B), a8, a8, 4, 4, 5, a8, None) == ivc.IVC_ERR_FORMAT
    assert fc(ref(f), ref(B), a8, a8, 4, 3, 5, a8, None) == ivc.IVC_ERR_ARG
    assert lib.ivc_f32_fr_flux_correction(ref(B), a8, a8, 4, 4, 0, a8, None) == ivc.IVC_ERR_ARG


def test_plan_workspace_too_small(lib):
    """ivc_plan_batched reports a workspace smaller than it needs before it
    touches the workspace or the device."""
    f = ivc.default_format()
    arr = (ivc.ivc_field * 3)()
    ws = ctypes.c_size_t(0)
    assert lib.ivc_plan_batched(ctypes.byref(f), ivc.IVC_OP_ADD, arr, 3, None, ctypes.byref(ws),
                                None, None, None) == ivc.IVC_OK
    assert ws.value > 0
    small = ctypes.c_size_t(ws.value - 8)
    plan = ctypes.c_void_p()
    fake = 4096          # never dereferenced: the size check comes first
    assert lib.ivc_plan_batched(ctypes.byref(f), ivc.IVC_OP_ADD, arr, 3, fake,
                                ctypes.byref(small), None, None,
                                ctypes.byref(plan)) == ivc.IVC_ERR_NOMEM
    assert not plan.value


@pytest.mark.parametrize("entry", ["add", "axpy", "compress", "decompress", "add_noalloc",
                                   "compress_exact", "plan_batched"])
def test_invalid_format_rejected_by_entry_points(lib, entry):
    """A format that fails validation is rejected by every entry point before
    any device work (IVC_ERR_FORMAT), whatever the pointers."""
    bad = ivc.make_format(exp_bits=9)
    B = ctypes.byref(bad)
    p = 4096
    calls = {
        "add": lambda: lib.ivc_add(B, p, p, p, 16, None),
        "axpy": lambda: lib.ivc_axpy(B, 0.5, p, p, 16, None),
        "compress": lambda: lib.ivc_compress(B, p, 0, 0, 16, p, None, None),
        "decompress": lambda: lib.ivc_decompress(B, p, 16, p, 0, 0, None),
        "add_noalloc": lambda: lib.ivc_add_noalloc(B, p, p, p, 16, None),
        "compress_exact": lambda: lib.ivc_compress_exact(B, p, 16, p, None, None),
    }
    if entry == "plan_batched":
        arr = (ivc.ivc_field * 1)()
        ws = ctypes.c_size_t(1 << 20)
        plan = ctypes.c_void_p()
        st = lib.ivc_plan_batched(B, ivc.IVC_OP_ADD, arr, 1, p, ctypes.byref(ws), None, None,
                                  ctypes.byref(plan))
    else:
        st = calls[entry]()
    assert st == ivc.IVC_ERR_FORMAT
