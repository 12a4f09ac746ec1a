"""GPU parity of the compressed flux divergence (Algorithm 1, Sec. 4; Table
fr_nse, step 10) against the oracle, through the C ABI: the tensor-core kernel
(ivc_flux_divergence: three TF32 products per FP32 term, FP32 accumulation)
and the CUDA-core one (ivc_flux_divergence_simt), both held to the bound below.

The oracle compresses the FP32 flux itself and the GPU is given the oracle's
words.  The GPU accumulates the 3 ns products of each output in FP32 (FMA,
order of its own); the oracle sums them in FP64.  Bound per output:
    |gpu - oracle| <= 2 (3 ns + 38) 2^-24 sum_{c,j} |D| |X|
(FP32 summation of 3 ns terms; the tensor-core kernel's TF32 split, whose
dropped tail products stay below 16 2^-24 of each term, and its plain-FP32
decode, within 22 2^-24 of each decoded component; a factor 2 of margin).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2003_02633_gb300 import ivc, synth  # noqa: E402
from parity_util import formats  # noqa: E402

DEV = "cuda:0"
U = 2.0 ** -24


def _flux(order, ne, nvars=5, E=16, scale=None):
    """TGV Euler flux rows (ns, nvars, ne, 3) float32 on the host."""
    F = synth.tgv_euler_flux(elements_per_axis=E, order=order, elements=ne).numpy()
    F = F[:, :nvars]
    if scale is not None:
        F = (F * scale).astype(np.float32)
    return np.ascontiguousarray(F)


def _bound(D, X, ns):
    absD = np.abs(D.astype(np.float64)).reshape(3, ns, ns)          # (c, j, k)
    t = np.einsum("cjk,jpec->kpe", absD, np.abs(X.astype(np.float64)))
    return 2.0 * (3 * ns + 38) * U * t + 1e-30


def _run(fname, order, ne, nvars=5, ld=None, h=2 * math.pi / 16, simt=False):
    fo, fg = formats(fname)
    F = _flux(order, ne, nvars)
    ns = F.shape[0]
    D = synth.fr_hex_operator(order, h)
    w = O.compress(fo, F.reshape(-1, 3)).reshape(ns, nvars, ne)
    ld = ne if ld is None else ld
    wpad = np.zeros((ns, nvars, ld), np.uint64)
    wpad[:, :, :ne] = w
    Wd = torch.from_numpy(wpad.view(np.int64)).to(DEV)
    Dd = torch.from_numpy(D).to(DEV)
    out = torch.full((ns, nvars, ld), 7.0, dtype=torch.float32, device=DEV)
    ivc.flux_divergence(fg, Wd, Dd, ne=ne, out=out, simt=simt)
    ivc.flux_divergence_check()   # no bounded wait ran out
    got = out.cpu().numpy()
    ref = O.flux_divergence(fo, w, D, ns, nvars)
    X = O.decompress(fo, w.reshape(-1)).reshape(ns, nvars, ne, 3)
    err = np.abs(got[:, :, :ne].astype(np.float64) - ref)
    bound = _bound(D, X, ns)
    assert np.all(err <= bound), (fname, float((err / bound).max()))
    # padding beyond ne untouched
    assert np.all(got[:, :, ne:] == 7.0)
    return err, bound


@pytest.mark.parametrize("simt", [False, True])
@pytest.mark.parametrize("fname", ["primary", "L1717", "tanh", "fracsplit"])
def test_fdiv_formats_ragged(fname, simt):
    # 3 full tiles of 64 elements and a ragged one (1 full tile of 128 and a
    # ragged one on the tensor-core kernel)
    _run(fname, 3, 3 * 64 + 37, simt=simt)


@pytest.mark.parametrize("simt", [False, True])
@pytest.mark.parametrize("order,nvars", [(1, 5), (2, 3), (3, 1), (3, 4)])
def test_fdiv_orders_and_rows(order, nvars, simt):
    _run("primary", order, 100, nvars=nvars, simt=simt)


@pytest.mark.parametrize("simt", [False, True])
def test_fdiv_padded_leading_dimension(simt):
    _run("primary", 3, 77, ld=80, simt=simt)


def test_fdiv_single_element_and_empty():
    _run("primary", 3, 1)
    fo, fg = formats("primary")
    W = torch.zeros((64, 5, 0), dtype=torch.int64, device=DEV)
    D = torch.zeros((192, 64), dtype=torch.float32, device=DEV)
    out = ivc.flux_divergence(fg, W, D)
    assert out.shape == (64, 5, 0)


@pytest.mark.parametrize("simt", [False, True])
def test_fdiv_many_tiles(simt):
    # 4096 + 37 elements: 65 tiles of 64 (more than one per block on small
    # grids), 33 of 128
    err, bound = _run("primary", 3, 4096 + 37, simt=simt)
    assert float((err / bound).max()) < 1.0


@pytest.mark.parametrize("simt", [False, True])
def test_f32_flux_divergence_baseline(simt):
    order, ne, nvars = 3, 200, 5
    F = _flux(order, ne, nvars)
    ns = F.shape[0]
    D = synth.fr_hex_operator(order, 0.3)
    Fc = np.ascontiguousarray(np.transpose(F, (3, 0, 1, 2)))        # (3, ns, nvars, ne)
    out = ivc.f32_flux_divergence(torch.from_numpy(Fc).to(DEV), torch.from_numpy(D).to(DEV),
                                  simt=simt)
    ivc.flux_divergence_check()
    got = out.cpu().numpy().astype(np.float64)
    Dd = D.astype(np.float64).reshape(3, ns, ns)
    ref = np.einsum("cjk,jpec->kpe", Dd, F.astype(np.float64))
    assert np.all(np.abs(got - ref) <= _bound(D, F, ns))


_MULTI = {}


@pytest.mark.parametrize("simt", [False, True])
def test_fdiv_several_tiles_per_block(simt):
    # 313 tiles of 128 elements (626 of 64): more tiles than SMs, so persistent
    # blocks walk several tiles (tile hand-over of the accumulators and of the
    # mbarrier phases); every output against the oracle
    if not _MULTI:
        ne = 313 * 128 - 91
        F = _flux(3, ne)
        D = synth.fr_hex_operator(3, 2 * math.pi / 16)
        fo, _ = formats("primary")
        w = O.compress(fo, F.reshape(-1, 3)).reshape(64, 5, ne)
        X = O.decompress(fo, w.reshape(-1)).reshape(64, 5, ne, 3)
        _MULTI.update(ne=ne, D=D, w=w, ref=O.flux_divergence(fo, w, D, 64, 5),
                      bound=_bound(D, X, 64))
    fo, fg = formats("primary")
    ne, D, w = _MULTI["ne"], _MULTI["D"], _MULTI["w"]
    Wd = torch.from_numpy(w.view(np.int64)).to(DEV)
    out = ivc.flux_divergence(fg, Wd, torch.from_numpy(D).to(DEV), simt=simt)
    ivc.flux_divergence_check()
    err = np.abs(out.cpu().numpy().astype(np.float64) - _MULTI["ref"])
    assert np.all(err <= _MULTI["bound"]), float((err / _MULTI["bound"]).max())


@pytest.mark.parametrize("simt", [False, True])
@pytest.mark.parametrize("comp", [0, 1, 2])
def test_fdiv_selector_operator_gives_decoded_components(simt, comp):
    """With D selecting one component (D[comp ns + k][k] = 1, every other entry
    0) each output is the decoded component X(k, p)_comp itself, so the kernels'
    decodes are compared value by value with the oracle's decompress.  CUDA-core
    kernel: exact decode and 1 x X plus zeros, bit-exact.  Tensor-core kernel:
    the plain FP32 pair decode (relative error at most 22 2^-24) plus the TF32
    truncation of the tail of the split (at most 4 2^-24), so within 26 2^-24
    relative; a wrong sign, table entry, fold or axis fails by orders of
    magnitude more.  Random directions and magnitudes 10^U(-3, 3), poles,
    seam, zero, saturating and FP32-subnormal vectors included."""
    fo, fg = formats("primary")
    ns, nv, ne = 64, 5, 3 * 128 + 11
    a, _ = synth.roundtrip_inputs(ns * nv * ne - 8 - 64, seed=57)   # + the 64 edge vectors
    edge = np.float32([[0, 0, 1.5], [0, 0, -2.5], [-3, 0, 0], [0, 0, 0],
                       [1e-3, -1e-30, 0], [4, 4, 4], [-1, 1e-8, 1], [0, -7, 0]])
    X = np.concatenate([a, edge])
    # finite rows only: with the selector, 0 x inf in another row of the same
    # element would turn its outputs into NaN
    X[~np.all(np.isfinite(X), axis=1)] = np.float32([1.0, -2.0, 3.0])
    X = X.reshape(ns, nv, ne, 3)
    with np.errstate(invalid="ignore", over="ignore"):
        w = O.compress(fo, X.reshape(-1, 3)).reshape(ns, nv, ne)
        want = O.decompress(fo, w.reshape(-1)).reshape(ns, nv, ne, 3)[..., comp]
    D = np.zeros((3 * ns, ns), np.float32)
    D[comp * ns + np.arange(ns), np.arange(ns)] = 1.0
    out = ivc.flux_divergence(fg, torch.from_numpy(w.view(np.int64)).to(DEV),
                              torch.from_numpy(D).to(DEV), simt=simt)
    ivc.flux_divergence_check()
    got = out.cpu().numpy()
    if simt:
        assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    else:
        err = np.abs(got.astype(np.float64) - want.astype(np.float64))
        tol = 26.0 * U * np.abs(want.astype(np.float64))
        assert np.all(err <= tol), float((err / np.maximum(tol, 1e-45)).max())
