"""GPU parity of the compressed flux divergence (Algorithm 1, Sec. 4; Table
fr_nse, step 10) against the oracle, through the C ABI: the tensor-core kernel
(ivc_flux_divergence: three TF32 products per FP32 term, FP32 accumulation)
and the CUDA-core one (ivc_flux_divergence_simt), both held to the bound below.

The oracle compresses the FP32 flux itself and the GPU is given the oracle's
words.  The GPU accumulates the 3 ns products of each output in FP32 (FMA,
order of its own); the oracle sums them in FP64.  Bound per output:
    |gpu - oracle| <= 2 (3 ns + 2) 2^-24 sum_{c,j} |D| |X|
(FP32 summation of 3 ns terms, plus one ulp of the decoded flux, with a
factor 2 of margin).
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
    return 2.0 * (3 * ns + 2) * U * t + 1e-30


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
