"""GPU parity of the flux-reconstruction steps 5-9 and 11 (Table fr_nse, Sec.
4) against the oracle (oracle/fr.py), through the C ABI, with compressed rows
(fast path of the primary layout, generic path of the fractional split, the
tanh map and the <0,7,23>-17-17 layout) and with FP32 rows.

Inputs: the seeded element data of synth.fr_case (a deformed periodic mesh,
Taylor-Green state with a smooth perturbation); rows are compressed by the
oracle, and every step gets the oracle's output of the previous one, so both
sides decode the same words.  The oracle evaluates in FP64 with the FP32
basis the kernels receive.

Bounds per output component:
  * linear steps (5, 6, 7, 11): 2 (t + 1) 2^-24 M, M the same contraction on
    absolute values, t its number of terms (FP32 FMA chain);
  * physics (8, 9): 64 2^-24 M, M the oracle's evaluation on magnitudes
    (every subtraction an addition), about 20 dependent roundings with a
    factor-2 margin;
  * compressed outputs add the format's worst-case row error eps |row|
    (half a bin of each angle and one unit of the magnitude field:
    1.2 pi hypot(1/N_theta, 1/(2 N_phi)) + 2^-m + 2^-23, the 1.2 covering
    the tanh map's widest bins).
Entries past ne (the padding of the leading dimension) must stay untouched.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from oracle import fr as R  # noqa: E402
from paper_2003_02633_gb300 import ivc, synth  # noqa: E402
from parity_util import formats  # noqa: E402

DEV = "cuda:0"
U = 2.0 ** -24
GAS = dict(gamma=1.4, mu=1.0 / 1600.0, prandtl=0.72)
SENT_W = 0x7FF0DEADBEEF0000
SENT_F = -7.0
FMTS = ["f32", "primary", "fracsplit", "tanh", "L1717"]


def _eps(fo):
    if fo is None:
        return 0.0
    N, M = O.nmax(fo)
    return 1.2 * math.pi * math.hypot(1.0 / N, 1.0 / (2 * M)) + 2.0 ** -fo.man_bits + 2.0 ** -23


class Case:
    def __init__(self, dims, order, pad=3):
        c = synth.fr_case(dims, order, deform=0.1, perturb=0.05)
        self.c = {k: (v.numpy() if hasattr(v, "numpy") else v) for k, v in c.items()}
        self.dims = dims
        self.order = order
        self.ne = int(np.prod(dims))
        self.ld = self.ne + pad
        b = synth.fr_basis(order)
        # the oracle works with the FP32 basis the kernels get
        self.B = {k: (np.asarray(b[k], np.float32).astype(np.float64)
                      if k in ("dm", "lm", "lp", "gl", "gr") else b[k]) for k in b}
        self.Bc = ivc.fr_basis(b)
        self.absB = {k: (np.abs(v) if isinstance(v, np.ndarray) else v) for k, v in self.B.items()}
        self.gas = ivc.fr_gas(**GAS)
        self.ns = (order + 1) ** 3
        self.nf = 6 * (order + 1) ** 2

    # --- host -> device
    def scal(self, x):
        x = np.asarray(x, np.float32)
        out = np.zeros(x.shape[:-1] + (self.ld,), np.float32)
        out[..., :self.ne] = x
        return torch.from_numpy(out).to(DEV)

    def rows_in(self, fo, rows):
        """Oracle-compressed words (or, fo None, the FP32 rows) on the device,
        and the values both sides see (decoded rows, FP64)."""
        rows = np.asarray(rows, np.float32)
        npts, nr = rows.shape[0], rows.shape[1]
        if fo is None:
            vals = rows.astype(np.float64)
            out = np.zeros((3, npts, nr, self.ld), np.float32)
            out[..., :self.ne] = np.moveaxis(rows, 3, 0)
            return torch.from_numpy(out).to(DEV), vals
        w = O.compress(fo, rows.reshape(-1, 3)).reshape(npts, nr, self.ne)
        vals = O.decompress(fo, w.reshape(-1)).reshape(npts, nr, self.ne, 3).astype(np.float64)
        out = np.zeros((npts, nr, self.ld), np.uint64)
        out[..., :self.ne] = w
        return torch.from_numpy(out.view(np.int64)).to(DEV), vals

    def rows_out(self, fg, npts, nr):
        if fg is None:
            return torch.full((3, npts, nr, self.ld), SENT_F, dtype=torch.float32, device=DEV)
        return torch.full((npts, nr, self.ld), SENT_W, dtype=torch.int64, device=DEV)

    def scal_out(self, npts, nv):
        return torch.full((npts, nv, self.ld), SENT_F, dtype=torch.float32, device=DEV)

    # --- device -> host
    def rows_back(self, fo, t, check_pad=True):
        a = t.cpu().numpy()
        if fo is None:
            assert not check_pad or np.all(a[..., self.ne:] == SENT_F)
            return np.moveaxis(a[..., :self.ne], 0, 3).astype(np.float64)
        w = a.view(np.uint64)
        assert not check_pad or np.all(w[..., self.ne:] == np.uint64(SENT_W))
        npts, nr = w.shape[0], w.shape[1]
        return O.decompress(fo, np.ascontiguousarray(w[..., :self.ne]).reshape(-1)).reshape(
            npts, nr, self.ne, 3).astype(np.float64)

    def scal_back(self, t):
        a = t.cpu().numpy()
        assert np.all(a[..., self.ne:] == SENT_F)
        return a[..., :self.ne].astype(np.float64)


_CASES = {}


def case(dims=(6, 5, 4), order=3):
    key = (dims, order)
    if key not in _CASES:
        _CASES[key] = Case(dims, order)
    return _CASES[key]


def _fmt(name):
    if name == "f32":
        return None, None
    return formats(name)


def _check_rows(got, ref, arith, eps, what):
    """|got - ref| <= arith + eps (|ref| + |arith|) per component (row norms)."""
    nrm = np.linalg.norm(ref, axis=-1, keepdims=True) + np.linalg.norm(arith, axis=-1,
                                                                       keepdims=True)
    tol = arith + eps * nrm + 1e-30
    r = np.abs(got - ref) / tol
    assert np.all(r <= 1.0), (what, float(r.max()), np.unravel_index(np.argmax(r), r.shape))
    return float(r.max())


def _check_scal(got, ref, arith, what):
    r = np.abs(got - ref) / (arith + 1e-30)
    assert np.all(r <= 1.0), (what, float(r.max()))
    return float(r.max())


# ------------------------------------------------------------------ step 5

@pytest.mark.parametrize("name", FMTS)
@pytest.mark.parametrize("dims,order", [((6, 5, 4), 3), ((3, 3, 3), 1), ((5, 2, 3), 2)])
def test_gradient(name, dims, order):
    C = case(dims, order)
    fo, fg = _fmt(name)
    w = C.c["w_s"]
    out = C.rows_out(fg, C.ns, 5)
    ivc.fr_gradient(fg, C.Bc, C.scal(w), ne=C.ne, out=out)
    got = C.rows_back(fo, out)
    ref = R.gradient(w, C.B)
    q = order + 1
    arith = 2 * (q + 1) * U * R.gradient(np.abs(w), C.absB)
    _check_rows(got, ref, arith, _eps(fo), ("grad", name))


# ------------------------------------------------------------------ step 6

@pytest.mark.parametrize("name", FMTS)
@pytest.mark.parametrize("inplace", [False, True])
def test_correct_gradient(name, inplace):
    C = case()
    fo, fg = _fmt(name)
    G0 = R.gradient(C.c["w_s"], C.B)
    Gd, Gv = C.rows_in(fo, G0)
    dw = C.c["dw_f"]
    out = Gd if inplace else C.rows_out(fg, C.ns, 5)
    ivc.fr_correct_gradient(fg, C.Bc, Gd, C.scal(dw), ne=C.ne, out=out)
    # in place, the padding holds the input's zeros
    got = C.rows_back(fo, out, check_pad=not inplace)
    ref = R.correct_gradient(Gv, dw, C.B)
    arith = 2 * 4 * U * R.correct_gradient(np.abs(Gv), np.abs(dw), C.absB)
    _check_rows(got, ref, arith, _eps(fo), ("correct", name, inplace))


# ------------------------------------------------------------------ step 7

@pytest.mark.parametrize("name", FMTS)
@pytest.mark.parametrize("dims,order", [((6, 5, 4), 3), ((4, 4, 1), 2)])
def test_interp_rows(name, dims, order):
    C = case(dims, order)
    fo, fg = _fmt(name)
    X0 = R.correct_gradient(R.gradient(C.c["w_s"], C.B), C.c["dw_f"], C.B)
    Xd, Xv = C.rows_in(fo, X0)
    out = C.rows_out(fg, C.nf, 5)
    ivc.fr_interp_rows(fg, C.Bc, Xd, ne=C.ne, out=out)
    got = C.rows_back(fo, out)
    ref = R.interp_rows(Xv, C.B)
    arith = 2 * (order + 2) * U * R.interp_rows(np.abs(Xv), C.absB)
    _check_rows(got, ref, arith, _eps(fo), ("interp", name))


# ------------------------------------------------------------------ step 9

# 20^3 elements: several (tile, point) items per warp at the full launch, so
# that each warp reuses its staging slots from one item to the next
MANY = (20, 20, 20)


@pytest.mark.parametrize("name,dims", [(n, (6, 5, 4)) for n in FMTS] +
                         [("primary", MANY), ("fracsplit", MANY)])
def test_solution_flux(name, dims):
    C = case(dims, 3)
    fo, fg = _fmt(name)
    Gc = R.correct_gradient(R.gradient(C.c["w_s"], C.B), C.c["dw_f"], C.B)
    Gd, Gv = C.rows_in(fo, Gc)
    Sd, Sv = C.rows_in(fo, C.c["S_s"])
    qs, det = C.c["q_s"], C.c["detJ_s"]
    out = C.rows_out(fg, C.ns, 5)
    ivc.fr_flux(fg, C.order, C.gas, C.scal(qs), Gd, Sd, C.scal(det), ne=C.ne, out=out)
    got = C.rows_back(fo, out)
    ref = R.solution_flux(qs, Gv, Sv, det, **GAS)
    arith = 64 * U * R.solution_flux(qs, Gv, Sv, det, mag=True, **GAS)
    _check_rows(got, ref, arith, _eps(fo), ("flux", name))


# ------------------------------------------------------------------ step 8

@pytest.mark.parametrize("name,dims", [(n, d) for n in FMTS for d in [(6, 5, 4), (1, 3, 2)]] +
                         [("primary", MANY), ("fracsplit", MANY)])
def test_common_viscous_flux(name, dims):
    C = case(dims, 3)
    fo, fg = _fmt(name)
    Gc = R.correct_gradient(R.gradient(C.c["w_s"], C.B), C.c["dw_f"], C.B)
    Gf = R.interp_rows(Gc, C.B)
    Gd, Gv = C.rows_in(fo, Gf)
    nd, nv = C.rows_in(fo, C.c["n_f"])
    Sd, Sv = C.rows_in(fo, C.c["S_f"])
    det, qf, nFi = C.c["detJ_f"], C.c["q_f"], C.c["nFinv_f"]
    out = C.scal_out(C.nf, 5)
    ivc.fr_common_viscous_flux(fg, 3, C.gas, dims, Gd, nd, Sd, C.scal(det), C.scal(qf),
                               C.scal(nFi), out=out)
    got = C.scal_back(out)
    ref = R.common_viscous(Gv, nv, Sv, det, qf, nFi, dims, **GAS)
    arith = 64 * U * R.common_viscous(Gv, nv, Sv, det, qf, nFi, dims, mag=True, **GAS)
    _check_scal(got, ref, arith, ("common viscous", name, dims))


# ------------------------------------------------------------------ step 11

@pytest.mark.parametrize("name", FMTS)
def test_flux_correction(name):
    C = case()
    fo, fg = _fmt(name)
    Gc = R.correct_gradient(R.gradient(C.c["w_s"], C.B), C.c["dw_f"], C.B)
    F = R.solution_flux(C.c["q_s"], Gc, C.c["S_s"], C.c["detJ_s"], **GAS)
    Fd, Fv = C.rows_in(fo, F)
    nF = np.asarray(C.c["nFinv_f"], np.float32).astype(np.float64)
    out = C.scal_out(C.nf, 5)
    ivc.fr_flux_correction(fg, C.Bc, Fd, C.scal(nF), ne=C.ne, out=out)
    got = C.scal_back(out)
    ref = R.flux_correction(Fv, nF, C.B)
    q = C.order + 1
    mag = np.abs(nF) + np.abs(R.flux_correction(np.abs(Fv), 0 * nF, C.absB))
    _check_scal(got, ref, 2 * (q + 2) * U * mag, ("flux correction", name))


def test_empty_calls():
    C = case()
    fo, fg = _fmt("primary")
    z = torch.zeros((C.ns, 5, 0), dtype=torch.float32, device=DEV)
    ivc.fr_gradient(fg, C.Bc, z, ne=0, out=torch.zeros((C.ns, 5, 0), dtype=torch.int64,
                                                        device=DEV))
