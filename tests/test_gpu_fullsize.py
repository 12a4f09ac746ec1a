"""GPU parity at the benchmark's full sizes, in the launch configuration the
benchmark times, on outputs the oracle computes one by one:

* compressed add, N = 2^28 vectors per operand (the headline workload: the same
  seeded device generator and seeds as bench.py), 2^16 sampled outputs;
* the flux divergence of Algorithm 1 on the 96^3 degree-3 mesh, 48 sampled
  elements;
* random-access decompression of 2^28 random indices into 2^28 words, 2^16
  sampled outputs.

The oracle's inputs are the sampled FP32 vectors (or words) copied to the host;
its expected values never come from the CUDA path.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2003_02633_gb300 import ivc, synth  # noqa: E402
from parity_util import check_decoded, check_words  # noqa: E402

DEV = "cuda:0"
FR_E = 96          # elements per axis of the FR mesh (the benchmark's)


def test_add_full_size_sampled():
    n = 1 << 28
    dev = torch.device(DEV)
    fmt = ivc.default_format()
    a = synth.device_vectors(n, 0, dev)
    b = synth.device_vectors(n, 1, dev)
    wa, wb = ivc.compress(fmt, a), ivc.compress(fmt, b)
    wc = ivc.add(fmt, wa, wb)
    torch.cuda.synchronize()
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(n, size=1 << 16, replace=False))
    it = torch.from_numpy(idx).to(dev)
    av, bv = a[it].cpu().numpy(), b[it].cpu().numpy()
    ga = wa[it].cpu().numpy().view(np.uint64)
    gb = wb[it].cpu().numpy().view(np.uint64)
    gc = wc[it].cpu().numpy().view(np.uint64)
    oa, ob = O.compress(O.PRIMARY, av), O.compress(O.PRIMARY, bv)
    check_words(O.PRIMARY, av, ga, oa, "compress a (N = 2^28)")
    check_words(O.PRIMARY, bv, gb, ob, "compress b (N = 2^28)")
    # the add of the GPU's own operand words (equal to the oracle's, or near a
    # boundary): the oracle adds the same words
    oc = O.add(O.PRIMARY, ga, gb)
    sums = O.decompress(O.PRIMARY, ga) + O.decompress(O.PRIMARY, gb)
    check_words(O.PRIMARY, sums.astype(np.float32), gc, oc, "add (N = 2^28)")


def test_flux_divergence_full_size_sampled():
    E = 96
    dev = torch.device(DEV)
    fmt = ivc.default_format()
    F = synth.tgv_euler_flux(E, 3, device=dev)
    ns, nv, ne = F.shape[0], F.shape[1], F.shape[2]
    W = ivc.compress(fmt, F.reshape(-1, 3)).reshape(ns, nv, ne)
    del F
    D = synth.fr_hex_operator(3, 2 * math.pi / E)
    out = ivc.flux_divergence(fmt, W, torch.from_numpy(D).to(dev))
    ivc.flux_divergence_check()
    rng = np.random.default_rng(7)
    sel = np.sort(rng.choice(ne, size=48, replace=False))
    st = torch.from_numpy(sel).to(dev)
    Wh = W[:, :, st].cpu().numpy().view(np.uint64)
    got = out[:, :, st].cpu().numpy().astype(np.float64)
    ref = O.flux_divergence(O.PRIMARY, Wh, D, ns, nv)
    X = O.decompress(O.PRIMARY, Wh.reshape(-1)).reshape(ns, nv, sel.size, 3).astype(np.float64)
    bound = 2.0 * (3 * ns + 2) * 2.0 ** -24 * np.einsum(
        "cjk,jpec->kpe", np.abs(D.astype(np.float64)).reshape(3, ns, ns), np.abs(X)) + 1e-30
    assert np.all(np.abs(got - ref) <= bound)


def test_gather_full_size_sampled():
    n = 1 << 28
    dev = torch.device(DEV)
    fmt = ivc.default_format()
    x = synth.device_vectors(n, 31, dev)
    w = ivc.compress(fmt, x)
    del x
    g = torch.Generator(device=dev)
    g.manual_seed(32)
    idx = torch.randint(0, n, (n,), generator=g, device=dev, dtype=torch.int64)
    out = ivc.gather_decompress(fmt, w, idx)
    rng = np.random.default_rng(5)
    s = torch.from_numpy(np.sort(rng.choice(n, size=1 << 16, replace=False))).to(dev)
    j = idx[s]
    words = w[j].cpu().numpy().view(np.uint64)
    check_decoded(out[s].cpu().numpy(), O.decompress(O.PRIMARY, words), "gather (N = 2^28)")


def _fr_sample_words(fmt_o, rows_dev, sel_t, what):
    """GPU-compressed words of synth rows, with the sampled elements' words
    checked against the oracle's compression of the same rows; as in the add
    above, the oracle then works on those (checked) words."""
    fmt = ivc.default_format()
    W = ivc.compress(fmt, rows_dev.reshape(-1, 3)).reshape(rows_dev.shape[:3])
    host = rows_dev[:, :, sel_t].cpu().numpy()                       # (npts, nr, ns, 3)
    wo = O.compress(fmt_o, host.reshape(-1, 3)).reshape(host.shape[:3])
    wg = W[:, :, sel_t].cpu().numpy().view(np.uint64)
    check_words(fmt_o, host.reshape(-1, 3), wg.reshape(-1), wo.reshape(-1), what)
    return W, wg


def test_fr_interp_and_interface_full_size_sampled():
    # steps 7 and 8 of Table fr_nse on the 96^3 degree-3 mesh of the benchmark
    # (synth.fr_case, same launch shapes), 24 sampled elements against the oracle
    from oracle import fr as R
    E, order = FR_E, 3
    dims = (E, E, E)
    dev = torch.device(DEV)
    fo = O.PRIMARY
    fmt = ivc.default_format()
    c = synth.fr_case(dims, order, device=dev)
    ne = E ** 3
    ns, nf = 64, 96
    bas = synth.fr_basis(order)
    B32 = {k: (np.asarray(v, np.float32).astype(np.float64) if k in ("dm", "lm", "lp", "gl", "gr")
               else v) for k, v in bas.items()}
    rng = np.random.default_rng(8)
    sel = np.sort(rng.choice(ne, size=24, replace=False))
    st = torch.from_numpy(sel).to(dev)
    # step 7 on gradient-like rows (the benchmark's vector distribution)
    X = synth.device_vectors(ns * 5 * ne, 41, dev).reshape(ns, 5, ne, 3)
    Wx, wx = _fr_sample_words(fo, X, st, "step 7 inputs")
    del X
    out = ivc.fr_interp_rows(fmt, ivc.fr_basis(bas), Wx)
    got = O.decompress(fo, out[:, :, st].cpu().numpy().view(np.uint64).reshape(-1)).reshape(
        nf, 5, sel.size, 3).astype(np.float64)
    Xv = O.decompress(fo, wx.reshape(-1)).reshape(ns, 5, sel.size, 3).astype(np.float64)
    ref = R.interp_rows(Xv, B32)
    arith = 2 * 5 * 2.0 ** -24 * R.interp_rows(np.abs(Xv), {k: (np.abs(v) if isinstance(
        v, np.ndarray) else v) for k, v in B32.items()})
    eps = 1.2 * math.pi * math.hypot(1 / 262143, 1 / (2 * 131071)) + 2.0 ** -22 + 2.0 ** -23
    nrm = np.linalg.norm(ref, axis=-1, keepdims=True) + np.linalg.norm(arith, axis=-1,
                                                                       keepdims=True)
    assert np.all(np.abs(got - ref) <= arith + eps * nrm + 1e-30)
    del Wx, out
    # step 8: interface flux of the sampled elements (every flux point, both sides)
    G = synth.device_vectors(nf * 5 * ne, 42, dev, lo=-2.0, hi=1.0).reshape(nf, 5, ne, 3)
    Wg, _ = _fr_sample_words(fo, G, st, "step 8 gradient rows")
    Wn = ivc.compress(fmt, c["n_f"].reshape(-1, 3)).reshape(nf, 1, ne)
    Ws = ivc.compress(fmt, c["S_f"].reshape(-1, 3)).reshape(nf, 3, ne)
    gas = dict(gamma=1.4, mu=1.0 / 1600.0, prandtl=0.72)
    res = ivc.fr_common_viscous_flux(fmt, order, ivc.fr_gas(**gas), dims, Wg, Wn, Ws,
                                     c["detJ_f"], c["q_f"], c["nFinv_f"])
    got8 = res[:, :, st].cpu().numpy().astype(np.float64)              # (nf, 5, ns)
    # the partners of the sampled elements' flux points, and the oracle on both sides
    pr = R.partner(dims, order + 1)                                     # (nf, ne) flat f' ne + e'
    pf, pe = pr[:, sel] // ne, pr[:, sel] % ne
    fidx = np.arange(nf)[:, None].repeat(sel.size, 1)

    def side(f_i, e_i):
        ft = torch.from_numpy(np.ascontiguousarray(f_i).reshape(-1)).to(dev)
        et = torch.from_numpy(np.ascontiguousarray(e_i).reshape(-1)).to(dev)
        g = O.decompress(fo, Wg[ft, :, et].cpu().numpy().view(np.uint64).reshape(-1)).reshape(
            -1, 5, 3).astype(np.float64)
        s = O.decompress(fo, Ws[ft, :, et].cpu().numpy().view(np.uint64).reshape(-1)).reshape(
            -1, 3, 3).astype(np.float64)
        det = c["detJ_f"][ft, et].cpu().numpy().astype(np.float64)
        qv = c["q_f"][ft, :, et].cpu().numpy().astype(np.float64).T      # (5, m)
        gx = R.physical_gradient(np.moveaxis(g, 1, 0), s, det)
        gxm = R.physical_gradient(np.moveaxis(g, 1, 0), s, det, mag=True)
        return (R.viscous_rows(qv, gx, gas["gamma"], gas["mu"], gas["prandtl"]),
                R.viscous_rows(qv, gxm, gas["gamma"], gas["mu"], gas["prandtl"], mag=True))

    Fo, Mo = side(fidx, np.broadcast_to(sel, fidx.shape))
    Fp, Mp = side(pf, pe)
    ft, et = torch.from_numpy(fidx.reshape(-1)).to(dev), torch.from_numpy(
        np.broadcast_to(sel, fidx.shape).reshape(-1).copy()).to(dev)
    n = O.decompress(fo, Wn[ft, 0, et].cpu().numpy().view(np.uint64)).astype(np.float64)
    nFi = c["nFinv_f"][ft, :, et].cpu().numpy().astype(np.float64).T   # (5, m)
    ref8 = nFi - 0.5 * ((Fo + Fp) * n[None]).sum(-1)
    mag8 = np.abs(nFi) + 0.5 * ((Mo + Mp) * np.abs(n)[None]).sum(-1)
    ref8 = np.moveaxis(ref8.reshape(5, nf, sel.size), 0, 1)
    mag8 = np.moveaxis(mag8.reshape(5, nf, sel.size), 0, 1)
    assert np.all(np.abs(got8 - ref8) <= 64 * 2.0 ** -24 * mag8 + 1e-30)
