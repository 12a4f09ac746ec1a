"""GPU parity of the random-access decompression (ivc_gather_decompress) and
its FP32 baseline, through the C ABI.  The oracle decodes the same words; the
gathered rows must equal the oracle's decoded rows at the same indices (the
decode rule of the streaming kernels: within 1 ulp, NaN where the oracle gives
NaN), and out-of-range indices give NaN rows."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2003_02633_gb300 import ivc, synth  # noqa: E402
from parity_util import check_decoded, formats  # noqa: E402

DEV = "cuda:0"


def _indices(nw, n, seed):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, nw, n).astype(np.int64)
    bad = rng.choice(n, size=min(n, 7), replace=False)
    idx[bad] = np.array([-1, nw, nw + 5, -(1 << 40), 1 << 62, -7, nw * 3])[: bad.size]
    return idx, bad


@pytest.mark.parametrize("fname", ["primary", "fracsplit", "L1717", "tanh"])
@pytest.mark.parametrize("offset", [0, 1])
def test_gather_decompress(fname, offset):
    fo, fg = formats(fname)
    a, _ = synth.roundtrip_inputs(1 << 16, seed=3)
    w = O.compress(fo, a)
    nw = w.shape[0]
    n = (1 << 17) + 3
    idx, bad = _indices(nw, n + offset, seed=11)
    Wd = torch.from_numpy(w.view(np.int64)).to(DEV)
    Id = torch.from_numpy(idx).to(DEV)[offset:]     # offset 1: 8-byte aligned, generic kernel
    got = ivc.gather_decompress(fg, Wd, Id).cpu().numpy()
    idx = idx[offset:]
    ref = O.decompress(fo, w)
    ok = (idx >= 0) & (idx < nw)
    want = np.full((n, 3), np.nan, np.float32)
    want[ok] = ref[idx[ok]]
    check_decoded(got, want, f"gather {fname}")
    assert np.all(np.isnan(got[~ok]))


def test_gather_small_and_empty():
    fo, fg = formats("primary")
    a, _ = synth.roundtrip_inputs(100, seed=4)
    w = O.compress(fo, a)
    Wd = torch.from_numpy(w.view(np.int64)).to(DEV)
    for n in (1, 2, 3):
        idx = np.arange(n, dtype=np.int64)[::-1].copy()
        got = ivc.gather_decompress(fg, Wd, torch.from_numpy(idx).to(DEV)).cpu().numpy()
        check_decoded(got, O.decompress(fo, w)[idx], "gather small")
    out = ivc.gather_decompress(fg, Wd, torch.zeros(0, dtype=torch.int64, device=DEV))
    assert out.shape == (0, 3)


@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_f32_gather(layout):
    rng = np.random.default_rng(5)
    nsrc, n = 5000, 20001
    x = rng.standard_normal((nsrc, 3)).astype(np.float32)
    idx, bad = _indices(nsrc, n, seed=6)
    Id = torch.from_numpy(idx).to(DEV)
    if layout == "aos":
        got = ivc.f32_gather(torch.from_numpy(x).to(DEV), Id).cpu().numpy()
    else:
        ld = nsrc + 3
        rows = np.zeros((3, ld), np.float32)
        rows[:, :nsrc] = x.T
        got = ivc.f32_gather(torch.from_numpy(rows).to(DEV), Id, layout=ivc.IVC_SOA, ld=ld,
                             nsrc=nsrc).cpu().numpy()
    ok = (idx >= 0) & (idx < nsrc)
    assert np.array_equal(got[ok], x[idx[ok]])
    assert np.all(np.isnan(got[~ok]))


@pytest.mark.parametrize("fname", ["primary", "fracsplit"])
def test_gather_pole_words_exact(fname):
    # words at the poles (n_phi = 0 or n_phi_max) with any n_theta and any
    # magnitude decode to exactly (+0, +0, +-r^), settled in the fast kernel
    fo, fg = formats(fname)
    N, M = O.nmax(fo)
    rng = np.random.default_rng(21)
    n = 4096
    E = rng.integers(0, 128, n).astype(np.uint64)          # includes 0 and non-finite 127
    m = rng.integers(0, 1 << 22, n).astype(np.uint64)
    nt = rng.integers(0, N + 1, n).astype(np.uint64)
    npv = np.where(rng.random(n) < 0.5, 0, M).astype(np.uint64)
    if fo.map == 2:
        low = npv * np.uint64(N + 1) + nt
    else:
        low = (npv << np.uint64(18)) | nt
    w = (E << np.uint64(57)) | (m << np.uint64(35)) | low
    Wd = torch.from_numpy(w.view(np.int64)).to(DEV)
    idx = torch.arange(n, dtype=torch.int64, device=DEV)
    got = ivc.gather_decompress(fg, Wd, idx).cpu().numpy()
    want = O.decompress(fo, w)
    fin = np.isfinite(want).all(1)
    assert np.array_equal(got[fin].view(np.uint32), want[fin].view(np.uint32))
    check_decoded(got, want, f"gather poles {fname}")
