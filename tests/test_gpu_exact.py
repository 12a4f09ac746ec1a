"""GPU parity of the exact-decision path (64/128-bit integer arithmetic, no
floating point wider than FP32): ivc_compress_exact / ivc_decompress_exact
take every rounding decision there, so these tests exercise on every vector
the code the fast kernels reach only near a boundary, against the oracle, for
every format (uniform layouts, fractional split, tanh map, a 16-bit layout,
flush-to-zero / infinite-code range handling), plus the edge vectors.  The
fast kernels must give the same words and vectors as the exact path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2003_02633_gb300 import ivc, synth  # noqa: E402
from parity_util import check_decoded, check_words, formats  # noqa: E402

DEV = "cuda:0"
NAMES = ["primary", "L1617", "L1717", "base", "fracsplit", "fracsplit_pow2", "tanh", "tiny",
         "ftz_inf"]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _host_words(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module")
def vecs():
    a, _ = synth.roundtrip_inputs((1 << 17) + 3, seed=21)
    return np.concatenate([a, synth.edge_vectors()])


@pytest.mark.parametrize("name", NAMES)
def test_compress_exact_matches_oracle(vecs, name):
    fo, fg = formats(name)
    with np.errstate(invalid="ignore", over="ignore"):
        want = O.compress(fo, vecs)
    got = _host_words(ivc.compress_exact(fg, _dev(vecs)))
    check_words(fo, vecs, got, want, f"compress_exact {name}")
    fast = _host_words(ivc.compress(fg, _dev(vecs)))
    check_words(fo, vecs, fast, got, f"compress vs compress_exact {name}")


@pytest.mark.parametrize("name", NAMES)
def test_decompress_exact_matches_oracle(vecs, name):
    fo, fg = formats(name)
    with np.errstate(invalid="ignore", over="ignore"):
        w = O.compress(fo, vecs)
        want = O.decompress(fo, w)
    wd = _dev(np.asarray(w, np.uint64).view(np.int64))
    got = ivc.decompress_exact(fg, wd).cpu().numpy()
    same = check_decoded(got, want, f"decompress_exact {name}")
    assert same == 1.0, f"{name}: {1 - same:.2e} of the exact decodes differ from the oracle"
    fast = ivc.decompress(fg, wd).cpu().numpy()
    check_decoded(fast, got, f"decompress vs decompress_exact {name}")


def test_decompress_exact_random_words():
    """Every 64-bit pattern of the primary layout (random words, non-canonical
    and non-finite ones included) decodes through the exact path to the
    oracle's vector."""
    fo, fg = formats("primary")
    w = synth.random_words(1 << 17, seed=23)
    with np.errstate(invalid="ignore", over="ignore"):
        want = O.decompress(fo, w)
    got = ivc.decompress_exact(fg, _dev(np.asarray(w, np.uint64).view(np.int64))).cpu().numpy()
    assert check_decoded(got, want, "decompress_exact random words") == 1.0


def test_exact_empty_and_errors():
    fg = ivc.default_format()
    e = torch.empty(0, 3, dtype=torch.float32, device=DEV)
    w = ivc.compress_exact(fg, e)
    assert w.shape[0] == 0
    L = ivc.load()
    s = torch.cuda.current_stream().cuda_stream
    import ctypes
    assert L.ivc_compress_exact(ctypes.byref(fg), None, 4, None, None, s) == ivc.IVC_ERR_ARG
    assert L.ivc_decompress_exact(ctypes.byref(fg), None, -1, None, s) == ivc.IVC_ERR_ARG
