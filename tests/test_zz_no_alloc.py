"""ivc_add_noalloc, the compressed add for callers that must not allocate
device memory (its tables sit in a fixed array inside the library instead of
cudaMalloc'd memory): through the C ABI it gives the words ivc_add gives, on
two calls in a row (the second with a different format, so the shared array
is rewritten), and rejects formats whose tables do not fit the array."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2003_02633_gb300 import ivc, synth  # noqa: E402
from parity_util import check_words, formats  # noqa: E402

DEV = "cuda:0"


def _words(w):
    return torch.from_numpy(np.asarray(w, np.uint64).view(np.int64)).to(DEV)


def _run(name, n, seed):
    fo, fg = formats(name)
    a, b = synth.roundtrip_inputs(n, seed=seed)
    wa, wb = _words(O.compress(fo, a)), _words(O.compress(fo, b))
    want = ivc.add(fg, wa, wb)
    got = torch.full_like(wa, -1)
    ivc.add_noalloc(fg, wa, wb, got)
    torch.cuda.synchronize()
    g = got.cpu().numpy().view(np.uint64)
    w = want.cpu().numpy().view(np.uint64)
    with np.errstate(invalid="ignore", over="ignore"):
        pre = O.decompress(fo, O.compress(fo, a)) + O.decompress(fo, O.compress(fo, b))
    check_words(fo, pre, g, w, f"noalloc vs ivc_add ({name})")
    return g


def test_noalloc_matches_ivc_add_twice():
    g1 = _run("primary", (1 << 18) + 3, seed=101)
    g2 = _run("fracsplit", (1 << 16) + 1, seed=102)
    g3 = _run("primary", 4097, seed=103)   # the array is rewritten back
    assert g1.shape[0] > 0 and g2.shape[0] > 0 and g3.shape[0] > 0


def test_noalloc_rejects_oversized_tables():
    L = ivc.load()
    s = torch.cuda.current_stream().cuda_stream
    x = torch.zeros(8, dtype=torch.int64, device=DEV)
    tanh = ivc.make_format(map=1, gamma=0.5)
    assert L.ivc_add_noalloc(ctypes.byref(tanh), x.data_ptr(), x.data_ptr(), x.data_ptr(), 8,
                             s) == ivc.IVC_ERR_UNSUPPORTED
    big = ivc.make_format(map=2, nphi_max_p1=(1 << 18) - 1, phi_bits=20, theta_bits=19)
    st = L.ivc_add_noalloc(ctypes.byref(big), x.data_ptr(), x.data_ptr(), x.data_ptr(), 8, s)
    assert st in (ivc.IVC_ERR_NOMEM, ivc.IVC_ERR_FORMAT)
    torch.cuda.synchronize()
