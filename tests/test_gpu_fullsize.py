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
