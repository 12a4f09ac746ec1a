"""Pins of the oracle's compressed flux divergence (Algorithm 1, Sec. 4;
Table fr_nse, step 10) against what mathematics fixes, independently of the
oracle's own arithmetic:

* the tensor-product Lagrange operator on 4^3 Gauss-Legendre points
  differentiates polynomials of degree <= 3 per variable exactly, so the
  divergence of such a flux is known in closed form; the oracle's result on the
  compressed flux must match it within the error that compression may add
  (Table 1: normalised error below 1.7187e-5 for <0,7,22>-17-18), summed
  through |D|;
* a constant flux has zero divergence (the same bound);
* swapping the operator's point indices or its axis blocks (plausible
  mistakes) breaks the first pin.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_02633_gb300 import synth

H = 0.5
EMAX = 1.72e-5 + 1e-7   # Table 1 ceiling plus the FP32 rounding of the inputs


def _points(order=3, h=H):
    q = order + 1
    xg, _ = np.polynomial.legendre.leggauss(q)
    ns = q ** 3
    j = np.arange(ns)
    jz, jy, jx = j // (q * q), (j // q) % q, j % q
    return 0.5 * h * xg[jx], 0.5 * h * xg[jy], 0.5 * h * xg[jz]


def _fluxes(x, y, z, shift):
    """Two flux rows of degree <= 3 per variable and their divergences."""
    x, y, z = x + shift[0], y + shift[1], z + shift[2]
    F0 = np.stack([x * x * y, y ** 3 * z, x * y * z * z], axis=-1)
    d0 = 2 * x * y + 3 * y * y * z + 2 * x * y * z
    F1 = np.stack([z ** 3 + 1.0, x * y * y - 2.0, x ** 3 + 0.5 * y], axis=-1)
    d1 = 2 * x * y
    return [F0, F1], [d0, d1]


def _setup(ne=6, seed=0):
    rng = np.random.default_rng(seed)
    x, y, z = _points()
    ns = x.size
    F = np.zeros((ns, 2, ne, 3))
    dv = np.zeros((ns, 2, ne))
    for e in range(ne):
        rows, divs = _fluxes(x, y, z, rng.uniform(-2, 2, 3))
        for p in range(2):
            F[:, p, e] = rows[p]
            dv[:, p, e] = divs[p]
    return ns, F, dv


def _bound(D, F):
    ns = F.shape[0]
    absD = np.abs(D.astype(np.float64)).reshape(3, ns, ns).sum(axis=0)   # (j, k)
    mag = np.linalg.norm(F, axis=-1)                                      # (j, p, e)
    return EMAX * np.einsum("jk,jpe->kpe", absD, mag) + 1e-12


def test_polynomial_flux_divergence_exact_up_to_compression():
    ns, F, dv = _setup()
    D = synth.fr_hex_operator(3, H)
    w = O.compress(O.PRIMARY, F.reshape(-1, 3).astype(np.float32))
    got = O.flux_divergence(O.PRIMARY, w, D, ns, 2)
    err = np.abs(got - dv)
    assert np.all(err <= _bound(D, F)), float((err / _bound(D, F)).max())
    # compression moves the result: the check is not vacuous
    assert err.max() > 0


def test_constant_flux_has_zero_divergence():
    x, y, z = _points()
    ns = x.size
    F = np.broadcast_to(np.array([0.3, -1.7, 2.5]), (ns, 1, 3, 3)).copy()
    D = synth.fr_hex_operator(3, H)
    w = O.compress(O.PRIMARY, F.reshape(-1, 3).astype(np.float32))
    got = O.flux_divergence(O.PRIMARY, w, D, ns, 1)
    # constant up to compression: the decoded rows are identical, so the
    # result is the operator's column sums times them (~1e-6 relative)
    assert np.abs(got).max() <= 1e-5 * np.abs(D).sum(axis=0).max() * 3.0


@pytest.mark.parametrize("mistake", ["transpose_points", "swap_axes"])
def test_plausible_operator_mistakes_fail(mistake):
    ns, F, dv = _setup()
    D = synth.fr_hex_operator(3, H).astype(np.float64).reshape(3, ns, ns)
    if mistake == "transpose_points":
        D = np.transpose(D, (0, 2, 1))
    else:
        D = D[[1, 0, 2]]
    D = D.reshape(3 * ns, ns).astype(np.float32)
    w = O.compress(O.PRIMARY, F.reshape(-1, 3).astype(np.float32))
    got = O.flux_divergence(O.PRIMARY, w, D, ns, 2)
    assert np.any(np.abs(got - dv) > _bound(D, F))
