"""Oracle of the flux-reconstruction steps 5-11 of Table fr_nse (Sec. 4) with
compressed gradient, metric, normal and flux rows.

TEST INFRASTRUCTURE ONLY: plain FP64 NumPy, written from the definitions;
only the tests, the smoke check and the benchmark's CPU baseline may use it.
It imports nothing from the CUDA package.

Rows (3-vectors) arrive decoded, as FP64 arrays with the components in the
last axis; the callers decode compressed rows with ``oracle.decompress`` first.
Element index e is the last axis before the components.  The one-dimensional
basis (``dm``, ``lm``, ``lp``, ``gl``, ``gr`` on the Gauss-Legendre points) is
an input; this module assembles the dense tensor-product operators from it and
applies them as plain contractions, without the sum factorisation the kernels
use:
  * ``grad_op``    (3, ns, ns): derivative along axis c at point k of the basis
                   function of point j;
  * ``interp_op``  (nf, ns): value at flux point f of the basis function of j;
  * ``lift_op``    (3, ns, nf): derivative along c at k of the correction
                   function of flux point f (zero unless f is on a face of
                   axis c and on the line of k).
Solution point j = (jz q + jy) q + jx; flux point f = (2 c + s) q^2 + b q + a
(face of axis c, side s = 0 at xi_c = -1; a, b the indices along the other
two axes in increasing order).

Readings (the paper lists the steps' operands, Table fr_nse, not their
formulas; these are the standard flux-reconstruction steps on those operands):
  * step 5: the reference-space gradient of the primitives (rho, u, v, w, p);
  * step 6: the gradient plus the lifted interface jump, the input at the flux
    points being the jump w^I - w^f of each primitive;
  * step 7: the corrected gradient rows interpolated to the flux points;
  * step 8: BR1 common viscous flux, the mean of both sides' viscous fluxes
    (physical gradient J^-T grad_xi w = S^T grad_xi w / |J| with S = |J| J^-1
    the metric rows), dotted with this side's scaled normal and subtracted from
    the inviscid normal flux of step 2: n.(F_inv - F_vis);
  * step 9: the reference flux S (F_inv - F_vis) of every equation at the
    solution points (compressible Navier-Stokes, Stokes hypothesis, constant
    viscosity mu and Prandtl number Pr);
  * step 11: the interface flux minus the interior normal flux interpolated to
    the flux point, sign(side) e_c . F.
The partner of flux point (e, f) for step 8 is the matching point of the face
on the other side in the next element along that axis of a periodic
Ex x Ey x Ez mesh, element e = (ez Ey + ey) Ex + ex.
"""
from __future__ import annotations

import numpy as np


def _q(basis) -> int:
    return len(basis["lm"])


def sol_index(q: int):
    """(ns, 3) per-axis indices (jx, jy, jz) of the solution points."""
    return np.array([[j % q, (j // q) % q, j // (q * q)] for j in range(q ** 3)])


def face_points(q: int):
    """(nf, 3) per-axis indices of the flux points (-1 / q for the ends) and
    the (nf,) face 2 c + s of each."""
    pts, face = [], []
    for c in range(3):
        oth = [d for d in range(3) if d != c]
        for s in range(2):
            for b in range(q):
                for a in range(q):
                    ijk = [0, 0, 0]
                    ijk[c] = -1 if s == 0 else q
                    ijk[oth[0]], ijk[oth[1]] = a, b
                    pts.append(ijk)
                    face.append(2 * c + s)
    return np.array(pts), np.array(face)


def grad_op(basis) -> np.ndarray:
    q = _q(basis)
    sj = sol_index(q)
    ns = q ** 3
    dm = np.asarray(basis["dm"], np.float64)
    G = np.zeros((3, ns, ns))
    for c in range(3):
        oth = [d for d in range(3) if d != c]
        for k in range(ns):
            for j in range(ns):
                if all(sj[k, d] == sj[j, d] for d in oth):
                    G[c, k, j] = dm[sj[k, c], sj[j, c]]
    return G


def interp_op(basis) -> np.ndarray:
    q = _q(basis)
    sj = sol_index(q)
    fp, face = face_points(q)
    lm = np.asarray(basis["lm"], np.float64)
    lp = np.asarray(basis["lp"], np.float64)
    I = np.zeros((len(fp), q ** 3))
    for f in range(len(fp)):
        c, s = face[f] // 2, face[f] % 2
        oth = [d for d in range(3) if d != c]
        for j in range(q ** 3):
            if all(sj[j, d] == fp[f, d] for d in oth):
                I[f, j] = (lm if s == 0 else lp)[sj[j, c]]
    return I


def lift_op(basis) -> np.ndarray:
    q = _q(basis)
    sj = sol_index(q)
    fp, face = face_points(q)
    gl = np.asarray(basis["gl"], np.float64)
    gr = np.asarray(basis["gr"], np.float64)
    C = np.zeros((3, q ** 3, len(fp)))
    for f in range(len(fp)):
        c, s = face[f] // 2, face[f] % 2
        oth = [d for d in range(3) if d != c]
        for k in range(q ** 3):
            if all(sj[k, d] == fp[f, d] for d in oth):
                C[c, k, f] = (gl if s == 0 else gr)[sj[k, c]]
    return C


# ------------------------------------------------------------------ steps 5-7


def gradient(w, basis) -> np.ndarray:
    """Step 5: grad w (ns, nv, ne, 3) of scalars w (ns, nv, ne)."""
    return np.einsum("ckj,jpe->kpec", grad_op(basis), np.asarray(w, np.float64))


def correct_gradient(G, dw, basis) -> np.ndarray:
    """Step 6: G (ns, nv, ne, 3) plus the lifted jumps dw (nf, nv, ne)."""
    return np.asarray(G, np.float64) + np.einsum("ckf,fpe->kpec", lift_op(basis),
                                                 np.asarray(dw, np.float64))


def interp_rows(X, basis) -> np.ndarray:
    """Step 7: rows X (ns, nv, ne, 3) at the flux points (nf, nv, ne, 3)."""
    return np.einsum("fj,jpec->fpec", interp_op(basis), np.asarray(X, np.float64))


def flux_correction(F, nF, basis) -> np.ndarray:
    """Step 11: nF (nf, nv, ne) minus sign(side) e_c . (F interpolated to f)."""
    q = _q(basis)
    _, face = face_points(q)
    Ff = interp_rows(F, basis)                                  # (nf, nv, ne, 3)
    sgn = np.where(face % 2 == 0, -1.0, 1.0)
    inner = sgn[:, None, None] * Ff[np.arange(len(face)), :, :, face // 2]
    return np.asarray(nF, np.float64) - inner


# ------------------------------------------------------------- physics (8, 9)


# Every physics function takes ``mag``: with it, the same expression is
# evaluated on absolute values with every subtraction turned into an addition,
# which bounds the size of the terms an FP32 evaluation rounds (the error
# scale of the parity tests).


def primitives(qv, gamma, mag=False):
    """rho, velocity (..., 3), p of conserved q (5, ...)."""
    if mag:
        qv = np.abs(qv)
    rho = qv[0]
    u = np.stack([qv[1] / rho, qv[2] / rho, qv[3] / rho], -1)
    ke = 0.5 * rho * (u * u).sum(-1)
    p = (gamma - 1.0) * (qv[4] + ke if mag else qv[4] - ke)
    return rho, u, p


def inviscid_rows(qv, gamma, mag=False) -> np.ndarray:
    """Euler flux rows (5, ..., 3) (Eq. eulerF)."""
    rho, u, p = primitives(qv, gamma, mag)
    if mag:
        qv = np.abs(qv)
    rows = [qv[0][..., None] * u]
    for i in range(3):
        r = qv[1 + i][..., None] * u
        r[..., i] += p
        rows.append(r)
    rows.append((qv[4] + p)[..., None] * u)
    return np.stack(rows, 0)


def physical_gradient(G, S, detJ, mag=False) -> np.ndarray:
    """grad_x of every primitive: (S^T G) / |J| per point; G (5, ..., 3) rows of
    reference gradients, S (..., 3 rows, 3)."""
    if mag:
        G, S, detJ = np.abs(G), np.abs(S), np.abs(detJ)
    return np.einsum("...ri,v...r->v...i", S, G) / detJ[None, ..., None]


def viscous_rows(qv, gx, gamma, mu, prandtl, mag=False) -> np.ndarray:
    """Viscous flux rows (5, ..., 3): 0, the stress tensor rows, and u . tau +
    kappa grad T, with kappa grad T = mu gamma / ((gamma - 1) Pr) grad(p / rho)
    and gx the physical gradients of (rho, u, v, w, p)."""
    rho, u, p = primitives(qv, gamma, mag)
    if mag:
        gx, u = np.abs(gx), np.abs(u)
    sg = 1.0 if mag else -1.0
    gu = gx[1:4]                                                # (3: u_b, ..., 3: a)
    div = gu[0][..., 0] + gu[1][..., 1] + gu[2][..., 2]
    tau = np.empty(gu.shape)                                    # tau[b][..., a]
    for b in range(3):
        for a in range(3):
            tau[b][..., a] = mu * (gu[b][..., a] + gu[a][..., b])
        tau[b][..., b] += sg * (2.0 / 3.0) * mu * div
    k = mu * gamma / ((gamma - 1.0) * prandtl)
    grad_t = (gx[4] + sg * (p / rho)[..., None] * gx[0]) / rho[..., None]
    energy = sum(u[..., b][..., None] * tau[b] for b in range(3)) + k * grad_t
    return np.stack([np.zeros(tau[0].shape), tau[0], tau[1], tau[2], energy], 0)


def solution_flux(qs, G, S, detJ, gamma, mu, prandtl, mag=False) -> np.ndarray:
    """Step 9: reference flux rows S (F_inv - F_vis) (ns, 5, ne, 3) from q^s
    (ns, 5, ne), gradient rows G (ns, 5, ne, 3), S (ns, 3, ne, 3), |J| (ns, ne)."""
    qv = np.moveaxis(np.asarray(qs, np.float64), 1, 0)           # (5, ns, ne)
    Gv = np.moveaxis(np.asarray(G, np.float64), 1, 0)            # (5, ns, ne, 3)
    Sm = np.moveaxis(np.asarray(S, np.float64), 1, 2)            # (ns, ne, 3, 3)
    gx = physical_gradient(Gv, Sm, np.asarray(detJ, np.float64), mag)
    Fi = inviscid_rows(qv, gamma, mag)
    Fv = viscous_rows(qv, gx, gamma, mu, prandtl, mag)
    Fp = Fi + Fv if mag else Fi - Fv
    Fr = np.einsum("...ri,v...i->v...r", np.abs(Sm) if mag else Sm, Fp)
    return np.moveaxis(Fr, 0, 1)


def partner(dims, q: int):
    """(nf, ne) flat index f' * ne + e' of the point across each flux point."""
    Ex, Ey, Ez = dims
    ne = Ex * Ey * Ez
    _, face = face_points(q)
    e = np.arange(ne)
    ec = [e % Ex, (e // Ex) % Ey, e // (Ex * Ey)]
    nf = len(face)
    out = np.empty((nf, ne), np.int64)
    for f in range(nf):
        c, s = face[f] // 2, face[f] % 2
        n = list(ec)
        n[c] = (ec[c] + (1 if s == 1 else -1)) % dims[c]
        en = (n[2] * Ey + n[1]) * Ex + n[0]
        fo = f + (q * q if s == 0 else -q * q)                   # same (a, b), other side
        out[f] = fo * ne + en
    return out


def common_viscous(Gf, nrm, Sf, detJf, qf, nFinv, dims, gamma, mu, prandtl,
                   mag=False) -> np.ndarray:
    """Step 8: n.(F_inv - F^I_vis) (nf, 5, ne) with F^I_vis the mean of the two
    sides' viscous fluxes (BR1).  Gf (nf, 5, ne, 3), nrm (nf, 1, ne, 3), Sf
    (nf, 3, ne, 3), |J| (nf, ne), qf and nFinv (nf, 5, ne)."""
    nf = Gf.shape[0]
    q = int(round((nf / 6) ** 0.5))
    qv = np.moveaxis(np.asarray(qf, np.float64), 1, 0)
    Gv = np.moveaxis(np.asarray(Gf, np.float64), 1, 0)
    Sm = np.moveaxis(np.asarray(Sf, np.float64), 1, 2)
    gx = physical_gradient(Gv, Sm, np.asarray(detJf, np.float64), mag)
    Fv = viscous_rows(qv, gx, gamma, mu, prandtl, mag)          # (5, nf, ne, 3)
    pr = partner(dims, q)
    Fo = Fv.reshape(5, -1, 3)[:, pr.reshape(-1)].reshape(Fv.shape)
    FI = 0.5 * (Fv + Fo)
    n = np.asarray(nrm, np.float64)[:, 0]                       # (nf, ne, 3)
    nF = np.asarray(nFinv, np.float64)
    if mag:
        return np.abs(nF) + np.moveaxis((FI * np.abs(n)[None]).sum(-1), 0, 1)
    return nF - np.moveaxis((FI * n[None]).sum(-1), 0, 1)
