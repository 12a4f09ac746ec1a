"""Pins of the oracle of the flux-reconstruction steps 5-11 (oracle/fr.py) and
of the one-dimensional basis the inputs carry (synth.fr_basis), against what
the mathematics fixes rather than against their own formulas:

* Lagrange basis: partition of unity, exact derivatives and end values of
  polynomials up to the degree;
* correction functions: the DG weak form (Gauss quadrature of the lifted
  derivative against every basis function gives the surface terms), which
  holds only for the Radau correction functions of Sec. 4's DG recovery;
* gradient, interpolation, lifting operators: exact on tensor-product
  polynomials, and the lifting reproduces the weak form line by line;
* physics: Euler rows of a fluid at rest, simple shear and pure conduction
  closed forms, a traceless symmetric stress, rotation and scaling covariance
  of the metric transform;
* step 8: the partner map joins points that carry the same physical state,
  and the interface flux is conservative (the two sides sum to zero);
* step 11: a flux that is one polynomial across the element, with the exact
  normal flux at the faces, needs no correction.

A plausible mistake (a transposed operator, a swapped side, a sign in the
stress or the heat flux, a wrong partner, S for S^T) fails one of them.
"""
import numpy as np
import pytest

from oracle import fr as R
from paper_2003_02633_gb300 import synth

GAS = dict(gamma=1.4, mu=6.25e-4, prandtl=0.72)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_lagrange_basis_exact_on_polynomials(order):
    B = synth.fr_basis(order)
    xg = B["xg"]
    for m in range(order + 1):
        v = xg ** m
        assert np.allclose(B["dm"] @ v, m * xg ** (m - 1) if m else 0 * xg, atol=1e-12)
        assert B["lm"] @ v == pytest.approx((-1.0) ** m, abs=1e-12)
        assert B["lp"] @ v == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_correction_functions_satisfy_dg_weak_form(order):
    # int g_L' phi = -phi(-1), int g_R' phi = phi(+1) for every phi of degree
    # <= order: Gauss quadrature on the q points is exact for these products
    B = synth.fr_basis(order)
    q = order + 1
    _, wq = np.polynomial.legendre.leggauss(q)
    for a in range(q):        # phi = l_a, the Lagrange basis function of point a
        assert wq[a] * B["gl"][a] == pytest.approx(-B["lm"][a], rel=1e-12, abs=1e-12)
        assert wq[a] * B["gr"][a] == pytest.approx(B["lp"][a], rel=1e-12, abs=1e-12)


def _poly_field(order, ne, seed, npts_idx):
    """Random tensor-product polynomial of degree <= order per axis at the
    given per-axis indices (-1 / q = ends), with its exact gradient."""
    rng = np.random.default_rng(seed)
    B = synth.fr_basis(order)
    q = order + 1
    C = rng.standard_normal((ne, q, q, q))            # coefficients of x^i y^j z^k

    def coord(i):
        return -1.0 if i < 0 else (1.0 if i >= q else B["xg"][i])

    vals = np.zeros((len(npts_idx), ne))
    grads = np.zeros((len(npts_idx), ne, 3))
    for p, (ix, iy, iz) in enumerate(npts_idx):
        x, y, z = coord(ix), coord(iy), coord(iz)
        for i in range(q):
            for j in range(q):
                for k in range(q):
                    c = C[:, i, j, k]
                    vals[p] += c * x ** i * y ** j * z ** k
                    if i:
                        grads[p, :, 0] += c * i * x ** (i - 1) * y ** j * z ** k
                    if j:
                        grads[p, :, 1] += c * j * x ** i * y ** (j - 1) * z ** k
                    if k:
                        grads[p, :, 2] += c * k * x ** i * y ** j * z ** (k - 1)
    return vals, grads


@pytest.mark.parametrize("order", [1, 2, 3])
def test_gradient_and_interpolation_exact(order):
    q = order + 1
    B = synth.fr_basis(order)
    ne = 3
    sol = R.sol_index(q)
    fp, face = R.face_points(q)
    ws, gs = _poly_field(order, ne, 1, sol)
    wf, gf = _poly_field(order, ne, 1, fp)
    G = R.gradient(ws[:, None, :], B)[:, 0]                      # (ns, ne, 3)
    assert np.allclose(G, gs, atol=1e-9)
    Xf = R.interp_rows(gs[:, None], B)[:, 0]                     # gradient rows to faces
    assert np.allclose(Xf, gf, atol=1e-9)
    # the interior normal value at each face point
    F = np.repeat(ws[:, None, :, None], 3, axis=3)
    nF = np.where(face % 2 == 0, -1.0, 1.0)[:, None, None] * wf[:, None, :]
    assert np.allclose(R.flux_correction(F, nF, B), 0.0, atol=1e-9)


@pytest.mark.parametrize("order", [1, 3])
def test_lifting_matches_weak_form(order):
    # with jumps d on the faces, Gauss quadrature of (Gc - G) against each
    # basis function of the line gives d_R l_a(+1) - d_L l_a(-1) along the
    # face's axis, and nothing along the others
    q = order + 1
    B = synth.fr_basis(order)
    _, wq = np.polynomial.legendre.leggauss(q)
    rng = np.random.default_rng(3)
    ns, nf = q ** 3, 6 * q * q
    dw = rng.standard_normal((nf, 1, 2))
    G = rng.standard_normal((ns, 1, 2, 3))
    D = R.correct_gradient(G, dw, B) - G                         # (ns, 1, 2, 3)
    sol = R.sol_index(q)
    fp, face = R.face_points(q)
    for k in range(ns):
        for c in range(3):
            oth = [d for d in range(3) if d != c]
            fL = [f for f in range(nf) if face[f] == 2 * c and
                  all(fp[f, d] == sol[k, d] for d in oth)][0]
            fR = fL + q * q
            a = sol[k, c]
            want = dw[fR, 0] * B["lp"][a] - dw[fL, 0] * B["lm"][a]
            assert np.allclose(wq[a] * D[k, 0, :, c], want, atol=1e-12)


def _state(n, rng, u=None):
    rho = 1.0 + rng.random(n)
    vel = rng.standard_normal((n, 3)) if u is None else np.broadcast_to(u, (n, 3))
    p = 50.0 + rng.random(n)
    E = p / (GAS["gamma"] - 1) + 0.5 * rho * (vel * vel).sum(1)
    return np.stack([rho, rho * vel[:, 0], rho * vel[:, 1], rho * vel[:, 2], E]), rho, vel, p


def test_euler_rows_fluid_at_rest():
    rng = np.random.default_rng(0)
    qv, rho, vel, p = _state(4, rng, u=np.zeros(3))
    F = R.inviscid_rows(qv, GAS["gamma"])
    assert np.allclose(F[0], 0) and np.allclose(F[4], 0)
    for i in range(3):
        want = np.zeros((4, 3))
        want[:, i] = p
        assert np.allclose(F[1 + i], want)


def test_viscous_simple_shear_and_conduction():
    mu, g, pr = GAS["mu"], GAS["gamma"], GAS["prandtl"]
    rng = np.random.default_rng(1)
    # shear u = (s y, 0, 0) at a point with u_x = 2, uniform rho and p
    s = 3.0
    qv, rho, vel, p = _state(1, rng, u=np.array([2.0, 0.0, 0.0]))
    gx = np.zeros((5, 1, 3))
    gx[1, 0, 1] = s                                             # du/dy
    F = R.viscous_rows(qv, gx, g, mu, pr)
    assert np.allclose(F[0], 0)
    assert np.allclose(F[1][0], [0, mu * s, 0]) and np.allclose(F[2][0], [mu * s, 0, 0])
    assert np.allclose(F[3][0], 0)
    assert np.allclose(F[4][0], [0, 2.0 * mu * s, 0])           # u . tau
    # conduction: fluid at rest, dp/dx = 5, uniform rho: k grad(p / rho)
    qv, rho, vel, p = _state(1, rng, u=np.zeros(3))
    gx = np.zeros((5, 1, 3))
    gx[4, 0, 0] = 5.0
    F = R.viscous_rows(qv, gx, g, mu, pr)
    kappa = mu * g / ((g - 1) * pr)
    assert np.allclose(F[4][0], [kappa * 5.0 / rho[0], 0, 0])
    assert np.allclose(F[1:4], 0)
    # density gradient at uniform pressure: T ~ p / rho falls where rho rises
    gx = np.zeros((5, 1, 3))
    gx[0, 0, 2] = 0.25
    F = R.viscous_rows(qv, gx, g, mu, pr)
    assert np.allclose(F[4][0], [0, 0, -kappa * p[0] * 0.25 / rho[0] ** 2])


def test_euler_energy_row_is_enthalpy_flux():
    # (E + p) u = rho H u with the total enthalpy H = c_p T + |u|^2 / 2 and
    # c_p T = gamma p / ((gamma - 1) rho)
    rng = np.random.default_rng(7)
    qv, rho, vel, p = _state(5, rng)
    g = GAS["gamma"]
    H = g * p / ((g - 1) * rho) + 0.5 * (vel * vel).sum(1)
    F = R.inviscid_rows(qv, g)
    assert np.allclose(F[4], (rho * H)[:, None] * vel)
    assert np.allclose(F[0], rho[:, None] * vel)


def test_stress_traceless_symmetric():
    rng = np.random.default_rng(2)
    qv, *_ = _state(6, rng)
    gx = rng.standard_normal((5, 6, 3))
    F = R.viscous_rows(qv, gx, GAS["gamma"], GAS["mu"], GAS["prandtl"])
    tau = F[1:4]                                                # tau[b][n, a]
    assert np.allclose(tau[0][:, 0] + tau[1][:, 1] + tau[2][:, 2], 0, atol=1e-15)
    for a in range(3):
        for b in range(3):
            assert np.allclose(tau[b][:, a], tau[a][:, b])


def _rotation(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return Q * np.sign(np.linalg.det(Q))


def test_flux_metric_rotation_and_scaling():
    # a rotated frame (J = Q^T, S = |J| J^-1 = Q) or a scaled one (J = h I,
    # S = h^2 I): the reference flux is S F(physical gradient)
    rng = np.random.default_rng(4)
    n = 7
    qs, *_ = _state(n, rng)
    gphys = rng.standard_normal((5, n, 3))
    Fphys = (R.inviscid_rows(qs, GAS["gamma"])
             - R.viscous_rows(qs, gphys, GAS["gamma"], GAS["mu"], GAS["prandtl"]))
    for S, det in ((_rotation(rng), 1.0), (np.eye(3) * 0.3 ** 2, 0.3 ** 3)):
        # reference gradient: J^T grad_x with J = det S^-1, i.e. det S^-T grad_x
        gref = det * np.einsum("ri,vnr->vni", np.linalg.inv(S), gphys)
        G = gref[None]                                          # (1, 5, n, 3)
        Sm = np.broadcast_to(S, (1, n, 3, 3)).transpose(0, 2, 1, 3)   # (1, 3 rows, n, 3)
        out = R.solution_flux(qs[None], G, Sm, np.full((1, n), det),
                              **GAS)[0]                         # (5, n, 3)
        want = np.einsum("ri,vni->vnr", S, Fphys)
        assert np.allclose(out, want, rtol=1e-12, atol=1e-9)


def test_partner_map_joins_matching_points():
    dims = (3, 2, 4)
    c = synth.fr_case(dims, order=2, deform=0.15)
    q = 3
    pr = R.partner(dims, q)
    ne = int(np.prod(dims))
    qf = c["q_f"].numpy().reshape(c["q_f"].shape[0], 5, ne)
    flat = np.moveaxis(qf, 1, 2).reshape(-1, 5)                 # (nf * ne, 5)
    mine = np.moveaxis(qf, 1, 2).reshape(-1, 5)
    # the same physical point (up to the FP64 rounding of its coordinates)
    assert np.allclose(flat[pr.reshape(-1)], mine, rtol=1e-6, atol=1e-6)
    assert np.array_equal(pr.reshape(-1)[pr.reshape(-1)], np.arange(pr.size))
    nrm = c["n_f"].numpy()[:, 0].reshape(-1, 3)
    assert np.allclose(nrm[pr.reshape(-1)], -nrm, rtol=1e-6, atol=1e-6)   # opposite normals


def test_common_viscous_conservative_and_inviscid_limit():
    dims = (3, 3, 2)
    c = synth.fr_case(dims, order=2, deform=0.1)
    rng = np.random.default_rng(5)
    nf, ne = c["q_f"].shape[0], c["q_f"].shape[2]
    a = lambda k: c[k].numpy().astype(np.float64)
    Gf = rng.standard_normal((nf, 5, ne, 3))
    out = R.common_viscous(Gf, a("n_f"), a("S_f"), a("detJ_f"), a("q_f"), a("nFinv_f"),
                           dims, **GAS)
    pr = R.partner(dims, 3).reshape(-1)
    flat = np.moveaxis(out, 1, 2).reshape(-1, 5)
    assert np.allclose(flat + flat[pr], 0.0, atol=1e-9)
    # no gradients: the inviscid normal flux alone
    out0 = R.common_viscous(0 * Gf, a("n_f"), a("S_f"), a("detJ_f"), a("q_f"), a("nFinv_f"),
                            dims, **GAS)
    assert np.array_equal(out0, a("nFinv_f"))


def test_mag_bounds_value():
    rng = np.random.default_rng(6)
    n = 7
    qs, *_ = _state(n, rng)
    G = rng.standard_normal((1, 5, n, 3))
    S = rng.standard_normal((1, 3, n, 3))
    det = 1.0 + rng.random((1, n))
    v = R.solution_flux(qs[None], G, S, det, **GAS)
    m = R.solution_flux(qs[None], G, S, det, mag=True, **GAS)
    assert np.all(np.abs(v) <= m * (1 + 1e-12))
