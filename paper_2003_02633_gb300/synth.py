"""Seeded synthetic inputs for the compressed-vector kernels.

This module only draws inputs.  It holds none of the compression arithmetic,
and both the CUDA path (tests, benchmark) and the oracle receive the same
arrays from it.

Every host generator uses ``numpy.random.default_rng(seed)`` (PCG64), works in
FP64 and casts to FP32 at the end, as the paper samples its test vectors
(Sec. 2.2: directions drawn in double precision, then converted to single).
The device generator (``device_vectors``) uses a seeded ``torch.Generator`` on
the target device for sizes where host generation would dominate the run.

Workloads (sizes and distributions):
  * ``roundtrip_inputs``: a then b, N = 2^20 each; direction = normalised
    three standard normals, magnitude 10^U(-3, 3); then the 64 edge vectors
    of ``edge_vectors`` appended to each.
  * ``bandwidth_vectors``: the same distribution at any N (the vector-add
    benchmark uses N = 2^28).
  * ``tgv_fields``: Taylor-Green vortex velocity and a pressure-gradient
    forcing at the 64 Gauss-Legendre solution points of each p = 3 hex
    element of a uniform mesh on [-pi, pi]^3.
  * ``batched_fields``: 256 fields, lengths floor(2^U(10, 24)), each with its
    own magnitude window inside [1e-6, 1e6].
  * ``precision_vectors``: magnitudes 10^U(-30, 30), 10% of directions
    within 1e-3 rad of a pole.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["unit_sphere", "unit_cube", "random_vectors", "edge_vectors",
           "roundtrip_inputs", "bandwidth_vectors", "device_vectors", "tgv_fields",
           "batched_lengths", "batched_fields", "precision_vectors", "random_words"]


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _directions(rng: np.random.Generator, n: int) -> np.ndarray:
    g = rng.standard_normal((n, 3))
    nrm = np.linalg.norm(g, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return g / nrm


def unit_sphere(n: int, seed: int = 0) -> np.ndarray:
    """n directions uniform on the unit sphere, drawn in FP64, stored as FP32."""
    return _f32(_directions(np.random.default_rng(seed), n))


def unit_cube(n: int, seed: int = 0) -> np.ndarray:
    """n points uniform in [-1, 1]^3 (FP64 draw, FP32 store)."""
    return _f32(np.random.default_rng(seed).uniform(-1.0, 1.0, (n, 3)))


def random_vectors(n: int, seed: int = 0, lo: float = -3.0, hi: float = 3.0,
                   rng: np.random.Generator | None = None) -> np.ndarray:
    """Uniform directions with magnitude 10^U(lo, hi)."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    d = _directions(rng, n)
    mag = 10.0 ** rng.uniform(lo, hi, (n, 1))
    return _f32(d * mag)


def edge_vectors() -> np.ndarray:
    """The 64 edge vectors: signed zeros, axis vectors over the magnitude range,
    exact poles, the theta seam, the theta and phi ties, range limits, FP32
    subnormals, non-finite components and exact-tie magnitudes."""
    inf, nan = float("inf"), float("nan")
    e = []
    e += [(0.0, 0.0, 0.0), (-0.0, 0.0, 0.0), (0.0, -0.0, 0.0), (0.0, 0.0, -0.0),
          (-0.0, -0.0, -0.0)]
    for r in (1.0, 1e-3, 1e3, 2.0 ** -79, float(np.nextafter(np.float32(2.0 ** 47),
                                                             np.float32(0)))):
        for ax in range(3):
            for s in (1.0, -1.0):
                v = [0.0, 0.0, 0.0]
                v[ax] = s * r
                e.append(tuple(v))
    e += [(0.0, 0.0, 2.5), (0.0, -0.0, -7e-5)]                 # exact poles
    e += [(-1.0, 0.0, 0.5), (-1.0, -0.0, 0.5), (-3.0, 0.0, -2.0), (-3.0, -0.0, -2.0)]  # seam
    e += [(2.0, 0.0, 1.0), (2.0, -0.0, -1.0), (5e-3, 0.0, 0.0)]  # theta tie
    e += [(1.0, 1.0, 0.0), (-2.0, 3.0, 0.0), (0.3, -0.7, -0.0)]  # phi tie
    e += [(3 * 2.0 ** -81, 4 * 2.0 ** -81, 0.0),                 # just above the lowest value
          (2.0 ** 47, 0.0, 0.0), (1e20, 1e20, 1e20),             # overflow
          (1e-30, 0.0, 0.0), (1e-25, 1e-25, 0.0)]                # underflow
    e += [(1e-40, 0.0, 0.0), (1.0, 1e-40, 0.0), (1.0, -1e-40, 0.0)]  # FP32 subnormals
    e += [(inf, 0.0, 0.0), (nan, 1.0, 1.0), (-inf, inf, 0.0)]    # non-finite
    e += [(3e38, 3e38, 0.0), (1e30, 2e30, -3e30)]                # squares overflow FP32
    # |(a, b, 0)| = c exactly, c an odd 25-bit integer: the FP32 norm is an exact
    # rounding tie (the first between an odd and an even mantissa, the second
    # between an even and an odd one).
    e += [(1221901.0, 16745580.0, 0.0)]
    e += [_pythagorean_tie(odd_low=True)]
    assert len(e) <= 64, len(e)
    while len(e) < 64:
        k = len(e)
        e.append((math.ldexp(1.0, k - 60), -math.ldexp(1.5, 20 - k), math.ldexp(1.25, k % 7)))
    return _f32(np.array(e, dtype=np.float64))


def _pythagorean_tie(odd_low: bool) -> tuple:
    """A vector (a, b, 0) with a, b < 2^24 and a^2 + b^2 = c^2, c odd in
    [2^24, 2^25): its norm is halfway between two FP32 numbers.  With odd_low
    the lower neighbour has an odd last mantissa bit (a primitive hypotenuse is
    1 mod 4, so that case scales a primitive triple by 3)."""
    k = 3 if odd_low else 1
    for u in range(800, 4300):
        for v in range(1, u):
            if (u - v) % 2 == 0 or math.gcd(u, v) != 1:
                continue
            c = k * (u * u + v * v)
            a, b = k * (u * u - v * v), k * 2 * u * v
            if not (1 << 24) <= c < (1 << 25) or max(a, b) >= (1 << 24):
                continue
            low_mant = ((c - 1) - (1 << 24)) // 2
            if (low_mant % 2 == 1) == odd_low:
                return (float(a), float(b), 0.0)
    raise RuntimeError("no tie vector found")


def roundtrip_inputs(n: int = 1 << 20, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(a, b): n vectors each (a drawn first, then b), magnitudes 10^U(-3,3),
    with the 64 edge vectors appended to both."""
    rng = np.random.default_rng(seed)
    a = random_vectors(n, rng=rng)
    b = random_vectors(n, rng=rng)
    e = edge_vectors()
    eb = np.roll(e, 7, axis=0)
    return (np.concatenate([a, e]), np.concatenate([b, eb]))


def bandwidth_vectors(n: int, seed: int = 0) -> np.ndarray:
    """The vector-add workload distribution (magnitude 10^U(-3,3)) at size n."""
    return random_vectors(n, seed=seed)


def device_vectors(n: int, seed: int, device, lo: float = -3.0, hi: float = 3.0):
    """Same distribution as ``random_vectors``, drawn on a torch device with a
    seeded torch.Generator (FP64 draw, FP32 store), generated in chunks.
    Returns an (n, 3) float32 tensor on ``device``."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty((n, 3), dtype=torch.float32, device=device)
    chunk = 1 << 24
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        d = torch.randn((m, 3), dtype=torch.float64, device=device, generator=g)
        d /= torch.linalg.vector_norm(d, dim=1, keepdim=True).clamp_min(1e-300)
        mag = 10.0 ** (lo + (hi - lo) * torch.rand((m, 1), dtype=torch.float64, device=device,
                                                   generator=g))
        out[s:s + m] = (d * mag).to(torch.float32)
    return out


def tgv_fields(elements_per_axis: int = 96, order: int = 3, p0: float = 100.0,
               rho0: float = 1.0, u0: float = 1.0):
    """Taylor-Green vortex (Sec. 4.2, Eq. tgv_xyz, k = 1) sampled at the
    (order+1)^3 Gauss-Legendre solution points of each hex element of a
    uniform mesh on [-pi, pi]^3; point index = element * (order+1)^3 + node.

    Returns (v, f, rho) as FP32: v the velocity, f = -grad(p)/rho the pointwise
    pressure-gradient forcing, rho = p rho0 / p0 (Boyle's law)."""
    q = order + 1
    xg, _ = np.polynomial.legendre.leggauss(q)
    h = 2.0 * math.pi / elements_per_axis
    ecent = -math.pi + h * (np.arange(elements_per_axis) + 0.5)
    # coordinates per axis: element-major, node-minor
    ax = (ecent[:, None] + 0.5 * h * xg[None, :])           # (E, q)
    E = elements_per_axis
    # element (ez, ey, ex) and node (kz, ky, kx) ordering
    X = ax[None, None, :, None, None, :]
    Y = ax[None, :, None, None, :, None]
    Z = ax[:, None, None, :, None, None]
    shape = (E, E, E, q, q, q)
    X = np.broadcast_to(X, shape)
    Y = np.broadcast_to(Y, shape)
    Z = np.broadcast_to(Z, shape)
    perm = (0, 1, 2, 3, 4, 5)
    X = np.transpose(X, perm).reshape(-1)
    Y = np.transpose(Y, perm).reshape(-1)
    Z = np.transpose(Z, perm).reshape(-1)
    u = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    c = rho0 * u0 * u0 / 16.0
    p = p0 + c * (np.cos(2 * X) + np.cos(2 * Y)) * (2 + np.cos(2 * Z))
    rho = p * rho0 / p0
    dpdx = c * (-2 * np.sin(2 * X)) * (2 + np.cos(2 * Z))
    dpdy = c * (-2 * np.sin(2 * Y)) * (2 + np.cos(2 * Z))
    dpdz = c * (np.cos(2 * X) + np.cos(2 * Y)) * (-2 * np.sin(2 * Z))
    f = -np.stack([dpdx, dpdy, dpdz], axis=1) / rho[:, None]
    vel = np.stack([u, v, w], axis=1)
    return _f32(vel), _f32(f), _f32(rho)


def batched_lengths(nfields: int = 256, seed: int = 0, lo_log2: float = 10.0,
                    hi_log2: float = 24.0) -> np.ndarray:
    """Field lengths floor(2^U(lo, hi))."""
    rng = np.random.default_rng(seed)
    return np.floor(2.0 ** rng.uniform(lo_log2, hi_log2, nfields)).astype(np.int64)


def batched_fields(nfields: int = 256, seed: int = 0, scale: float = 1.0):
    """Lengths and per-field magnitude windows: field i has magnitudes
    10^U(c - w/2, c + w/2) with w ~ U(1, 4) decades and c ~ U(-6 + w/2, 6 - w/2).
    ``scale`` < 1 shrinks every length (for tests).  Returns (lengths, windows)
    with windows an (nfields, 2) array of log10 bounds."""
    rng = np.random.default_rng(seed)
    lens = np.floor(2.0 ** rng.uniform(10.0, 24.0, nfields))
    lens = np.maximum(1, np.floor(lens * scale)).astype(np.int64)
    w = rng.uniform(1.0, 4.0, nfields)
    c = rng.uniform(-6.0 + w / 2, 6.0 - w / 2)
    return lens, np.stack([c - w / 2, c + w / 2], axis=1)


def precision_vectors(n: int, seed: int = 0, polar_fraction: float = 0.1,
                      cap: float = 1e-3) -> np.ndarray:
    """Magnitudes 10^U(-30, 30); 90% of directions uniform on the sphere, 10%
    with polar angle within ``cap`` of 0 or pi (uniform on the cap) and uniform
    azimuth."""
    rng = np.random.default_rng(seed)
    d = _directions(rng, n)
    k = int(round(polar_fraction * n))
    idx = rng.permutation(n)[:k]
    cosd = rng.uniform(math.cos(cap), 1.0, k)
    sind = np.sqrt(np.maximum(0.0, 1.0 - cosd * cosd))
    az = rng.uniform(-math.pi, math.pi, k)
    sgn = np.where(rng.uniform(0, 1, k) < 0.5, -1.0, 1.0)
    d[idx] = np.stack([sind * np.cos(az), sind * np.sin(az), sgn * cosd], axis=1)
    mag = 10.0 ** rng.uniform(-30.0, 30.0, (n, 1))
    return _f32(d * mag)


def random_words(n: int, seed: int = 0, exp_bits: int = 7, man_bits: int = 22,
                 phi_bits: int = 17, theta_bits: int = 18) -> np.ndarray:
    """Uniformly random bit fields (exponent in 1 .. 2^e-2) packed MSB-first
    as exponent | mantissa | n_phi | n_theta.  Includes non-canonical words."""
    rng = np.random.default_rng(seed)
    E = rng.integers(1, (1 << exp_bits) - 1, n, dtype=np.uint64)
    m = rng.integers(0, 1 << man_bits, n, dtype=np.uint64)
    p = rng.integers(0, 1 << phi_bits, n, dtype=np.uint64)
    t = rng.integers(0, 1 << theta_bits, n, dtype=np.uint64)
    sm = np.uint64(theta_bits + phi_bits)
    se = np.uint64(theta_bits + phi_bits + man_bits)
    return (E << se) | (m << sm) | (p << np.uint64(theta_bits)) | t


def tgv_fields_device(elements_per_axis: int, device, order: int = 3, p0: float = 100.0,
                      rho0: float = 1.0, u0: float = 1.0):
    """``tgv_fields`` evaluated on a torch device (FP64, stored FP32), for mesh
    sizes where the host version would be slow.  Same point ordering."""
    import torch
    q = order + 1
    xg, _ = np.polynomial.legendre.leggauss(q)
    E = elements_per_axis
    h = 2.0 * math.pi / E
    ecent = -math.pi + h * (torch.arange(E, dtype=torch.float64, device=device) + 0.5)
    ax = (ecent[:, None] + 0.5 * h * torch.tensor(xg, dtype=torch.float64, device=device)[None, :])
    shape = (E, E, E, q, q, q)
    X = ax[None, None, :, None, None, :].expand(shape).reshape(-1)
    Y = ax[None, :, None, None, :, None].expand(shape).reshape(-1)
    Z = ax[:, None, None, :, None, None].expand(shape).reshape(-1)
    u = u0 * torch.sin(X) * torch.cos(Y) * torch.cos(Z)
    v = -u0 * torch.cos(X) * torch.sin(Y) * torch.cos(Z)
    w = torch.zeros_like(u)
    c = rho0 * u0 * u0 / 16.0
    p = p0 + c * (torch.cos(2 * X) + torch.cos(2 * Y)) * (2 + torch.cos(2 * Z))
    rho = p * rho0 / p0
    f = -torch.stack([c * (-2 * torch.sin(2 * X)) * (2 + torch.cos(2 * Z)),
                      c * (-2 * torch.sin(2 * Y)) * (2 + torch.cos(2 * Z)),
                      c * (torch.cos(2 * X) + torch.cos(2 * Y)) * (-2 * torch.sin(2 * Z))],
                     dim=1) / rho[:, None]
    vel = torch.stack([u, v, w], dim=1)
    return vel.float().contiguous(), f.float().contiguous(), rho.float().contiguous()


def fr_hex_operator(order: int = 3, h: float = 1.0) -> np.ndarray:
    """Divergence operator of a flux-reconstruction hex element (Sec. 4,
    Algorithm 1): D[c * ns + j, k] = d l_j / d x_c at solution point k, with
    l_j the tensor-product Lagrange basis on the (order+1)^3 Gauss-Legendre
    points of a cube of side h (reference [-1, 1]^3, scaled by 2 / h).
    Point j = (jz q + jy) q + jx, q = order + 1.  Returns float32 (3 ns, ns)."""
    q = order + 1
    xg, _ = np.polynomial.legendre.leggauss(q)
    # 1-D derivative matrix L[b, a] = l_b'(xi_a)
    L = np.zeros((q, q))
    for b in range(q):
        others = np.delete(xg, b)
        coef = np.polynomial.polynomial.polyfromroots(others) / np.prod(xg[b] - others)
        L[b] = np.polynomial.polynomial.polyval(xg, np.polynomial.polynomial.polyder(coef))
    ns = q ** 3
    D = np.zeros((3 * ns, ns))
    eye = np.eye(q)
    for j in range(ns):
        jz, jy, jx = j // (q * q), (j // q) % q, j % q
        for k in range(ns):
            kz, ky, kx = k // (q * q), (k // q) % q, k % q
            D[0 * ns + j, k] = L[jx, kx] * eye[jy, ky] * eye[jz, kz]
            D[1 * ns + j, k] = eye[jx, kx] * L[jy, ky] * eye[jz, kz]
            D[2 * ns + j, k] = eye[jx, kx] * eye[jy, ky] * L[jz, kz]
    return (D * (2.0 / h)).astype(np.float32)


def tgv_euler_flux(elements_per_axis: int = 96, order: int = 3, p0: float = 100.0,
                   rho0: float = 1.0, u0: float = 1.0, gamma: float = 1.4, device="cpu",
                   elements=None):
    """Inviscid (Euler) flux of the Taylor-Green vortex initial state (Sec. 4.2,
    Eq. tgv_xyz, k = 1) at the (order+1)^3 Gauss-Legendre solution points of the
    hex elements of a uniform mesh on [-pi, pi]^3, as the five flux rows of the
    conserved variables: rho u, rho u u + p e_x, rho u v + p e_y, rho u w + p e_z,
    (E + p) u with E = p / (gamma - 1) + rho |u|^2 / 2 and rho = p rho0 / p0.

    Layout for the divergence kernel: float32 torch tensor (ns, 5, ne, 3),
    element index fastest; element e = (ez E + ey) E + ex.  ``elements`` limits
    the count to the first ones (tests).  Computed in FP64 on ``device``."""
    import torch
    q = order + 1
    ns = q ** 3
    E = elements_per_axis
    ne = E ** 3 if elements is None else int(elements)
    xg, _ = np.polynomial.legendre.leggauss(q)
    h = 2.0 * math.pi / E
    dev = torch.device(device)
    e = torch.arange(ne, device=dev, dtype=torch.int64)
    ez, ey, ex = e // (E * E), (e // E) % E, e % E
    xgt = torch.tensor(xg, device=dev, dtype=torch.float64)
    out = torch.empty((ns, 5, ne, 3), device=dev, dtype=torch.float32)
    c = rho0 * u0 * u0 / 16.0
    for j in range(ns):
        jz, jy, jx = j // (q * q), (j // q) % q, j % q
        X = -math.pi + h * (ex.double() + 0.5) + 0.5 * h * xgt[jx]
        Y = -math.pi + h * (ey.double() + 0.5) + 0.5 * h * xgt[jy]
        Z = -math.pi + h * (ez.double() + 0.5) + 0.5 * h * xgt[jz]
        u = u0 * torch.sin(X) * torch.cos(Y) * torch.cos(Z)
        v = -u0 * torch.cos(X) * torch.sin(Y) * torch.cos(Z)
        w = torch.zeros_like(u)
        p = p0 + c * (torch.cos(2 * X) + torch.cos(2 * Y)) * (2 + torch.cos(2 * Z))
        rho = p * rho0 / p0
        Et = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
        vel = torch.stack([u, v, w], dim=1)
        rows = [rho[:, None] * vel,
                rho[:, None] * u[:, None] * vel + torch.stack([p, 0 * p, 0 * p], dim=1),
                rho[:, None] * v[:, None] * vel + torch.stack([0 * p, p, 0 * p], dim=1),
                rho[:, None] * w[:, None] * vel + torch.stack([0 * p, 0 * p, p], dim=1),
                (Et + p)[:, None] * vel]
        out[j] = torch.stack(rows, dim=0).to(torch.float32)
    return out


# ----------------------------------------------------------------------------
# Flux-reconstruction element data for the steps of Table fr_nse (Sec. 4)


def fr_basis(order: int = 3) -> dict:
    """One-dimensional flux-reconstruction basis on the order+1 Gauss-Legendre
    points xi_i of [-1, 1] (Sec. 4: tensor-product Gauss-Legendre solution and
    flux points), FP64:
      xg  the points;
      dm  dm[i, a] = l_a'(xi_i), derivative of the Lagrange basis function a;
      lm, lp  l_a(-1), l_a(+1): interpolation to the two ends;
      gl, gr  g_L'(xi_i), g_R'(xi_i): derivatives of the DG correction
              functions (right and left Radau polynomials of degree order+1,
              g_L(-1) = 1, g_L(1) = 0, g_R(xi) = g_L(-xi))."""
    q = order + 1
    xg, _ = np.polynomial.legendre.leggauss(q)
    P = np.polynomial.polynomial
    dm = np.zeros((q, q))
    lm = np.zeros(q)
    lp = np.zeros(q)
    for a in range(q):
        others = np.delete(xg, a)
        coef = P.polyfromroots(others) / np.prod(xg[a] - others)
        dm[:, a] = P.polyval(xg, P.polyder(coef))
        lm[a] = P.polyval(-1.0, coef)
        lp[a] = P.polyval(1.0, coef)
    L = np.polynomial.legendre
    ek = np.zeros(q + 1)
    ek[order] = 1.0
    ek1 = np.zeros(q + 1)
    ek1[order + 1] = 1.0
    sgn = (-1.0) ** (order + 1) / 2.0
    gL = sgn * (ek1 - ek)                      # Legendre coefficients of g_L
    gl = L.legval(xg, L.legder(gL))
    gr = -L.legval(-xg, L.legder(gL))           # g_R(xi) = g_L(-xi)
    return {"order": order, "xg": xg, "dm": dm, "lm": lm, "lp": lp, "gl": gl, "gr": gr}


def fr_face_points(order: int):
    """Flux-point numbering of a hex: face = 2 c + s (axis c = 0, 1, 2 for x,
    y, z; side s = 0 at xi_c = -1, 1 at +1), point f = face q^2 + b q + a with
    (a, b) the point's indices along the other two axes in increasing order.
    Returns an (nf, 3) int array of per-axis indices with -1 / q standing for
    the ends xi_c = -1 / +1, and the (nf,) face of each point."""
    q = order + 1
    pts, face = [], []
    for c in range(3):
        oth = [d for d in range(3) if d != c]
        for s in range(2):
            for b in range(q):
                for a in range(q):
                    ijk = [0, 0, 0]
                    ijk[c] = -1 if s == 0 else q
                    ijk[oth[0]] = a
                    ijk[oth[1]] = b
                    pts.append(ijk)
                    face.append(2 * c + s)
    return np.array(pts), np.array(face)


def _euler_rows_t(qv, gamma):
    """Inviscid flux rows (5, ..., 3) of conserved q (5, ...) (Eq. eulerF)."""
    import torch
    rho = qv[0]
    u = torch.stack([qv[1] / rho, qv[2] / rho, qv[3] / rho], dim=-1)
    p = (gamma - 1.0) * (qv[4] - 0.5 * rho * (u * u).sum(-1))
    rows = [qv[0][..., None] * u]
    for i in range(3):
        r = qv[1 + i][..., None] * u
        r[..., i] = r[..., i] + p
        rows.append(r)
    rows.append((qv[4] + p)[..., None] * u)
    return torch.stack(rows, dim=0)


def fr_case(dims=(4, 4, 4), order: int = 3, deform: float = 0.1, perturb: float = 0.05,
            p0: float = 100.0, rho0: float = 1.0, u0: float = 1.0, gamma: float = 1.4,
            device="cpu") -> dict:
    """Element data of the flux-reconstruction steps 5-11 of Table fr_nse on a
    periodic mesh of Ex x Ey x Ez hexes covering [-pi, pi]^3, mapped by
    x = P + deform (sin Py sin Pz, sin Pz sin Px, sin Px sin Py) (a smooth
    periodic deformation of the uniform mesh; 0 gives the uniform mesh of the
    paper's Taylor-Green runs).  Element e = (ez Ey + ey) Ex + ex.

    Flow: the Taylor-Green vortex initial state (Sec. 4.2, p0 = 100) plus a
    smooth periodic perturbation of relative size `perturb` in every primitive
    (so that no gradient row is identically zero, as in the developed flow):
      u = u0 (sin X cos Y cos Z + perturb sin(Y + Z)),
      v = u0 (-cos X sin Y cos Z + perturb sin(Z + X)),
      w = u0 perturb sin(X + Y),
      p = p0 + rho0 u0^2 ((cos 2X + cos 2Y)(2 + cos 2Z) / 16 + perturb cos(X + Y + Z)),
      rho = p rho0 / p0.

    Returns FP32 torch tensors on `device` (FP64 arithmetic), element index
    fastest; "row" tensors hold 3-vectors in the last axis:
      w_s  (ns, 5, ne)     primitives rho, u, v, w, p at the solution points
      q_s  (ns, 5, ne)     conserved rho, rho u, rho v, rho w, E
      S_s  (ns, 3, ne, 3)  rows of S = |J| J^-1 (J = dx/dxi), the metric terms
      detJ_s (ns, ne)      |J|
      q_f, S_f, detJ_f     the same at the flux points (nf in place of ns)
      n_f  (nf, 1, ne, 3)  scaled outward normal, sign(side) * row c of S
      dw_f (nf, 5, ne)     jump w(x_f) - (interpolated w^s) of the primitives
      nFinv_f (nf, 5, ne)  n_f . F_inv(q_f), the inviscid normal flux
    plus "dims", "order", "gamma"."""
    import torch
    dev = torch.device(device)
    Ex, Ey, Ez = dims
    ne = Ex * Ey * Ez
    B = fr_basis(order)
    q = order + 1
    ns = q ** 3
    xg = B["xg"]
    e = torch.arange(ne, device=dev, dtype=torch.int64)
    eidx = [e % Ex, (e // Ex) % Ey, e // (Ex * Ey)]
    hs = [2.0 * math.pi / Ex, 2.0 * math.pi / Ey, 2.0 * math.pi / Ez]
    t64 = dict(device=dev, dtype=torch.float64)

    def ref_coord(idx):                    # index -1 / q = end, else GL point
        if idx < 0:
            return -1.0
        if idx >= q:
            return 1.0
        return float(xg[idx])

    def geometry(ijk):
        """Mapped coordinates (3, npts, ne), S (npts, 3, ne, 3), |J| (npts, ne)."""
        npts = len(ijk)
        xi = torch.tensor([[ref_coord(i) for i in p] for p in ijk], **t64)   # (npts, 3)
        P = [(-math.pi + hs[c] * (eidx[c].double()[None, :] + 0.5)
              + 0.5 * hs[c] * xi[:, c:c + 1]) for c in range(3)]            # (npts, ne)
        sx, sy, sz = torch.sin(P[0]), torch.sin(P[1]), torch.sin(P[2])
        cx, cy, cz = torch.cos(P[0]), torch.cos(P[1]), torch.cos(P[2])
        A = deform
        X = [P[0] + A * sy * sz, P[1] + A * sz * sx, P[2] + A * sx * sy]
        one = torch.ones_like(sx)
        dM = [[one, A * cy * sz, A * sy * cz],
              [A * sz * cx, one, A * cz * sx],
              [A * cx * sy, A * sx * cy, one]]
        # columns of J = dx/dxi; S = |J| J^-1 is the adjugate, whose row r is
        # the cross product of columns r + 1 and r + 2
        cols = [torch.stack([dM[i][j] * (0.5 * hs[j]) for i in range(3)], -1) for j in range(3)]
        S = torch.stack([torch.linalg.cross(cols[(r + 1) % 3], cols[(r + 2) % 3], dim=-1)
                         for r in range(3)], 1)                             # (npts, 3, ne, 3)
        det = (cols[0] * S[:, 0]).sum(-1)
        return X, S.contiguous(), det

    def flow(X):
        x, y, z = X
        u = u0 * (torch.sin(x) * torch.cos(y) * torch.cos(z) + perturb * torch.sin(y + z))
        v = u0 * (-torch.cos(x) * torch.sin(y) * torch.cos(z) + perturb * torch.sin(z + x))
        w = u0 * perturb * torch.sin(x + y)
        p = p0 + rho0 * u0 * u0 * ((torch.cos(2 * x) + torch.cos(2 * y)) * (2 + torch.cos(2 * z))
                                   / 16.0 + perturb * torch.cos(x + y + z))
        rho = p * rho0 / p0
        prim = torch.stack([rho, u, v, w, p], 0)                           # (5, npts, ne)
        En = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
        cons = torch.stack([rho, rho * u, rho * v, rho * w, En], 0)
        return prim, cons

    sol = [[jx, jy, jz] for jz in range(q) for jy in range(q) for jx in range(q)]
    Xs, S_s, det_s = geometry(sol)
    w_s, q_s = flow(Xs)
    fpts, face = fr_face_points(order)
    Xf, S_f, det_f = geometry(fpts.tolist())
    w_f, q_f = flow(Xf)
    nf = len(fpts)
    # scaled normals: sign(side) * row c of S
    cf = torch.tensor(face // 2, device=dev)
    sg = torch.tensor(np.where(face % 2 == 0, -1.0, 1.0), **t64)
    n_f = sg[:, None, None] * S_f[torch.arange(nf, device=dev), cf]        # (nf, ne, 3)
    # interpolated interior primitives at the flux points
    wsr = w_s.reshape(5, q, q, q, ne)                                      # (v, jz, jy, jx, e)
    wint = torch.empty((5, nf, ne), **t64)
    lm = torch.tensor(B["lm"], **t64)
    lp = torch.tensor(B["lp"], **t64)
    for f in range(nf):
        c, s = face[f] // 2, face[f] % 2
        ijk = fpts[f]
        wl = lm if s == 0 else lp
        sel = [ijk[2], ijk[1], ijk[0]]                                     # (jz, jy, jx)
        sel[2 - c] = slice(None)
        line = wsr[:, sel[0], sel[1], sel[2]]                              # (5, q, ne)
        wint[:, f] = (wl[None, :, None] * line).sum(1)
    dw_f = w_f - wint
    Finv = _euler_rows_t(q_f, gamma)                                       # (5, nf, ne, 3)
    nFinv = (Finv * n_f[None]).sum(-1)
    f32 = lambda t: t.to(torch.float32).contiguous()
    return {
        "dims": tuple(dims), "order": order, "gamma": gamma,
        "w_s": f32(w_s.permute(1, 0, 2)), "q_s": f32(q_s.permute(1, 0, 2)),
        "S_s": f32(S_s), "detJ_s": f32(det_s),
        "q_f": f32(q_f.permute(1, 0, 2)), "S_f": f32(S_f), "detJ_f": f32(det_f),
        "n_f": f32(n_f[:, None]), "dw_f": f32(dw_f.permute(1, 0, 2)),
        "nFinv_f": f32(nFinv.permute(1, 0, 2)),
    }
