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
