"""Seeded synthetic inputs for the domain-wall solver (gauge links, sources, weights).

This module is shared by the CUDA path's tests/benchmarks and by the CPU oracle's
tests. It holds none of the solver's arithmetic: only random-number generation and
the construction of the input fields the paper's workloads need (Sec. 2.1, Sec. 4).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), turned into 53-bit uniforms and
then into normals by the Box-Muller transform. The generator is counter based, so
each field is a pure function of (seed, tag) and of the lattice size.

Host layouts (Sec. 3.1, "Vector Index Conversion"):
  * 5D spinor: real index c + 24*s + 24*Ns*site, site = x + Nx*(y + Ny*(z + Nz*t)),
    with c = reim + 2*(colour + 3*spin).  A complex view has shape
    (V4, Ns, 4, 3).
  * gauge field: U_mu(x) as a 3x3 complex matrix, layout
    [t][z][y][x][mu][a][b]{re,im}, mu = 0..3 for x, y, z, t.  A complex view has
    shape (V4, 4, 3, 3).
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream tags: each kind of field draws from its own counter stream.
TAG_GAUGE = 1
TAG_SOURCE = 2
TAG_GAUGE_TRANSFORM = 3
TAG_ARRIVALS = 4
TAG_MISC = 5


def _stream_seed(seed: int, tag: int) -> np.uint64:
    return np.uint64(((int(seed) & 0xFFFFFFFFFFFF) << 8 | (tag & 0xFF)) & 0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, tag: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 sequence for (seed, tag)."""
    base = _stream_seed(seed, tag)
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = base + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, tag: int, count: int, offset: int = 0) -> np.ndarray:
    """53-bit uniforms in [0, 1)."""
    z = splitmix64(seed, tag, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normals(seed: int, tag: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller, two per pair of uniforms."""
    npair = (count + 1) // 2
    u = uniforms(seed, tag, 2 * npair)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * npair)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:count]


# ---------------------------------------------------------------- geometry

def volume(dims) -> int:
    nx, ny, nz, nt = dims
    return nx * ny * nz * nt


def site_parity(dims) -> np.ndarray:
    """Parity (x+y+z+t) mod 2 of every site, in lexicographic order (x fastest)."""
    nx, ny, nz, nt = dims
    t, z, y, x = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx),
                             indexing="ij")
    return ((x + y + z + t) & 1).reshape(-1)


# ---------------------------------------------------------------- gauge field

def su3_from_normals(g: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*H) for H = traceless Hermitian part of a Gaussian complex matrix.

    g: (..., 18) normals in (a, b, re/im) order.  Returns (..., 3, 3) complex.
    """
    a = g[..., 0::2] + 1j * g[..., 1::2]
    a = a.reshape(g.shape[:-1] + (3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[..., None, None] * np.eye(3)
    lam, vec = np.linalg.eigh(h)
    ph = np.exp(1j * eps * lam)
    return (vec * ph[..., None, :]) @ np.conj(np.swapaxes(vec, -1, -2))


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Random SU(3) links U_mu(x) = exp(i*eps*H), host layout, float64 (V4*4*18,)."""
    v4 = volume(dims)
    g = normals(seed, TAG_GAUGE, v4 * 4 * 18).reshape(v4, 4, 18)
    u = su3_from_normals(g, eps)
    return np.ascontiguousarray(u).view(np.float64).reshape(-1).copy()


def unit_gauge(dims) -> np.ndarray:
    """Free field U_mu(x) = 1."""
    v4 = volume(dims)
    u = np.zeros((v4, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u.view(np.float64).reshape(-1).copy()


def gauge_transform(dims, seed: int) -> np.ndarray:
    """Random SU(3) matrix Omega(x) per site, complex (V4, 3, 3)."""
    v4 = volume(dims)
    g = normals(seed, TAG_GAUGE_TRANSFORM, v4 * 18).reshape(v4, 18)
    return su3_from_normals(g, 1.0)


# ---------------------------------------------------------------- sources

def gaussian_source(dims, ns: int, seed: int, parity: int | None = None) -> np.ndarray:
    """Complex Gaussian 5D spinor in host layout, float64 (V4*Ns*24,).

    parity=None fills every site; parity=0/1 zeroes the sites of the other parity.
    """
    v4 = volume(dims)
    x = normals(seed, TAG_SOURCE, v4 * ns * 24).reshape(v4, ns * 24)
    if parity is not None:
        x[site_parity(dims) != parity] = 0.0
    return x.reshape(-1).copy()


def point_source(dims, ns: int, spin: int, colour: int) -> np.ndarray:
    """Point source e_{spin,colour} at x = 0.

    Placed on the s-slice where the chirality's wall sits: s = 0 (first slice) for
    spin 0, 1 (P+), s = Ns-1 (last slice) for spin 2, 3 (P-).
    """
    v4 = volume(dims)
    x = np.zeros((v4, ns, 4, 3, 2))
    s = 0 if spin < 2 else ns - 1
    x[0, s, spin, colour, 0] = 1.0
    return x.reshape(-1)


# ---------------------------------------------------------------- 5th-dimension weights

def weights(kind: str, ns: int):
    """(omega, sigma) arrays of length Ns for a named weight set (Sec. 2.1).

    shamir: sigma = 0, omega = 1.  borici: sigma = omega = 1.
    cosine: omega = sigma = 1 + 0.5*cos(pi*(s - 1/2)/Ns), s = 1..Ns (a general
    sigma = omega set with s-dependent weights).
    """
    if kind == "shamir":
        return np.ones(ns), np.zeros(ns)
    if kind == "borici":
        return np.ones(ns), np.ones(ns)
    if kind == "cosine":
        s = np.arange(1, ns + 1)
        w = 1.0 + 0.5 * np.cos(np.pi * (s - 0.5) / ns)
        return w.copy(), w.copy()
    if kind == "symmetric":
        # an R5-symmetric sigma = omega set (omega_s = omega_{Ns+1-s})
        s = np.arange(1, ns + 1)
        w = 1.0 + 0.4 * np.cos(np.pi * (2 * s - ns - 1) / (2 * ns))
        return w.copy(), w.copy()
    raise ValueError(f"unknown weight set {kind!r}")
