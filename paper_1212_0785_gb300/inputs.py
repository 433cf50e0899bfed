"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the HMC arithmetic: it only draws numbers (numpy
PCG64) in the canonical host layouts

  gauge    complex128 (V, 4, 3, 3)   [site][mu][row][col]
  spinor   complex128 (V, 4, 3)      [site][spin][color]
  momentum float64    (V, 4, 8)      [site][mu][Gell-Mann coefficient]

with the site index lexicographic, i = x + Lx(y + Ly(z + Lz t)).  The start
configurations of the benchmarked workloads (exp(i eps H) with Philox Gaussians)
are produced by the library's own gauge-start call, not here.
"""
from __future__ import annotations

import numpy as np


def volume(dims) -> int:
    return int(np.prod(dims))


def parity_of_sites(dims) -> np.ndarray:
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return ((x + y + z + t) % 2).reshape(-1).astype(np.int8)


def random_unitary3(rng: np.random.Generator, n: int, spread: float = 1.0) -> np.ndarray:
    """n random 3x3 special-unitary matrices.  spread=1 gives a broad (Haar-like)
    distribution; small spread gives matrices near the identity.  Built by a QR
    factorisation of identity + spread * complex Gaussian, with the phases of R's
    diagonal moved into Q and the determinant divided out."""
    g = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2)
    a = np.eye(3)[None] + spread * g
    q, r = np.linalg.qr(a)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return q


def random_gauge(dims, seed: int, spread: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    V = volume(dims)
    return random_unitary3(rng, V * 4, spread).reshape(V, 4, 3, 3)


def random_spinor(dims, seed: int, parity: int | None = None) -> np.ndarray:
    """complex Gaussian spinor; parity 0/1 zeroes the sites of the other parity"""
    rng = np.random.default_rng(seed)
    V = volume(dims)
    s = (rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))) / np.sqrt(2)
    if parity is not None:
        s[parity_of_sites(dims) != parity] = 0
    return s


def random_momentum(dims, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal((volume(dims), 4, 8))


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return random_unitary3(rng, volume(dims), 1.0)
