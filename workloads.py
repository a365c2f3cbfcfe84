"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no arithmetic of the method: it only draws the point sets
and the input vectors of the paper's experiments (Sec. 6) with numpy's seeded
generator, so that both implementations see identical arrays.

Recipes (seed = 16050361600 + workload id unless a test passes its own):
* 1D NUFFT-type, Sec. 6.1: x_j iid U[0,1) sorted, xi_k = k - N/2.
* 1D FIO, Sec. 6.2: x_j = j/N, xi_k = k - N/2.
* 2D FIO, Sec. 6.3: x on the n x n grid of [0,1)^2, xi on [-n/2, n/2)^2.
* g: real and imaginary parts iid N(0,1).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 16050361600


def rng(seed: int | None = None, workload: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + workload if seed is None else seed)


def uniform_x(N: int) -> np.ndarray:
    """x_j = j/N (eq. 1D-xandxi)."""
    return np.arange(N, dtype=np.float64) / N


def random_sorted_x(N: int, gen: np.random.Generator) -> np.ndarray:
    """N iid U[0,1) points, sorted ascending (Sec. 6.1)."""
    return np.sort(gen.random(N))


def random_unsorted_x(N: int, gen: np.random.Generator) -> np.ndarray:
    return gen.random(N)


def omega_1d(N: int) -> np.ndarray:
    """xi_k = k - N/2 for k = 0..N-1 (eq. Omega)."""
    return np.arange(N, dtype=np.float64) - N / 2


def grid_x_2d(n: int) -> np.ndarray:
    """(n*n, 2) points (n1/n, n2/n), row-major in (n1, n2) (eq. X)."""
    a = np.arange(n, dtype=np.float64) / n
    X1, X2 = np.meshgrid(a, a, indexing="ij")
    return np.stack([X1.ravel(), X2.ravel()], axis=1)


def omega_2d(n: int) -> np.ndarray:
    """(n*n, 2) integer frequencies in [-n/2, n/2)^2, row-major (eq. Omega)."""
    a = np.arange(n, dtype=np.float64) - n / 2
    K1, K2 = np.meshgrid(a, a, indexing="ij")
    return np.stack([K1.ravel(), K2.ravel()], axis=1)


def complex_normal(shape, gen: np.random.Generator, dtype=np.complex128) -> np.ndarray:
    """Real and imaginary parts iid N(0,1)."""
    re = gen.standard_normal(shape)
    im = gen.standard_normal(shape)
    return (re + 1j * im).astype(dtype)
