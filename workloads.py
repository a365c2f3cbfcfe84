"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no arithmetic of the method: it only draws the point sets
and the input vectors of the paper's experiments (Sec. 6) with numpy's seeded
generator, so that both implementations see identical arrays.

Recipes (seed = 16050361600 + workload id unless a test passes its own):
* 1D NUFFT-type, Sec. 6.1: x_j iid U[0,1) sorted, xi_k = k - N/2.
* 1D FIO, Sec. 6.2: x_j = j/N, xi_k = k - N/2.
* 2D FIO, Sec. 6.3: x on the n x n grid of [0,1)^2, xi on [-n/2, n/2)^2.
* g: real and imaginary parts iid N(0,1).
* amplitude factors (non-unit a(x, xi), Sec. 1): ``separated_amplitude``.
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


def separated_amplitude(x, xi, q: int, gen: np.random.Generator, dtype=np.complex128):
    """Factors (alpha, beta) of a synthetic smooth amplitude
    a(x, xi) = sum_t alpha_t(x) beta_t(xi), t < q (Sec. 1: a smooth symbol of
    order zero in xi).  alpha_0 = beta_0 = 1; for t >= 1,
    alpha_t(x) = c_t cos(2 pi t (x_1 + .. + x_d)) + i s_t sin(2 pi t x_1) with
    c_t, s_t iid U(-1/2, 1/2), and beta_t(xi) = (xi_1 / sqrt(1 + |xi|^2))^t.
    x: (nx,) or (nx, d); xi: (N,) or (N, d).  Returns column-major factor
    arrays of shapes (nx, q) and (N, q)."""
    xs = np.asarray(x, np.float64).reshape(len(x), -1)
    ks = np.asarray(xi, np.float64).reshape(len(xi), -1)
    alpha = np.ones((xs.shape[0], q), np.complex128)
    beta = np.ones((ks.shape[0], q), np.complex128)
    c = gen.uniform(-0.5, 0.5, q)
    s = gen.uniform(-0.5, 0.5, q)
    w = ks[:, 0] / np.sqrt(1.0 + (ks * ks).sum(axis=1))
    for t in range(1, q):
        alpha[:, t] = c[t] * np.cos(2 * np.pi * t * xs.sum(axis=1)) + 1j * s[t] * np.sin(2 * np.pi * t * xs[:, 0])
        beta[:, t] = w ** t
    return alpha.astype(dtype), beta.astype(dtype)
