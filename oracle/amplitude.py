"""Non-unit amplitude a(x, xi) (Sec. 1, eq. FIO), in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the product path never
imports it.

The paper's kernels are K(x, xi) = a(x, xi) e(Phi(x, xi)).  It takes a = 1
for the rest of the paper after observing that a smooth amplitude is
numerically low rank jointly on X x Omega, so that it adds little work.  The
reading followed here: the amplitude is given as a separated sum of q terms,

    a(x, xi) = sum_t alpha_t(x) beta_t(xi),   t = 0 .. q-1,

so that the amplitude operator is

    A = sum_t diag(alpha_t) K_Phi diag(beta_t),

each K_Phi applied by the phase-only IBF.  Factor arrays are column-major:
``alpha`` is (len(x), q), ``beta`` is (N, q).

* ``dense_1d`` / ``dense_2d``: the matrix of eq. DFIO with the amplitude,
  A[n, k] = a(x_n, xi_k) e(Phi(x_n, xi_k)), entrywise (small sizes only).
* ``apply`` / ``adjoint``: A g through any phase-only apply (the oracle's
  IBF, MIBF or direct sum) on the q stacked, scaled copies of g, and the
  conjugate transpose sum_t diag(conj beta_t) K_Phi^* diag(conj alpha_t).
"""
from __future__ import annotations

import numpy as np

from . import direct_1d, direct_2d


def _cols(v, n):
    v = np.asarray(v, np.complex128)
    vec = v.ndim == 1
    return v.reshape(n, -1), vec


def dense_1d(phase_id: int, x, xi, alpha, beta) -> np.ndarray:
    """A[n, k] = (sum_t alpha[n, t] beta[k, t]) e(Phi(x_n, xi_k)) (eq. DFIO
    with a(x, xi)); the phase factor is column k of the direct sum applied to
    the k-th unit vector."""
    xi = np.asarray(xi, np.float64)
    K = direct_1d(phase_id, x, xi, np.eye(xi.size, dtype=np.complex128))
    return (np.asarray(alpha) @ np.asarray(beta).T) * K


def dense_2d(phase_id: int, x, xi, alpha, beta) -> np.ndarray:
    """2D counterpart of ``dense_1d``; x: (nx, 2), xi: (nxi, 2)."""
    xi = np.asarray(xi, np.float64).reshape(-1, 2)
    K = direct_2d(phase_id, x, xi, np.eye(xi.shape[0], dtype=np.complex128))
    return (np.asarray(alpha) @ np.asarray(beta).T) * K


def apply(phase_apply, alpha, beta, g) -> np.ndarray:
    """u = sum_t alpha_t .* K_Phi (beta_t .* g).

    ``phase_apply(G)`` applies the phase-only operator to the columns of an
    (N, m) array; it is called once on the q scaled copies of g side by side
    (copy t in columns t*nrhs .. t*nrhs + nrhs - 1)."""
    alpha = np.asarray(alpha, np.complex128)
    beta = np.asarray(beta, np.complex128)
    q = beta.shape[1]
    g2, vec = _cols(g, beta.shape[0])
    nrhs = g2.shape[1]
    G = np.concatenate([beta[:, t, None] * g2 for t in range(q)], axis=1)
    U = np.asarray(phase_apply(G)).reshape(alpha.shape[0], q * nrhs)
    u = sum(alpha[:, t, None] * U[:, t * nrhs:(t + 1) * nrhs] for t in range(q))
    return u[:, 0] if vec else u


def adjoint(phase_adjoint, alpha, beta, y) -> np.ndarray:
    """g = sum_t conj(beta_t) .* K_Phi^* (conj(alpha_t) .* y), the conjugate
    transpose of ``apply``."""
    alpha = np.asarray(alpha, np.complex128)
    beta = np.asarray(beta, np.complex128)
    q = alpha.shape[1]
    y2, vec = _cols(y, alpha.shape[0])
    nrhs = y2.shape[1]
    Y = np.concatenate([np.conj(alpha[:, t, None]) * y2 for t in range(q)], axis=1)
    Gq = np.asarray(phase_adjoint(Y)).reshape(beta.shape[0], q * nrhs)
    g = sum(np.conj(beta[:, t, None]) * Gq[:, t * nrhs:(t + 1) * nrhs] for t in range(q))
    return g[:, 0] if vec else g
