"""Pins of the oracle's non-unit amplitude (Sec. 1, eq. FIO with a(x, xi)).

The amplitude operator sum_t diag(alpha_t) K_Phi diag(beta_t) is checked
against the dense matrix a(x_n, xi_k) e(Phi(x_n, xi_k)) written entrywise
(exact through the direct sum; exact through the IBF for the separable test
phase, whose butterfly is exact), against the plain IBF for a = 1 and for a
constant amplitude, and its adjoint against the dot-product identity and the
dense conjugate transpose.  Swapping alpha and beta, dropping a conjugate or
an amplitude term, or shifting the stacked columns fails one of them."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import amplitude as A


def _setup_1d(phase, N, q, seed, nrhs=3):
    gen = W.rng(seed)
    x = W.random_sorted_x(N, gen) if phase == O.PHASE_NUFFT else W.uniform_x(N)
    xi = W.omega_1d(N)
    alpha, beta = W.separated_amplitude(x, xi, q, gen)
    g = W.complex_normal((N, nrhs), gen)
    return x, xi, alpha, beta, g


def test_direct_route_equals_dense_definition():
    N, q = 128, 4
    x, xi, alpha, beta, g = _setup_1d(O.PHASE_FIO1D, N, q, 901)
    D = A.dense_1d(O.PHASE_FIO1D, x, xi, alpha, beta)
    u = A.apply(lambda G: O.direct_1d(O.PHASE_FIO1D, x, xi, G), alpha, beta, g)
    assert O.rel_l2(u, D @ g) < 1e-13
    # the amplitude is not trivial: it changes the result at O(1)
    assert O.rel_l2(O.direct_1d(O.PHASE_FIO1D, x, xi, g), D @ g) > 0.1


def test_unit_and_constant_amplitude_reduce_to_ibf():
    N, r = 256, 9
    x, xi, _, _, g = _setup_1d(O.PHASE_FIO1D, N, 1, 902)
    ibf = lambda G: O.ibf_apply_1d(O.PHASE_FIO1D, N, r, x, G)
    one = np.ones((N, 1))
    assert np.array_equal(A.apply(ibf, one, one, g), ibf(g))
    c = np.array([0.5 + 0.25j, -1.5, 2j])
    d = np.array([2.0, 1 - 1j, 0.5j])
    u = A.apply(ibf, np.tile(c, (N, 1)), np.tile(d, (N, 1)), g)
    assert O.rel_l2(u, (c @ d) * ibf(g)) < 1e-14


@pytest.mark.parametrize("phase", [O.PHASE_SEPARABLE, O.PHASE_NUFFT])
def test_ibf_route_against_dense(phase):
    """Separable phase: the IBF is exact, so the amplitude IBF equals the
    dense definition to rounding.  NUFFT phase at r = 9: within the IBF's own
    interpolation error (about 5e-7 at this r)."""
    N, r, q = 64 if phase == O.PHASE_SEPARABLE else 256, 9, 3
    x, xi, alpha, beta, g = _setup_1d(phase, N, q, 903)
    D = A.dense_1d(phase, x, xi, alpha, beta)
    u = A.apply(lambda G: O.ibf_apply_1d(phase, N, r, x, G), alpha, beta, g)
    err = O.rel_l2(u, D @ g)
    assert err < (1e-12 if phase == O.PHASE_SEPARABLE else 1e-5)


def test_fio_error_tracks_the_phase_only_ibf():
    N, r, q = 256, 9, 3
    x, xi, alpha, beta, g = _setup_1d(O.PHASE_FIO1D, N, q, 904)
    D = A.dense_1d(O.PHASE_FIO1D, x, xi, alpha, beta)
    u = A.apply(lambda G: O.ibf_apply_1d(O.PHASE_FIO1D, N, r, x, G), alpha, beta, g)
    e_amp = O.rel_l2(u, D @ g)
    e_one = O.rel_l2(O.ibf_apply_1d(O.PHASE_FIO1D, N, r, x, g), O.direct_1d(O.PHASE_FIO1D, x, xi, g))
    assert e_amp < 1e-4 and e_amp < 4 * e_one


def test_adjoint_identity_and_dense_transpose():
    N, r, q = 256, 9, 3
    x, xi, alpha, beta, g = _setup_1d(O.PHASE_FIO1D, N, q, 905, nrhs=2)
    y = W.complex_normal((N, 2), W.rng(906))
    fwd = lambda G: O.ibf_apply_1d(O.PHASE_FIO1D, N, r, x, G)
    adj = lambda Y: O.ibf_adjoint_1d(O.PHASE_FIO1D, N, r, x, Y)
    lhs = np.vdot(y, A.apply(fwd, alpha, beta, g))
    rhs = np.vdot(A.adjoint(adj, alpha, beta, y), g)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # exact case: separable phase, against the dense conjugate transpose
    N = 64
    x, xi, alpha, beta, _ = _setup_1d(O.PHASE_SEPARABLE, N, q, 907)
    y = W.complex_normal((N, 2), W.rng(908))
    D = A.dense_1d(O.PHASE_SEPARABLE, x, xi, alpha, beta)
    ga = A.adjoint(lambda Y: O.ibf_adjoint_1d(O.PHASE_SEPARABLE, N, 9, x, Y), alpha, beta, y)
    assert O.rel_l2(ga, D.conj().T @ y) < 1e-12


def test_2d_mibf_separable_exact():
    n, r, q = 32, 5, 3
    gen = W.rng(910)
    x, xi = W.grid_x_2d(n), W.omega_2d(n)
    alpha, beta = W.separated_amplitude(x, xi, q, gen)
    g = W.complex_normal((n * n, 2), gen)
    y = W.complex_normal((n * n, 2), gen)
    D = A.dense_2d(O.PHASE_SEPARABLE, x, xi, alpha, beta)
    u = A.apply(lambda G: O.mibf_apply_2d(O.PHASE_SEPARABLE, n, r, x, G), alpha, beta, g)
    assert O.rel_l2(u, D @ g) < 1e-12
    ga = A.adjoint(lambda Y: O.mibf_adjoint_2d(O.PHASE_SEPARABLE, n, r, x, Y), alpha, beta, y)
    assert O.rel_l2(ga, D.conj().T @ y) < 1e-12
