"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself through a retyped formula:
* the direct sum against numpy's inverse FFT on the uniform grid, and Parseval;
* the Chebyshev grid and Lagrange basis against numpy's Chebyshev points and
  polynomial fitting (partition of unity, cardinality, exact reproduction);
* the IBF with a separable phase, where the remainder R^{AB} of eq. RAB
  vanishes and the factorization is exact (Sec. 2.1);
* the explicit factors multiplied as dense matrices in the paper's own vector
  orderings (Sec. 3: j-major in the first half, i-major after the switch);
* convergence in r, N-independence, and the error levels printed in Tables 1
  and 3 (tests/golden);
* the adjoint by the dot-product identity and against the dense K^*.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import read_golden


def _x_for(phase, N, seed=2):
    return W.random_sorted_x(N, W.rng(seed)) if phase == O.PHASE_NUFFT else W.uniform_x(N)


# ---------------------------------------------------------------- direct sum
@pytest.mark.parametrize("N", [16, 256, 1024])
def test_direct_equals_dft_closed_form(N):
    """Phi = x.xi on x_j = j/N, xi_k = k - N/2: u_j = (-1)^j N ifft(g)_j."""
    g = W.complex_normal((N, 2), W.rng(3))
    u = O.direct_1d(O.PHASE_NUFFT, W.uniform_x(N), W.omega_1d(N), g)
    ref = ((-1.0) ** np.arange(N))[:, None] * N * np.fft.ifft(g, axis=0)
    assert O.rel_l2(u, ref) < 1e-13
    # Parseval: ||u||^2 = N ||g||^2 column by column
    np.testing.assert_allclose(np.sum(np.abs(u) ** 2, 0), N * np.sum(np.abs(g) ** 2, 0), rtol=1e-12)


def test_direct_2d_equals_dft_closed_form():
    n = 16
    x = W.grid_x_2d(n)
    xi = W.omega_2d(n)
    g = W.complex_normal(n * n, W.rng(4))
    u = O.direct_2d(O.PHASE_NUFFT, x, xi, g).reshape(n, n)
    sgn = ((-1.0) ** np.arange(n))
    ref = np.outer(sgn, sgn) * n * n * np.fft.ifft2(g.reshape(n, n))
    assert O.rel_l2(u, ref) < 1e-13


# ------------------------------------------------------------- phase shapes
# the series of tests/golden/phase_values.txt, kind 4
SERIES_GOLDEN_A, SERIES_GOLDEN_B = [0.25, 0.0, 0.125], [0.0, 0.125, 0.0]
# the 2D series of tests/golden/phase_values.txt, kind 5: rows (p, q, al1, be1, al2, be2)
SERIES2_GOLDEN = [[0, 0, 0.25, 0, 0.125, 0], [1, 0, 0, 0.125, 0, 0], [1, 1, 0.0625, 0, 0, 0],
                  [0, 1, 0, 0, 0.0625, 0], [1, -1, 0, 0, 0, 0.03125]]
# Sec. 6.3's coefficients (constants /16) as a series: sin a sin b = (cos(a-b) - cos(a+b))/2
SERIES2_SEC63 = [[0, 0, 0.125, 0, 0.125, 0], [1, -1, 1 / 32, 0, 1 / 32, 0], [1, 1, -1 / 32, 0, 1 / 32, 0]]
# smooth positive coefficients with six terms (c1 >= 0.136, c2 >= 0.072)
SERIES2_SMOOTH = [[0, 0, 0.2, 0, 0.12, 0], [1, 0, 0.02, 0.015, 0, 0.01], [0, 1, -0.01, 0, 0.015, -0.005],
                  [1, 1, 0, 0.01, 0.005, 0], [1, -1, 0.005, 0, 0, 0.008], [2, 1, 0, -0.004, 0.003, 0.002]]
# a smooth positive coefficient with five terms (|c - 1/4| <= 0.11)
SERIES_SMOOTH_A = [0.25, 0.04, -0.02, 0.01, 0.005]
SERIES_SMOOTH_B = [0.0, 0.03, 0.015, -0.01, 0.004]


def test_phase_values_match_hand_computed():
    """The phases of Sec. 6 at points where they are exact rationals
    (tests/golden/phase_values.txt, each value worked out by hand): c(x) of
    the 1D FIO and c1, c2 of the 2D FIO at quarter and twelfth points, where
    sin and cos take the values 0, +-1/2, +-1.  A phase-shifted coefficient
    (cos for sin) or c1 and c2 exchanged moves several rows by >= 1."""
    kinds = {0: O.PHASE_NUFFT, 1: O.PHASE_FIO1D, 2: O.PHASE_FIO2D, 3: O.PHASE_FIO2D_32, 4: O.PHASE_FIO1D_SERIES,
             5: O.PHASE_FIO2D_SERIES}
    O.set_series(SERIES_GOLDEN_A, SERIES_GOLDEN_B)
    O.set_series2(SERIES2_GOLDEN)
    rows = read_golden("phase_values.txt")
    assert len(rows) >= 37
    for kind, x1, x2, k1, k2, want in rows:
        ph = kinds[int(kind)]
        got = O.phi_1d(ph, x1, k1) if int(kind) in (0, 1, 4) else O.phi_2d(ph, x1, x2, k1, k2)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (kind, x1, x2, k1, k2, got, want)


# ------------------------------------------------------- grids and Lagrange
@pytest.mark.parametrize("r", [3, 5, 7, 9, 12])
def test_chebyshev_grid_matches_numpy(r):
    z = O.cheb_grid(r)
    ref = 0.5 * np.polynomial.chebyshev.chebpts2(r)[::-1]
    np.testing.assert_allclose(z, ref, atol=1e-15)


@pytest.mark.parametrize("r", [3, 6, 9, 11])
def test_lagrange_identities(r):
    z = O.cheb_grid(r)
    # cardinality M_t(z_s) = delta_ts
    for t in range(r):
        for s in range(r):
            assert abs(O.lagrange(r, t, z[s]) - (1.0 if s == t else 0.0)) < 1e-13
    # partition of unity and exact reproduction of degree r-1 polynomials
    u = np.linspace(-0.75, 0.75, 17)  # includes the child-grid range used by the butterfly
    coef = W.rng(7).standard_normal(r)
    for uu in u:
        Mt = np.array([O.lagrange(r, t, uu) for t in range(r)])
        assert abs(Mt.sum() - 1.0) < 1e-12
        assert abs(Mt @ np.polyval(coef, z) - np.polyval(coef, uu)) < 1e-10


# ------------------------------------------------- IBF structural exactness
@pytest.mark.parametrize("N,r,h", [(16, 3, 2), (64, 5, 3), (256, 9, 4), (256, 4, 0), (512, 7, 5), (1024, 9, 5)])
def test_separable_phase_is_exact(N, r, h):
    """Phi = f(x) + h(xi) makes R^{AB} = 0 (eq. RAB), so every interpolation
    is exact and the IBF must reproduce the direct sum to rounding."""
    x = W.random_unsorted_x(N, W.rng(11))
    g = W.complex_normal(N, W.rng(12))
    ud = O.direct_1d(O.PHASE_SEPARABLE, x, W.omega_1d(N), g)
    ui = O.ibf_apply_1d(O.PHASE_SEPARABLE, N, r, x, g, h=h)
    assert O.rel_l2(ui, ud) < 1e-12


def _dense_ibf(E: O.ExplicitIBF, xleaf):
    """Assemble U G^{L-1}..G^h M^h (H^h)^*..(H^1)^* (V^0)^* as dense matrices
    in the orderings of Sec. 3: Lambda^l = [Lambda^l_j]_j with
    Lambda^l_j = [Lambda^l_{i,j}]_i up to the switch, i-major after it."""
    N, r, L, h = E.N, E.r, E.L, E.h
    nx = E.x.size

    def pH(l, i, j):  # position of pair (i,j) at level l, first half
        return j * (1 << l) + i

    def pG(l, i, j):  # second half
        return i * (1 << (L - l)) + j

    V = E.V()
    Vs = np.zeros((r * N, N), complex)
    for k in range(N):
        for t in range(r):
            Vs[pH(0, 0, k) * r + t, k] = V[k, t]
    mats = [Vs]
    for l in range(1, L + 1):
        B = E.blocks(l)
        D = np.zeros((r * N, r * N), complex)
        first = l <= h
        for i in range(1 << l):
            for j in range(1 << (L - l)):
                p = i * (1 << (L - l)) + j
                for c in range(2):
                    if first:
                        row, col = pH(l, i, j), pH(l - 1, i // 2, 2 * j + c)
                    else:
                        row, col = pG(l, i, j), pG(l - 1, i // 2, 2 * j + c)
                    D[row * r:(row + 1) * r, col * r:(col + 1) * r] = B[p, c]
        mats.append(D)
        if l == h:
            Mb = E.M()
            Ms = np.zeros((r * N, r * N), complex)
            for i in range(1 << h):
                for j in range(1 << (L - h)):
                    p = i * (1 << (L - h)) + j
                    row, col = pG(h, i, j), pH(h, i, j)
                    Ms[row * r:(row + 1) * r, col * r:(col + 1) * r] = Mb[p]
            mats.append(Ms)
    U = E.U()
    Us = np.zeros((nx, r * N), complex)
    for n in range(nx):
        i = xleaf[n]
        Us[n, pG(L, i, 0) * r:(pG(L, i, 0) + 1) * r] = U[n]
    mats.append(Us)
    K = mats[0]
    for m in mats[1:]:
        K = m @ K
    return K


@pytest.mark.parametrize("N,r,phase", [(4, 3, O.PHASE_FIO1D), (16, 5, O.PHASE_FIO1D), (64, 6, O.PHASE_NUFFT),
                                       (16, 4, O.PHASE_NUFFT), (64, 7, O.PHASE_FIO1D)])
def test_dense_factor_product_matches_apply(N, r, phase):
    """Tiny N brute force: the product of the dense factors equals the
    factor-by-factor apply, the matrix-free butterfly, and approximates K."""
    x = _x_for(phase, N)
    E = O.ExplicitIBF(phase, N, r, x)
    xleaf = np.minimum(np.floor(x * N).astype(int), N - 1)
    K = _dense_ibf(E, xleaf)
    G = W.complex_normal((N, 3), W.rng(5))
    ue = E.apply(G)
    um = O.ibf_apply_1d(phase, N, r, x, G)
    assert O.rel_l2(ue, K @ G) < 1e-13
    assert O.rel_l2(um, K @ G) < 1e-13
    Kd = O.direct_1d(phase, x, W.omega_1d(N), np.eye(N))
    assert O.rel_l2(K, Kd) < 0.05  # interpolation error only (r small)


@pytest.mark.parametrize("phase", [O.PHASE_FIO1D, O.PHASE_NUFFT])
def test_unit_vector_gives_column(phase):
    N, r = 256, 9
    x = _x_for(phase, N)
    for k in (0, 77, N // 2, N - 1):
        e = np.zeros(N, complex)
        e[k] = 1
        col = O.direct_1d(phase, x, W.omega_1d(N), e)
        ui = O.ibf_apply_1d(phase, N, r, x, e)
        assert O.rel_l2(ui, col) < 1e-3


# ---------------------------------------------------------- approximation
@pytest.mark.parametrize("phase", [O.PHASE_FIO1D, O.PHASE_NUFFT])
def test_error_falls_with_r_and_is_flat_in_N(phase):
    errs = {}
    for N in (256, 1024):
        x = _x_for(phase, N)
        g = W.complex_normal(N, W.rng(1))
        ud = O.direct_1d(phase, x, W.omega_1d(N), g)
        errs[N] = [O.rel_l2(O.ibf_apply_1d(phase, N, r, x, g), ud) for r in range(4, 13)]
        assert all(a > 2 * b for a, b in zip(errs[N], errs[N][1:])), errs[N]
        assert errs[N][-1] < 1e-6
    ratio = np.array(errs[1024]) / np.array(errs[256])
    assert np.all((ratio > 1 / 3) & (ratio < 3)), ratio


def test_nufft_error_matches_table1():
    """Table 1 is the type-I transform sum_j e^{-2 pi i x_j xi} u(x_j), i.e.
    the adjoint of K = e(+x xi): the oracle's adjoint error against the dense
    K^* must sit at the printed level (within a factor 3)."""
    for N, r, eps in read_golden("table1_nufft_1d.txt"):
        N, r = int(N), int(r)
        if N > 1024:
            continue
        x = W.random_sorted_x(N, W.rng(21))
        y = W.complex_normal(N, W.rng(22))
        ga = O.ibf_adjoint_1d(O.PHASE_NUFFT, N, r, x, y)
        # K^* y = conj(K conj(y)) row by row: K^*_{k n} = conj(e(x_n xi_k))
        ref = O.direct_1d(O.PHASE_NUFFT, W.omega_1d(N), x, np.conj(y)).conj()
        err = O.rel_l2(ga, ref)
        assert eps / 3 < err < eps * 3, (N, r, err, eps)


def test_fio_error_below_table3():
    """Table 3's optimal-IBF errors bound the preliminary IBF's from above;
    the preliminary error is the same order for r = 7 and r = 10."""
    for N, r, eps in read_golden("table3_fio_1d.txt"):
        N, r = int(N), int(r)
        if N > 1024:
            continue
        x = W.uniform_x(N)
        g = W.complex_normal(N, W.rng(23))
        ud = O.direct_1d(O.PHASE_FIO1D, x, W.omega_1d(N), g)
        err = O.rel_l2(O.ibf_apply_1d(O.PHASE_FIO1D, N, r, x, g), ud)
        assert eps / 30 < err < eps, (N, r, err, eps)


@pytest.mark.parametrize("N", [128, 2048])
def test_odd_depth_both_switch_levels(N):
    L = N.bit_length() - 1
    x = W.uniform_x(N)
    g = W.complex_normal(N, W.rng(31))
    ud = O.direct_1d(O.PHASE_FIO1D, x, W.omega_1d(N), g)
    for h in (L // 2, L // 2 + 1):
        err = O.rel_l2(O.ibf_apply_1d(O.PHASE_FIO1D, N, 9, x, g, h=h), ud)
        assert err < 1e-4, (h, err)


def test_point_order_is_irrelevant():
    N = 512
    x = W.random_sorted_x(N, W.rng(41))
    perm = W.rng(42).permutation(N)
    g = W.complex_normal(N, W.rng(43))
    u = O.ibf_apply_1d(O.PHASE_NUFFT, N, 7, x, g)
    up = O.ibf_apply_1d(O.PHASE_NUFFT, N, 7, x[perm], g)
    np.testing.assert_allclose(up, u[perm], rtol=0, atol=1e-13 * np.abs(u).max())


# --------------------------------------------------------------- adjoint
@pytest.mark.parametrize("phase,N", [(O.PHASE_FIO1D, 256), (O.PHASE_NUFFT, 512), (O.PHASE_FIO1D, 128)])
def test_adjoint_dot_product_identity(phase, N):
    x = _x_for(phase, N)
    g = W.complex_normal((N, 2), W.rng(51))
    y = W.complex_normal((N, 2), W.rng(52))
    Kg = O.ibf_apply_1d(phase, N, 9, x, g)
    Ksy = O.ibf_adjoint_1d(phase, N, 9, x, y)
    lhs = np.vdot(y, Kg)
    rhs = np.vdot(Ksy, g)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs) * 10
    E = O.ExplicitIBF(phase, N, 9, x)
    np.testing.assert_allclose(E.adjoint(y), Ksy, rtol=0, atol=1e-12 * np.abs(Ksy).max())


def test_adjoint_matches_dense_conjugate_transpose():
    N, r = 256, 9
    x = W.uniform_x(N)
    Kd = O.direct_1d(O.PHASE_FIO1D, x, W.omega_1d(N), np.eye(N))
    y = W.complex_normal(N, W.rng(61))
    ga = O.ibf_adjoint_1d(O.PHASE_FIO1D, N, r, x, y)
    assert O.rel_l2(ga, Kd.conj().T @ y) < 1e-4
    # and the separable phase makes it exact
    Ks = O.direct_1d(O.PHASE_SEPARABLE, x, W.omega_1d(N), np.eye(N))
    gs = O.ibf_adjoint_1d(O.PHASE_SEPARABLE, N, r, x, y)
    assert O.rel_l2(gs, Ks.conj().T @ y) < 1e-12


# ------------------------------------------------- the series-coefficient FIO
def test_series_phase_reduces_to_sec62_fio():
    """With c(x) = 1/4 + sin(2 pi x)/8 the series phase is Sec. 6.2's: the
    direct sums and the IBFs agree to rounding."""
    O.set_series([0.25, 0.0], [0.0, 0.125])
    N, r = 256, 9
    x = W.uniform_x(N)
    g = W.complex_normal((N, 2), W.rng(40))
    a = O.ibf_apply_1d(O.PHASE_FIO1D_SERIES, N, r, x, g)
    b = O.ibf_apply_1d(O.PHASE_FIO1D, N, r, x, g)
    assert O.rel_l2(a, b) < 1e-13
    xi = W.omega_1d(N)
    assert O.rel_l2(O.direct_1d(O.PHASE_FIO1D_SERIES, x, xi, g), O.direct_1d(O.PHASE_FIO1D, x, xi, g)) < 1e-13


def test_series_phase_ibf_converges_in_r():
    """A five-term smooth coefficient: the IBF error against the direct sum
    falls monotonically in r, to the FIO's level at r = 9, and stays flat in N."""
    O.set_series(SERIES_SMOOTH_A, SERIES_SMOOTH_B)
    errs = {}
    for N in (256, 1024):
        x = W.uniform_x(N)
        g = W.complex_normal(N, W.rng(41))
        ref = O.direct_1d(O.PHASE_FIO1D_SERIES, x, W.omega_1d(N), g)
        errs[N] = [O.rel_l2(O.ibf_apply_1d(O.PHASE_FIO1D_SERIES, N, r, x, g), ref) for r in (5, 7, 9, 11)]
    for N, e in errs.items():
        assert all(e[i + 1] < e[i] for i in range(len(e) - 1)), (N, e)
        assert e[2] < 1e-4, (N, e)
    assert max(errs[1024][2], errs[256][2]) < 5 * min(errs[1024][2], errs[256][2])
