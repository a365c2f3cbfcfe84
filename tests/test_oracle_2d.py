"""Pins of the oracle's 2D butterfly (Sec. 5.1) and multiscale IBF (Sec. 5.2).

* separable phase => R^{AB} = 0 => the 2D butterfly on one box and the whole
  MIBF (every corona box plus the direct centre) reproduce the direct sum to
  rounding: this also proves the corona boxes and the centre cover Omega
  exactly once;
* the 2D NUFFT (Phi = x.xi, smooth everywhere) on the whole grid as one box
  converges in r;
* the FIO of Sec. 6.3 with the paper's constants (/32) reproduces the errors
  printed in Table 4 (tests/golden/table4_fio_2d.txt) within 3x;
* the workload's FIO (constants /16) converges in r.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import read_golden


@pytest.mark.parametrize("n,r", [(16, 5), (32, 7)])
def test_separable_2d_box_and_mibf_exact(n, r):
    x = W.grid_x_2d(n)
    xi = W.omega_2d(n)
    g = W.complex_normal((n * n, 2), W.rng(501))
    ud = O.direct_2d(O.PHASE_SEPARABLE, x, xi, g)
    ub = O.ibf_apply_2d_box(O.PHASE_SEPARABLE, n, r, x, -n / 2, -n / 2, g)
    assert O.rel_l2(ub, ud) < 1e-12
    center = 8 if n == 16 else 16
    um = O.mibf_apply_2d(O.PHASE_SEPARABLE, n, r, x, g, center_side=center // 2 if n == 16 else center)
    assert O.rel_l2(um, ud) < 1e-12


def test_nufft_2d_single_box_converges():
    n = 32
    x = W.grid_x_2d(n)
    g = W.complex_normal(n * n, W.rng(502))
    ud = O.direct_2d(O.PHASE_NUFFT, x, W.omega_2d(n), g)
    errs = [O.rel_l2(O.ibf_apply_2d_box(O.PHASE_NUFFT, n, r, x, -n / 2, -n / 2, g), ud) for r in (4, 5, 6, 7)]
    assert all(a > 2 * b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-3


def test_mibf_matches_table4():
    for n, r, eps in read_golden("table4_fio_2d.txt"):
        n, r = int(n), int(r)
        if n > 32:
            continue
        x = W.grid_x_2d(n)
        g = W.complex_normal(n * n, W.rng(503))
        ud = O.direct_2d(O.PHASE_FIO2D_32, x, W.omega_2d(n), g)
        err = O.rel_l2(O.mibf_apply_2d(O.PHASE_FIO2D_32, n, r, x, g), ud)
        assert eps / 3 < err < eps * 3, (n, r, err, eps)


def test_mibf_workload_phase_converges():
    n = 32
    x = W.grid_x_2d(n)
    g = W.complex_normal(n * n, W.rng(504))
    ud = O.direct_2d(O.PHASE_FIO2D, x, W.omega_2d(n), g)
    errs = [O.rel_l2(O.mibf_apply_2d(O.PHASE_FIO2D, n, r, x, g), ud) for r in (5, 7, 9)]
    assert errs[0] > 5 * errs[1] > 25 * errs[2], errs
    assert errs[1] < 1e-3


def test_2d_adjoint_dot_product_identity_and_separable_exactness():
    """The 2D adjoints are the conjugate transposes of the forward maps: the
    dot-product identity holds to rounding for one box and for the
    multiscale sum, and for a separable phase the MIBF adjoint equals the
    conjugate-transposed direct sum."""
    n, r = 32, 7
    x = W.grid_x_2d(n)
    g = W.complex_normal(n * n, W.rng(970))
    y = W.complex_normal(n * n, W.rng(971))
    m, q1, q2 = 8, -16.0, 8.0
    gq = W.complex_normal(m * m, W.rng(972))
    lhs = np.vdot(y, O.ibf_apply_2d_box(O.PHASE_FIO2D, m, r, x, q1, q2, gq))
    rhs = np.vdot(O.ibf_adjoint_2d_box(O.PHASE_FIO2D, m, r, x, q1, q2, y), gq)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    lhs = np.vdot(y, O.mibf_apply_2d(O.PHASE_FIO2D, n, r, x, g))
    rhs = np.vdot(O.mibf_adjoint_2d(O.PHASE_FIO2D, n, r, x, y), g)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # separable phase: e(Phi(x_p, xi_k)) = e(Phi(x_p, xi_0)) e(Phi(x_0, xi_k)) e(-Phi(x_0, xi_0)),
    # so K^* y is rank one: conj(e(Phi(x_0, xi_k))) e(Phi(x_0, xi_0)) sum_p conj(e(Phi(x_p, xi_0))) y_p
    ga = O.mibf_adjoint_2d(O.PHASE_SEPARABLE, n, 5, x, y)
    xi = W.omega_2d(n)
    ph = lambda a, b: O.phi_2d(O.PHASE_SEPARABLE, a[0], a[1], b[0], b[1])
    col0 = np.exp(2j * np.pi * np.array([ph(a, xi[0]) for a in x]))
    row0 = np.exp(2j * np.pi * np.array([ph(x[0], b) for b in xi]))
    exact = np.conj(row0) * np.exp(2j * np.pi * ph(x[0], xi[0])) * np.vdot(col0, y)
    assert O.rel_l2(ga, exact) < 1e-12


def test_series2_phase_reduces_to_sec63_fio():
    """With c1 = 1/8 + (cos 2 pi (x1 - x2) - cos 2 pi (x1 + x2))/32 and
    c2 = 1/8 + (cos 2 pi (x1 - x2) + cos 2 pi (x1 + x2))/32 the series phase is
    Sec. 6.3's (constants /16): phases, direct sums and MIBFs agree to
    rounding."""
    from test_oracle import SERIES2_SEC63

    O.set_series2(SERIES2_SEC63)
    gen = W.rng(510)
    for _ in range(50):
        x1, x2 = gen.random(2)
        k1, k2 = gen.uniform(-64, 64, 2)
        a = O.phi_2d(O.PHASE_FIO2D_SERIES, x1, x2, k1, k2)
        b = O.phi_2d(O.PHASE_FIO2D, x1, x2, k1, k2)
        assert abs(a - b) < 1e-13 * max(1.0, abs(b))
    n, r = 32, 7
    x = W.grid_x_2d(n)
    g = W.complex_normal((n * n, 2), W.rng(511))
    ua = O.mibf_apply_2d(O.PHASE_FIO2D_SERIES, n, r, x, g)
    ub = O.mibf_apply_2d(O.PHASE_FIO2D, n, r, x, g)
    assert O.rel_l2(ua, ub) < 1e-12


def test_series2_phase_mibf_converges_in_r():
    """Six-term smooth coefficients: the MIBF error against the direct sum
    falls by a factor > 3 per step of r and reaches the workload FIO's level."""
    from test_oracle import SERIES2_SMOOTH

    O.set_series2(SERIES2_SMOOTH)
    n = 32
    x = W.grid_x_2d(n)
    g = W.complex_normal(n * n, W.rng(512))
    ud = O.direct_2d(O.PHASE_FIO2D_SERIES, x, W.omega_2d(n), g)
    errs = [O.rel_l2(O.mibf_apply_2d(O.PHASE_FIO2D_SERIES, n, r, x, g), ud) for r in (5, 7, 9)]
    assert errs[0] > 3 * errs[1] > 9 * errs[2], errs
    assert errs[1] < 1e-3, errs
