"""Pins of the optimal-IBF oracle (sweep-out compression, Sec. 4.2) against
facts the compression must respect, independent of its own arithmetic:

* at full rank (r0 = r) every truncated SVD is exact, so the compressed
  product must equal the preliminary IBF it started from (structure,
  indexing and the V-side stacking are all exercised);
* a separable phase Phi = f(x) + h(xi) makes the kernel rank one on every
  domain pair (eq. RAB vanishes), so r0 = 1 must reproduce the direct sum;
* the error against the direct sum cannot grow with r0, and the adjoint
  must satisfy the dot-product identity."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.optimal import OptimalIBF, split_svd


def test_split_svd_is_the_truncated_svd():
    Z = W.complex_normal((9, 10), W.rng(950))
    for k in (1, 4, 9):
        A, B = split_svd(Z, k)
        s = np.linalg.svd(Z, compute_uv=False)
        # Eckart-Young: the spectral error of the best rank-k approximation is s[k]
        err = np.linalg.norm(Z - A @ B, 2)
        assert abs(err - (s[k] if k < s.size else 0.0)) < 1e-12 * s[0]
        # both factors carry the square roots of the singular values
        assert np.allclose(np.linalg.norm(A, axis=0), np.sqrt(s[:k]))
        assert np.allclose(np.linalg.norm(B, axis=1), np.sqrt(s[:k]))


@pytest.mark.parametrize("phase,N,r", [(O.PHASE_FIO1D, 256, 9), (O.PHASE_NUFFT, 256, 7), (O.PHASE_FIO1D, 128, 5)])
def test_full_rank_equals_preliminary(phase, N, r):
    x = W.random_sorted_x(N, W.rng(951)) if phase == O.PHASE_NUFFT else W.uniform_x(N)
    g = W.complex_normal((N, 2), W.rng(952))
    opt = OptimalIBF(phase, N, r, x, r0=r)
    ref = O.ExplicitIBF(phase, N, r, x).apply(g)
    assert O.rel_l2(opt.apply(g), ref) < 1e-12


def test_separable_phase_rank_one_is_exact():
    N, r = 512, 7
    x = W.uniform_x(N)
    g = W.complex_normal(N, W.rng(953))
    opt = OptimalIBF(O.PHASE_SEPARABLE, N, r, x, r0=1)
    ud = O.direct_1d(O.PHASE_SEPARABLE, x, W.omega_1d(N), g)
    assert O.rel_l2(opt.apply(g), ud) < 1e-12


def test_error_does_not_grow_with_rank_and_adjoint():
    N, r = 1024, 9
    x = W.uniform_x(N)
    g = W.complex_normal(N, W.rng(954))
    ud = O.direct_1d(O.PHASE_FIO1D, x, W.omega_1d(N), g)
    errs = []
    for r0 in (3, 5, 7, 9):
        errs.append(O.rel_l2(OptimalIBF(O.PHASE_FIO1D, N, r, x, r0=r0).apply(g), ud))
    print("\noptimal IBF FIO N=1024 r=9, r0 = 3,5,7,9: " + ", ".join("%.2e" % e for e in errs))
    assert all(b <= a * 1.05 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-4
    opt = OptimalIBF(O.PHASE_FIO1D, N, r, x, r0=6)
    y = W.complex_normal(N, W.rng(955))
    lhs = np.vdot(y, opt.apply(g))
    rhs = np.vdot(opt.adjoint(y), g)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
