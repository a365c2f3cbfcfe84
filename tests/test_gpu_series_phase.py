"""The FIOs with series coefficients.  1D (IBF_PHASE_FIO1D_SERIES; the FIO
class of Sec. 1, Assumption 1.1, Phi = x xi + c(x)|xi| with a caller-given
smooth periodic c): GPU parity with the oracle's preliminary IBF (Algorithm
2.1 / Sec. 3) and its adjoint, FP64 explicit at the FIO phase's conditioning
floor and FP32 structured at 1e-5; and with Sec. 6.2's coefficient the plan
equals the IBF_PHASE_FIO1D plan.  2D (IBF_PHASE_FIO2D_SERIES, Sec. 6.3's
generalized-Radon form with caller-given c1, c2): parity of the multiscale
IBF (Sec. 5) and its adjoint with the oracle's, and with Sec. 6.3's
coefficients the plan equals the IBF_PHASE_FIO2D plan."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from test_oracle import SERIES2_SEC63, SERIES2_SMOOTH, SERIES_SMOOTH_A, SERIES_SMOOTH_B


def series_floor(N, a, b):
    """FP64 parity floor of the series phase: each term's cosine or sine may
    differ by 2 ulp between CUDA and libm, so c(x) by up to
    sum_m (|a_m| + |b_m|) 2^-51 and the phase by |xi| <= N/2 times that; a
    phase error d moves a unit-modulus factor by 2 pi d.  4x that bound, and
    never below 1e-12."""
    return max(1e-12, 4 * 2 * np.pi * (N / 2) * (np.sum(np.abs(a)) + np.sum(np.abs(b))) * 2.0 ** -51)

def series2_floor(n, rows):
    """The same bound in 2D: |xi| <= n / sqrt(2) on the grid of Sec. 5, each
    coefficient off by sum_t (|al| + |be|) 2^-51 at most."""
    rows = np.asarray(rows, dtype=np.float64)
    return max(1e-12, 4 * 2 * np.pi * (n / np.sqrt(2)) * np.abs(rows[:, 2:]).sum() * 2.0 ** -51)


pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ibf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_03616_gb300 as m
    return m


@pytest.mark.parametrize("N,r,nrhs,random_x", [(256, 9, 2, False), (4096, 9, 3, False), (2048, 7, 2, True)])
def test_series_phase_matches_oracle(ibf, N, r, nrhs, random_x):
    O.set_series(SERIES_SMOOTH_A, SERIES_SMOOTH_B)
    coef = (SERIES_SMOOTH_A, SERIES_SMOOTH_B)
    x = W.random_sorted_x(N, W.rng(51)) if random_x else W.uniform_x(N)
    g = W.complex_normal((N, nrhs), W.rng(52))
    y = W.complex_normal((N, nrhs), W.rng(53))
    ref = O.ibf_apply_1d(O.PHASE_FIO1D_SERIES, N, r, x, g)
    refa = O.ibf_adjoint_1d(O.PHASE_FIO1D_SERIES, N, r, x, y)
    xa = x if random_x else None
    for dt, cdt, tol in ((ibf.C128, np.complex128, series_floor(N, *coef)), (ibf.C64_FP32, np.complex64, 1e-5)):
        plan = ibf.Plan(ibf.PHASE_FIO1D_SERIES, N, r, dt, x=xa, coef=coef)
        u = plan.apply(torch.from_numpy(g.astype(cdt)).cuda()).cpu().numpy()
        ga = plan.adjoint(torch.from_numpy(y.astype(cdt)).cuda()).cpu().numpy()
        ef, ea = O.rel_l2(u, ref), O.rel_l2(ga, refa)
        print("\nseries phase N=%d r=%d dtype=%d: fwd %.3e adj %.3e (tol %.1e)" % (N, r, dt, ef, ea, tol))
        assert ef < tol and ea < tol
        plan.close()


def test_series_with_sec62_coefficient_equals_fio1d_plan(ibf):
    N, r = 1 << 12, 9
    g = torch.from_numpy(W.complex_normal((N, 2), W.rng(54))).cuda()
    a = ibf.Plan(ibf.PHASE_FIO1D_SERIES, N, r, ibf.C128, coef=([0.25, 0.0], [0.0, 0.125])).apply(g)
    b = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C128).apply(g)
    assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) < 1e-13


@pytest.mark.parametrize("n,r,nrhs", [(32, 7, 2), (64, 9, 1), (64, 5, 3)])
def test_series2_phase_matches_oracle(ibf, n, r, nrhs):
    O.set_series2(SERIES2_SMOOTH)
    x = W.grid_x_2d(n)
    g = W.complex_normal((n * n, nrhs), W.rng(55))
    y = W.complex_normal((n * n, nrhs), W.rng(56))
    ref = O.mibf_apply_2d(O.PHASE_FIO2D_SERIES, n, r, x, g)
    refa = O.mibf_adjoint_2d(O.PHASE_FIO2D_SERIES, n, r, x, y)
    for dt, cdt, tol in ((ibf.C128, np.complex128, series2_floor(n, SERIES2_SMOOTH)),
                         (ibf.C64_FP32, np.complex64, 1e-5)):
        plan = ibf.Plan(ibf.PHASE_FIO2D_SERIES, n * n, r, dt, d=2, coef=SERIES2_SMOOTH)
        u = plan.apply(torch.from_numpy(g.astype(cdt)).cuda()).cpu().numpy()
        ga = plan.adjoint(torch.from_numpy(y.astype(cdt)).cuda()).cpu().numpy()
        ef, ea = O.rel_l2(u, ref), O.rel_l2(ga, refa)
        print("\nseries2 phase n=%d r=%d dtype=%d: fwd %.3e adj %.3e (tol %.1e)" % (n, r, dt, ef, ea, tol))
        assert ef < tol and ea < tol
        plan.close()


def test_series2_with_sec63_coefficients_equals_fio2d_plan(ibf):
    n, r = 64, 7
    g = torch.from_numpy(W.complex_normal((n * n, 2), W.rng(57))).cuda()
    a = ibf.Plan(ibf.PHASE_FIO2D_SERIES, n * n, r, ibf.C128, d=2, coef=SERIES2_SEC63).apply(g)
    b = ibf.Plan(ibf.PHASE_FIO2D, n * n, r, ibf.C128, d=2).apply(g)
    assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) < 1e-13

