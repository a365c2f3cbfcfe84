"""GPU parity of the CUDA IBF against the FP64 oracle (element by element).

Tolerances (relative L2 over all outputs):
* FP64 explicit form vs the oracle's IBF: 1e-12, or for the 1D FIO phase
  the conditioning floor fp64_floor(N) if that is larger.  The FIO phase
  contains c(x)|xi| with c = (2 + sin 2 pi x)/8; the CUDA and libm sines may
  differ by up to 2 ulp, so c differs by up to 2^-52/8 and the phase by up
  to |xi| 2^-55 <= N 2^-56.  A phase error d moves a unit-modulus factor by
  2 pi d, so the relative result error is bounded by about 2 pi N 2^-56;
  we allow 4x that (N = 2^14: 5.6e-12; N <= 2^12 stays at 1e-12).
* FP64 structured form: 1e-11.  It uses the universal transfer matrices
  T_c (exact child offsets) where the paper's formula evaluates the Lagrange
  weight at the rounded grid point c_C + w_C z_s; for Omega boxes far from
  0 that rounding is ~N eps relative to the box width, so the two FP64
  results may differ at the 1e-12 level.
* FP32 structured form: 1e-5 (the single-precision bar).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

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


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()


def fp64_floor(phase, N):
    if phase != O.PHASE_FIO1D:
        return 1e-12
    return max(1e-12, 4 * 2 * np.pi * N * 2.0 ** -56)


def _x(phase, N, seed):
    return W.random_sorted_x(N, W.rng(seed)) if phase == O.PHASE_NUFFT else W.uniform_x(N)


CASES_64 = [
    # phase, N, r, nrhs
    (O.PHASE_FIO1D, 4, 3, 1),
    (O.PHASE_FIO1D, 256, 9, 1),
    (O.PHASE_FIO1D, 4096, 9, 3),
    (O.PHASE_NUFFT, 1024, 9, 1),      # random sorted x: empty and multi-point leaves
    (O.PHASE_SEPARABLE, 512, 7, 2),
    (O.PHASE_FIO1D, 2048, 5, 2),      # odd L
    (O.PHASE_FIO1D, 1 << 14, 9, 1),
]


@pytest.mark.parametrize("phase,N,r,nrhs", CASES_64)
def test_fp64_explicit_matches_oracle(ibf, phase, N, r, nrhs):
    x = _x(phase, N, 5)
    g = W.complex_normal((N, nrhs), W.rng(6))
    y = W.complex_normal((N, nrhs), W.rng(7))
    plan = ibf.Plan(phase, N, r, ibf.C128, x=None if phase != O.PHASE_NUFFT else x)
    u = plan.apply(_dev(g, np.complex128)).cpu().numpy()
    ga = plan.adjoint(_dev(y, np.complex128)).cpu().numpy()
    ref = O.ibf_apply_1d(phase, N, r, x, g)
    refa = O.ibf_adjoint_1d(phase, N, r, x, y)
    tol = fp64_floor(phase, N)
    print("\nparity fp64-explicit phase=%d N=%d r=%d nrhs=%d fwd %.3e adj %.3e tol %.1e" % (
        phase, N, r, nrhs, O.rel_l2(u, ref), O.rel_l2(ga, refa), tol))
    assert O.rel_l2(u, ref) < tol
    assert O.rel_l2(ga, refa) < tol


@pytest.mark.parametrize("phase,N,r,nrhs", CASES_64)
def test_fp64_structured_matches_oracle(ibf, phase, N, r, nrhs):
    if r not in (5, 7, 9, 11):
        pytest.skip("structured form supports r in {5,7,9,11}")
    x = _x(phase, N, 5)
    g = W.complex_normal((N, nrhs), W.rng(6))
    y = W.complex_normal((N, nrhs), W.rng(7))
    plan = ibf.Plan(phase, N, r, ibf.C128, x=None if phase != O.PHASE_NUFFT else x, form=ibf.FORM_STRUCTURED)
    u = plan.apply(_dev(g, np.complex128)).cpu().numpy()
    ga = plan.adjoint(_dev(y, np.complex128)).cpu().numpy()
    tol = max(1e-11, fp64_floor(phase, N))
    ef, ea = O.rel_l2(u, O.ibf_apply_1d(phase, N, r, x, g)), O.rel_l2(ga, O.ibf_adjoint_1d(phase, N, r, x, y))
    print("\nparity fp64-structured phase=%d N=%d r=%d nrhs=%d fwd %.3e adj %.3e tol %.1e" % (
        phase, N, r, nrhs, ef, ea, tol))
    assert ef < tol
    assert ea < tol


@pytest.mark.parametrize("phase,N,r,nrhs,kw", [
    (O.PHASE_FIO1D, 4096, 9, 1, {}),
    (O.PHASE_FIO1D, 4096, 9, 37, {}),                              # ragged rhs tile
    (O.PHASE_FIO1D, 1 << 13, 7, 16, dict(levels_per_launch=3)),    # several launches per half
    (O.PHASE_FIO1D, 2048, 9, 70, dict(max_nrhs=32)),               # nrhs sliced
    (O.PHASE_NUFFT, 1024, 9, 5, {}),
    (O.PHASE_SEPARABLE, 256, 5, 3, dict(rhs_tile=2, levels_per_launch=1)),
    (O.PHASE_FIO1D, 8, 5, 2, {}),
])
def test_fp32_structured_matches_oracle(ibf, phase, N, r, nrhs, kw):
    x = _x(phase, N, 8)
    g = W.complex_normal((N, nrhs), W.rng(9))
    y = W.complex_normal((N, nrhs), W.rng(10))
    plan = ibf.Plan(phase, N, r, ibf.C64_FP32, x=None if phase != O.PHASE_NUFFT else x, **kw)
    u = plan.apply(_dev(g, np.complex64)).cpu().numpy()
    ga = plan.adjoint(_dev(y, np.complex64)).cpu().numpy()
    ef, ea = O.rel_l2(u, O.ibf_apply_1d(phase, N, r, x, g)), O.rel_l2(ga, O.ibf_adjoint_1d(phase, N, r, x, y))
    print("\nparity fp32-structured phase=%d N=%d r=%d nrhs=%d %s fwd %.3e adj %.3e" % (
        phase, N, r, nrhs, kw, ef, ea))
    assert ef < 1e-5
    assert ea < 1e-5


def test_unsorted_points_follow_caller_order(ibf):
    N, r = 1024, 9
    x = W.random_unsorted_x(N, W.rng(12))
    g = W.complex_normal(N, W.rng(13))
    ref = O.ibf_apply_1d(O.PHASE_NUFFT, N, r, x, g)
    for dt, cdt, tol in ((ibf.C128, np.complex128, 1e-12), (ibf.C64_FP32, np.complex64, 1e-5)):
        plan = ibf.Plan(ibf.PHASE_NUFFT, N, r, dt, x=x)
        u = plan.apply(_dev(g, cdt)).cpu().numpy()
        assert O.rel_l2(u, ref) < tol


def test_bad_arguments_return_errors(ibf):
    plan = ibf.Plan(ibf.PHASE_FIO1D, 256, 9, ibf.C64_FP32)
    g = torch.zeros(256, dtype=torch.complex64, device="cuda")
    lib = ibf.load_library()
    import ctypes
    # misaligned pointer
    rc = lib.ibf_apply(plan._p, ctypes.c_void_p(g.data_ptr() + 4), ctypes.c_void_p(g.data_ptr() + 4096), 1, None)
    assert rc == 1
    # overlapping input and output
    rc = lib.ibf_apply(plan._p, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(g.data_ptr()), 1, None)
    assert rc == 1
    assert lib.ibf_apply(plan._p, ctypes.c_void_p(g.data_ptr()), None, 1, None) == 1
    assert lib.ibf_apply(plan._p, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(g.data_ptr()), 0, None) == 1
    with pytest.raises(ibf.IBFError):
        ibf.Plan(ibf.PHASE_FIO1D, 256, 9, ibf.C64_FP32, x=np.full(256, 1.5))
    with pytest.raises(ibf.IBFError):
        ibf.Plan(ibf.PHASE_FIO1D, 256, 9, ibf.C64_FP32, h=8)


def test_plan_queries(ibf):
    plan = ibf.Plan(ibf.PHASE_FIO1D, 1 << 12, 9, ibf.C128)
    assert plan.query(ibf.Q_L) == 12 and plan.query(ibf.Q_H) == 6
    assert plan.query(ibf.Q_NNZ) == 9 * 4096 + 12 * 4096 * 162 + 4096 * 81 + 9 * 4096
    assert plan.query(ibf.Q_FACTOR_BYTES) == 16 * plan.query(ibf.Q_NNZ)
    p32 = ibf.Plan(ibf.PHASE_FIO1D, 1 << 12, 9, ibf.C64_FP32)
    assert p32.query(ibf.Q_LAUNCHES) >= 2
