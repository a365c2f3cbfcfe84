"""GPU parity of the CUDA IBF against the FP64 oracle (element by element).

Tolerances (relative L2 over all outputs):
* FP64 explicit form vs the oracle's IBF: 1e-12.
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
    assert O.rel_l2(u, ref) < 1e-12
    assert O.rel_l2(ga, refa) < 1e-12


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
    assert O.rel_l2(u, O.ibf_apply_1d(phase, N, r, x, g)) < 1e-11
    assert O.rel_l2(ga, O.ibf_adjoint_1d(phase, N, r, x, y)) < 1e-11


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
    assert O.rel_l2(u, O.ibf_apply_1d(phase, N, r, x, g)) < 1e-5
    assert O.rel_l2(ga, O.ibf_adjoint_1d(phase, N, r, x, y)) < 1e-5


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
