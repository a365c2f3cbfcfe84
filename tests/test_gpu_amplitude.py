"""GPU parity of ibf_apply_amplitude, the non-unit amplitude
a(x, xi) = sum_t alpha_t(x) beta_t(xi) (Sec. 1, eq. FIO), with the oracle's
amplitude operator sum_t diag(alpha_t) K diag(beta_t) on the oracle's IBF or
MIBF: FP32 structured and FP64 explicit 1D plans, a 2D plan, forward and
adjoint, ragged column counts, several passes through a small work buffer,
the unit amplitude, argument errors, and the full 1D size (N = 2^20) on
sampled rows of the defining sum."""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import amplitude as A

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


def _cuda(a, cdt):
    return torch.from_numpy(np.ascontiguousarray(a.astype(cdt))).cuda()


def _gpu(plan, cdt, alpha, beta, v, adjoint=False, work=None):
    out = plan.apply_amplitude(_cuda(v, cdt), _cuda(alpha, cdt), _cuda(beta, cdt), adjoint=adjoint, work=work)
    return out.cpu().numpy()


@pytest.mark.parametrize("phase,N,r,dtype,nrhs,q", [
    (O.PHASE_FIO1D, 1 << 12, 9, "fp32", 5, 3),
    (O.PHASE_NUFFT, 1 << 12, 9, "fp32", 1, 4),
    (O.PHASE_NUFFT, 1 << 10, 9, "fp64", 3, 3),
])
def test_1d_matches_oracle(ibf, phase, N, r, dtype, nrhs, q):
    gen = W.rng(1201)
    x = W.random_sorted_x(N, gen) if phase == O.PHASE_NUFFT else W.uniform_x(N)
    xi = W.omega_1d(N)
    alpha, beta = W.separated_amplitude(x, xi, q, gen)
    g = W.complex_normal((N, nrhs), gen)
    y = W.complex_normal((N, nrhs), gen)
    fp64 = dtype == "fp64"
    cdt = np.complex128 if fp64 else np.complex64
    plan = ibf.Plan(phase, N, r, ibf.C128 if fp64 else ibf.C64_FP32, x=None if phase != O.PHASE_NUFFT else x,
                    form=ibf.FORM_EXPLICIT if fp64 else ibf.FORM_AUTO)
    ref = A.apply(lambda G: O.ibf_apply_1d(phase, N, r, x, G), alpha, beta, g)
    refa = A.adjoint(lambda Y: O.ibf_adjoint_1d(phase, N, r, x, Y), alpha, beta, y)
    u = _gpu(plan, cdt, alpha, beta, g)
    ga = _gpu(plan, cdt, alpha, beta, y, adjoint=True)
    tol = 1e-11 if fp64 else 1e-5
    ef, ea = O.rel_l2(u, ref), O.rel_l2(ga, refa)
    print("\nparity amplitude phase=%d N=%d %s nrhs=%d q=%d fwd %.3e adj %.3e" % (phase, N, dtype, nrhs, q, ef, ea))
    assert ef < tol and ea < tol
    plan.close()


def test_2d_matches_oracle(ibf):
    n, r, q, nrhs = 32, 7, 3, 2
    gen = W.rng(1202)
    x, xi = W.grid_x_2d(n), W.omega_2d(n)
    alpha, beta = W.separated_amplitude(x, xi, q, gen)
    g = W.complex_normal((n * n, nrhs), gen)
    plan = ibf.Plan(ibf.PHASE_FIO2D, n * n, r, ibf.C64_FP32, d=2)
    ref = A.apply(lambda G: O.mibf_apply_2d(O.PHASE_FIO2D, n, r, x, G), alpha, beta, g)
    refa = A.adjoint(lambda Y: O.mibf_adjoint_2d(O.PHASE_FIO2D, n, r, x, Y), alpha, beta, g)
    ef = O.rel_l2(_gpu(plan, np.complex64, alpha, beta, g), ref)
    ea = O.rel_l2(_gpu(plan, np.complex64, alpha, beta, g, adjoint=True), refa)
    print("\nparity amplitude 2d n=%d fwd %.3e adj %.3e" % (n, ef, ea))
    assert ef < 1e-5 and ea < 1e-5
    plan.close()


def test_passes_unit_amplitude_and_errors(ibf):
    N, q, nrhs = 1 << 11, 3, 7
    gen = W.rng(1203)
    x, xi = W.uniform_x(N), W.omega_1d(N)
    alpha, beta = W.separated_amplitude(x, xi, q, gen)
    g = W.complex_normal((N, nrhs), gen)
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=16)
    one_pass = _gpu(plan, np.complex64, alpha, beta, g)
    for m in (1, 2):                      # three and two passes (accumulating gather)
        work = torch.empty(2 * N * nrhs * m + 3, dtype=torch.complex64, device="cuda")
        assert np.abs(_gpu(plan, np.complex64, alpha, beta, g, work=work) - one_pass).max() \
            < 1e-6 * np.abs(one_pass).max()
    # a = 1: the scaling and accumulation are exact, so the result is the plain apply's
    one = np.ones((N, 1))
    gd = _cuda(g, np.complex64)
    assert torch.equal(plan.apply_amplitude(gd, _cuda(one, np.complex64), _cuda(one, np.complex64)),
                       plan.apply(gd))
    # work below 2 N nrhs elements is rejected before any launch
    small = torch.empty(2 * N * nrhs - 1, dtype=torch.complex64, device="cuda")
    with pytest.raises(ibf.IBFError) as ei:
        plan.apply_amplitude(gd, _cuda(alpha, np.complex64), _cuda(beta, np.complex64), work=small)
    assert ei.value.code == 1
    # q = 0 and an output aliasing alpha are rejected
    lib = ibf.load_library()
    a = _cuda(alpha, np.complex64).t().contiguous()
    b = _cuda(beta, np.complex64).t().contiguous()
    src = gd.t().contiguous()
    dst = torch.empty_like(src)
    wk = torch.empty(2 * N * nrhs * q, dtype=torch.complex64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = ctypes.c_void_p
    assert lib.ibf_apply_amplitude(plan._p, P(a.data_ptr()), P(b.data_ptr()), 0, P(src.data_ptr()),
                                   P(dst.data_ptr()), nrhs, 0, P(wk.data_ptr()), wk.numel(), s) == 1
    assert lib.ibf_apply_amplitude(plan._p, P(a.data_ptr()), P(b.data_ptr()), q, P(src.data_ptr()),
                                   P(a.data_ptr()), nrhs, 0, P(wk.data_ptr()), wk.numel(), s) == 1
    assert lib.ibf_apply_amplitude(plan._p, P(a.data_ptr()), P(b.data_ptr()), q, P(src.data_ptr()),
                                   P(dst.data_ptr()), nrhs, 0, P(src.data_ptr()), wk.numel(), s) == 1
    plan.close()


def test_full_size_sampled_rows_of_the_definition(ibf):
    """N = 2^20, FP32 structured plan, q = 3, 2 columns: 64 sampled rows of u
    against the defining sum with the amplitude (the oracle's direct sum on
    those rows), within the IBF's own interpolation error at r = 9."""
    N, r, q, nrhs = 1 << 20, 9, 3, 2
    gen = W.rng(1204)
    x, xi = W.uniform_x(N), W.omega_1d(N)
    alpha, beta = W.separated_amplitude(x, xi, q, gen)
    g = W.complex_normal((N, nrhs), gen)
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C64_FP32, max_nrhs=nrhs * q)
    u = _gpu(plan, np.complex64, alpha, beta, g)
    rows = np.sort(W.rng(1205).choice(N, 64, replace=False))
    ref = A.apply(lambda G: O.direct_1d(O.PHASE_FIO1D, x[rows], xi, G), alpha[rows], beta, g)
    err = O.rel_l2(u[rows], ref)
    print("\namplitude full size N=2^20 sampled rows rel err %.3e" % err)
    assert err < 1e-4
    plan.close()
