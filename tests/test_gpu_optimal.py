"""GPU optimal IBF (sweep-out stage of Sec. 4.2, FP64): the compression on
the GPU (one-sided Jacobi SVDs) against the oracle's compression (LAPACK
SVDs) on the same preliminary factors.  A rank-r0 truncation is unique when
the r0-th and (r0+1)-th singular values differ, so both must give the same
operator to rounding; at full rank both equal the preliminary IBF, and for a
separable phase rank one is exact.

Tolerance: 1e-10, or 1e-3 of the compression's own effect (optimal vs
preliminary) when that is larger.  All cuts here have a gap of at least 2
between the r0-th and (r0+1)-th singular values, but at r = 12 the cut lies
near rounding level (sigma_{r0+1} / sigma_1 ~ 1e-13), where any normwise
stable SVD fixes the smallest kept directions only to about
eps sigma_1 / sigma_r0: two LAPACK drivers then differ by 3e-11 and the
Jacobi SVD by 3e-9, against a compression effect of 1.7e-5."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.optimal import OptimalIBF

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex128)).cuda()


@pytest.mark.parametrize("phase,N,r,r0,nrhs", [
    (O.PHASE_FIO1D, 256, 9, 9, 2),        # full rank: the preliminary IBF itself
    (O.PHASE_FIO1D, 1024, 9, 6, 2),
    (O.PHASE_NUFFT, 1024, 9, 5, 3),       # random points: leaves with 0, 1, several points
    (O.PHASE_FIO1D, 2048, 12, 9, 1),      # odd L
    (O.PHASE_SEPARABLE, 512, 7, 1, 2),    # rank one is exact
])
def test_optimal_matches_oracle(ibf, phase, N, r, r0, nrhs):
    x = W.random_sorted_x(N, W.rng(960)) if phase == O.PHASE_NUFFT else W.uniform_x(N)
    g = W.complex_normal((N, nrhs), W.rng(961))
    y = W.complex_normal((N, nrhs), W.rng(962))
    plan = ibf.Plan(phase, N, r, ibf.C128, x=x if phase == O.PHASE_NUFFT else None, form=ibf.FORM_OPTIMAL, rank=r0)
    assert plan.query(ibf.Q_RANK) == r0 and plan.query(ibf.Q_FORM) == ibf.FORM_OPTIMAL
    u = plan.apply(_dev(g)).cpu().numpy()
    ga = plan.adjoint(_dev(y)).cpu().numpy()
    ref = OptimalIBF(phase, N, r, x, r0)
    uo, go = ref.apply(g), ref.adjoint(y)
    ef, ea = O.rel_l2(u, uo), O.rel_l2(ga, go)
    ud = O.direct_1d(phase, x, W.omega_1d(N), g)
    trunc = O.rel_l2(uo, O.ExplicitIBF(phase, N, r, x).apply(g))
    tol = max(1e-10, 1e-3 * trunc)
    print("\noptimal phase=%d N=%d r=%d r0=%d: gpu vs oracle fwd %.2e adj %.2e (tol %.1e); oracle vs direct %.2e"
          % (phase, N, r, r0, ef, ea, tol, O.rel_l2(uo, ud)))
    assert ef < tol
    assert ea < tol
    if phase == O.PHASE_SEPARABLE:
        assert O.rel_l2(u, ud) < 1e-12
    plan.close()


def test_optimal_rejects_bad_options(ibf):
    for kw, code in [(dict(dtype=ibf.C128, rank=0), 1), (dict(dtype=ibf.C128, rank=10), 1),
                     (dict(dtype=ibf.C64_BF16X3, rank=4), 4)]:
        with pytest.raises(ibf.IBFError) as e:
            ibf.Plan(ibf.PHASE_FIO1D, 256, 9, form=ibf.FORM_OPTIMAL, **kw)
        assert e.value.code == code
    with pytest.raises(ibf.IBFError) as e:
        ibf.Plan(ibf.PHASE_FIO1D, 256, 13, ibf.C128, form=ibf.FORM_OPTIMAL, rank=6)
    assert e.value.code == 4
    for kw, code in [(dict(dtype=ibf.C64_BF16X3, rank=4), 4), (dict(dtype=ibf.C128, rank=0), 1)]:
        with pytest.raises(ibf.IBFError) as e:
            ibf.Plan(ibf.PHASE_FIO1D, 256, 9, form=ibf.FORM_OPTIMAL_IN, **kw)
        assert e.value.code == code
    with pytest.raises(ibf.IBFError) as e:
        ibf.Plan(ibf.PHASE_FIO2D, 32 * 32, 7, ibf.C128, d=2, form=ibf.FORM_OPTIMAL_IN, rank=4)
    assert e.value.code == 4


@pytest.mark.parametrize("phase,N,r,r0,nrhs", [
    (O.PHASE_FIO1D, 1024, 9, 6, 2),
    (O.PHASE_NUFFT, 1024, 9, 5, 3),       # random points: the leaf ranks follow the fullest leaf
    (O.PHASE_FIO1D, 2048, 12, 9, 1),
    (O.PHASE_FIO1D, 64, 9, 9, 2),         # both sides of the sweep-in reach the middle factor
])
def test_sweep_in_matches_oracle_and_keeps_the_operator(ibf, phase, N, r, r0, nrhs):
    """Sweep-in (Sec. 4.3) on the GPU: its splits are exact, so the plan must
    give the sweep-out plan's results to rounding with fewer stored entries,
    exactly as many as the oracle's sweep-in, and match the oracle's optimal
    IBF like the sweep-out form does."""
    x = W.random_sorted_x(N, W.rng(963)) if phase == O.PHASE_NUFFT else W.uniform_x(N)
    g = W.complex_normal((N, nrhs), W.rng(964))
    y = W.complex_normal((N, nrhs), W.rng(965))
    kw = dict(x=x if phase == O.PHASE_NUFFT else None, rank=r0)
    pin = ibf.Plan(phase, N, r, ibf.C128, form=ibf.FORM_OPTIMAL_IN, **kw)
    pout = ibf.Plan(phase, N, r, ibf.C128, form=ibf.FORM_OPTIMAL, **kw)
    assert pin.query(ibf.Q_FORM) == ibf.FORM_OPTIMAL_IN and pin.query(ibf.Q_RANK) == r0
    ui, uo = pin.apply(_dev(g)).cpu().numpy(), pout.apply(_dev(g)).cpu().numpy()
    gi, go = pin.adjoint(_dev(y)).cpu().numpy(), pout.adjoint(_dev(y)).cpu().numpy()
    ref = OptimalIBF(phase, N, r, x, r0, sweep_in=True)
    e_io, e_ioa = O.rel_l2(ui, uo), O.rel_l2(gi, go)
    ef, ea = O.rel_l2(ui, ref.apply(g)), O.rel_l2(gi, ref.adjoint(y))
    trunc = O.rel_l2(ref.apply(g), O.ExplicitIBF(phase, N, r, x).apply(g))
    tol = max(1e-10, 1e-3 * trunc)
    print("\nsweep-in phase=%d N=%d r=%d r0=%d: vs sweep-out fwd %.2e adj %.2e; vs oracle fwd %.2e adj %.2e "
          "(tol %.1e); nnz %d -> %d" % (phase, N, r, r0, e_io, e_ioa, ef, ea, tol, pout.query(ibf.Q_NNZ),
                                         pin.query(ibf.Q_NNZ)))
    assert pin.query(ibf.Q_NNZ) == ref.nnz() < pout.query(ibf.Q_NNZ)
    assert e_io < 1e-11 and e_ioa < 1e-11
    assert ef < tol and ea < tol
    pin.close()
    pout.close()


@pytest.mark.parametrize("form,phase,N,r,r0,nrhs", [
    ("optimal_in", O.PHASE_FIO1D, 1024, 9, 6, 3),
    ("optimal_in", O.PHASE_NUFFT, 1024, 9, 5, 2),
    ("optimal", O.PHASE_FIO1D, 2048, 12, 9, 2),
    ("explicit", O.PHASE_FIO1D, 1024, 9, 0, 5),
    ("explicit", O.PHASE_NUFFT, 512, 7, 0, 1),
    # the bulk-copy level kernel (4..32 columns): partial chunks at N = 16,
    # 8 / 12 / 16 / 24 columns, sweep-in ranks 1..9, and 40 columns (the
    # warp-per-pair kernel)
    ("explicit", O.PHASE_FIO1D, 16, 5, 0, 4),
    ("optimal_in", O.PHASE_FIO1D, 2048, 12, 9, 8),
    ("optimal", O.PHASE_FIO1D, 1024, 9, 6, 12),
    ("explicit", O.PHASE_NUFFT, 1024, 9, 0, 16),
    ("explicit", O.PHASE_FIO1D, 512, 7, 0, 24),
    ("explicit", O.PHASE_FIO1D, 256, 7, 0, 40),
])
def test_fp32_explicit_and_optimal_forms(ibf, form, phase, N, r, r0, nrhs):
    """FP32 plans of the explicit and optimal forms: factors built (and
    compressed) in FP64, stored and applied in FP32.  Against the oracle's
    IBF of the same form: the FP32 bar 1e-5 (plus the compression's
    tolerance); against the FP64 plan of the same form: 1e-5."""
    x = W.random_sorted_x(N, W.rng(966)) if phase == O.PHASE_NUFFT else W.uniform_x(N)
    g = W.complex_normal((N, nrhs), W.rng(967))
    y = W.complex_normal((N, nrhs), W.rng(968))
    fm = {"optimal_in": ibf.FORM_OPTIMAL_IN, "optimal": ibf.FORM_OPTIMAL, "explicit": ibf.FORM_EXPLICIT}[form]
    kw = dict(x=x if phase == O.PHASE_NUFFT else None, form=fm, rank=r0)
    p32 = ibf.Plan(phase, N, r, ibf.C64_FP32, **kw)
    p64 = ibf.Plan(phase, N, r, ibf.C128, **kw)
    assert p32.query(ibf.Q_FACTOR_BYTES) == 8 * p32.query(ibf.Q_NNZ) and p32.query(ibf.Q_NNZ) == p64.query(ibf.Q_NNZ)
    d32 = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).cuda()
    u32 = p32.apply(d32(g)).cpu().numpy()
    g32 = p32.adjoint(d32(y)).cpu().numpy()
    u64 = p64.apply(_dev(g)).cpu().numpy()
    g64 = p64.adjoint(_dev(y)).cpu().numpy()
    if form == "explicit":
        ref = O.ExplicitIBF(phase, N, r, x)
        tol = 1e-5
    else:
        ref = OptimalIBF(phase, N, r, x, r0, sweep_in=form == "optimal_in")
        tol = 1e-5 + 1e-3 * O.rel_l2(ref.apply(g), O.ExplicitIBF(phase, N, r, x).apply(g))
    ef, ea = O.rel_l2(u32, ref.apply(g)), O.rel_l2(g32, ref.adjoint(y))
    print("\nfp32 %s phase=%d N=%d r=%d r0=%d: vs oracle fwd %.2e adj %.2e (tol %.1e); vs fp64 plan %.2e %.2e"
          % (form, phase, N, r, r0, ef, ea, tol, O.rel_l2(u32, u64), O.rel_l2(g32, g64)))
    assert ef < tol and ea < tol
    assert O.rel_l2(u32, u64) < 1e-5 and O.rel_l2(g32, g64) < 1e-5
    assert p32.status() == 0          # no bounded device-side wait expired
    p32.close()
    p64.close()


def test_fp32_optimal_full_size_matches_fp64(ibf):
    """The configuration the benchmark times: optimal IBF with sweep-in,
    N = 2^16, r = 12 -> r0 = 9, 8 columns, complex64 through the bulk-copy
    level kernel (chunks of 8 output pairs, 5 consumer groups).  Its FP64
    plan holds the same compressed factors, so the two differ by FP32
    rounding only: relative L2 <= 1e-5 on every column, every element within
    1e-4 of the FP64 result's RMS; forward and adjoint; and no bounded wait
    expired."""
    N, r, r0, nrhs = 1 << 16, 12, 9, 8
    kw = dict(form=ibf.FORM_OPTIMAL_IN, rank=r0)
    p32 = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C64_FP32, **kw)
    p64 = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C128, **kw)
    g = W.complex_normal((N, nrhs), W.rng(980))
    y = W.complex_normal((N, nrhs), W.rng(981))
    for fwd in (True, False):
        src = g if fwd else y
        run32 = p32.apply if fwd else p32.adjoint
        run64 = p64.apply if fwd else p64.adjoint
        a = run32(torch.from_numpy(src.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
        b = run64(_dev(src)).cpu().numpy()
        for c in range(nrhs):
            assert O.rel_l2(a[:, c], b[:, c]) < 1e-5, (fwd, c)
        rms = np.sqrt(np.mean(np.abs(b) ** 2))
        assert np.max(np.abs(a - b)) / rms < 1e-4, fwd
    assert p32.status() == 0
    p32.close()
    p64.close()
