"""GPU parity of the 2D multiscale IBF (Sec. 5) with the oracle's MIBF on
the same corona decomposition, and at the full workload size (n = 512,
nrhs = 32, complex64) against the FP64 GPU form and sampled direct sums."""
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


def _run(ibf, phase, n, r, dtype, g):
    plan = ibf.Plan(phase, n * n, r, dtype, d=2)
    cdt = np.complex128 if dtype == ibf.C128 else np.complex64
    u = plan.apply(torch.from_numpy(g.astype(cdt)).cuda()).cpu().numpy()
    plan.close()
    return u


@pytest.mark.parametrize("phase,n,r,nrhs", [(O.PHASE_SEPARABLE, 32, 5, 2), (O.PHASE_FIO2D, 32, 7, 3),
                                            (O.PHASE_FIO2D, 64, 5, 1), (O.PHASE_NUFFT, 64, 7, 2),
                                            (O.PHASE_FIO2D, 64, 9, 2), (O.PHASE_FIO2D, 64, 7, 37),
                                            (O.PHASE_FIO2D, 128, 7, 1)])   # rings of side-32 boxes: odd depth
def test_2d_matches_oracle_mibf(ibf, phase, n, r, nrhs):
    x = W.grid_x_2d(n)
    g = W.complex_normal((n * n, nrhs), W.rng(601))
    ref = O.mibf_apply_2d(phase, n, r, x, g)
    u64 = _run(ibf, phase, n, r, ibf.C128, g)
    u32 = _run(ibf, phase, n, r, ibf.C64_FP32, g)
    e64, e32 = O.rel_l2(u64, ref), O.rel_l2(u32, ref)
    print("\nparity 2d phase=%d n=%d r=%d nrhs=%d fp64 %.3e fp32 %.3e" % (phase, n, r, nrhs, e64, e32))
    assert e64 < 1e-12
    assert e32 < 1e-5
    if phase == O.PHASE_SEPARABLE:
        ud = O.direct_2d(phase, x, W.omega_2d(n), g)
        assert O.rel_l2(u64, ud) < 1e-12


def test_2d_full_size_fp32_vs_fp64_and_sampled_direct(ibf):
    n, r, nrhs = 512, 7, 32
    N = n * n
    g = W.complex_normal((nrhs, N), W.rng(602), dtype=np.complex64)   # rows = columns of g
    p32 = ibf.Plan(ibf.PHASE_FIO2D, N, r, ibf.C64_FP32, d=2)
    p64 = ibf.Plan(ibf.PHASE_FIO2D, N, r, ibf.C128, d=2, max_nrhs=8)
    gd = torch.from_numpy(g).cuda()
    u32 = torch.empty_like(gd)
    p32.apply_raw(gd.data_ptr(), u32.data_ptr(), nrhs, torch.cuda.current_stream().cuda_stream)
    g64 = gd[:4].to(torch.complex128).contiguous()
    u64 = torch.empty_like(g64)
    p64.apply_raw(g64.data_ptr(), u64.data_ptr(), 4, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    e = float(torch.linalg.vector_norm(u32[:4].to(torch.complex128) - u64) / torch.linalg.vector_norm(u64))
    # sampled rows of the direct sum (Sec. 6, eq. relativeerr)
    rows = W.rng(603).choice(N, 64, replace=False)
    x = W.grid_x_2d(n)[rows]
    ud = O.direct_2d(O.PHASE_FIO2D, x, W.omega_2d(n), g[:2].T.astype(np.complex128))
    ei = O.rel_l2(u64[:2].cpu().numpy().T[rows], ud)
    print("\n2d n=512 r=7: fp32 vs fp64 %.3e, fp64 vs direct (64 rows) %.3e" % (e, ei))
    assert e < 1e-5
    assert ei < 5e-3
    # the adjoint at full size: FP32 against FP64, and <K g, y> = <g, K^* y> in FP64
    y64 = torch.from_numpy(W.complex_normal((4, N), W.rng(604))).cuda()
    ga64 = torch.empty_like(y64)
    p64.adjoint_raw(y64.data_ptr(), ga64.data_ptr(), 4, torch.cuda.current_stream().cuda_stream)
    y32 = y64.to(torch.complex64).contiguous()
    ga32 = torch.empty_like(y32)
    p32.adjoint_raw(y32.data_ptr(), ga32.data_ptr(), 4, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ea = float(torch.linalg.vector_norm(ga32.to(torch.complex128) - ga64) / torch.linalg.vector_norm(ga64))
    lhs = torch.vdot(y64.flatten(), u64.flatten()).item()
    rhs = torch.vdot(ga64.flatten(), g64.flatten()).item()
    print("2d n=512 adjoint: fp32 vs fp64 %.3e, dot-product identity %.1e" % (ea, abs(lhs - rhs) / abs(lhs)))
    assert ea < 1e-5
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


@pytest.mark.parametrize("phase,n,r,nrhs,max_nrhs", [(O.PHASE_FIO2D, 32, 7, 3, 32), (O.PHASE_SEPARABLE, 64, 5, 2, 32),
                                                     (O.PHASE_FIO2D, 64, 9, 6, 4)])   # slices of 4 and 2
def test_2d_adjoint_matches_oracle(ibf, phase, n, r, nrhs, max_nrhs):
    """g = K^* y of the 2D multiscale IBF against the oracle's adjoint, FP64
    and FP32, with the dot-product identity against the GPU forward apply."""
    x = W.grid_x_2d(n)
    y = W.complex_normal((n * n, nrhs), W.rng(980))
    ref = O.mibf_adjoint_2d(phase, n, r, x, y)
    out = {}
    for dt, cdt in ((ibf.C128, np.complex128), (ibf.C64_FP32, np.complex64)):
        plan = ibf.Plan(phase, n * n, r, dt, d=2, max_nrhs=max_nrhs)
        yd = torch.from_numpy(y.astype(cdt)).cuda()
        out[dt] = plan.adjoint(yd).cpu().numpy()
        if dt == ibf.C128:
            g = W.complex_normal((n * n, nrhs), W.rng(981))
            u = plan.apply(torch.from_numpy(g).cuda()).cpu().numpy()
            lhs, rhs = np.vdot(y, u), np.vdot(out[dt], g)
            assert abs(lhs - rhs) < 1e-11 * abs(lhs)
        plan.close()
    e64, e32 = O.rel_l2(out[ibf.C128], ref), O.rel_l2(out[ibf.C64_FP32], ref)
    print("\nadjoint 2d phase=%d n=%d r=%d nrhs=%d fp64 %.3e fp32 %.3e" % (phase, n, r, nrhs, e64, e32))
    assert e64 < 1e-12
    assert e32 < 1e-5
