"""The tensor-core form IBF_C64_TF32X3: the transfer products of the G-form
levels (forward G levels, adjoint H levels) on the tcgen05 tensor cores in
TF32 with both operands split in two terms (Sec. 2.1's Lagrange transfer
inside eq. PIBF3's butterfly level), everything else as the FP32 form.
Element-by-element parity with the FP64 oracle's preliminary IBF (Algorithm
2.1 / Sec. 3) and its adjoint at the FP32 bar of 1e-5 relative L2; at the
bench shape (N = 2^20, 64 columns) four sampled columns against the oracle;
and the device status word of the bounded waits stays clear."""
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


def _x(phase, N, seed):
    return W.random_sorted_x(N, W.rng(seed)) if phase == O.PHASE_NUFFT else W.uniform_x(N)


@pytest.mark.parametrize("phase,N,r,nrhs", [
    (O.PHASE_FIO1D, 256, 9, 32),
    (O.PHASE_FIO1D, 4096, 9, 40),        # a full and a ragged 32-column tile
    (O.PHASE_NUFFT, 2048, 9, 33),        # random points, odd L, one column in the last tile
    (O.PHASE_SEPARABLE, 1024, 7, 32),
    (O.PHASE_FIO1D, 1 << 13, 5, 32),
    (O.PHASE_FIO1D, 1 << 12, 11, 32),
])
def test_tf32x3_matches_oracle(ibf, phase, N, r, nrhs):
    x = _x(phase, N, 5)
    g = W.complex_normal((N, nrhs), W.rng(16))
    y = W.complex_normal((N, nrhs), W.rng(17))
    plan = ibf.Plan(phase, N, r, ibf.C64_TF32X3, x=None if phase != O.PHASE_NUFFT else x, max_nrhs=nrhs)
    assert plan.query(ibf.Q_RHS_TILE) == 32
    u = plan.apply(torch.from_numpy(g.astype(np.complex64)).cuda()).cpu().numpy()
    ga = plan.adjoint(torch.from_numpy(y.astype(np.complex64)).cuda()).cpu().numpy()
    torch.cuda.synchronize()
    assert plan.status() == 0
    ref = O.ibf_apply_1d(phase, N, r, x, g)
    refa = O.ibf_adjoint_1d(phase, N, r, x, y)
    ef, ea = O.rel_l2(u, ref), O.rel_l2(ga, refa)
    print("\ntf32x3 phase=%d N=%d r=%d nrhs=%d: fwd %.3e adj %.3e" % (phase, N, r, nrhs, ef, ea))
    assert ef < 1e-5 and ea < 1e-5
    plan.close()


def test_tf32x3_full_size_sampled_columns(ibf):
    N, r, nrhs = 1 << 20, 9, 64
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C64_TF32X3, max_nrhs=nrhs)
    g = W.complex_normal((nrhs, N), W.rng(workload=2), dtype=np.complex64)   # rows = columns of g
    gd = torch.from_numpy(g).cuda()
    u = torch.empty_like(gd)
    plan.apply_raw(gd.data_ptr(), u.data_ptr(), nrhs, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert plan.status() == 0
    u = u.cpu().numpy()
    cols = [0, 31, 32, nrhs - 1]
    ref = O.ibf_apply_1d(O.PHASE_FIO1D, N, r, W.uniform_x(N), g[cols].T.astype(np.complex128))
    err = O.rel_l2(u[cols].T, ref)
    emax = float(np.max(np.abs(u[cols].T - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)))
    print("\ntf32x3 full size N=2^20 nrhs=64: %.3e vs oracle (max element %.3e of rms)" % (err, emax))
    assert err < 1e-5 and emax < 1e-4
    plan.close()
