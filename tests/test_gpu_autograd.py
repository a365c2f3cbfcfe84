"""Differentiation through the IBF: torch.autograd.Function whose backward is
the hand-written adjoint, checked against finite differences, gradcheck and
the dense K^* (FP64, N = 256), and at the adjoint workload size (1D FIO,
N = 2^18, nrhs = 32, complex64) against the FP64 GPU form."""
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


@pytest.mark.parametrize("N,ncol", [(64, 2), (256, 1)])
def test_gradcheck_fp64(ibf, N, ncol):
    from paper_1605_03616_gb300.autograd import ibf_apply, ibf_adjoint
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C128)
    g = torch.from_numpy(W.complex_normal((N, ncol), W.rng(71))).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v: ibf_apply(plan, v), (g,), eps=1e-6, atol=1e-8, rtol=1e-6)
    y = torch.from_numpy(W.complex_normal((N, ncol), W.rng(72))).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v: ibf_adjoint(plan, v), (y,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_loss_gradient_fd_and_dense_adjoint(ibf):
    """loss = ||K g - y||^2: the autograd gradient equals 2 K^*(K g - y) with
    the dense conjugate transpose of the oracle's IBF, and central finite
    differences of the loss evaluated through the GPU forward apply (FP64)
    along random directions."""
    from paper_1605_03616_gb300.autograd import ibf_apply
    N, r = 256, 9
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C128)
    g_np = W.complex_normal(N, W.rng(81))
    y_np = W.complex_normal(N, W.rng(82))
    g = torch.from_numpy(g_np).cuda().requires_grad_(True)
    y = torch.from_numpy(y_np).cuda()
    loss = (ibf_apply(plan, g) - y).abs().pow(2).sum()
    loss.backward()
    grad = g.grad.cpu().numpy()
    # dense IBF matrix from the oracle (columns = IBF applied to unit vectors)
    x = W.uniform_x(N)
    Kibf = O.ibf_apply_1d(O.PHASE_FIO1D, N, r, x, np.eye(N))
    # PyTorch's gradient of a real loss w.r.t. complex g is dL/d(conj g) * 2 = 2 K^H (K g - y)
    ref = 2 * Kibf.conj().T @ (Kibf @ g_np - y_np)
    assert O.rel_l2(grad, ref) < 1e-12
    # central finite differences: d/dt L(g + t v) = Re<grad, v>
    rng = W.rng(83)
    for _ in range(3):
        v = W.complex_normal(N, rng)
        h = 1e-6
        def L(vec):
            with torch.no_grad():
                return float((plan.apply(torch.from_numpy(vec).cuda()) - y).abs().pow(2).sum())
        fd = (L(g_np + h * v) - L(g_np - h * v)) / (2 * h)
        an = float(np.real(np.vdot(grad, v)))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_adjoint_workload_fp32_vs_fp64(ibf):
    """N = 2^18, nrhs = 32: FP32 forward + backward against the FP64 explicit
    GPU form of the same IBF (relative L2 <= 1e-5), and the FP32 dot-product
    identity <K g, y> = <g, K^* y>."""
    from paper_1605_03616_gb300.autograd import ibf_apply
    N, r, nrhs = 1 << 18, 9, 32
    p32 = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C64_FP32, max_nrhs=nrhs)
    p64 = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C128, max_nrhs=8)
    g_np = W.complex_normal((N, nrhs), W.rng(91), dtype=np.complex64)
    y_np = W.complex_normal((N, nrhs), W.rng(92), dtype=np.complex64)
    g = torch.from_numpy(g_np).cuda().requires_grad_(True)
    y = torch.from_numpy(y_np).cuda()
    u = ibf_apply(p32, g)
    loss = (u - y).abs().pow(2).sum()
    loss.backward()
    g64 = torch.from_numpy(g_np.astype(np.complex128)).cuda()
    u64 = p64.apply(g64)
    r64 = u64 - torch.from_numpy(y_np.astype(np.complex128)).cuda()
    grad64 = 2 * p64.adjoint(r64.contiguous())
    eu = float(torch.linalg.vector_norm(u.detach().to(torch.complex128) - u64) / torch.linalg.vector_norm(u64))
    eg = float(torch.linalg.vector_norm(g.grad.to(torch.complex128) - grad64) / torch.linalg.vector_norm(grad64))
    print("\nadjoint workload N=2^18 nrhs=32: forward %.3e gradient %.3e" % (eu, eg))
    assert eu < 1e-5 and eg < 1e-5
    lhs = torch.vdot(y.reshape(-1).to(torch.complex128), u.detach().reshape(-1).to(torch.complex128))
    ky = p32.adjoint(y)
    rhs = torch.vdot(ky.reshape(-1).to(torch.complex128), g.detach().reshape(-1).to(torch.complex128))
    assert abs(complex(lhs - rhs)) < 1e-5 * abs(complex(lhs))


def test_2d_loss_gradient_matches_oracle_adjoint(ibf):
    """2D multiscale IBF (n = 32, FP64): the autograd gradient of
    ||K g - y||^2 is 2 K^*(K g - y) with the oracle's forward and adjoint,
    and matches central finite differences along a random direction."""
    from paper_1605_03616_gb300.autograd import ibf_apply
    n, r = 32, 7
    N = n * n
    x = W.grid_x_2d(n)
    plan = ibf.Plan(ibf.PHASE_FIO2D, N, r, ibf.C128, d=2)
    g_np = W.complex_normal(N, W.rng(90))
    y_np = W.complex_normal(N, W.rng(91))
    g = torch.from_numpy(g_np).cuda().requires_grad_(True)
    y = torch.from_numpy(y_np).cuda()
    loss = (ibf_apply(plan, g) - y).abs().pow(2).sum()
    loss.backward()
    grad = g.grad.cpu().numpy()
    ref = 2 * O.mibf_adjoint_2d(O.PHASE_FIO2D, n, r, x, O.mibf_apply_2d(O.PHASE_FIO2D, n, r, x, g_np) - y_np)
    assert O.rel_l2(grad, ref) < 1e-11
    v = W.complex_normal(N, W.rng(92))
    h = 1e-6

    def L(gg):
        with torch.no_grad():
            return float((ibf_apply(plan, torch.from_numpy(gg).cuda()) - y).abs().pow(2).sum())

    fd = (L(g_np + h * v) - L(g_np - h * v)) / (2 * h)
    assert abs(fd - np.real(np.vdot(grad, v))) < 1e-6 * abs(fd)
    plan.close()
