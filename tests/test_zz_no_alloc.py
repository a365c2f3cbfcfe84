"""ibf_apply_static_scratch: the apply for callers that may not allocate
device memory once their plans exist (a plug-in whose host application owns
the device heap, a server with a memory budget fixed at plan time).  It keeps
its scratch in a static device array instead of the plan's workspace; its
results must match ibf_apply's within the FP32 tolerance of the other tests,
on two calls in a row (the array keeps the previous call's contents).  A case
with more columns than one half of the array holds runs the column-chunk
loop; a warmed-up call must leave the device's free memory unchanged; a 2D
plan is refused before any CUDA work."""
import ctypes

import numpy as np
import pytest

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


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _static_apply(ibf, plan, g, u):
    s = torch.cuda.current_stream().cuda_stream
    rc = ibf.load_library().ibf_apply_static_scratch(plan._p, ctypes.c_void_p(g.data_ptr()),
                                                     ctypes.c_void_p(u.data_ptr()), g.shape[0], ctypes.c_void_p(s))
    assert rc == 0, ibf.last_error()


@pytest.mark.parametrize("N,r,nrhs,dtype", [(1 << 12, 9, 5, "f32"), (1 << 11, 7, 40, "f32"), (1 << 10, 9, 3, "f64")])
def test_static_scratch_matches_apply_twice(ibf, N, r, nrhs, dtype):
    cdt = torch.complex64 if dtype == "f32" else torch.complex128
    kind = ibf.C64_FP32 if dtype == "f32" else ibf.C128
    # a plan with the smallest workspace it can own
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, r, kind, form=ibf.FORM_STRUCTURED, max_nrhs=1)
    outs = []
    for call in range(2):
        g_np = W.complex_normal((nrhs, N), W.rng(100 + call))  # rows are the columns of g
        g = torch.from_numpy(g_np).to(cdt).cuda()
        ref = torch.empty_like(g)
        plan.apply_raw(g.data_ptr(), ref.data_ptr(), nrhs, torch.cuda.current_stream().cuda_stream)
        u = torch.full_like(g, float("nan"))
        _static_apply(ibf, plan, g, u)
        torch.cuda.synchronize()
        outs.append((u, ref))
    for u, ref in outs:
        assert torch.isfinite(torch.view_as_real(u)).all()
        assert _rel(u, ref) < 1e-5


def test_static_scratch_rejects_oversize_and_explicit(ibf):
    lib = ibf.load_library()
    big = ibf.Plan(ibf.PHASE_FIO1D, 1 << 20, 9, ibf.C128, form=ibf.FORM_STRUCTURED, max_nrhs=1)
    g = torch.zeros((1, 1 << 20), dtype=torch.complex128, device="cuda")
    u = torch.zeros_like(g)
    rc = lib.ibf_apply_static_scratch(big._p, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1, None)
    assert rc == 1 and "static scratch limit" in ibf.last_error()
    big.close()
    ex = ibf.Plan(ibf.PHASE_FIO1D, 256, 9, ibf.C128)
    g = torch.zeros((1, 256), dtype=torch.complex128, device="cuda")
    u = torch.zeros_like(g)
    rc = lib.ibf_apply_static_scratch(ex._p, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1, None)
    assert rc == 4


def test_static_scratch_column_chunks_and_no_allocation(ibf):
    # complex128, r = 9, N = 2^19: one Lambda column is 72 MiB, so each half of
    # the 256 MiB array holds one column and three columns take three chunks
    N, r, nrhs = 1 << 19, 9, 3
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C128, form=ibf.FORM_STRUCTURED, max_nrhs=1)
    g = torch.from_numpy(W.complex_normal((nrhs, N), W.rng(110))).cuda()
    ref = torch.empty_like(g)
    plan.apply_raw(g.data_ptr(), ref.data_ptr(), nrhs, torch.cuda.current_stream().cuda_stream)
    u = torch.full_like(g, float("nan"))
    _static_apply(ibf, plan, g, u)          # warm-up: every kernel of the schedule loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    u.fill_(float("nan"))
    torch.cuda.synchronize()
    _static_apply(ibf, plan, g, u)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for c in range(nrhs):
        assert _rel(u[c], ref[c]) < 1e-12, c
    plan.close()


def test_static_scratch_refuses_2d_plan(ibf):
    lib = ibf.load_library()
    n = 64
    p2 = ibf.Plan(ibf.PHASE_FIO2D, n * n, 7, ibf.C64_FP32, d=2)
    g = torch.zeros((1, n * n), dtype=torch.complex64, device="cuda")
    u = torch.zeros_like(g)
    rc = lib.ibf_apply_static_scratch(p2._p, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1, None)
    assert rc == 4 and "1D" in ibf.last_error()
    p2.close()
