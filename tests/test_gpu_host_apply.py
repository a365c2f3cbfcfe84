"""ibf_apply_host: the apply with host-resident vectors, the columns split into
chunks whose copies overlap the apply.  Its outputs must equal the device
apply's bit for bit (the same kernels run on the same columns), for ragged
column counts, the adjoint, pageable memory, 2D and explicit plans, and back
to back calls that reuse the staging slots."""
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


def _device(plan, g, adjoint=False):
    """The device apply of the (nrhs, N) array g, as an (nrhs, N) CPU tensor."""
    gd = torch.from_numpy(g).cuda().t()          # (N, nrhs), the binding's layout
    res = plan.adjoint(gd) if adjoint else plan.apply(gd)
    return res.t().contiguous().cpu()


@pytest.mark.parametrize("adjoint", [False, True])
def test_host_apply_equals_device_apply_fp32(ibf, adjoint):
    N, nrhs = 1 << 12, 37                      # chunks of 32 and 5 columns
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=64)
    g = W.complex_normal((nrhs, N), W.rng(801 + adjoint), dtype=np.complex64)
    src = torch.from_numpy(g).pin_memory()
    dst = torch.full_like(src, float("nan")).pin_memory()
    plan.apply_host(src, dst, adjoint=adjoint)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(dst, _device(plan, g, adjoint))
    plan.close()


def test_host_apply_back_to_back_and_pageable(ibf):
    N = 1 << 11
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=8)   # chunks of 8 columns
    gs = [W.complex_normal((29, N), W.rng(810 + i), dtype=np.complex64) for i in range(3)]
    outs = [np.full_like(g, np.nan) for g in gs]                          # pageable numpy arrays
    for g, o in zip(gs, outs):
        plan.apply_host(g, o)
    torch.cuda.current_stream().synchronize()
    for g, o in zip(gs, outs):
        assert np.array_equal(o, _device(plan, g).numpy())
    plan.close()


def test_host_apply_2d_and_explicit(ibf):
    n = 32
    p2 = ibf.Plan(ibf.PHASE_FIO2D, n * n, 7, ibf.C64_FP32, d=2, max_nrhs=32)
    g2 = W.complex_normal((20, n * n), W.rng(820), dtype=np.complex64)    # chunks of 16 and 4
    o2 = torch.empty_like(torch.from_numpy(g2)).pin_memory()
    p2.apply_host(torch.from_numpy(g2).pin_memory(), o2)
    a2 = torch.empty_like(torch.from_numpy(g2)).pin_memory()
    p2.apply_host(torch.from_numpy(g2).pin_memory(), a2, adjoint=True)
    pe = ibf.Plan(ibf.PHASE_FIO1D, 256, 9, ibf.C128, form=ibf.FORM_EXPLICIT, max_nrhs=4)
    ge = W.complex_normal((3, 256), W.rng(821))
    oe = torch.empty_like(torch.from_numpy(ge)).pin_memory()
    pe.apply_host(torch.from_numpy(ge).pin_memory(), oe)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(o2, _device(p2, g2))
    assert torch.equal(a2, _device(p2, g2, adjoint=True))
    assert torch.equal(oe, _device(pe, ge))
    p2.close()
    pe.close()


def test_host_apply_pipelined_calls(ibf):
    """IBF_HOST_PIPELINE: back-to-back calls whose copy-in may overlap the
    previous call's last apply give the device apply's results bit for bit,
    also when one call's output is the next call's input (then the copy-in
    waits for the previous copy-outs) and with an unflagged call in between."""
    N, nrhs = 1 << 12, 70                      # chunks of 32, 32 and 6 columns
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=64)
    gs = [W.complex_normal((nrhs, N), W.rng(830 + i), dtype=np.complex64) for i in range(4)]
    src = [torch.from_numpy(g).pin_memory() for g in gs]
    dst = [torch.full_like(s, float("nan")).pin_memory() for s in src]
    for i in range(4):
        plan.apply_host(src[i], dst[i], pipeline=(i != 2))
    # chained: the output of one call is the input of the next
    c1 = torch.full_like(src[0], float("nan")).pin_memory()
    c2 = torch.full_like(src[0], float("nan")).pin_memory()
    plan.apply_host(src[0], c1, pipeline=True)
    plan.apply_host(c1, c2, pipeline=True)
    torch.cuda.current_stream().synchronize()
    for g, d in zip(gs, dst):
        assert torch.equal(d, _device(plan, g))
    ref1 = _device(plan, gs[0])
    assert torch.equal(c1, ref1)
    assert torch.equal(c2, _device(plan, ref1.numpy()))
    lib = ibf.load_library()
    assert lib.ibf_apply_host(plan._p, src[0].data_ptr(), dst[0].data_ptr(), 1, 8, None) == 1   # unknown flag
    plan.close()


def test_host_apply_deferred_copy_outs(ibf):
    """IBF_HOST_DEFER: a stream of calls whose last copy-outs are ordered with
    the stream only by a later unflagged call or ibf_host_flush gives the
    device apply's results bit for bit: separate outputs (3 chunks per call,
    so both staging slots are reused across calls), a chain where one call's
    output is the next call's input, an adjoint call, and both ways of
    closing the stream."""
    N, nrhs = 1 << 12, 70                      # chunks of 32, 32 and 6 columns
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=64)
    gs = [W.complex_normal((nrhs, N), W.rng(850 + i), dtype=np.complex64) for i in range(4)]
    src = [torch.from_numpy(g).pin_memory() for g in gs]
    dst = [torch.full_like(s, float("nan")).pin_memory() for s in src]
    for i in range(4):
        plan.apply_host(src[i], dst[i], pipeline=True, defer=True)
    plan.host_flush()
    torch.cuda.current_stream().synchronize()
    for g, d in zip(gs, dst):
        assert torch.equal(d, _device(plan, g))
    # chain and adjoint under deferral, closed by an unflagged call
    c1 = torch.full_like(src[0], float("nan")).pin_memory()
    c2 = torch.full_like(src[0], float("nan")).pin_memory()
    a1 = torch.full_like(src[0], float("nan")).pin_memory()
    last = torch.full_like(src[0], float("nan")).pin_memory()
    plan.apply_host(src[0], c1, pipeline=True, defer=True)
    plan.apply_host(c1, c2, pipeline=True, defer=True)
    plan.apply_host(src[1], a1, adjoint=True, pipeline=True, defer=True)
    plan.apply_host(src[2], last, pipeline=True)
    torch.cuda.current_stream().synchronize()
    ref1 = _device(plan, gs[0])
    assert torch.equal(c1, ref1)
    assert torch.equal(c2, _device(plan, ref1.numpy()))
    assert torch.equal(last, _device(plan, gs[2]))
    assert torch.equal(a1, _device(plan, gs[1], adjoint=True))
    lib = ibf.load_library()
    assert lib.ibf_host_flush(None, None) == 1
    assert lib.ibf_host_flush(plan._p, None) == 0      # nothing outstanding
    plan.close()
