"""Batched apply of many uneven plans (one launch per fused chunk index),
its CUDA-graph capture, and the launch-shape autotuner."""
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


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _make(ibf, count, seed, emin=6, emax=12, nmax=40):
    rng = W.rng(seed)
    Ns = [1 << int(e) for e in rng.integers(emin, emax + 1, count)]
    nrhs = [int(v) for v in rng.integers(1, nmax + 1, count)]
    plans = [ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=k) for N, k in zip(Ns, nrhs)]
    ins = [torch.from_numpy(W.complex_normal((k, N), rng, dtype=np.complex64)).cuda() for N, k in zip(Ns, nrhs)]
    outs = [torch.full_like(t, float("nan")) for t in ins]
    return Ns, nrhs, plans, ins, outs


@pytest.mark.parametrize("adjoint", [False, True])
def test_batch_matches_per_plan_and_oracle(ibf, adjoint):
    Ns, nrhs, plans, ins, outs = _make(ibf, 12, 200 + adjoint)
    batch = ibf.Batch(plans, ins, outs, adjoint=adjoint)
    assert batch.query(ibf.BQ_LAUNCHES) <= 12 * (max(p.query(ibf.Q_LAUNCHES) for p in plans) + 2)
    batch.apply()
    torch.cuda.synchronize()
    for b, (p, g, u) in enumerate(zip(plans, ins, outs)):
        ref = torch.empty_like(g)
        raw = p.adjoint_raw if adjoint else p.apply_raw
        raw(g.data_ptr(), ref.data_ptr(), g.shape[0], torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert _rel(u, ref) < 1e-6, b
        if b < 3:
            x = W.uniform_x(Ns[b])
            gn = g.cpu().numpy().T.astype(np.complex128)
            fn = O.ibf_adjoint_1d if adjoint else O.ibf_apply_1d
            assert O.rel_l2(u.cpu().numpy().T, fn(O.PHASE_FIO1D, Ns[b], 9, x, gn)) < 1e-5


def test_batch_graph_capture(ibf):
    Ns, nrhs, plans, ins, outs = _make(ibf, 8, 300)
    batch = ibf.Batch(plans, ins, outs)
    batch.apply()
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        batch.apply(stream=s)
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, first):
        assert torch.equal(a, b)


def test_autotune_keeps_results(ibf):
    N, nrhs = 1 << 12, 24
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=nrhs)
    g = torch.from_numpy(W.complex_normal((N, nrhs), W.rng(400), dtype=np.complex64)).cuda()
    before = plan.apply(g)
    k, rt, ms = plan.autotune(nrhs)
    assert 2 <= k <= 10 and rt in (8, 16, 32) and ms > 0
    assert plan.query(ibf.Q_LEVELS_PER_LAUNCH) == k and plan.query(ibf.Q_RHS_TILE) == rt
    after = plan.apply(g)
    assert _rel(after, before) < 1e-6


def test_persistent_single_launch_matches(ibf):
    Ns, nrhs, plans, ins, outs = _make(ibf, 10, 700)
    batch = ibf.Batch(plans, ins, outs)
    batch.apply_persistent()
    assert batch.status() == 0
    torch.cuda.synchronize()
    for b, (p, g, u) in enumerate(zip(plans, ins, outs)):
        ref = torch.empty_like(g)
        p.apply_raw(g.data_ptr(), ref.data_ptr(), g.shape[0], torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert _rel(u, ref) < 1e-6, b
    # adjoint, and replay inside a CUDA graph
    Ns, nrhs, plans, ins, outs = _make(ibf, 6, 701)
    batch = ibf.Batch(plans, ins, outs, adjoint=True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.apply_persistent(stream=s)
    s.synchronize()
    first = [o.clone() for o in outs]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        batch.apply_persistent(stream=s)
    for o in outs:
        o.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert batch.status() == 0
    for a, b in zip(outs, first):
        assert torch.equal(a, b)


@pytest.mark.parametrize("adjoint", [False, True])
def test_persistent_single_launch_matches_oracle(ibf, adjoint):
    """The one-launch batch against the oracle's preliminary IBF (Algorithm
    2.1 / Sec. 3) and its adjoint, on plans that reach 4-level work items
    (N = 2^16: chunks of 4 levels on both sides of the switch), odd depth
    (N = 2^11) and a small plan (N = 2^8)."""
    Ns, nrhs = [1 << 16, 1 << 11, 1 << 8], [2, 5, 3]
    rng = W.rng(720 + adjoint)
    plans = [ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=k) for N, k in zip(Ns, nrhs)]
    ins = [torch.from_numpy(W.complex_normal((k, N), rng, dtype=np.complex64)).cuda() for N, k in zip(Ns, nrhs)]
    outs = [torch.full_like(t, float("nan")) for t in ins]
    batch = ibf.Batch(plans, ins, outs, adjoint=adjoint)
    batch.apply_persistent()
    torch.cuda.synchronize()
    assert batch.status() == 0
    fn = O.ibf_adjoint_1d if adjoint else O.ibf_apply_1d
    for N, g, u in zip(Ns, ins, outs):
        ref = fn(O.PHASE_FIO1D, N, 9, W.uniform_x(N), g.cpu().numpy().T.astype(np.complex128))
        e = O.rel_l2(u.cpu().numpy().T, ref)
        print("\npersistent %s N=%d: %.3e vs oracle" % ("adjoint" if adjoint else "forward", N, e))
        assert e < 1e-5, N


@pytest.mark.parametrize("adjoint", [False, True])
def test_persistent_packed_items_match_oracle(ibf, adjoint):
    """Narrow and shallow plans: a persistent item runs several blocks side by
    side (1, 2 and 3 columns: tiles of 1, 2 and 4 columns, groups of fewer
    than 32 threads on a named barrier; N = 2^6 leaves items with spare
    groups), next to a 40-column plan (two 32-column tiles, one block per
    item).  Forward and adjoint against the oracle's preliminary IBF."""
    Ns, nrhs = [1 << 6, 1 << 7, 1 << 9, 1 << 10], [1, 2, 3, 40]
    rng = W.rng(730 + adjoint)
    plans = [ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=k) for N, k in zip(Ns, nrhs)]
    ins = [torch.from_numpy(W.complex_normal((k, N), rng, dtype=np.complex64)).cuda() for N, k in zip(Ns, nrhs)]
    outs = [torch.full_like(t, float("nan")) for t in ins]
    batch = ibf.Batch(plans, ins, outs, adjoint=adjoint)
    batch.apply_persistent()
    torch.cuda.synchronize()
    assert batch.status() == 0
    fn = O.ibf_adjoint_1d if adjoint else O.ibf_apply_1d
    for N, g, u in zip(Ns, ins, outs):
        ref = fn(O.PHASE_FIO1D, N, 9, W.uniform_x(N), g.cpu().numpy().T.astype(np.complex128))
        e = O.rel_l2(u.cpu().numpy().T, ref)
        print("\npersistent packed %s N=%d nrhs=%d: %.3e vs oracle" % ("adjoint" if adjoint else "forward", N,
                                                                       g.shape[0], e))
        assert e < 1e-5, N


def test_persistent_wait_expires_without_hanging(ibf):
    """A dependency that is never satisfied (test hook) makes the bounded waits
    run out: the kernel returns, the batch reports IBF_ERR_TIMEOUT, and the
    context stays usable for a correct run afterwards."""
    import time
    Ns, nrhs, plans, ins, outs = _make(ibf, 4, 702, emin=8, emax=10)
    batch = ibf.Batch(plans, ins, outs)
    lib = ibf.load_library()
    assert lib.ibf_batch_set_wait_limit(batch._b, 1 << 12) == 0
    assert lib.ibf_batch_test_withhold(batch._b, 0, 1) == 0
    t0 = time.time()
    batch.apply_persistent()
    assert batch.status() == 5          # IBF_ERR_TIMEOUT
    assert time.time() - t0 < 30
    # every plan of the batch holds the timeout in its sticky status until read
    assert [p.status() for p in plans] == [5] * len(plans)
    assert [p.status() for p in plans] == [0] * len(plans)
    assert lib.ibf_batch_test_withhold(batch._b, 0, 0) == 0
    assert lib.ibf_batch_set_wait_limit(batch._b, 1 << 21) == 0
    batch.apply_persistent()
    assert batch.status() == 0
    torch.cuda.synchronize()
    for p, g, u in zip(plans, ins, outs):
        ref = torch.empty_like(g)
        p.apply_raw(g.data_ptr(), ref.data_ptr(), g.shape[0], torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert _rel(u, ref) < 1e-6


def test_batch_fp64_graph_and_persistent(ibf):
    """FP64 structured plans: the batched launches and the persistent launch
    equal the per-plan apply (forward and adjoint)."""
    rng = W.rng(710)
    Ns = [1 << int(e) for e in rng.integers(6, 11, 6)]
    nrhs = [int(v) for v in rng.integers(1, 12, 6)]
    for adjoint in (False, True):
        plans = [ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C128, form=ibf.FORM_STRUCTURED, max_nrhs=k)
                 for N, k in zip(Ns, nrhs)]
        ins = [torch.from_numpy(W.complex_normal((k, N), rng)).cuda() for N, k in zip(Ns, nrhs)]
        outs = [torch.full_like(t, float("nan")) for t in ins]
        batch = ibf.Batch(plans, ins, outs, adjoint=adjoint)
        refs = []
        for p, g in zip(plans, ins):
            ref = torch.empty_like(g)
            raw = p.adjoint_raw if adjoint else p.apply_raw
            raw(g.data_ptr(), ref.data_ptr(), g.shape[0], torch.cuda.current_stream().cuda_stream)
            refs.append(ref)
        batch.apply()
        torch.cuda.synchronize()
        for u, ref in zip(outs, refs):
            assert _rel(u, ref) < 1e-13
        for o in outs:
            o.fill_(float("nan"))
        batch.apply_persistent()
        torch.cuda.synchronize()
        assert batch.status() == 0
        for u, ref in zip(outs, refs):
            assert _rel(u, ref) < 1e-13
