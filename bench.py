"""Benchmark of the IBF apply on GB300 (one JSON line on rank 0).

Workload (default): 1D FIO, Phi(x,xi) = x xi + c(x)|xi|, c = (2 + sin 2 pi x)/8
(Sec. 6.2), x_j = j/N, xi_k = k - N/2, N = 2^20, r = 9 Chebyshev points,
nrhs = 64 complex64 right-hand sides with iid N(0,1) real and imaginary
parts, FP32 structured fused apply.  A step is one u = K g over the 64
vectors.  Inputs (512 MB) and the two Lambda buffers (4.8 GB each) exceed
the 129 MB L2, so no flush is needed between steps.

Reported next to it: the plain FP64 explicit single-vector form on the same
GPU (the form the fast path is measured against) with the relative L2
difference of the FP32 result from it, per-kernel CUDA-event timing of the
dominant kernel against its roofline, and the FP64 CPU oracle timed on the
host cores.

--impl reference times the FP64 CPU oracle (the method as the paper states
it, matrix-free, all host cores) on one vector of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

FP32_LANES_PER_SM = 128

# DRAM bytes (read + write) per launch of the fused kernels, from one
# single-pass ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of
# this benchmark at N = 2^20, r = 9, nrhs = 64, 4 levels per launch, tile 32
# (the ncu DRAM capture of the fused kernels).  Keyed by the launch's level
# range; valid only while the kernel sources hash to KERNEL_SRC_SHA.
KERNEL_SRC_SHA = "c023499f6816bede"
TRAFFIC_N20_R9_NRHS64_K4 = {
    (0, 4, "H"): 1216580608 + 4771279104,
    (4, 7, "H"): 5284974592 + 4777747968,
    (7, 10, "H"): 5964532992 + 4782129408,
    (10, 14, "G"): 5436852224 + 4781660672,
    (14, 17, "G"): 5285030400 + 4780770560,
    (17, 20, "G"): 5369789184 + 527908096,
}


def kernel_src_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("paper_1605_03616_gb300/csrc/ibf_fused.cuh", "paper_1605_03616_gb300/csrc/ibf_fused_f32.cu"):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]
METRIC = "IBF apply vectors/s (rel.err <= 1e-5 vs plain FP64 GPU form)"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def workload_name(a):
    return "1D FIO Phi=x*xi+c(x)|xi| N=2^%d r=%d nrhs=%d complex64 (FP32 structured)" % (
        int(np.log2(a.N)), a.r, a.nrhs)


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index: int):
        self.dev = dev_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [v.strip() for v in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- multi-GPU helpers
def max_over_ranks(value_ms: float, world: int, dist=None, device=None) -> float:
    """Largest per-rank time: the whole job is as slow as its slowest rank."""
    if world <= 1 or dist is None:
        return value_ms
    import torch
    t = torch.tensor([float(value_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(vectors_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Weak scaling: every rank applies its own batch of vectors per step, so
    the job processes world * vectors_per_rank * steps vectors in max_ms."""
    return world * vectors_per_rank * steps / (max_ms / 1e3)


# ------------------------------------------------------------ CPU oracle arm
def oracle_vectors_per_s(a, threads: int):
    """Time the FP64 oracle (matrix-free butterfly) on one vector of the
    workload; returns (vectors/s, seconds)."""
    import oracle as O
    O.set_threads(threads)
    g = W.complex_normal((a.N, 1), W.rng(workload=2))
    x = W.uniform_x(a.N)
    t0 = time.perf_counter()
    O.ibf_apply_1d(O.PHASE_FIO1D, a.N, a.r, x, g)
    dt = time.perf_counter() - t0
    return 1.0 / dt, dt


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    # warm-up steps run the same code on a 2^12 problem: the CPU oracle has no
    # state to warm beyond its first touch of the code and the thread pool
    small = argparse.Namespace(**{**vars(a), "N": 1 << 12})
    for _ in range(a.warmup):
        oracle_vectors_per_s(small, cores)
    times = []
    for _ in range(a.steps):
        times.append(oracle_vectors_per_s(a, cores)[1])
    tot = sum(times)
    v = a.steps / tot
    sample = "one of the %d vectors per step (N=2^%d, matrix-free FP64 oracle, %d threads)" % (
        a.nrhs, int(np.log2(a.N)), cores)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "vectors/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "N": a.N, "r": a.r, "nrhs": a.nrhs, "phase": "FIO1D"},
            "cpu_baseline": {"value": v, "unit": "vectors/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------- batched workload
def run_nufft_latency(ibf, torch, N=1024, reps=200):
    """Latency of a small nonuniform transform: phase x xi with N = 1024 sorted iid uniform
    points, one vector: apply latency in microseconds, FP64 explicit and FP32
    structured, as a sequence of launches and replayed from a CUDA graph."""
    gen = W.rng(workload=1)
    x = W.random_sorted_x(N, gen)
    g64 = torch.from_numpy(W.complex_normal(N, gen)).cuda()
    out = {"workload": "NUFFT phase x*xi, N=1024 random sorted x, r=9, one vector"}
    stream = torch.cuda.Stream()
    for name, dtype, gv in [("fp64_explicit", ibf.C128, g64), ("fp32_structured", ibf.C64_FP32,
                                                               g64.to(torch.complex64))]:
        p = ibf.Plan(ibf.PHASE_NUFFT, N, 9, dtype, x=x, max_nrhs=1)
        u = torch.empty_like(gv)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(10):
                p.apply_raw(gv.data_ptr(), u.data_ptr(), 1, stream.cuda_stream)
            e0.record(stream)
            for _ in range(reps):
                p.apply_raw(gv.data_ptr(), u.data_ptr(), 1, stream.cuda_stream)
            e1.record(stream)
        stream.synchronize()
        t_launch = e0.elapsed_time(e1) / reps * 1e3
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            p.apply_raw(gv.data_ptr(), u.data_ptr(), 1, stream.cuda_stream)
        for _ in range(10):
            graph.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"us_per_apply": t_launch, "us_per_apply_graph": e0.elapsed_time(e1) / reps * 1e3,
                     "launches": p.query(ibf.Q_LAUNCHES)}
        del graph
        if dtype == ibf.C64_FP32:
            k, rt, ms = p.autotune(1)
            out[name]["autotuned"] = {"levels_per_launch": k, "rhs_tile": rt, "us_per_apply": ms * 1e3,
                                      "launches": p.query(ibf.Q_LAUNCHES)}
        p.close()
    return out


def run_optimal(ibf, torch, N=1 << 16, nrhs=8, reps=3, variants=None):
    """Optimal IBF (sweep-out stage, Sec. 4.2, and with the sweep-in stage,
    Sec. 4.3) against the preliminary IBF, explicit factors in FP64 and in
    FP32 (built in FP64, stored and applied in FP32), 1D FIO N = 2^16,
    8 columns: construction time, apply vectors/s, stored entries, and the
    relative L2 difference from the r = 12 FP64 preliminary IBF (itself
    ~7e-8 from the direct sum)."""
    gen = W.rng(workload=6)
    g = torch.from_numpy(W.complex_normal((N, nrhs), gen)).cuda()
    g32 = g.to(torch.complex64)
    out, ref = [], None
    names = {ibf.FORM_EXPLICIT: "preliminary", ibf.FORM_OPTIMAL: "optimal (sweep-out)",
             ibf.FORM_OPTIMAL_IN: "optimal (sweep-out + sweep-in)",
             ibf.FORM_STRUCTURED: "preliminary, structured (the fast FP32 form)"}
    C128, C64 = ibf.C128, ibf.C64_FP32
    variants = variants or [(12, ibf.FORM_EXPLICIT, 0, C128), (9, ibf.FORM_EXPLICIT, 0, C128),
                            (12, ibf.FORM_OPTIMAL, 9, C128), (12, ibf.FORM_OPTIMAL_IN, 9, C128),
                            (12, ibf.FORM_OPTIMAL, 7, C128), (12, ibf.FORM_OPTIMAL_IN, 7, C128),
                            (9, ibf.FORM_OPTIMAL, 7, C128),
                            (12, ibf.FORM_EXPLICIT, 0, C64), (12, ibf.FORM_OPTIMAL_IN, 9, C64),
                            (12, ibf.FORM_OPTIMAL_IN, 7, C64), (9, ibf.FORM_STRUCTURED, 0, C64)]
    for r, form, r0, dt in variants:
        gin = g if dt == C128 else g32
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p = ibf.Plan(ibf.PHASE_FIO1D, N, r, dt, form=form, rank=r0, max_nrhs=nrhs)
        if form == ibf.FORM_STRUCTURED:
            p.autotune(nrhs)
        torch.cuda.synchronize()
        tc = (time.perf_counter() - t0) * 1e3
        u = p.apply(gin)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            p.apply(gin)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        u = u.to(torch.complex128)
        if ref is None:
            ref = u.clone()
        rec = {"form": names[form], "dtype": "f64" if dt == C128 else "f32", "r": r,
               "r0": r0 or r, "construct_ms": tc, "apply_ms": ms, "vectors_per_s": nrhs / (ms / 1e3),
               "nnz": p.query(ibf.Q_NNZ),
               "rel_diff_vs_r12_preliminary": float(torch.linalg.vector_norm(u - ref) / torch.linalg.vector_norm(ref))}
        out.append(rec)
        p.close()
    return {"workload": "1D FIO N=2^%d, %d columns, explicit factors (FP64, and FP32 copies)" % (int(np.log2(N)), nrhs),
            "variants": out}


def run_autograd(ibf, torch, N=1 << 18, nrhs=32, reps=5):
    """Training-style step: loss ||K g - y||^2 at N = 2^18, 32 columns, complex64; one
    step = forward apply + backward (the hand-written adjoint) through
    torch.autograd, CUDA events."""
    from paper_1605_03616_gb300.autograd import ibf_apply
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=nrhs)
    gen = W.rng(workload=5)
    g0 = torch.from_numpy(W.complex_normal((N, nrhs), gen, dtype=np.complex64)).cuda()
    y = torch.from_numpy(W.complex_normal((N, nrhs), gen, dtype=np.complex64)).cuda()

    def step():
        g = g0.clone().requires_grad_(True)
        loss = (ibf_apply(plan, g) - y).abs().pow(2).sum()
        loss.backward()
        return g.grad

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    rec = {"workload": "loss ||K g - y||^2, 1D FIO N=2^18 r=9, 32 columns complex64, forward + adjoint via autograd",
           "ms_per_step": ms, "vectors_per_s": nrhs / (ms / 1e3)}
    plan.close()
    return rec


def run_tensorcore(ibf, torch, N=1 << 20, nrhs=64, k=4, reps=5, profile=True):
    """Tensor-core form against the packed-FP32 SIMT form on the same workload
    (1D FIO, r = 9, 32-column tiles, k levels per launch): per-apply and
    per-launch CUDA-event times, and the relative difference of the results.
    Each plan runs one warm-up apply, `reps` timed applies and (profile) one
    apply with per-launch events."""
    g = torch.from_numpy(W.complex_normal((nrhs, N), W.rng(workload=2), dtype=np.complex64)).cuda()
    out, rec = {}, {"workload": "1D FIO N=%d r=9 nrhs=%d complex64, %d levels per launch, tile 32" % (N, nrhs, k)}
    s = torch.cuda.current_stream().cuda_stream
    for dt, name in ((ibf.C64_FP32, "fp32_simt"), (ibf.C64_TF32X3, "tf32x3_tensor")):
        p = ibf.Plan(ibf.PHASE_FIO1D, N, 9, dt, max_nrhs=nrhs, levels_per_launch=k, rhs_tile=32)
        u = torch.empty_like(g)
        p.apply_raw(g.data_ptr(), u.data_ptr(), nrhs, s)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            p.apply_raw(g.data_ptr(), u.data_ptr(), nrhs, s)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        r = {"ms_per_apply": ms, "vectors_per_s": nrhs / ms * 1e3}
        if profile:
            p.profile_begin(64)
            p.apply_raw(g.data_ptr(), u.data_ptr(), nrhs, s)
            prof = p.profile_end()
            r["launch_ms"] = [round(m, 4) for _, m in prof]
            r["launch_kind"] = ["H" if kk == ibf.K_FUSED_H else "G" for kk, _ in prof]
        torch.cuda.synchronize()
        r["status"] = p.status()
        out[name] = u
        rec[name] = r
        p.close()
    a, b = out["tf32x3_tensor"], out["fp32_simt"]
    rec["tf32x3_rel_diff_vs_fp32"] = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    rec["tensor_over_simt_time"] = rec["tf32x3_tensor"]["ms_per_apply"] / rec["fp32_simt"]["ms_per_apply"]
    return rec


def run_amplitude(ibf, torch, N=1 << 20, nrhs=16, q=3, reps=5):
    """Non-unit amplitude a(x, xi) = sum_t alpha_t(x) beta_t(xi) (Sec. 1),
    1D FIO N = 2^20, r = 9, 16 columns complex64, q = 3 terms (one pass: the
    phase-only apply runs on 48 columns), against the phase-only apply of the
    same 16 and of 48 columns on the same plan; CUDA events."""
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=nrhs * q)
    gen = W.rng(workload=7)
    x, xi = W.uniform_x(N), W.omega_1d(N)
    alpha, beta = W.separated_amplitude(x, xi, q, gen, dtype=np.complex64)
    # (N, m) views of contiguous (m, N) tensors: the column-major layout of
    # the C ABI, so the binding passes them on without a copy
    al = torch.from_numpy(alpha.T.copy()).cuda().t()
    be = torch.from_numpy(beta.T.copy()).cuda().t()
    g = torch.from_numpy(W.complex_normal((nrhs, N), gen, dtype=np.complex64)).cuda().t()
    g3 = torch.from_numpy(W.complex_normal((nrhs * q, N), gen, dtype=np.complex64)).cuda().t()
    work = torch.empty(2 * N * nrhs * q, dtype=torch.complex64, device="cuda")

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_amp = timed(lambda: plan.apply_amplitude(g, al, be, work=work))
    ms_1 = timed(lambda: plan.apply(g))
    ms_q = timed(lambda: plan.apply(g3))
    rec = {"workload": "1D FIO N=2^%d r=9, %d columns complex64, amplitude of q=%d separated terms"
                       % (int(np.log2(N)), nrhs, q),
           "ms": ms_amp, "vectors_per_s": nrhs / (ms_amp / 1e3), "phase_only_ms_16_columns": ms_1,
           "phase_only_ms_48_columns": ms_q, "scaling_kernels_ms": ms_amp - ms_q}
    plan.close()
    return rec


def run_batch(ibf, torch, reps=5, count=256, seed=4):
    """256 independent 1D FIO transforms, N = 2^e with e uniform in 10..16,
    nrhs uniform in 1..64, complex64, r = 9: the batched launch captured in a
    CUDA graph vs a loop of per-transform applies, both with CUDA events."""
    gen = W.rng(workload=seed)
    es = gen.integers(10, 17, count)
    nr = gen.integers(1, 65, count)
    plans = [ibf.Plan(ibf.PHASE_FIO1D, 1 << int(e), 9, ibf.C64_FP32, max_nrhs=int(k)) for e, k in zip(es, nr)]
    ins = [torch.from_numpy(W.complex_normal((int(k), 1 << int(e)), gen, dtype=np.complex64)).cuda()
           for e, k in zip(es, nr)]
    outs = [torch.empty_like(t) for t in ins]
    batch = ibf.Batch(plans, ins, outs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(2):
            batch.apply(stream=stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        batch.apply(stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    t_graph = e0.elapsed_time(e1) / reps
    ref = [o.clone() for o in outs]
    cs = torch.cuda.current_stream().cuda_stream

    def loop():
        for p, g, u in zip(plans, ins, outs):
            p.apply_raw(g.data_ptr(), u.data_ptr(), g.shape[0], cs)
    loop()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        loop()
    e1.record()
    torch.cuda.synchronize()
    t_loop = e0.elapsed_time(e1) / reps
    err = max(float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) for a, b in zip(outs, ref))
    # the same batch as one persistent launch, also replayed from a CUDA graph
    with torch.cuda.stream(stream):
        batch.apply_persistent(stream=stream)
    stream.synchronize()
    pgraph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(pgraph, stream=stream):
        batch.apply_persistent(stream=stream)
    for _ in range(2):
        pgraph.replay()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        pgraph.replay()
    e1.record()
    torch.cuda.synchronize()
    t_pers = e0.elapsed_time(e1) / reps
    perr = max(float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) for a, b in zip(outs, ref))
    pstatus = batch.status()
    vec = int(nr.sum())
    # algorithmic FP32 flops of the whole batch (independent of the fusion depth)
    flops = sum(apply_flops(int(e), 9, 1 << int(e), int(k)) for e, k in zip(es, nr))
    g_launches = batch.query(ibf.BQ_LAUNCHES)
    batch.close()
    # the graph again with every plan's launch shape picked by the autotuner
    for p, k in zip(plans, nr):
        p.autotune(int(k))
    tbatch = ibf.Batch(plans, ins, outs)
    with torch.cuda.stream(stream):
        tbatch.apply(stream=stream)
    stream.synchronize()
    tgraph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(tgraph, stream=stream):
        tbatch.apply(stream=stream)
    for _ in range(2):
        tgraph.replay()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        tgraph.replay()
    e1.record()
    torch.cuda.synchronize()
    t_tuned = e0.elapsed_time(e1) / reps
    terr = max(float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) for a, b in zip(outs, ref))
    t_launches = tbatch.query(ibf.BQ_LAUNCHES)
    tbatch.close()
    pk, _ = peaks()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_peak = nsm * FP32_LANES_PER_SM * 2 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    res = {"workload": "256 x 1D FIO, N=2^e e~U{10..16}, nrhs~U{1..64}, r=9, complex64",
           "vectors": vec, "graph_ms": t_graph, "loop_ms": t_loop,
           "graph_vectors_per_s": vec / (t_graph / 1e3), "loop_vectors_per_s": vec / (t_loop / 1e3),
           "speedup_vs_loop": t_loop / t_graph, "launches_graph": g_launches,
           "launches_loop": sum(p.query(ibf.Q_LAUNCHES) for p in plans), "max_rel_diff_graph_vs_loop": err,
           "persistent_ms": t_pers, "persistent_vectors_per_s": vec / (t_pers / 1e3), "persistent_launches": 1,
           "persistent_max_rel_diff": perr, "persistent_status": pstatus,
           "tuned_graph_ms": t_tuned, "tuned_graph_vectors_per_s": vec / (t_tuned / 1e3),
           "tuned_launches_graph": t_launches, "tuned_max_rel_diff": terr,
           "alg_gflop": flops / 1e9, "fp32_peak_tflops": fp32_peak,
           "graph_alu_frac": flops / (t_graph / 1e3) / 1e12 / fp32_peak,
           "tuned_graph_alu_frac": flops / (t_tuned / 1e3) / 1e12 / fp32_peak,
           "persistent_alu_frac": flops / (t_pers / 1e3) / 1e12 / fp32_peak}
    for p in plans:
        p.close()
    return res


# ------------------------------------------------------------ 2D workload
def run_2d(ibf, torch, n=512, r=7, nrhs=32, reps=5):
    """2D FIO (Sec. 6.3 form, constants /16) on the n x n grid, multiscale IBF
    with a 16 x 16 centre, r = 7 per dimension, nrhs complex64 vectors."""
    N = n * n
    plan = ibf.Plan(ibf.PHASE_FIO2D, N, r, ibf.C64_FP32, d=2, max_nrhs=nrhs)
    g = torch.from_numpy(W.complex_normal((nrhs, N), W.rng(workload=3), dtype=np.complex64)).cuda()
    u = torch.empty_like(g)
    cs = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        plan.apply_raw(g.data_ptr(), u.data_ptr(), nrhs, cs)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.apply_raw(g.data_ptr(), u.data_ptr(), nrhs, cs)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    for _ in range(2):
        plan.adjoint_raw(u.data_ptr(), g.data_ptr(), nrhs, cs)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        plan.adjoint_raw(u.data_ptr(), g.data_ptr(), nrhs, cs)
    e1.record()
    torch.cuda.synchronize()
    ms_adj = e0.elapsed_time(e1) / reps
    res = {"workload": "2D FIO n=%d (N=%d) r=%d nrhs=%d complex64, MIBF with 16x16 centre" % (n, N, r, nrhs),
           "ms_per_apply": ms, "vectors_per_s": nrhs / (ms / 1e3), "adjoint_ms_per_apply": ms_adj,
           "launches": plan.query(ibf.Q_LAUNCHES), "factor_bytes": plan.query(ibf.Q_FACTOR_BYTES)}
    plan.close()
    return res


# ------------------------------------------------------------------ GPU arm
def structured_flops(kind_levels, r, N, nc, pro, epi, kind_g):
    """Algorithmic FP32 flops of one fused launch of the even/odd structured
    form, per butterfly unit (two outputs) and right-hand side:
    H form 8 r^2 + 36 r (two complex phase products, the even/odd sums and
    r^2 real multiply-adds per output), G form 8 r^2 + 44 r (even/odd parts
    of both inputs, r^2 multiply-adds per input shared by both outputs, four
    complex phase products per output index)."""
    unit = 8 * r * r + (44 if kind_g else 36) * r
    f = unit * (N // 2) * kind_levels * nc
    if pro == "V":
        f += 6 * r * N * nc
    if epi == "switch":
        f += 8 * r * r * N * nc
    if epi == "U":
        f += 8 * r * N * nc
    return f


def fused_schedule(L, h, kfuse):
    """Level ranges (lo, hi, kind) of the structured apply's fused launches in
    launch order: levels 1..h and h+1..L split into balanced chunks of at most
    kfuse levels (the library's schedule)."""
    sched = []

    def split(lo, hi, kind):
        n = hi - lo
        nch = (n + kfuse - 1) // kfuse
        for c in range(nch):
            ln = n // nch + (1 if c < n % nch else 0)
            sched.append((lo, lo + ln, kind))
            lo += ln
    split(0, h, "H")
    split(h, L, "G")
    return sched


def dominant_roofline(prof, L, h, kfuse, r, N, nrhs, fp32_peak, hbm_peak):
    """Roofline of the launch with the largest total time in a per-launch
    profile (list of (kind, ms) in launch order, whole applies): algorithmic
    flops (structured_flops) and bytes (Lambda or g/u in and out, the phase
    tables, the switch blocks) per launch over its mean CUDA-event time."""
    sched = fused_schedule(L, h, kfuse)
    per_launch = {}
    for idx, (_, t_ms) in enumerate(prof):
        per_launch.setdefault(sched[idx % len(sched)], []).append(t_ms)
    tot = {k: sum(v) for k, v in per_launch.items()}
    lo, hi, kd = max(tot, key=tot.get)
    pro = "V" if lo == 0 else None
    epi = "U" if hi == L else ("switch" if hi == h else None)
    avg_ms = statistics.mean(per_launch[(lo, hi, kd)])
    flops = structured_flops(hi - lo, r, N, nrhs, pro, epi, kd == "G")
    esz = 8
    bytes_alg = (N * nrhs * esz) if pro == "V" else (N * r * nrhs * esz)
    bytes_alg += (N * nrhs * esz) if epi == "U" else (N * r * nrhs * esz)
    bytes_alg += (hi - lo) * 2 * N * r * esz
    if epi == "switch":
        bytes_alg += N * r * r * esz
    ach_tf = flops / (avg_ms / 1e3) / 1e12
    ach_gb = bytes_alg / (avg_ms / 1e3) / 1e9
    return {"lo": lo, "hi": hi, "kind": kd, "pro": pro, "epi": epi, "avg_ms": avg_ms, "n": len(per_launch[(lo, hi, kd)]),
            "flops": flops, "bytes": bytes_alg, "tflops": ach_tf, "gbs": ach_gb, "alu_frac": ach_tf / fp32_peak,
            "hbm_frac": ach_gb / hbm_peak,
            "launch_ms": {"%s %d..%d" % (kk, a0 + 1, b0): round(statistics.mean(v), 4)
                          for (a0, b0, kk), v in per_launch.items()}}


# Series coefficients of the phases with caller-given coefficients: 1D,
# c(x) = sum_m a_m cos(2 pi m x) + b_m sin(2 pi m x) (Sec. 6.2's c plus three
# harmonics); 2D, rows (p, q, al1, be1, al2, be2) of c1, c2 (Sec. 6.3's form).
SERIES1D = ([0.25, 0.01, -0.02, 0.01], [0.0, 0.125, 0.015, -0.01])
SERIES2D = [[0, 0, 0.2, 0, 0.12, 0], [1, 0, 0.02, 0.015, 0, 0.01], [0, 1, -0.01, 0, 0.015, -0.005],
            [1, 1, 0, 0.01, 0.005, 0], [1, -1, 0.005, 0, 0, 0.008], [2, 1, 0, -0.004, 0.003, 0.002]]


def run_series(ibf, torch, reps=5):
    """The FIOs with series coefficients: plan construction (wall clock) and
    FP32 apply at the workload sizes -- 1D N=2^20, r=9, 64 columns (tile and
    depth of the FIO1D workload) and 2D n=512, r=7, 32 columns -- beside the
    fixed-coefficient phases of Sec. 6.2 / 6.3 at the same sizes."""
    cs = torch.cuda.current_stream().cuda_stream
    out = {"workload": "1D N=2^20 r=9 64 columns; 2D n=512 r=7 32 columns; complex64 structured",
           "series1d_terms": len(SERIES1D[0]), "series2d_terms": len(SERIES2D)}

    def timed(plan, nrhs, N):
        g = torch.from_numpy(W.complex_normal((nrhs, N), W.rng(workload=7), dtype=np.complex64)).cuda()
        u = torch.empty_like(g)
        for _ in range(2):
            plan.apply_raw(g.data_ptr(), u.data_ptr(), nrhs, cs)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.apply_raw(g.data_ptr(), u.data_ptr(), nrhs, cs)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for tag, phase, d, N, r, nrhs, kw in (
            ("fio1d", ibf.PHASE_FIO1D, 1, 1 << 20, 9, 64, {}),
            ("series1d", ibf.PHASE_FIO1D_SERIES, 1, 1 << 20, 9, 64, {"coef": SERIES1D}),
            ("fio2d", ibf.PHASE_FIO2D, 2, 512 * 512, 7, 32, {}),
            ("series2d", ibf.PHASE_FIO2D_SERIES, 2, 512 * 512, 7, 32, {"coef": SERIES2D})):
        extra = {"levels_per_launch": 4, "rhs_tile": 32} if d == 1 else {}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = ibf.Plan(phase, N, r, ibf.C64_FP32, d=d, max_nrhs=nrhs, **extra, **kw)
        torch.cuda.synchronize()
        t_build = (time.perf_counter() - t0) * 1e3
        ms = timed(plan, nrhs, N)
        out[tag] = {"construct_ms": t_build, "apply_ms": ms, "vectors_per_s": nrhs * 1e3 / ms}
        plan.close()
    return out


def run_config2_sweep(ibf, torch, fp32_peak, hbm_peak, Ns=(1 << 16, 1 << 18, 1 << 20), nrhss=(1, 16, 64), reps=5):
    """1D FIO grid N x nrhs: the FP32 structured apply in its autotuned launch
    shape (vectors/s, the dominant launch's roofline fraction) against the
    plain FP64 explicit single-vector form on the same GPU (vectors/s, and the
    FP32 result's relative L2 difference from it on the first column)."""
    s = torch.cuda.current_stream().cuda_stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pts = []
    for N in Ns:
        g = torch.from_numpy(W.complex_normal((max(nrhss), N), W.rng(workload=2), dtype=np.complex64)).cuda()
        p64 = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C128, max_nrhs=1)
        g64 = g[0:1].to(torch.complex128).contiguous()
        u64 = torch.empty_like(g64)
        for _ in range(2):
            p64.apply_raw(g64.data_ptr(), u64.data_ptr(), 1, s)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(3):
            p64.apply_raw(g64.data_ptr(), u64.data_ptr(), 1, s)
        e1.record()
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 3
        p64.close()
        for nrhs in nrhss:
            plan = ibf.Plan(ibf.PHASE_FIO1D, N, 9, ibf.C64_FP32, max_nrhs=nrhs)
            k, rt, _ = plan.autotune(nrhs)
            gg = g[:nrhs].contiguous()
            u = torch.empty_like(gg)
            for _ in range(2):
                plan.apply_raw(gg.data_ptr(), u.data_ptr(), nrhs, s)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                plan.apply_raw(gg.data_ptr(), u.data_ptr(), nrhs, s)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            plan.profile_begin(4 * plan.query(ibf.Q_LAUNCHES) + 8)
            for _ in range(3):
                plan.apply_raw(gg.data_ptr(), u.data_ptr(), nrhs, s)
            prof = plan.profile_end()
            dom = dominant_roofline(prof, plan.L, plan.h, plan.query(ibf.Q_LEVELS_PER_LAUNCH), 9, N, nrhs,
                                    fp32_peak, hbm_peak)
            err = float(torch.linalg.vector_norm(u[0].to(torch.complex128) - u64[0]) /
                        torch.linalg.vector_norm(u64[0]))
            v32 = nrhs / ms * 1e3
            pts.append({"N": N, "nrhs": nrhs, "vectors_per_s": v32, "ms_per_apply": ms, "levels_per_launch": k,
                        "rhs_tile": rt, "launches": plan.query(ibf.Q_LAUNCHES),
                        "dominant_launch": "%s %d..%d" % (dom["kind"], dom["lo"] + 1, dom["hi"]),
                        "dominant_ms": dom["avg_ms"], "alu_frac": dom["alu_frac"], "hbm_frac": dom["hbm_frac"],
                        "fp64_plain_vectors_per_s": 1e3 / t64, "speedup_vs_fp64_plain": v32 / (1e3 / t64),
                        "rel_err_vs_fp64": err})
            plan.close()
        del g
    return {"workload": "1D FIO Phi=x*xi+c(x)|xi| r=9 complex64 (FP32 structured, autotuned per point) vs "
                        "plain FP64 explicit single-vector form", "fp32_peak_tflops": fp32_peak,
            "hbm_peak_gbs": hbm_peak, "points": pts}


def apply_flops(L, r, N, nc):
    """Algorithmic FP32 flops of one structured apply (switch at h = L // 2):
    h H levels, L - h G levels, the V^0 prologue, the switch and U^L."""
    h = L // 2
    return (structured_flops(h, r, N, nc, "V", "switch", False) +
            structured_flops(L - h, r, N, nc, None, "U", True))


def run_gpu(a):
    import torch
    import torch.distributed as dist

    import paper_1605_03616_gb300 as ibf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    N, r, nrhs = a.N, a.r, a.nrhs
    torch.cuda.synchronize()
    t_c0 = time.perf_counter()
    plan = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C64_FP32, max_nrhs=nrhs)   # returns after construction
    t_struct = (time.perf_counter() - t_c0) * 1e3
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    g_host = W.complex_normal((nrhs, N), W.rng(workload=2 + 1000 * rank), dtype=np.complex64)  # row = column
    g = torch.from_numpy(g_host).to(dev)            # column-major N x nrhs
    u = torch.empty_like(g)
    tuned = None
    if a.levels_per_launch or a.rhs_tile:
        plan.close()
        plan = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C64_FP32, max_nrhs=nrhs, levels_per_launch=a.levels_per_launch,
                        rhs_tile=a.rhs_tile)
        tuned = {"levels_per_launch": a.levels_per_launch, "rhs_tile": a.rhs_tile, "ms": None, "forced": True}
    elif not a.no_autotune:
        k_, rt_, ms_ = plan.autotune(nrhs)
        tuned = {"levels_per_launch": k_, "rhs_tile": rt_, "ms": ms_}
    launches = plan.query(ibf.Q_LAUNCHES)

    def step():
        plan.apply_raw(g.data_ptr(), u.data_ptr(), nrhs, stream.cuda_stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    plan.profile_begin(a.steps * launches + 8)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    prof = plan.profile_end()
    ms = max_over_ranks(ms, world, dist if world > 1 else None, dev)
    value = job_throughput(nrhs, a.steps, world, ms)

    # ---- dominant kernel and its roofline (per-launch CUDA events, timed region)
    sched = []
    L, h = plan.L, plan.h
    kfuse = plan.query(ibf.Q_LEVELS_PER_LAUNCH)
    rtile = plan.query(ibf.Q_RHS_TILE)

    def split(lo, hi, kind):
        n = hi - lo
        nch = (n + kfuse - 1) // kfuse
        for c in range(nch):
            ln = n // nch + (1 if c < n % nch else 0)
            sched.append((lo, lo + ln, kind))
            lo += ln
    split(0, h, ibf.K_FUSED_H)
    split(h, L, ibf.K_FUSED_G)
    per_launch = {}
    for idx, (kind, t_ms) in enumerate(prof):
        lo, hi, kd = sched[idx % len(sched)]
        per_launch.setdefault((lo, hi, kd), []).append(t_ms)
    tot = {k: sum(v) for k, v in per_launch.items()}
    dom = max(tot, key=tot.get)
    lo, hi, kd = dom
    pro = "V" if lo == 0 else None
    epi = "U" if hi == L else ("switch" if hi == h else None)
    avg_ms = statistics.mean(per_launch[dom])
    flops = structured_flops(hi - lo, r, N, nrhs, pro, epi, kd == ibf.K_FUSED_G)
    esz = 8
    bytes_alg = 0
    bytes_alg += (N * nrhs * esz) if pro == "V" else (N * r * nrhs * esz)          # input
    bytes_alg += (N * nrhs * esz) if epi == "U" else (N * r * nrhs * esz)          # output
    bytes_alg += (hi - lo) * 2 * N * r * esz                                       # phase tables
    if epi == "switch":
        bytes_alg += N * r * r * esz
    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12      # TFLOP/s at max clock
    ach_tf = flops / (avg_ms / 1e3) / 1e12
    ach_gb = bytes_alg / (avg_ms / 1e3) / 1e9
    frac_alu = ach_tf / fp32_peak
    frac_hbm = ach_gb / float(pk["hbm_gbs"])
    kname = "k_fused<float,%d,fwd,%s,tile %d> levels %d..%d" % (r, "H" if kd == ibf.K_FUSED_H else "G", rtile,
                                                                 lo + 1, hi)
    if frac_alu >= frac_hbm:
        roof = {"bound": "alu", "achieved": ach_tf, "peak": fp32_peak, "unit": "TFLOP/s", "frac": frac_alu,
                "traffic": None}
    else:
        roof = {"bound": "hbm", "achieved": ach_gb, "peak": float(pk["hbm_gbs"]), "unit": "GB/s",
                "frac": frac_hbm, "traffic": None}
    traffic = None
    if (N, r, nrhs, kfuse, rtile) == (1 << 20, 9, 64, 4, 32) and kernel_src_sha() == KERNEL_SRC_SHA:
        traffic = TRAFFIC_N20_R9_NRHS64_K4.get((lo, hi, "H" if kd == ibf.K_FUSED_H else "G"))
    roof["traffic"] = traffic
    roof.update({"kernel": kname, "avg_launch_ms": avg_ms, "launches_timed": len(per_launch[dom]),
                 "launch_ms": {"%s %d..%d" % ("H" if kk == ibf.K_FUSED_H else "G", a0 + 1, b0):
                               round(statistics.mean(v), 4) for (a0, b0, kk), v in per_launch.items()},
                 "peak_source": ("FP32 lanes x SMs x 2 x max SM clock (%s clock)" % pk_kind) if roof["bound"] == "alu"
                 else "%s hbm_gbs" % pk_kind,
                 "alu_frac": frac_alu, "hbm_frac": frac_hbm, "alg_flops": flops, "alg_bytes": bytes_alg})

    # ---- end to end through the public API with host buffers
    gh = torch.from_numpy(g_host).pin_memory()
    uh = torch.empty_like(gh).pin_memory()

    def e2e_step():
        # ibf_apply_host: chunked copies in and out overlap the apply; the
        # inputs are host-written, so a step's copy-in may overlap the
        # previous step's last apply (IBF_HOST_PIPELINE), and a step's last
        # copy-out runs under the next step's applies (IBF_HOST_DEFER; the
        # flush after the last step orders the stream after every copy-out)
        plan.apply_host(gh, uh, stream=stream, pipeline=True, defer=True)

    for _ in range(max(1, a.warmup)):
        e2e_step()
    plan.host_flush(stream)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for _ in range(a.steps):
        e2e_step()
    plan.host_flush(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dist if world > 1 else None, dev)
    e2e = {"value": job_throughput(nrhs, a.steps, world, e2e_ms), "unit": "vectors/s",
           "h2d_bytes_per_step": int(gh.numel() * 8), "d2h_bytes_per_step": int(uh.numel() * 8),
           "api": "ibf_apply_host (page-locked host buffers, copies overlapped with the apply, IBF_HOST_PIPELINE | "
                  "IBF_HOST_DEFER, ibf_host_flush after the last step)"}

    # ---- plain FP64 explicit single-vector form on the same GPU, and accuracy
    fp64 = None
    if not a.skip_fp64 and rank == 0:
        t_c0 = time.perf_counter()
        p64 = ibf.Plan(ibf.PHASE_FIO1D, N, r, ibf.C128, max_nrhs=1)
        t_expl = (time.perf_counter() - t_c0) * 1e3
        g64 = g[0:1].to(torch.complex128).contiguous()
        u64 = torch.empty_like(g64)
        for _ in range(2):
            p64.apply_raw(g64.data_ptr(), u64.data_ptr(), 1, stream.cuda_stream)
        torch.cuda.synchronize()
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            p64.apply_raw(g64.data_ptr(), u64.data_ptr(), 1, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / reps
        ucmp = u[0:4].to(torch.complex128)
        g4 = g[0:4].to(torch.complex128).contiguous()
        u4 = torch.empty_like(g4)
        for c in range(4):
            p64.apply_raw(g4[c].data_ptr(), u4[c].data_ptr(), 1, stream.cuda_stream)
        plan.apply_raw(g.data_ptr(), u.data_ptr(), nrhs, stream.cuda_stream)
        torch.cuda.synchronize()
        ucmp = u[0:4].to(torch.complex128)
        err = float(torch.linalg.vector_norm(ucmp - u4) / torch.linalg.vector_norm(u4))
        fp64 = {"value": 1e3 / t64, "unit": "vectors/s", "ms_per_vector": t64, "form": "explicit FP64, nrhs=1",
                "rel_err_fp32_vs_fp64": err, "speedup": value / world / (1e3 / t64)}
        p64.close()
        del g64, u64, g4, u4

    # ---- batched uneven workload (rank 0)
    batch = None
    if rank == 0 and not a.skip_batch:
        batch = run_batch(ibf, torch)

    # ---- construction: plan build time and the number of phase evaluations
    # of the explicit factors, (3 r L + r^2 + 2 r) N, FP64 on the GPU
    L = int(round(np.log2(N)))
    n_phase = (3 * r * L + r * r + 2 * r) * N
    construction = {"structured_fp32_plan_ms": t_struct,
                    "phase_evaluations": n_phase,
                    "phase_evaluations_per_s_structured": n_phase / (t_struct / 1e3),
                    "note": "wall clock of plan creation (host set-up, FP64 phase kernels, uploads), one run"}
    if fp64 is not None:
        construction["explicit_fp64_plan_ms"] = t_expl

    grad5 = None
    if rank == 0 and not a.skip_batch:
        grad5 = run_autograd(ibf, torch)
    amplitude = None
    if rank == 0 and not a.skip_batch:
        amplitude = run_amplitude(ibf, torch)
    optimal = nufft = None
    if rank == 0 and not a.skip_fp64:
        optimal = run_optimal(ibf, torch)
        nufft = run_nufft_latency(ibf, torch)

    fio2d = None
    if rank == 0 and not a.skip_2d:
        fio2d = run_2d(ibf, torch)

    series = None
    if rank == 0 and not a.skip_2d:
        series = run_series(ibf, torch)

    tensorcore = None
    if rank == 0 and not a.skip_tc:
        tensorcore = run_tensorcore(ibf, torch, N=N, nrhs=nrhs)

    sweep = None
    if rank == 0 and not a.skip_sweep:
        sweep = run_config2_sweep(ibf, torch, fp32_peak, float(pk["hbm_gbs"]))

    # ---- CPU oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not a.skip_cpu:
        cores = os.cpu_count() or 1
        v, dt = oracle_vectors_per_s(a, cores)
        cpu = {"value": v, "unit": "vectors/s", "cores": cores, "kind": "oracle",
               "sample": "1 of the %d vectors (full N=2^%d, matrix-free FP64 oracle, %.1f s)" % (
                   nrhs, int(np.log2(N)), dt)}
        # one core, on a 2^16 vector (the full size would take minutes)
        small = argparse.Namespace(**{**vars(a), "N": 1 << 16})
        v1, dt1 = oracle_vectors_per_s(small, 1)
        cpu["single_core"] = {"vectors_per_s_at_N_2e16": v1, "seconds": dt1, "cores": 1}
        oracle_vectors_per_s(small, cores)   # leave the thread count at all cores

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "vectors/s", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name(a), "N": N, "r": r, "nrhs_per_gpu": nrhs, "phase": "FIO1D",
                           "form": "structured, %d fused launches/apply" % launches,
                           "autotuned_shape": tuned,
                           "l2": "inputs and workspace larger than L2 (no flush)",
                           "parallelism": "independent rhs batches per GPU (dp%d)" % world},
                "clocks": clk, "e2e": e2e, "gpu_launches": a.steps * launches, "roofline": roof,
                "fp64_plain": fp64, "construction": construction, "batch256": batch, "autograd": grad5, "optimal_ibf": optimal, "nufft1024_latency": nufft,
                "amplitude": amplitude, "tensorcore": tensorcore, "config2_sweep": sweep,
                "fio2d": fio2d, "series_phases": series, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ibf", choices=["ibf", "reference"])
    ap.add_argument("--N", type=int, default=1 << 20)
    ap.add_argument("--r", type=int, default=9)
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-2d", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--levels-per-launch", type=int, default=0, help="force the fused depth (skips autotuning)")
    ap.add_argument("--rhs-tile", type=int, default=0, help="force the rhs tile (skips autotuning)")
    ap.add_argument("--only-2d", type=int, default=0, metavar="n",
                    help="profiling aid: time only the 2D apply on the n x n grid and print its record")
    ap.add_argument("--only-batch", action="store_true",
                    help="profiling aid: time only the 256-transform batch and print its record")
    ap.add_argument("--only-optimal", type=int, default=0, metavar="N",
                    help="profiling aid: time only the FP32 optimal IBF with sweep-in (r = 12 -> 9) at size N")
    ap.add_argument("--only-amplitude", type=int, default=0, metavar="N",
                    help="profiling aid: time only the amplitude apply (q = 3, 16 columns) at size N")
    ap.add_argument("--only-tc", type=int, default=0, metavar="N",
                    help="profiling aid: one warm-up and one timed apply of an FP32 and a TF32X3 plan at size N "
                         "(--nrhs columns, --levels-per-launch levels, default 4)")
    ap.add_argument("--skip-tc", action="store_true")
    ap.add_argument("--only-series", action="store_true",
                    help="profiling aid: construction and apply of the series-coefficient phases only")
    ap.add_argument("--skip-sweep", action="store_true")
    ap.add_argument("--only-sweep", action="store_true", help="profiling aid: run only the config-2 grid")
    a = ap.parse_args()
    if a.warmup < 3 and a.impl == "ibf":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if a.impl == "reference":
        return run_reference(a)
    if a.only_2d or a.only_batch or a.only_optimal or a.only_amplitude or a.only_tc or a.only_sweep or a.only_series:
        import torch
        import paper_1605_03616_gb300 as ibf
        if a.only_2d:
            name, rec = "fio2d", run_2d(ibf, torch, n=a.only_2d)
        elif a.only_series:
            name, rec = "series_phases", run_series(ibf, torch)
        elif a.only_batch:
            name, rec = "batch256", run_batch(ibf, torch)
        elif a.only_optimal:
            name, rec = "optimal_ibf", run_optimal(ibf, torch, N=a.only_optimal,
                                                   variants=[(12, ibf.FORM_OPTIMAL_IN, 9, ibf.C64_FP32)])
        elif a.only_sweep:
            pk, _ = peaks()
            nsm = torch.cuda.get_device_properties(0).multi_processor_count
            fp32_peak = nsm * FP32_LANES_PER_SM * 2 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
            name, rec = "config2_sweep", run_config2_sweep(ibf, torch, fp32_peak, float(pk["hbm_gbs"]))
        elif a.only_tc:
            name, rec = "tensorcore", run_tensorcore(ibf, torch, N=a.only_tc, nrhs=a.nrhs,
                                                     k=a.levels_per_launch or 4, reps=1, profile=False)
        else:
            name, rec = "amplitude", run_amplitude(ibf, torch, N=a.only_amplitude)
        print(json.dumps({"profile_only": name, **rec}), flush=True)
        return 0
    return run_gpu(a)


if __name__ == "__main__":
    sys.exit(main())
