"""GB300 (sm_103a) interpolative butterfly factorization -- Python binding.

Thin ctypes binding of the C ABI in ``include/ibf.h`` (argument marshalling
only: every step of construction and apply runs in the library's CUDA
kernels).  PyTorch provides device memory and streams.

    plan = Plan(PHASE_FIO1D, N=1 << 16, r=9, dtype=C64_FP32)
    u = plan.apply(g)            # g: complex64 CUDA tensor (N,) or (N, nrhs)
    gy = plan.adjoint(y)         # K^* y
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH

PHASE_NUFFT = 0
PHASE_FIO1D = 1
PHASE_FIO2D = 2
PHASE_FIO1D_SERIES = 4     # Phi = x xi + c(x)|xi|, c(x) a trigonometric series (coef=(a, b))
PHASE_FIO2D_SERIES = 5     # Phi = x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2), c1, c2 2D series (coef=rows of 6)
PHASE_SEPARABLE = 100

C128 = 0
C64_FP32 = 1
C64_BF16X3 = 2
C64_TF32X3 = 3             # tensor-core G-form levels (tcgen05 kind::tf32, two-term splits)

HOST_ADJOINT, HOST_PIPELINE, HOST_DEFER = 1, 2, 4   # ibf_apply_host flags

FORM_AUTO = 0
FORM_EXPLICIT = 1
FORM_STRUCTURED = 2
FORM_OPTIMAL = 3
FORM_OPTIMAL_IN = 4         # sweep-out then sweep-in (Sec. 4.3)

Q_N, Q_L, Q_H, Q_R, Q_DTYPE, Q_FORM, Q_FACTOR_BYTES, Q_WORKSPACE_BYTES, Q_MAX_NRHS, Q_NNZ, Q_LAUNCHES, \
    Q_LEVELS_PER_LAUNCH, Q_RHS_TILE, Q_RANK = range(14)

STATUS = {0: "IBF_OK", 1: "IBF_ERR_INVALID", 2: "IBF_ERR_OOM", 3: "IBF_ERR_CUDA", 4: "IBF_ERR_UNSUPPORTED",
          5: "IBF_ERR_TIMEOUT"}

# every symbol include/ibf.h declares
EXPORTS = ("ibf_plan_create", "ibf_plan_create_ex", "ibf_apply", "ibf_apply_adjoint", "ibf_plan_destroy",
           "ibf_plan_query", "ibf_get_last_error", "ibf_plan_profile_begin", "ibf_plan_profile_end",
           "ibf_apply_static_scratch", "ibf_batch_create", "ibf_batch_apply", "ibf_batch_query",
           "ibf_batch_destroy", "ibf_plan_autotune", "ibf_batch_apply_persistent", "ibf_batch_status",
           "ibf_batch_set_wait_limit", "ibf_batch_test_withhold", "ibf_apply_host", "ibf_apply_amplitude",
           "ibf_plan_status", "ibf_host_flush")

BQ_LAUNCHES, BQ_WORKSPACE_BYTES, BQ_COUNT, BQ_PERSIST_ITEMS = range(4)

K_EXPLICIT_INIT, K_EXPLICIT_LEVEL, K_EXPLICIT_SWITCH, K_EXPLICIT_TERM, K_FUSED_H, K_FUSED_G = range(6)


class IBFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("h", ctypes.c_int), ("max_nrhs", ctypes.c_int),
                ("levels_per_launch", ctypes.c_int), ("rhs_tile", ctypes.c_int), ("rank", ctypes.c_int),
                ("phase_coef", ctypes.c_void_p), ("phase_ncoef", ctypes.c_int)]


_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load_library(path: str | None = None):
    """Load the compiled library; raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("IBF CUDA library not built (%s); run __graft_entry__.build()" % p)
    L = ctypes.CDLL(p)
    P = ctypes.c_void_p
    I = ctypes.c_int
    I64 = ctypes.c_int64
    L.ibf_plan_create.argtypes = [I, I, I64, I, I, ctypes.POINTER(P)]
    L.ibf_plan_create_ex.argtypes = [I, I, I64, I, I, P, ctypes.POINTER(Options), ctypes.POINTER(P)]
    L.ibf_apply.argtypes = [P, P, P, I, P]
    L.ibf_apply_adjoint.argtypes = [P, P, P, I, P]
    L.ibf_plan_destroy.argtypes = [P]
    L.ibf_plan_query.argtypes = [P, I, ctypes.POINTER(I64)]
    L.ibf_get_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    L.ibf_apply_static_scratch.argtypes = [P, P, P, I, P]
    L.ibf_batch_create.argtypes = [P, I, P, P, P, I, ctypes.POINTER(P)]
    L.ibf_batch_apply.argtypes = [P, P]
    L.ibf_batch_query.argtypes = [P, I, ctypes.POINTER(I64)]
    L.ibf_batch_destroy.argtypes = [P]
    L.ibf_plan_autotune.argtypes = [P, I, P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float)]
    L.ibf_batch_apply_persistent.argtypes = [P, P]
    L.ibf_batch_status.argtypes = [P]
    L.ibf_batch_set_wait_limit.argtypes = [P, ctypes.c_longlong]
    L.ibf_batch_test_withhold.argtypes = [P, I, I]
    L.ibf_plan_profile_begin.argtypes = [P, I]
    L.ibf_apply_amplitude.argtypes = [P, P, P, I, P, P, I, I, P, I64, P]
    L.ibf_plan_profile_end.argtypes = [P, P, P, I, ctypes.POINTER(I)]
    L.ibf_plan_status.argtypes = [P]
    L.ibf_host_flush.argtypes = [P, P]
    for nm in EXPORTS:
        getattr(L, nm).restype = I
    if path is None:
        _lib = L
    return L


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    load_library().ibf_get_last_error(buf, 512)
    return buf.value.decode()


def _check(rc: int):
    if rc != 0:
        raise IBFError(rc, last_error())


def _torch():
    import torch
    return torch


def _host_buffers(src, dst, N: int, double: bool):
    """Checks the host buffers of ibf_apply_host, which the library cannot
    size itself: CPU tensors or numpy arrays, C-contiguous, of the plan's
    complex dtype, both of shape (nrhs, N) (or (N,) for one column).
    Returns (src address, dst address, nrhs)."""
    want = "complex128" if double else "complex64"
    shapes = []
    for name, a in (("src", src), ("dst", dst)):
        if hasattr(a, "data_ptr"):
            if a.is_cuda:
                raise TypeError("%s: ibf_apply_host takes host buffers; use apply() for CUDA tensors" % name)
            if str(a.dtype) != "torch." + want or not a.is_contiguous():
                raise TypeError("%s: expected a contiguous torch.%s tensor" % (name, want))
        elif isinstance(a, np.ndarray):
            if a.dtype != np.dtype(want) or not a.flags["C_CONTIGUOUS"]:
                raise TypeError("%s: expected a C-contiguous numpy.%s array" % (name, want))
        else:
            raise TypeError("%s: expected a CPU tensor or a numpy array" % name)
        shapes.append(tuple(a.shape))
    if shapes[0] != shapes[1]:
        raise ValueError("src and dst shapes differ: %s vs %s" % (shapes[0], shapes[1]))
    shp = shapes[0]
    if not ((len(shp) == 2 and shp[1] == N and shp[0] >= 1) or shp == (N,)):
        raise ValueError("expected shape (nrhs, %d) or (%d,), got %s" % (N, N, shp))
    addr = [a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data for a in (src, dst)]
    return addr[0], addr[1], (shp[0] if len(shp) == 2 else 1)


class Plan:
    """An IBF plan (include/ibf.h: ibf_plan_create_ex / ibf_plan_destroy)."""

    def __init__(self, phase: int, N: int, r: int = 9, dtype: int = C64_FP32, x=None, d: int = 1,
                 form: int = FORM_AUTO, h: int = 0, max_nrhs: int = 0, levels_per_launch: int = 0,
                 rhs_tile: int = 0, rank: int = 0, coef=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("the IBF library runs on a CUDA GPU only; none is available")
        torch.cuda.init()
        self._lib = load_library()
        self.N, self.r, self.dtype, self.phase = int(N), int(r), int(dtype), int(phase)
        opt = Options(form, h, max_nrhs, levels_per_launch, rhs_tile, rank)
        if coef is not None and self.phase == PHASE_FIO2D_SERIES:
            # rows (p, q, al1, be1, al2, be2): c_d(x) = sum_t al_d cos(2 pi (p x1 + q x2)) + be_d sin(...)
            self._coef = np.ascontiguousarray(coef, dtype=np.float64)
            if self._coef.ndim != 2 or self._coef.shape[1] != 6:
                raise ValueError("coef: rows of (p, q, al1, be1, al2, be2)")
            opt.phase_coef = self._coef.ctypes.data
            opt.phase_ncoef = self._coef.shape[0]
        elif coef is not None:
            # PHASE_FIO1D_SERIES: coef = (a, b), c(x) = sum_m a[m] cos(2 pi m x) + b[m] sin(2 pi m x)
            a, b = (np.ascontiguousarray(v, dtype=np.float64).ravel() for v in coef)
            if a.shape != b.shape:
                raise ValueError("coef: a and b must have the same length")
            self._coef = np.concatenate([a, b])
            opt.phase_coef = self._coef.ctypes.data
            opt.phase_ncoef = a.size
        xa = None
        if x is not None:
            xa = np.ascontiguousarray(x, dtype=np.float64)
            if xa.size != N * d:
                raise ValueError("x must hold N*d doubles")
        out = ctypes.c_void_p()
        with torch.cuda.device(torch.cuda.current_device()):
            _check(self._lib.ibf_plan_create_ex(self.phase, d, self.N, self.r, self.dtype,
                                                xa.ctypes.data_as(ctypes.c_void_p) if xa is not None else None,
                                                ctypes.byref(opt), ctypes.byref(out)))
        self._p = out
        self.cdtype = torch.complex128 if self.dtype == C128 else torch.complex64

    def close(self):
        if getattr(self, "_p", None):
            self._lib.ibf_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, what: int) -> int:
        v = ctypes.c_int64()
        _check(self._lib.ibf_plan_query(self._p, what, ctypes.byref(v)))
        return v.value

    def status(self) -> int:
        """The plan's sticky status, read and cleared (ibf_plan_status)."""
        return self._lib.ibf_plan_status(self._p)

    @property
    def L(self) -> int:
        return self.query(Q_L)

    @property
    def h(self) -> int:
        return self.query(Q_H)

    def _prep(self, v):
        torch = _torch()
        if not isinstance(v, torch.Tensor) or not v.is_cuda:
            raise TypeError("expected a CUDA tensor")
        if v.dtype != self.cdtype:
            raise TypeError("expected %s, got %s" % (self.cdtype, v.dtype))
        if v.shape[0] != self.N or v.dim() not in (1, 2):
            raise ValueError("expected shape (N,) or (N, nrhs)")
        nrhs = 1 if v.dim() == 1 else v.shape[1]
        # column-major N x nrhs == row-major (nrhs, N)
        colmajor = v.reshape(self.N, nrhs).t().contiguous()
        return colmajor, nrhs

    def _run(self, fn, v, out, stream):
        torch = _torch()
        src, nrhs = self._prep(v)
        dst = torch.empty((nrhs, self.N), dtype=self.cdtype, device=v.device) if out is None else out
        if dst.shape != (nrhs, self.N) or not dst.is_contiguous():
            raise ValueError("out must be a contiguous (nrhs, N) tensor")
        s = (stream or torch.cuda.current_stream(v.device)).cuda_stream
        _check(fn(self._p, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), nrhs,
                  ctypes.c_void_p(s)))
        res = dst.t()
        return res[:, 0] if v.dim() == 1 else res

    def apply(self, g, out=None, stream=None):
        """u = K g (ibf_apply)."""
        return self._run(self._lib.ibf_apply, g, out, stream)

    def adjoint(self, y, out=None, stream=None):
        """g = K^* y (ibf_apply_adjoint)."""
        return self._run(self._lib.ibf_apply_adjoint, y, out, stream)

    def profile_begin(self, cap: int) -> None:
        """Record per-kernel CUDA events for the next `cap` kernels."""
        _check(self._lib.ibf_plan_profile_begin(self._p, cap))

    def profile_end(self, cap: int = 1 << 16):
        """-> list of (kernel kind, milliseconds) recorded since profile_begin."""
        ms = np.zeros(cap, np.float32)
        kind = np.zeros(cap, np.int32)
        n = ctypes.c_int()
        _check(self._lib.ibf_plan_profile_end(self._p, ms.ctypes.data_as(ctypes.c_void_p),
                                              kind.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(n)))
        m = min(n.value, cap)
        return list(zip(kind[:m].tolist(), ms[:m].tolist()))

    def autotune(self, nrhs: int, stream=None):
        """Time every launch shape for `nrhs` columns and keep the fastest
        (ibf_plan_autotune).  Returns (levels_per_launch, rhs_tile, ms)."""
        torch = _torch()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        k, rt, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        _check(self._lib.ibf_plan_autotune(self._p, nrhs, ctypes.c_void_p(s), ctypes.byref(k), ctypes.byref(rt),
                                           ctypes.byref(ms)))
        return k.value, rt.value, ms.value

    def apply_raw(self, g_ptr: int, u_ptr: int, nrhs: int, stream_ptr: int = 0) -> None:
        """Pointer-level ibf_apply for callers that manage their own buffers."""
        _check(self._lib.ibf_apply(self._p, ctypes.c_void_p(g_ptr), ctypes.c_void_p(u_ptr), nrhs,
                                   ctypes.c_void_p(stream_ptr)))

    def adjoint_raw(self, y_ptr: int, g_ptr: int, nrhs: int, stream_ptr: int = 0) -> None:
        _check(self._lib.ibf_apply_adjoint(self._p, ctypes.c_void_p(y_ptr), ctypes.c_void_p(g_ptr), nrhs,
                                           ctypes.c_void_p(stream_ptr)))

    def apply_host(self, src, dst, adjoint: bool = False, stream=None, pipeline: bool = False,
                   defer: bool = False) -> None:
        """ibf_apply_host: `src` and `dst` are CPU tensors (or numpy arrays) of
        shape (nrhs, N), complex64 or complex128 to match the plan; page-locked
        tensors (`pin_memory()`) overlap the copies with the apply.  Queued on
        `stream` (default: the current CUDA stream); synchronise it before
        reading `dst`.  pipeline=True (IBF_HOST_PIPELINE) declares that `src`
        is written only by the host, so the copy-in may overlap the previous
        call's last apply.  defer=True (IBF_HOST_DEFER) leaves the copy-outs
        unordered with `stream` until a later call without it or
        `host_flush`, so the last copy-out overlaps the next call's applies."""
        torch = _torch()
        ps, pd, nrhs = _host_buffers(src, dst, self.N, self.dtype == C128)
        s = (stream or torch.cuda.current_stream()).cuda_stream
        _check(self._lib.ibf_apply_host(self._p, ctypes.c_void_p(ps), ctypes.c_void_p(pd), nrhs,
                                        (HOST_ADJOINT if adjoint else 0) | (HOST_PIPELINE if pipeline else 0) |
                                        (HOST_DEFER if defer else 0), ctypes.c_void_p(s)))

    def host_flush(self, stream=None) -> None:
        """ibf_host_flush: orders `stream` after the copy-outs of earlier
        deferred host applies (their `dst` is complete once `stream` is)."""
        torch = _torch()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        _check(self._lib.ibf_host_flush(self._p, ctypes.c_void_p(s)))

    def apply_amplitude(self, v, alpha, beta, adjoint: bool = False, out=None, work=None, stream=None):
        """u = A g (or g = A^* y with adjoint=True) for the amplitude
        a(x, xi) = sum_t alpha[:, t] beta[:, t] (ibf_apply_amplitude).

        `alpha`, `beta`: CUDA tensors of shape (N, q) and the plan's complex
        dtype (rows: points in the caller's x order, resp. xi_k).  `v`: as in
        `apply`.  `work`: optional 1-D scratch tensor of the plan's dtype; by
        default 2 N q nrhs elements are allocated here (one pass)."""
        torch = _torch()
        src, nrhs = self._prep(v)
        fa = [f.t().contiguous() for f in (alpha, beta)]      # column-major N x q == row-major (q, N)
        q = fa[0].shape[0]
        for f in fa:
            if not f.is_cuda or f.dtype != self.cdtype or f.shape != (q, self.N):
                raise ValueError("alpha and beta must be CUDA tensors of shape (N, q) and the plan's dtype")
        if work is None:
            work = torch.empty(2 * self.N * q * nrhs, dtype=self.cdtype, device=v.device)
        elif not work.is_cuda or work.dtype != self.cdtype or not work.is_contiguous():
            raise ValueError("work must be a contiguous CUDA tensor of the plan's dtype")
        dst = torch.empty((nrhs, self.N), dtype=self.cdtype, device=v.device) if out is None else out
        if dst.shape != (nrhs, self.N) or not dst.is_contiguous():
            raise ValueError("out must be a contiguous (nrhs, N) tensor")
        s = (stream or torch.cuda.current_stream(v.device)).cuda_stream
        _check(self._lib.ibf_apply_amplitude(self._p, ctypes.c_void_p(fa[0].data_ptr()),
                                             ctypes.c_void_p(fa[1].data_ptr()), q, ctypes.c_void_p(src.data_ptr()),
                                             ctypes.c_void_p(dst.data_ptr()), nrhs, 1 if adjoint else 0,
                                             ctypes.c_void_p(work.data_ptr()), work.numel(), ctypes.c_void_p(s)))
        res = dst.t()
        return res[:, 0] if v.dim() == 1 else res


class Batch:
    """Many structured plans applied together (ibf_batch_create/apply).

    `inputs[b]` / `outputs[b]` are CUDA tensors of shape (nrhs_b, N_b) -- the
    column-major N_b x nrhs_b layout of the C ABI -- bound at creation."""

    def __init__(self, plans, inputs, outputs, adjoint: bool = False):
        self._lib = load_library()
        n = len(plans)
        if not (len(inputs) == len(outputs) == n):
            raise ValueError("plans, inputs and outputs must have the same length")
        self.plans, self.inputs, self.outputs = list(plans), list(inputs), list(outputs)
        P = ctypes.c_void_p
        parr = (P * n)(*[p._p for p in plans])
        nr = (ctypes.c_int * n)(*[int(t.shape[0]) for t in inputs])
        iarr = (P * n)(*[t.data_ptr() for t in inputs])
        oarr = (P * n)(*[t.data_ptr() for t in outputs])
        for p, t, o in zip(plans, inputs, outputs):
            if t.shape != o.shape or t.shape[1] != p.N or not (t.is_contiguous() and o.is_contiguous()):
                raise ValueError("each input/output must be a contiguous (nrhs, N) tensor")
        out = P()
        _check(self._lib.ibf_batch_create(parr, n, nr, iarr, oarr, 1 if adjoint else 0, ctypes.byref(out)))
        self._b = out

    def apply(self, stream=None):
        torch = _torch()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        _check(self._lib.ibf_batch_apply(self._b, ctypes.c_void_p(s)))

    def apply_persistent(self, stream=None):
        """The whole batch in one persistent launch (ibf_batch_apply_persistent)."""
        torch = _torch()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        _check(self._lib.ibf_batch_apply_persistent(self._b, ctypes.c_void_p(s)))

    def status(self) -> int:
        """IBF_OK (0) or IBF_ERR_TIMEOUT (5) for the last persistent apply."""
        return self._lib.ibf_batch_status(self._b)

    def query(self, what: int) -> int:
        v = ctypes.c_int64()
        _check(self._lib.ibf_batch_query(self._b, what, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "_b", None):
            self._lib.ibf_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
