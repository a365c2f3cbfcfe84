"""Plain FP64 CPU oracle of the interpolative butterfly factorization.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_1605_03616_gb300``) never does.  The oracle shares no code with the
CUDA library.

The arithmetic lives in ``oracle.c`` (complex128, one loop per formula of the
paper); this module compiles it with gcc and wraps it with ctypes/numpy:

* ``direct_1d`` / ``direct_2d`` -- the defining sum u = K g (Sec. 1, eq. DFIO).
* ``ibf_apply_1d`` / ``ibf_adjoint_1d`` -- the butterfly algorithm (Algorithm
  2.1; equals the preliminary IBF of Sec. 3) and its conjugate transpose.
* ``ExplicitIBF`` -- the preliminary IBF with explicit block factors V^0, H^l,
  M^h, G^l, U^L (Sec. 3, eqs. PIBF1-PIBF3, switchlocM, PIBFbf3).
* ``ibf_apply_2d_box`` / ``mibf_apply_2d`` -- the 2D butterfly on one square
  frequency box (Sec. 5.1) and the multiscale sum over a corona
  decomposition with a directly summed centre (Sec. 5.2); with
  ``ibf_adjoint_2d_box`` / ``mibf_adjoint_2d``, their conjugate transposes.
* ``optimal.OptimalIBF`` (numpy, module ``oracle.optimal``) -- the optimal
  IBF's sweep-out compression of the explicit factors (Sec. 4.2) and,
  optionally, its sweep-in stage (Sec. 4.3).
* ``amplitude`` (numpy, module ``oracle.amplitude``) -- a non-unit amplitude
  a(x, xi) given as a separated sum (Sec. 1, eq. FIO): the dense definition
  and the sum of diagonally scaled phase-only applies, with its adjoint.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

PHASE_NUFFT = 0
PHASE_FIO1D = 1
PHASE_FIO2D = 2
PHASE_FIO2D_32 = 3      # the 2D FIO with the constants /32 printed in Sec. 6.3
PHASE_FIO1D_SERIES = 4   # Phi = x xi + c(x)|xi|, c a trigonometric series (set_series)
PHASE_FIO2D_SERIES = 5   # Phi = x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2), c1, c2 2D series (set_series2)
PHASE_SEPARABLE = 100

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (no FMA contraction, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-std=gnu11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declare the argument and result types of the library's functions."""
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    Ci = ctypes.c_int
    lib.orc_phi_1d.restype = ctypes.c_double
    lib.orc_phi_1d.argtypes = [Ci, ctypes.c_double, ctypes.c_double]
    lib.orc_set_series.restype = Ci
    lib.orc_set_series.argtypes = [Ci, P, P]
    lib.orc_set_series2.restype = Ci
    lib.orc_set_series2.argtypes = [Ci, P]
    lib.orc_phi_2d.restype = ctypes.c_double
    lib.orc_phi_2d.argtypes = [Ci] + [ctypes.c_double] * 4
    lib.orc_cheb_grid.argtypes = [Ci, P]
    lib.orc_lagrange.restype = ctypes.c_double
    lib.orc_lagrange.argtypes = [Ci, P, Ci, ctypes.c_double]
    lib.orc_direct_1d.argtypes = [Ci, I64, P, I64, P, P, Ci, P]
    lib.orc_direct_2d.argtypes = [Ci, I64, P, I64, P, P, Ci, P]
    lib.orc_ibf_apply_1d.argtypes = [Ci, I64, Ci, Ci, I64, P, P, Ci, P]
    lib.orc_ibf_adjoint_1d.argtypes = [Ci, I64, Ci, Ci, I64, P, P, Ci, P]
    lib.orc_ibf_build_1d.restype = P
    lib.orc_ibf_build_1d.argtypes = [Ci, I64, Ci, Ci, I64, P]
    lib.orc_ibf_free.argtypes = [P]
    lib.orc_ibf_explicit_apply.argtypes = [P, P, Ci, P]
    lib.orc_ibf_explicit_adjoint.argtypes = [P, P, Ci, P]
    for nm in ("orc_ibf_get_V", "orc_ibf_get_U", "orc_ibf_get_M"):
        getattr(lib, nm).argtypes = [P, P]
    lib.orc_ibf_get_blk.argtypes = [P, Ci, P]
    D = ctypes.c_double
    lib.orc_ibf_apply_2d.argtypes = [Ci, I64, Ci, Ci, I64, P, D, D, P, Ci, P]
    lib.orc_mibf_apply_2d.argtypes = [Ci, I64, Ci, Ci, I64, P, P, Ci, P]
    lib.orc_ibf_adjoint_2d.argtypes = [Ci, I64, Ci, Ci, I64, P, D, D, P, Ci, P]
    lib.orc_mibf_adjoint_2d.argtypes = [Ci, I64, Ci, Ci, I64, P, P, Ci, P]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle's level loops use."""
    lib = _load()
    try:
        f = lib.omp_set_num_threads
    except AttributeError:  # pragma: no cover
        f = ctypes.CDLL("libgomp.so.1").omp_set_num_threads
    f.argtypes = [ctypes.c_int]
    f(int(n))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _cols(g: np.ndarray, n: int) -> tuple[np.ndarray, int, bool]:
    """(n,) or (n, nrhs) -> column-major buffer, nrhs, was_vector"""
    g = np.asarray(g)
    vec = g.ndim == 1
    g2 = g.reshape(n, -1)
    return _c128(g2.T), g2.shape[1], vec


def _uncols(buf: np.ndarray, n: int, nrhs: int, vec: bool) -> np.ndarray:
    out = buf.reshape(nrhs, n).T.copy()
    return out[:, 0] if vec else out


def set_series(a, b) -> None:
    """Coefficients of PHASE_FIO1D_SERIES: c(x) = sum_m a[m] cos(2 pi m x) +
    b[m] sin(2 pi m x), m < len(a) (len(b) == len(a), 1..16 terms)."""
    a = _f64(a)
    b = _f64(b)
    if a.shape != b.shape or not 1 <= a.size <= 16:
        raise ValueError("a and b: the same length, 1..16")
    assert _load().orc_set_series(a.size, _ptr(a), _ptr(b)) == 0


def set_series2(terms) -> None:
    """Coefficients of PHASE_FIO2D_SERIES: rows (p, q, al1, be1, al2, be2),
    1..16 of them; c_d(x) = sum_t al_d cos(2 pi (p x1 + q x2)) +
    be_d sin(2 pi (p x1 + q x2))."""
    t = _f64(terms)
    if t.ndim != 2 or t.shape[1] != 6 or not 1 <= t.shape[0] <= 16:
        raise ValueError("terms: 1..16 rows of 6")
    t = np.ascontiguousarray(t)
    assert _load().orc_set_series2(t.shape[0], _ptr(t)) == 0


def phi_1d(phase_id: int, x: float, xi: float) -> float:
    return _load().orc_phi_1d(phase_id, float(x), float(xi))


def phi_2d(phase_id: int, x1: float, x2: float, k1: float, k2: float) -> float:
    return _load().orc_phi_2d(phase_id, float(x1), float(x2), float(k1), float(k2))


def cheb_grid(r: int) -> np.ndarray:
    z = np.zeros(r)
    _load().orc_cheb_grid(r, _ptr(z))
    return z


def lagrange(r: int, t: int, u: float) -> float:
    z = cheb_grid(r)
    return _load().orc_lagrange(r, _ptr(z), t, float(u))


def omega_1d(N: int) -> np.ndarray:
    """xi_k = k - N/2, k = 0..N-1 (eq. Omega)."""
    return np.arange(N, dtype=np.float64) - N / 2


def direct_1d(phase_id: int, x, xi, g) -> np.ndarray:
    x = _f64(x)
    xi = _f64(xi)
    gb, nrhs, vec = _cols(g, xi.size)
    u = np.zeros(x.size * nrhs, np.complex128)
    _load().orc_direct_1d(phase_id, x.size, _ptr(x), xi.size, _ptr(xi), _ptr(gb), nrhs, _ptr(u))
    return _uncols(u, x.size, nrhs, vec)


def direct_2d(phase_id: int, x, xi, g) -> np.ndarray:
    """x: (nx, 2), xi: (nxi, 2)."""
    x = _f64(x).reshape(-1, 2)
    xi = _f64(xi).reshape(-1, 2)
    gb, nrhs, vec = _cols(g, xi.shape[0])
    u = np.zeros(x.shape[0] * nrhs, np.complex128)
    _load().orc_direct_2d(phase_id, x.shape[0], _ptr(x), xi.shape[0], _ptr(xi), _ptr(gb), nrhs, _ptr(u))
    return _uncols(u, x.shape[0], nrhs, vec)


def default_h(L: int) -> int:
    """Switch level: floor(L/2) (Sec. 3 assumes L even; odd L takes the floor)."""
    return L // 2


def ibf_apply_1d(phase_id: int, N: int, r: int, x, g, h: int | None = None) -> np.ndarray:
    L = int(N).bit_length() - 1
    h = default_h(L) if h is None else h
    x = _f64(x)
    gb, nrhs, vec = _cols(g, N)
    u = np.zeros(x.size * nrhs, np.complex128)
    rc = _load().orc_ibf_apply_1d(phase_id, N, r, h, x.size, _ptr(x), _ptr(gb), nrhs, _ptr(u))
    if rc:
        raise ValueError("orc_ibf_apply_1d failed (%d)" % rc)
    return _uncols(u, x.size, nrhs, vec)


def ibf_adjoint_1d(phase_id: int, N: int, r: int, x, y, h: int | None = None) -> np.ndarray:
    L = int(N).bit_length() - 1
    h = default_h(L) if h is None else h
    x = _f64(x)
    yb, nrhs, vec = _cols(y, x.size)
    g = np.zeros(N * nrhs, np.complex128)
    rc = _load().orc_ibf_adjoint_1d(phase_id, N, r, h, x.size, _ptr(x), _ptr(yb), nrhs, _ptr(g))
    if rc:
        raise ValueError("orc_ibf_adjoint_1d failed (%d)" % rc)
    return _uncols(g, N, nrhs, vec)


def ibf_apply_2d_box(phase_id: int, m: int, r: int, x, q1: float, q2: float, g, h: int | None = None):
    """2D butterfly (Sec. 5.1) for frequencies xi = (q1 + k1, q2 + k2), k < m,
    g of shape (m*m,) or (m*m, nrhs) row-major in (k1, k2); x of shape (nx, 2)."""
    L = int(m).bit_length() - 1
    h = L // 2 if h is None else h
    x = _f64(x).reshape(-1, 2)
    gb, nrhs, vec = _cols(g, m * m)
    u = np.zeros(x.shape[0] * nrhs, np.complex128)
    rc = _load().orc_ibf_apply_2d(phase_id, m, r, h, x.shape[0], _ptr(x), float(q1), float(q2), _ptr(gb), nrhs,
                                  _ptr(u))
    if rc:
        raise ValueError("orc_ibf_apply_2d failed (%d)" % rc)
    return _uncols(u, x.shape[0], nrhs, vec)


def mibf_apply_2d(phase_id: int, n: int, r: int, x, g, center_side: int = 16):
    """Multiscale IBF (Sec. 5.2) on the n x n frequency grid; g (n*n,) or
    (n*n, nrhs) row-major in (k1, k2) with xi = (k1 - n/2, k2 - n/2)."""
    x = _f64(x).reshape(-1, 2)
    gb, nrhs, vec = _cols(g, n * n)
    u = np.zeros(x.shape[0] * nrhs, np.complex128)
    rc = _load().orc_mibf_apply_2d(phase_id, n, r, center_side, x.shape[0], _ptr(x), _ptr(gb), nrhs, _ptr(u))
    if rc:
        raise ValueError("orc_mibf_apply_2d failed (%d)" % rc)
    return _uncols(u, x.shape[0], nrhs, vec)


def ibf_adjoint_2d_box(phase_id: int, m: int, r: int, x, q1: float, q2: float, y, h: int | None = None):
    """Adjoint of ibf_apply_2d_box: g = K_Q^* y, y of shape (nx,) or (nx, nrhs)."""
    L = int(m).bit_length() - 1
    h = L // 2 if h is None else h
    x = _f64(x).reshape(-1, 2)
    yb, nrhs, vec = _cols(y, x.shape[0])
    g = np.zeros(m * m * nrhs, np.complex128)
    rc = _load().orc_ibf_adjoint_2d(phase_id, m, r, h, x.shape[0], _ptr(x), float(q1), float(q2), _ptr(yb), nrhs,
                                    _ptr(g))
    if rc:
        raise ValueError("orc_ibf_adjoint_2d failed (%d)" % rc)
    return _uncols(g, m * m, nrhs, vec)


def mibf_adjoint_2d(phase_id: int, n: int, r: int, x, y, center_side: int = 16):
    """Adjoint of mibf_apply_2d: g = K^* y on the n x n frequency grid."""
    x = _f64(x).reshape(-1, 2)
    yb, nrhs, vec = _cols(y, x.shape[0])
    g = np.zeros(n * n * nrhs, np.complex128)
    rc = _load().orc_mibf_adjoint_2d(phase_id, n, r, center_side, x.shape[0], _ptr(x), _ptr(yb), nrhs, _ptr(g))
    if rc:
        raise ValueError("orc_mibf_adjoint_2d failed (%d)" % rc)
    return _uncols(g, n * n, nrhs, vec)


class ExplicitIBF:
    """Preliminary IBF with explicit factors (Sec. 3), built by the oracle."""

    def __init__(self, phase_id: int, N: int, r: int, x, h: int | None = None):
        self.N, self.r = int(N), int(r)
        self.L = self.N.bit_length() - 1
        self.h = default_h(self.L) if h is None else h
        self.x = _f64(x)
        self._lib = _load()
        self._h = self._lib.orc_ibf_build_1d(phase_id, self.N, self.r, self.h, self.x.size, _ptr(self.x))
        if not self._h:
            raise ValueError("orc_ibf_build_1d failed")

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.orc_ibf_free(self._h)
            self._h = None

    def apply(self, g) -> np.ndarray:
        gb, nrhs, vec = _cols(g, self.N)
        u = np.zeros(self.x.size * nrhs, np.complex128)
        self._lib.orc_ibf_explicit_apply(self._h, _ptr(gb), nrhs, _ptr(u))
        return _uncols(u, self.x.size, nrhs, vec)

    def adjoint(self, y) -> np.ndarray:
        yb, nrhs, vec = _cols(y, self.x.size)
        g = np.zeros(self.N * nrhs, np.complex128)
        self._lib.orc_ibf_explicit_adjoint(self._h, _ptr(yb), nrhs, _ptr(g))
        return _uncols(g, self.N, nrhs, vec)

    # block accessors (for dense assembly in the tests)
    def V(self) -> np.ndarray:
        o = np.zeros((self.N, self.r), np.complex128)
        self._lib.orc_ibf_get_V(self._h, _ptr(o))
        return o

    def U(self) -> np.ndarray:
        o = np.zeros((self.x.size, self.r), np.complex128)
        self._lib.orc_ibf_get_U(self._h, _ptr(o))
        return o

    def M(self) -> np.ndarray:
        o = np.zeros((self.N, self.r, self.r), np.complex128)
        self._lib.orc_ibf_get_M(self._h, _ptr(o))
        return o

    def blocks(self, level: int) -> np.ndarray:
        """(N, 2, r, r): blocks[p, c, t, s] for output pair p = i*2^(L-l)+j."""
        o = np.zeros((self.N, 2, self.r, self.r), np.complex128)
        if self._lib.orc_ibf_get_blk(self._h, level, _ptr(o)):
            raise ValueError("bad level")
        return o


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
