"""CPU-side checks of the C ABI library: it builds, loads, exports every
symbol include/ibf.h declares, and rejects bad arguments before touching the
GPU.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1605_03616_gb300 import build as B
    import paper_1605_03616_gb300 as ibf
    B.build()
    return ibf.load_library()


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*int\s+(ibf_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "ibf_apply" in names and "ibf_plan_create" in names
    for nm in names:
        assert hasattr(lib, nm), nm


def test_python_binding_lists_every_symbol():
    import paper_1605_03616_gb300 as ibf
    assert set(declared_symbols()) <= set(ibf.EXPORTS) | set(getattr(ibf, "EXTRA_EXPORTS", ()))


def _create(lib, phase=1, d=1, N=1024, r=9, dtype=1):
    out = ctypes.c_void_p()
    rc = lib.ibf_plan_create(phase, d, N, r, dtype, ctypes.byref(out))
    return rc, out


def test_argument_validation_without_gpu(lib):
    import paper_1605_03616_gb300 as ibf
    assert lib.ibf_plan_status(None) == 1
    assert _create(lib, N=1000)[0] == 1           # not a power of two
    assert _create(lib, N=2)[0] == 1              # too small
    assert _create(lib, r=2)[0] == 1
    assert _create(lib, r=17)[0] == 1
    assert _create(lib, phase=7)[0] == 1
    assert _create(lib, d=3)[0] == 1
    assert _create(lib, dtype=9)[0] == 1
    assert _create(lib, d=2)[0] == 1              # 1D phase id in 2D
    assert _create(lib, d=2, phase=2, r=11)[0] == 4   # 2D supports r in {5, 7, 9}
    assert _create(lib, d=2, phase=2, N=1000)[0] == 1
    assert _create(lib, d=2, phase=2, N=256)[0] == 1  # n = 16 < 32
    assert _create(lib, r=6)[0] == 4              # structured form: r in {5,7,9,11}
    assert "r" in ibf.last_error()
    assert lib.ibf_plan_create(1, 1, 1024, 9, 1, None) == 1
    # NULL plan and NULL pointers are rejected before any CUDA call
    assert lib.ibf_apply(None, None, None, 1, None) == 1
    assert lib.ibf_apply_adjoint(None, None, None, 1, None) == 1
    assert lib.ibf_apply_host(None, None, None, 1, 0, None) == 1
    assert lib.ibf_host_flush(None, None) == 1                                 # NULL plan, no CUDA call
    assert lib.ibf_apply_amplitude(None, None, None, 1, None, None, 1, 0, None, 0, None) == 1
    assert lib.ibf_plan_destroy(None) == 0
    v = ctypes.c_int64()
    assert lib.ibf_plan_query(None, 0, ctypes.byref(v)) == 1


def test_form_options_validated_without_gpu(lib):
    """Plan options of the optimal forms are checked before any CUDA call."""
    import paper_1605_03616_gb300 as ibf

    def create(form, dtype=ibf.C128, r=9, rank=4, d=1, phase=ibf.PHASE_FIO1D, N=1024):
        o = ibf.Options()
        o.form, o.rank = form, rank
        out = ctypes.c_void_p()
        return lib.ibf_plan_create_ex(phase, d, N, r, dtype, None, ctypes.byref(o), ctypes.byref(out))

    assert create(5) == 1                                            # unknown form
    for form in (ibf.FORM_OPTIMAL, ibf.FORM_OPTIMAL_IN):
        assert create(form, rank=0) == 1                             # rank below 1
        assert create(form, rank=10) == 1                            # rank above r
        assert create(form, r=13, rank=6) == 4                       # r above 12
        assert create(form, dtype=ibf.C64_BF16X3) == 4               # no split-BF16 form
        assert create(form, d=2, phase=ibf.PHASE_FIO2D, N=64 * 64) == 4   # 1D only


def test_tensor_core_dtype_validated_without_gpu(lib):
    """IBF_C64_TF32X3 is the 1D structured form only; the split-BF16 dtype is
    not built.  Both are refused before any CUDA call."""
    import paper_1605_03616_gb300 as ibf

    def create(form, dtype, d=1, phase=ibf.PHASE_FIO1D, N=1024, r=9):
        o = ibf.Options()
        o.form, o.rank = form, 4
        out = ctypes.c_void_p()
        return lib.ibf_plan_create_ex(phase, d, N, r, dtype, None, ctypes.byref(o), ctypes.byref(out))

    assert create(ibf.FORM_EXPLICIT, ibf.C64_TF32X3) == 4
    assert create(ibf.FORM_OPTIMAL, ibf.C64_TF32X3) == 4
    assert create(ibf.FORM_STRUCTURED, ibf.C64_TF32X3, d=2, phase=ibf.PHASE_FIO2D, N=64 * 64, r=7) == 4
    assert create(ibf.FORM_STRUCTURED, ibf.C64_BF16X3) == 4
    assert create(ibf.FORM_STRUCTURED, 4) == 1                       # unknown dtype


def test_series_phase_validated_without_gpu(lib):
    """IBF_PHASE_FIO1D_SERIES needs 1..16 finite coefficients and is 1D only;
    every refusal comes before a CUDA call."""
    import numpy as np
    import paper_1605_03616_gb300 as ibf

    def create(coef, ncoef, d=1, N=1024, r=9):
        o = ibf.Options()
        o.form = ibf.FORM_STRUCTURED
        if coef is not None:
            o.phase_coef = coef.ctypes.data
        o.phase_ncoef = ncoef
        out = ctypes.c_void_p()
        return lib.ibf_plan_create_ex(ibf.PHASE_FIO1D_SERIES, d, N, r, ibf.C64_FP32, None, ctypes.byref(o),
                                      ctypes.byref(out))

    ok = np.array([0.25, 0.0, 0.0, 0.125])
    assert create(None, 2) == 1
    assert create(ok, 0) == 1
    assert create(ok, 17) == 1
    assert create(np.array([0.25, np.nan, 0.0, 0.1]), 2) == 1
    assert create(ok, 2, d=2, N=64 * 64, r=7) == 1          # no 2D form
    out = ctypes.c_void_p()
    assert lib.ibf_plan_create(ibf.PHASE_FIO1D_SERIES, 1, 1024, 9, ibf.C64_FP32, ctypes.byref(out)) == 1


def test_series2_phase_validated_without_gpu(lib):
    """IBF_PHASE_FIO2D_SERIES needs 1..16 finite rows of 6 whose constant
    terms bound each coefficient away from zero, and is 2D only; every
    refusal comes before a CUDA call."""
    import numpy as np
    import paper_1605_03616_gb300 as ibf

    def create(rows, nrows, d=2, N=64 * 64, r=7):
        o = ibf.Options()
        o.form = ibf.FORM_STRUCTURED
        if rows is not None:
            rows = np.ascontiguousarray(rows, dtype=np.float64)
            o.phase_coef = rows.ctypes.data
        o.phase_ncoef = nrows
        out = ctypes.c_void_p()
        return lib.ibf_plan_create_ex(ibf.PHASE_FIO2D_SERIES, d, N, r, ibf.C64_FP32, None, ctypes.byref(o),
                                      ctypes.byref(out))

    ok = [[0, 0, 0.125, 0, 0.125, 0], [1, -1, 1 / 32, 0, 1 / 32, 0], [1, 1, -1 / 32, 0, 1 / 32, 0]]
    assert create(None, 3) == 1
    assert create(ok, 0) == 1
    assert create(ok, 17) == 1
    assert create([[0, 0, 0.125, 0, 0.125, np.inf]], 1) == 1
    assert create([[0, 0, 0.05, 0, 0.125, 0], [1, 0, 0.03, 0.02, 0, 0]], 2) == 1     # c1 may vanish
    assert create([[0, 0, 0.125, 0, 0.05, 0], [0, 1, 0, 0, 0.05, 0]], 2) == 1        # c2 may vanish
    assert create([[0, 0, 0.125, 0, -0.125, 0]], 1) == 1                             # c2 < 0
    assert create(ok, 3, d=1, N=1024, r=9) == 1                                      # no 1D form

