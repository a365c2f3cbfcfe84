"""CPU checks of the binding's host-buffer validation for ibf_apply_host: the
library copies nrhs * N elements from and to the given addresses and cannot
size the buffers itself, so the binding refuses anything that is not a
contiguous host array of the plan's dtype and shape (nrhs, N)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1605_03616_gb300 import _host_buffers  # noqa: E402

N = 64


def test_accepts_numpy_and_cpu_tensors():
    a = np.zeros((3, N), np.complex64)
    b = np.zeros((3, N), np.complex64)
    ps, pd, nrhs = _host_buffers(a, b, N, False)
    assert (ps, pd, nrhs) == (a.ctypes.data, b.ctypes.data, 3)
    t = torch.zeros((2, N), dtype=torch.complex128)
    u = torch.zeros((2, N), dtype=torch.complex128)
    assert _host_buffers(t, u, N, True) == (t.data_ptr(), u.data_ptr(), 2)
    v = np.zeros(N, np.complex128)
    assert _host_buffers(v, v.copy(), N, True)[2] == 1


@pytest.mark.parametrize("bad", [
    lambda: (np.zeros((3, N), np.complex128), np.zeros((3, N), np.complex64)),      # dtype of src
    lambda: (np.zeros((3, N), np.complex64), np.zeros((4, N), np.complex64)),       # shapes differ
    lambda: (np.zeros((3, N + 1), np.complex64), np.zeros((3, N + 1), np.complex64)),  # wrong N
    lambda: (np.zeros((N, 3), np.complex64).T, np.zeros((3, N), np.complex64)),     # not contiguous
    lambda: (np.zeros((0, N), np.complex64), np.zeros((0, N), np.complex64)),       # no columns
    lambda: (torch.zeros((3, N), dtype=torch.complex64), np.zeros((3, N), np.complex128)),
    lambda: ([0.0] * N, np.zeros(N, np.complex64)),                                 # not an array
])
def test_refuses_mismatched_buffers(bad):
    src, dst = bad()
    with pytest.raises((TypeError, ValueError)):
        _host_buffers(src, dst, N, False)
