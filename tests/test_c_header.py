"""The boundary is a C ABI: include/ibf.h must compile as plain C99 (no C++
or torch types), a C program must link against the library and get its
argument checks without a GPU, and (on a GPU) a C program with no PyTorch in
it must create a plan, apply it to host buffers and match the oracle."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "ibf.h"

int main(void)
{
    char msg[256];
    ibf_plan* plan = (ibf_plan*)0;
    ibf_options o;
    memset(&o, 0, sizeof(o));
    o.form = IBF_FORM_OPTIMAL_IN;
    o.rank = 0;                                   /* invalid: rank below 1 */
    int rc1 = ibf_plan_create_ex(IBF_PHASE_FIO1D, 1, 1024, 9, IBF_C128, NULL, &o, &plan);
    int rc2 = ibf_apply(NULL, NULL, NULL, 1, NULL);
    int rc3 = ibf_apply_amplitude(NULL, NULL, NULL, 1, NULL, NULL, 1, 0, NULL, 0, NULL);
    int rc4 = ibf_plan_destroy(NULL);
    int last = ibf_get_last_error(msg, sizeof(msg));
    printf("%d %d %d %d %d %s\n", rc1, rc2, rc3, rc4, last, plan == NULL ? "null" : "set");
    return 0;
}
"""


def test_header_is_c99_and_links(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1605_03616_gb300 import build as B
    B.build()
    src = tmp_path / "use_ibf.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_ibf"
    libdir = os.path.dirname(B.LIB)
    name = os.path.basename(B.LIB)[3:-3]          # libX.so -> X
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L", libdir, "-l" + name, "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    rc1, rc2, rc3, rc4, last, plan = out.stdout.split()
    assert (rc1, rc2, rc3, rc4, last, plan) == ("1", "1", "1", "0", "1", "null")


APPLY_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime_api.h>
#include "ibf.h"

/* usage: apply_ibf dtype N nrhs in.bin out.bin  (column-major complex values) */
int main(int argc, char** argv)
{
    if (argc != 6) return 2;
    const int dtype = atoi(argv[1]);
    const long long N = atoll(argv[2]);
    const int nrhs = atoi(argv[3]);
    const size_t esz = dtype == IBF_C128 ? 16 : 8;
    const size_t bytes = esz * (size_t)N * (size_t)nrhs;
    void* g = malloc(bytes);
    void* u = malloc(bytes);
    FILE* f = fopen(argv[4], "rb");
    if (!g || !u || !f || fread(g, 1, bytes, f) != bytes) return 3;
    fclose(f);
    ibf_plan* plan = NULL;
    char msg[256];
    int rc = ibf_plan_create(IBF_PHASE_FIO1D, 1, (int64_t)N, 9, dtype, &plan);
    if (rc != IBF_OK) {
        ibf_get_last_error(msg, sizeof(msg));
        printf("create %d %s\n", rc, msg);
        return 4;
    }
    rc = ibf_apply_host(plan, g, u, nrhs, 0, NULL);
    cudaError_t e = cudaDeviceSynchronize();
    int st = ibf_plan_status(plan);
    ibf_plan_destroy(plan);
    f = fopen(argv[5], "wb");
    if (!f || fwrite(u, 1, bytes, f) != bytes) return 5;
    fclose(f);
    printf("%d %d %d\n", rc, (int)e, st);
    free(g);
    free(u);
    return 0;
}
"""


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [0, 1])      # IBF_C128 (explicit form), IBF_C64_FP32 (structured form)
def test_c_program_applies_on_gpu(tmp_path, dtype):
    import numpy as np
    import oracle as O
    import workloads as W
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1605_03616_gb300 import build as B
    B.build()
    cuda_home = os.path.dirname(os.path.dirname(B.nvcc()))
    src = tmp_path / "apply_ibf.c"
    src.write_text(APPLY_PROGRAM)
    exe = tmp_path / "apply_ibf"
    libdir = os.path.dirname(B.LIB)
    name = os.path.basename(B.LIB)[3:-3]
    cudalib = next((d for d in (os.path.join(cuda_home, "lib64"), os.path.join(cuda_home, "lib"))
                    if os.path.exists(os.path.join(d, "libcudart.so"))), None)
    if cudalib is None:
        pytest.skip("no libcudart.so in the CUDA toolkit")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda_home, "include"), str(src), "-o", str(exe), "-L", libdir, "-l" + name,
           "-L", cudalib, "-lcudart", "-Wl,-rpath," + libdir, "-Wl,-rpath," + cudalib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    N, nrhs = 1024, 3
    g = W.complex_normal((nrhs, N), W.rng(31))            # rows = columns of g
    cdt = np.complex128 if dtype == 0 else np.complex64
    (tmp_path / "in.bin").write_bytes(g.astype(cdt).tobytes())
    out = subprocess.run([str(exe), str(dtype), str(N), str(nrhs), str(tmp_path / "in.bin"),
                          str(tmp_path / "out.bin")], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, (out.stdout, out.stderr)
    assert out.stdout.split() == ["0", "0", "0"], out.stdout
    u = np.frombuffer((tmp_path / "out.bin").read_bytes(), dtype=cdt).reshape(nrhs, N)
    ref = O.ibf_apply_1d(O.PHASE_FIO1D, N, 9, W.uniform_x(N), g.T.astype(cdt).astype(np.complex128))
    err = O.rel_l2(u.T.astype(np.complex128), ref)
    assert err < (1e-12 if dtype == 0 else 1e-5), err
