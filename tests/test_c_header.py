"""The boundary is a C ABI: include/ibf.h must compile as plain C99 (no C++
or torch types), and a C program must link against the library and get its
argument checks without a GPU."""
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
