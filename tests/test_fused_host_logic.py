"""Host logic of the fused structured apply, compiled and run on the CPU
(nvcc, no GPU needed): the level schedule (chunks tile levels 1..L, at most
k levels each, balanced per side, none spanning the switch level h, so H
chunks never reach level L and G chunks never start at level 0 -- the facts
the persistent kernel relies on when it compiles in only the prologues and
epilogues of its level kind), the paired layout of the staged phase tables
(a bijection onto the unit's 4r entries; the two diagonals a level step reads
together side by side at an even offset, so one 16-byte load returns both),
and the fusion-depth choice against the shared-memory budget."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1605_03616_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "ibf_fused.cuh"
using namespace ibf;
static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { ++fails; if (fails < 20) { printf("FAIL: " __VA_ARGS__); printf("\n"); } } } while (0)

template <int RP, int KIND>
static void check_tab()
{
    int seen[4 * RP] = {0};
    for (int ac = 0; ac < 4; ++ac)
        for (int t = 0; t < RP; ++t) {
            const int o = tab_off<RP, KIND>(ac, t);
            CHECK(o >= 0 && o < 4 * RP, "tab_off out of range r=%d kind=%d", RP, KIND);
            if (o >= 0 && o < 4 * RP) seen[o]++;
        }
    for (int o = 0; o < 4 * RP; ++o) CHECK(seen[o] == 1, "tab_off not a bijection r=%d kind=%d", RP, KIND);
    // the two diagonals a level step reads together sit side by side, the first at an even offset
    const int pa[2][2] = {{0, 2}, {1, 3}}, pg[2][2] = {{0, 1}, {2, 3}};
    for (int p = 0; p < 2; ++p)
        for (int t = 0; t < RP; ++t) {
            const int a = KIND == 0 ? pa[p][0] : pg[p][0], b = KIND == 0 ? pa[p][1] : pg[p][1];
            const int oa = tab_off<RP, KIND>(a, t), ob = tab_off<RP, KIND>(b, t);
            CHECK(ob == oa + 1 && oa % 2 == 0, "pair not adjacent r=%d kind=%d", RP, KIND);
            CHECK(oa == p * 2 * RP + 2 * t, "pair %d at index %d not at 2r p + 2t", p, t);
        }
}

int main()
{
    check_tab<5, 0>(); check_tab<5, 1>(); check_tab<7, 0>(); check_tab<7, 1>();
    check_tab<9, 0>(); check_tab<9, 1>(); check_tab<11, 0>(); check_tab<11, 1>();
    int ncase = 0;
    for (int L = 2; L <= 26; ++L)
        for (int h = 1; h <= L - 1; ++h)
            for (int km = 1; km <= kMaxFuse; ++km) {
                std::vector<Chunk> s = fused_schedule(L, h, km);
                int at = 0, smin[2] = {1 << 30, 1 << 30}, smax[2] = {0, 0};
                for (const Chunk& c : s) {
                    ++ncase;
                    const int n = c.hi - c.lo;
                    CHECK(c.lo == at && n >= 1 && n <= km, "chunks do not tile the levels L=%d h=%d k=%d", L, h, km);
                    at = c.hi;
                    // no chunk spans h; H chunks end at or before h < L, G chunks start at h >= 1
                    if (c.kind == 0) CHECK(c.hi <= h && c.lo < h && c.hi < L, "H chunk L=%d h=%d", L, h);
                    else CHECK(c.kind == 1 && c.lo >= h && c.lo >= 1 && c.hi > h, "G chunk L=%d h=%d", L, h);
                    smin[c.kind] = std::min(smin[c.kind], n);
                    smax[c.kind] = std::max(smax[c.kind], n);
                }
                CHECK(at == L, "schedule ends at %d of L=%d", at, L);
                for (int kd = 0; kd < 2; ++kd) CHECK(smax[kd] - smin[kd] <= 1, "unbalanced chunks L=%d h=%d", L, h);
            }
    const int rts[6] = {1, 2, 4, 8, 16, 32}, rps[4] = {5, 7, 9, 11};
    for (int rt : rts)
        for (int rp : rps)
            for (size_t esz : {(size_t)8, (size_t)16}) {
                const int k = fused_kmax(rt, rp, esz);
                CHECK(k >= 1 && k <= kMaxFuse, "kmax range");
                CHECK(k == 1 || fused_smem_bytes(k, rt, rp, esz) <= 100 * 1024, "kmax over budget");
                CHECK(k == kMaxFuse || fused_smem_bytes(k + 1, rt, rp, esz) > 100 * 1024, "kmax not maximal");
                for (int kk = 1; kk <= kMaxFuse; ++kk)
                    // the table region starts 16-byte aligned (pair loads) after the tile
                    CHECK(((((size_t)1 << kk) * ((size_t)rp * rt + 1)) * esz) % 16 == 0, "table region alignment");
            }
    printf("%s %d %d\n", fails ? "FAILED" : "OK", fails, ncase);
    return fails ? 1 : 0;
}
"""


def test_fused_host_logic(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no CUDA toolkit")
    src = tmp_path / "fused_host_logic.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "fused_host_logic"
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a", "--expt-relaxed-constexpr",
           "-I", CSRC, str(src), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout[-2000:]
