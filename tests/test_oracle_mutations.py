"""The oracle's pins must be sensitive: each test here plants one plausible
mistake in a copy of the oracle -- the C source recompiled with gcc, or a
Python module re-executed from its edited source -- runs one of the real pin
tests against the copy, and requires that pin to fail.  Mistakes: a sign of
the phase factor, a phase-shifted 1D FIO coefficient, the sine terms of the
series coefficient dropped, the 2D FIO coefficients exchanged, the 2D
series' frequencies exchanged, its sine terms dropped or c2 used for c1, the Chebyshev
grid, a dropped Lagrange factor, the child
centre or a phase sign of a butterfly level, a transposed switch block, a
wrong box width in U^L, a dropped phase factor in V^0, a skipped corona box
in 2D, a dropped conjugate in an adjoint level, swapped amplitude factors, a missing conjugate in the amplitude
adjoint, a swapped pencil in the sweep-in, a rank one short, and a truncated
SVD split without the square roots."""
import ctypes
import os
import subprocess
import types

import pytest

import oracle as O
import oracle.amplitude as OA
import oracle.optimal as OO
import test_oracle as T
import test_oracle_2d as T2
import test_oracle_amplitude as TA
import test_oracle_optimal as TO

LP = "                    const cplx* lp = prev + (ip * ((int64_t)1 << (L - l + 1)) + C) * r;\n"

# (name, text in oracle.c, replacement, pin that must fail)
C_MUTATIONS = [
    ("phase factor sign", "return cos(a) + I * sin(a);", "return cos(a) - I * sin(a);",
     lambda: T.test_direct_equals_dft_closed_form(16)),
    ("Chebyshev grid", "z[t] = 0.5 * cos(t * M_PI / (r - 1));", "z[t] = 0.5 * cos(t * M_PI / r);",
     lambda: T.test_chebyshev_grid_matches_numpy(5)),
    ("Lagrange factor dropped", "        if (m != t)\n            p *=", "        if (m != t && m != 0)\n            p *=",
     lambda: T.test_lagrange_identities(6)),
    ("H-level child centre", "double cC = wbox_c(N, L - l + 1, C);\n" + LP + "                    for (int s = 0; s < r; ++s) {",
     "double cC = wbox_c(N, L - l + 1, 2 * j + 1 - c);\n" + LP + "                    for (int s = 0; s < r; ++s) {",
     lambda: T.test_separable_phase_is_exact(64, 5, 3)),
    # the separable phase cancels the G-level child centre, so the matrix-free
    # levels are held against the explicit factors built by separate code
    ("G-level child centre", "double cC = wbox_c(N, L - l + 1, C);\n" + LP + "                    cplx inner = 0;",
     "double cC = wbox_c(N, L - l + 1, 2 * j + 1 - c);\n" + LP + "                    cplx inner = 0;",
     lambda: T.test_dense_factor_product_matches_apply(16, 5, O.PHASE_FIO1D)),
    ("H-level phase sign", "next[(i * nj + j) * r + t] = e2pi(-orc_phi_1d(ph, cA, gBt)) * acc;",
     "next[(i * nj + j) * r + t] = e2pi(orc_phi_1d(ph, cA, gBt)) * acc;",
     lambda: T.test_separable_phase_is_exact(64, 5, 3)),
    ("switch block transposed",
     "acc += e2pi(orc_phi_1d(ph, gridpt(cA, wA, z, t), gridpt(cB, wB, z, s))) * old[s];",
     "acc += e2pi(orc_phi_1d(ph, gridpt(cA, wA, z, s), gridpt(cB, wB, z, t))) * old[s];",
     lambda: T.test_separable_phase_is_exact(64, 5, 3)),
    ("U^L box width", "acc += orc_lagrange(r, z, t, (x[n] - cA) / wA) * e2pi(-orc_phi_1d(ph, gridpt(cA, wA, z, t), cB)) *",
     "acc += orc_lagrange(r, z, t, (x[n] - cA) / (2 * wA)) * e2pi(-orc_phi_1d(ph, gridpt(cA, wA, z, t), cB)) *",
     # partition of unity hides an x-interpolation point from the separable
     # phase; the explicit factors (separate code) expose it
     lambda: T.test_dense_factor_product_matches_apply(16, 5, O.PHASE_FIO1D)),
    ("V^0 phase factor dropped",
     "orc_lagrange(r, z, t, (xi - cB) / wB) * e2pi(orc_phi_1d(ph, cA, xi)) * g[k];",
     "orc_lagrange(r, z, t, (xi - cB) / wB) * g[k];",
     lambda: T.test_separable_phase_is_exact(64, 5, 3)),
    ("2D corona ring box skipped", "if (b1 >= 1 && b1 <= 2 && b2 >= 1 && b2 <= 2) continue;   /* inner",
     "if (b1 >= 1 && b1 <= 2 && b2 >= 1 && b2 <= 3) continue;   /* inner",
     lambda: T2.test_separable_2d_box_and_mibf_exact(32, 7)),
    ("1D FIO coefficient phase-shifted (cos for sin)",
     "double c = (2.0 + sin(2.0 * M_PI * x)) / 8.0;", "double c = (2.0 + cos(2.0 * M_PI * x)) / 8.0;",
     T.test_phase_values_match_hand_computed),
    ("series coefficient without its sine terms",
     "c += orc_ca[m] * cos(arg) + orc_cb[m] * sin(arg);", "c += orc_ca[m] * cos(arg);",
     T.test_phase_values_match_hand_computed),
    ("2D FIO coefficients c1 and c2 exchanged",
     "double c1 = (2.0 + sin(2.0 * M_PI * x1) * sin(2.0 * M_PI * x2)) / den;\n"
     "        double c2 = (2.0 + cos(2.0 * M_PI * x1) * cos(2.0 * M_PI * x2)) / den;",
     "double c2 = (2.0 + sin(2.0 * M_PI * x1) * sin(2.0 * M_PI * x2)) / den;\n"
     "        double c1 = (2.0 + cos(2.0 * M_PI * x1) * cos(2.0 * M_PI * x2)) / den;",
     T.test_phase_values_match_hand_computed),
    ("2D series: p and q exchanged",
     "double arg = 2.0 * M_PI * (orc_pq[t][0] * x1 + orc_pq[t][1] * x2);",
     "double arg = 2.0 * M_PI * (orc_pq[t][1] * x1 + orc_pq[t][0] * x2);",
     T.test_phase_values_match_hand_computed),
    ("2D series: sine terms dropped",
     "c += orc_al[d][t] * cos(arg) + orc_be[d][t] * sin(arg);", "c += orc_al[d][t] * cos(arg);",
     T.test_phase_values_match_hand_computed),
    ("2D series: c2 used in place of c1",
     "double a = orc_series2(0, x1, x2) * k1;", "double a = orc_series2(1, x1, x2) * k1;",
     T.test_phase_values_match_hand_computed),
    ("adjoint conjugate dropped", "                                 e2pi(-orc_phi_1d(ph, gPs, cC));\n"
     "                        acc += conj(w) * ln[t];",
     "                                 e2pi(-orc_phi_1d(ph, gPs, cC));\n                        acc += w * ln[t];",
     lambda: T.test_adjoint_dot_product_identity(O.PHASE_FIO1D, 256)),
]


@pytest.mark.parametrize("name,old,new,pin", C_MUTATIONS, ids=[m[0] for m in C_MUTATIONS])
def test_c_oracle_mistake_is_caught(tmp_path, monkeypatch, name, old, new, pin):
    src = open(O._SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / "oracle_mut.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", "-std=gnu11",
                           str(path), "-o", str(lib), "-lm"])
    monkeypatch.setattr(O, "_lib", O._configure(ctypes.CDLL(str(lib))))
    with pytest.raises(AssertionError):
        pin()


def _mutated_module(mod, old, new):
    src = open(mod.__file__).read()
    assert src.count(old) == 1, old
    m = types.ModuleType(mod.__name__ + "_mutated")
    m.__package__ = "oracle"
    m.__file__ = mod.__file__
    exec(compile(src.replace(old, new), mod.__file__, "exec"), m.__dict__)
    return m


# (name, module, text, replacement, names to swap in (module, attribute), pin that must fail)
PY_MUTATIONS = [
    ("amplitude factors swapped", OA, "G = np.concatenate([beta[:, t, None] * g2",
     "G = np.concatenate([alpha[:, t, None] * g2", [(OA, "apply")],
     lambda: TA.test_ibf_route_against_dense(O.PHASE_SEPARABLE)),
    ("amplitude adjoint conjugate dropped", OA, "Y = np.concatenate([np.conj(alpha[:, t, None]) * y2",
     "Y = np.concatenate([alpha[:, t, None] * y2", [(OA, "adjoint")],
     lambda: TA.test_adjoint_identity_and_dense_transpose()),
    ("sweep-in G pencil outputs swapped", OO,
     "Z = np.vstack([C[p0] @ self.blocks[l][p0, c], C[p1] @ self.blocks[l][p1, c]])",
     "Z = np.vstack([C[p1] @ self.blocks[l][p0, c], C[p0] @ self.blocks[l][p1, c]])", [(TO, "OptimalIBF")],
     lambda: TO.test_sweep_in_full_rank_equals_preliminary(O.PHASE_FIO1D, 64, 9, 9, False)),
    ("sweep-in H rank one short", OO, "KH = {l: min(1 << l, r0)", "KH = {l: min(max(1, (1 << l) - 1), r0)",
     [(TO, "OptimalIBF")],
     lambda: TO.test_sweep_in_full_rank_equals_preliminary(O.PHASE_FIO1D, 64, 9, 9, False)),
    ("split without square roots", OO, "A[:, :k] = U[:, :k] * sq", "A[:, :k] = U[:, :k]", [(TO, "split_svd")],
     lambda: TO.test_split_svd_is_the_truncated_svd()),
]


@pytest.mark.parametrize("name,mod,old,new,swaps,pin", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_python_oracle_mistake_is_caught(monkeypatch, name, mod, old, new, swaps, pin):
    m = _mutated_module(mod, old, new)
    for target, attr in swaps:
        monkeypatch.setattr(target, attr, getattr(m, attr))
    with pytest.raises(AssertionError):
        pin()
    # the unmutated oracle passes the same pin
    monkeypatch.undo()
    pin()
