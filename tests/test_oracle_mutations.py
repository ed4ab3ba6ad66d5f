"""The oracle's pins must fail when a plausible mistake is planted in the oracle.

Each case copies dwf_oracle.c to a temporary directory, applies one source edit (a
flipped sign, a dropped dagger, a wrong link site, a transposed operand, ...),
compiles the copy with gcc and runs the pins that should notice, with the mutated
library swapped in.  At least one of them must fail; the committed oracle is
never modified.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "dwf_oracle.c")

# (name, old text, new text, pins that must catch it)
MUTATIONS = [
    ("forward projector sign", "one_pm_gamma(mu, -1, Sm);\n        one_pm_gamma(mu, +1, Sp);\n        long xf",
     "one_pm_gamma(mu, +1, Sm);\n        one_pm_gamma(mu, +1, Sp);\n        long xf",
     [lambda: pins.test_free_field_momentum_closed_form((4, 6, 2, 8))]),
    ("backward link not daggered", "link_at(U, xb, mu), 1, cspinor_at", "link_at(U, xb, mu), 0, cspinor_at",
     [lambda: pins.test_gamma5_hermiticity_of_dw((2, 4, 6, 4)),
      lambda: pins.test_gauge_covariance((2, 4, 6, 4))]),
    ("backward link at x instead of x-mu", "link_at(U, xb, mu), 1, cspinor_at", "link_at(U, x, mu), 1, cspinor_at",
     [lambda: pins.test_gauge_covariance((2, 4, 6, 4))]),
    ("backward hop 1/2 dropped", "add_block(acc, -0.5, Sp,", "add_block(acc, -1.0, Sp,",
     [lambda: pins.test_free_field_momentum_closed_form((4, 6, 2, 8))]),
    ("mass term dropped", "acc[i] = (DIM - m0) * p[i];", "acc[i] = DIM * p[i];",
     [lambda: pins.test_free_field_momentum_closed_form((4, 6, 2, 8))]),
    ("corner of L+ sign", "else Lp[(s - 1) * Ns + (Ns - 1)] += -mq / (2.0 * m0);",
     "else Lp[(s - 1) * Ns + (Ns - 1)] += mq / (2.0 * m0);",
     [lambda: pins.test_m5_shamir_closed_form(4, 0.05), pins.test_lmat_is_eq4,
      lambda: pins.test_m5_borici_spectrum(4, 0.4)]),
    ("chiralities swapped", "spin < 2 ? Mp : Mm", "spin < 2 ? Mm : Mp",
     [lambda: pins.test_dfull_matches_dense_assembly((2, 2, 2, 4), 3, "cosine")]),
    ("c applied on the column side", "A[i * Ns + j] = (i == j ? 1.0 : 0.0) + c_i * L[i * Ns + j];",
     "A[i * Ns + j] = (i == j ? 1.0 : 0.0) + sigma[j] / omega[j] * L[i * Ns + j];",
     [lambda: pins.test_m5_two_forms_of_eq8("mixed")]),
    ("omega^{-1/2} on one side only", "B[i * Ns + j] / sqrt(omega[i] * omega[j])", "B[i * Ns + j] / omega[i]",
     [lambda: pins.test_m5_two_forms_of_eq8("cosine")]),
    ("sigma replaced by omega in Eq. 1", "sigma[s] * DLpsi[o + c]", "omega[s] * DLpsi[o + c]",
     [lambda: pins.test_dfull_matches_dense_assembly((2, 2, 2, 2), 4, "shamir")]),
    ("M5 not transposed in C^dagger", "if (or_apply_s(dims, Ns, M5p, M5m, 1, p, v, a)) goto done;",
     "if (or_apply_s(dims, Ns, M5p, M5m, 0, p, v, a)) goto done;",
     [lambda: pins.test_cdag_is_adjoint_and_gamma5_identity(1)]),
    ("S2 uses omega instead of sqrt(omega)", "S2[i * Ns + j] = Yi[i * Ns + j] * sqrt(omega[j]);",
     "S2[i * Ns + j] = Yi[i * Ns + j] * omega[j];",
     [lambda: pins.test_schur_solve_matches_dense_lu((2, 2, 2, 4), 3, "cosine", 1)]),
    ("CG beta inverted", "double beta = rr_new / rr;", "double beta = rr / rr_new;",
     [lambda: pins.test_cg_iterates_are_the_krylov_galerkin_solutions(7)]),
    ("CG x stepped along the next direction",
     "for (size_t i = 0; i < n; ++i) x[i] += alpha * pv[i];\n        for (size_t i = 0; i < n; ++i) pv[i] = r[i] + beta * pv[i];",
     "for (size_t i = 0; i < n; ++i) pv[i] = r[i] + beta * pv[i];\n        for (size_t i = 0; i < n; ++i) x[i] += alpha * pv[i];",
     [lambda: pins.test_cg_iterates_are_the_krylov_galerkin_solutions(7)]),
    ("L+ and L- swapped in D", "spin < 2 ? Mp : Mm", "spin < 2 ? Mm : Mp",
     [lambda: pins.test_free_5d_operator_momentum_block((4, 6, 2, 8), 4)]),
]


@pytest.mark.parametrize("name,old,new,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, monkeypatch, name, old, new, checks):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mutated = src.replace(old, new, 1)
    csrc = tmp_path / "dwf_oracle.c"
    csrc.write_text(mutated)
    (tmp_path / "dwf_oracle.h").write_text(open(SRC.replace(".c", ".h")).read())
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(csrc), "-lm"])
    monkeypatch.setattr(oracle, "_lib", oracle.bind(ctypes.CDLL(str(so))))
    caught = 0
    for check in checks:
        try:
            check()
        except AssertionError:
            caught += 1
    assert caught > 0, f"no pin caught the planted mistake: {name}"
