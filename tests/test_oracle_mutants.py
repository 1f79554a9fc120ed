"""Plants plausible mistakes in copies of the oracle and checks that the pins catch each.

Each mutant is a textual change to ``oracle/oqr_oracle.c`` (a dropped term, a
wrong sign, a wrong or transposed index), compiled to a temporary library; the
pin suite is then run against it in a subprocess and must fail.  Nothing here
touches the real oracle build.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oqr_oracle.c")

MUTANTS = {
    "chol_diag_sign": ("s -= AT(C, k, j, ldc) * AT(C, k, j, ldc);", "s += AT(C, k, j, ldc) * AT(C, k, j, ldc);"),
    "chol_offdiag_index": ("t -= AT(C, k, i, ldc) * AT(C, k, j, ldc);", "t -= AT(C, k, i, ldc) * AT(C, k, i, ldc);"),
    "sym_reads_upper": ("return i >= j ? AT(A, i, j, lda) : AT(A, j, i, lda);", "return AT(A, i, j, lda);"),
    "symm_dropped_term": ("for (long k = 0; k < m; ++k)\n                s += sym_lower", "for (long k = 1; k < m; ++k)\n                s += sym_lower"),
    "trsm_dropped_term": ("for (long k = 0; k < j; ++k)\n                t -= AT(Q, i, k, ldq)", "for (long k = 0; k + 1 < j; ++k)\n                t -= AT(Q, i, k, ldq)"),
    "trsm_transposed_R": ("t -= AT(Q, i, k, ldq) * AT(R, k, j, ldr);", "t -= AT(Q, i, k, ldq) * AT(R, j, k, ldr);"),
    "householder_reflector": ("const double f = 2.0 * d / s;", "const double f = d / s;"),
    "no_sign_normalisation": ("if (AT(R, j, j, ldr) < 0.0) {", "if (0) {"),
    "cz_dropped_diagonal": ("for (long k = i; k < m; ++k)\n                s += AT(C, i, k, m)", "for (long k = i + 1; k < m; ++k)\n                s += AT(C, i, k, m)"),
    "backsub_transposed_C": ("AT(Q, i, c, ldq) -= AT(C, i, k, m) * qk;", "AT(Q, i, c, ldq) -= AT(C, k, i, m) * qk;"),
    "rprod_dropped_term": ("for (long k = i; k <= j; ++k)", "for (long k = i; k < j; ++k)"),
    "orth_no_identity": ("(r == c ? 1.0L : 0.0L)", "(r == c ? 0.0L : 0.0L)"),
    "repres_dropped_term": ("for (long k = 0; k <= j; ++k)", "for (long k = 0; k < j; ++k)"),
    "householder_missing_reflector": ("for (long k = n - 1; k >= 0; --k) {", "for (long k = n - 1; k >= 1; --k) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique or missing"
    msrc = tmp_path / "mutant.c"
    msrc.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c99",
                    str(msrc), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, OQR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
