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
    "no_sign_normalisation": ("if (AT(R, j, j, ldr) < 0.0) {", "if (0) {", 0),
    "cz_dropped_diagonal": ("for (long k = i; k < m; ++k)\n                s += AT(C, i, k, m)", "for (long k = i + 1; k < m; ++k)\n                s += AT(C, i, k, m)"),
    "backsub_transposed_C": ("AT(Q, i, c, ldq) -= AT(C, i, k, m) * qk;", "AT(Q, i, c, ldq) -= AT(C, k, i, m) * qk;"),
    "rprod_dropped_term": ("for (long k = i; k <= j; ++k)", "for (long k = i; k < j; ++k)"),
    "orth_no_identity": ("(r == c ? 1.0L : 0.0L)", "(r == c ? 0.0L : 0.0L)", 0),
    "repres_dropped_term": ("for (long k = 0; k <= j; ++k)", "for (long k = 0; k < j; ++k)"),
    "householder_missing_reflector": ("for (long k = n - 1; k >= 0; --k) {", "for (long k = n - 1; k >= 1; --k) {"),
    # the tridiagonal oracle (third element: which occurrence of a site that the dense oracle shares)
    "tri_chol_pivot": ("p -= cu[i - 1] * cu[i - 1];", "p -= cu[i - 1];"),
    "tri_cz_dropped_superdiagonal": ("((i + 1 < m) ? cu[i] * AT(Z, i + 1, c, ldz) : 0.0)", "0.0"),
    "tri_backsub_sign": ("t -= cu[i] * AT(Q, i + 1, c, ldq);", "t += cu[i] * AT(Q, i + 1, c, ldq);"),
    "tri_no_sign_normalisation": ("if (AT(R, j, j, ldr) < 0.0) {", "if (0) {", 1),
    "tri_orth_dropped_subdiagonal": ("s += (long double)e[i - 1] * (long double)AT(Q, i - 1, c, ldq);", "s += 0.0L;"),
    "tri_orth_no_identity": ("(r == c ? 1.0L : 0.0L)", "(r == c ? 0.0L : 0.0L)", 1),
}
CPU_METHOD = os.path.join(ROOT, "oracle", "cpu_method.c")


def plant(src, old, new, occurrence):
    """src with the occurrence-th (0-based) instance of old replaced by new."""
    at = -1
    for _ in range(occurrence + 1):
        at = src.index(old, at + 1)
    return src[:at] + new + src[at + len(old):]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new, occ = (MUTANTS[name] + (None,))[:3]
    src = open(SRC).read()
    if occ is None:
        assert src.count(old) == 1, f"mutation site for {name} not unique or missing"
        occ = 0
    else:
        assert src.count(old) > occ, f"mutation site for {name} missing"
    msrc = tmp_path / "mutant.c"
    msrc.write_text(plant(src, old, new, occ))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c99",
                    str(msrc), CPU_METHOD, "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, OQR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"


def test_unmutated_build_passes_the_pins(tmp_path):
    """The control: the same build of the unchanged sources passes every pin, so each mutant above fails
    for its planted mistake, not for the way it is built or loaded."""
    lib = tmp_path / "libcontrol.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c99",
                    SRC, CPU_METHOD, "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, OQR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
