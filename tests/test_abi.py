"""The C-ABI library builds, loads and exports every function include/*.h declares.

Runs without a GPU: no compute entry point is called, only the ones that
answer from the host (status strings, defaults, argument checks).
"""
import ctypes
import subprocess

import pytest

from paper_1401_5171_gb300 import oqr


def test_library_exports_every_declared_function():
    lib = oqr.load()
    names = oqr.declared_functions()
    assert {"oqr_cholqr", "oqr_cholqr2", "oqr_cgs2", "oqr_create", "oqr_destroy"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", oqr.LIB_PATH], capture_output=True, text=True, check=True)
    exported = {ln.split()[-1] for ln in out.stdout.splitlines() if " T " in ln}
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in names:
        assert hasattr(lib, n)


def test_status_strings_and_defaults():
    for s in range(8):
        assert oqr.status_string(s).startswith("OQR_")
    o = oqr.make_opts()
    assert (o.passes, o.shifted, o.prec, o.block, o.check) == (2, 0, oqr.OQR_FP64, 64, 0)
    assert o.shift_c == 11.0 and o.spin_limit == 4_000_000_000


def test_host_side_argument_checks():
    lib = oqr.load()
    assert lib.oqr_create(None, 0) == oqr.OQR_ERR_INVALID_ARG
    size = ctypes.c_size_t()
    assert lib.oqr_workspace_size(None, 0, 10, 5, None, ctypes.byref(size)) == oqr.OQR_ERR_INVALID_ARG
    assert lib.oqr_cholqr2(None, 10, 5, None, 10, None, 10, None, 10, None, 5, None, None, None) == \
        oqr.OQR_ERR_INVALID_ARG
    assert lib.oqr_destroy(None) == oqr.OQR_OK


def test_no_cpu_fallback_in_binding():
    # the binding only marshals: every compute name maps to the C library
    src = open(oqr.__file__).read()
    assert "import oracle" not in src and "from oracle" not in src
