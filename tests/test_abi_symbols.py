"""The C-ABI library loads and exports every entry point include/hosc.h declares (no GPU needed;
no compute calls are made)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hosc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(hosc_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2411_06563_gb300 import build, hosc
    if not os.path.exists(hosc.LIB_PATH):
        build.build()
    return hosc.LIB_PATH


def test_header_declares_the_entry_points():
    names = _declared()
    for core in ("hosc_create", "hosc_step", "hosc_solve_steady", "hosc_diagnostics",
                 "hosc_destroy", "hosc_get_field", "hosc_set_field", "hosc_strerror"):
        assert core in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_names(libpath):
    from paper_2411_06563_gb300 import hosc
    lib = hosc.lib()
    for n in _declared():
        assert hasattr(lib, n)
        assert hasattr(hosc, n), n


def test_host_only_calls_without_gpu(libpath):
    """Parameter helpers need no device: defaults, validation and workspace sizing."""
    from paper_2411_06563_gb300 import hosc
    p = hosc.hosc_default_params(21, 1e3, 1.0, 1.0)
    assert p.N == 21 and p.dt == 0.02 and p.max_lin_iter == 1000
    assert abs(p.lambda_ - 0.25 * (1 / 20) ** 2 / 0.02) < 1e-15
    n3 = 21 ** 3
    assert hosc.hosc_workspace_bytes(p) >= 60 * n3 * 8
    bad = hosc.hosc_default_params(21, 1e3, 1.0, 0.75)
    bad.I2_eps = 0.0
    assert hosc.hosc_workspace_bytes(bad) == 0
    bad = hosc.hosc_default_params(21, 1e3, 1.0, 1.0)
    bad.N = 3
    assert hosc.hosc_workspace_bytes(bad) == 0
    assert hosc.hosc_strerror(hosc.HOSC_ENOCONV).startswith("BiCGSTAB")
