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


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a C program compiled here with gcc."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "hosc.h"', "int main(void) {",
            '  printf("%%zu\\n", sizeof(%s));' % struct]
    prog += ['  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields]
    prog += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-x", "c", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True, timeout=120)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True,
                         timeout=60).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("name", ["hosc_params", "hosc_info", "hosc_diag", "hosc_pool_info"])
def test_binding_structs_match_the_header(name, tmp_path):
    """The ctypes structures of the binding have the header's size and field offsets (the
    header is C; it is compiled here as C, without the CUDA toolkit)."""
    from paper_2411_06563_gb300 import hosc
    cls = getattr(hosc, name)
    fields = [f[0] for f in cls._fields_]
    cnames = ["lambda" if f == "lambda_" else f for f in fields]
    size, offs = _c_layout(name, cnames, tmp_path)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs


def test_box_and_solver_validation_on_the_host(libpath):
    """Box lengths and the solver option are checked without a device; BiCGSTAB(2) adds three
    N^3 vectors per system to the workspace."""
    from paper_2411_06563_gb300 import hosc
    p = hosc.hosc_default_params(21, 1e3, 1.0, 1.0)
    assert p.Ly == 1.0 and p.Lz == 1.0 and p.solver == 0
    base = hosc.hosc_workspace_bytes(p)
    for Ly, Lz, ok in ((0.0, 0.0, True), (0.5, 2.0, True), (-1.0, 1.0, False),
                       (1.0, 65.0, False), (0.01, 1.0, False)):
        p.Ly, p.Lz = Ly, Lz
        assert (hosc.hosc_workspace_bytes(p) > 0) == ok, (Ly, Lz)
    p.Ly = p.Lz = 1.0
    p.solver = 1
    assert hosc.hosc_workspace_bytes(p) >= base + 12 * 21 ** 3 * 8
    p.precision = hosc.HOSC_MIXED
    assert hosc.hosc_workspace_bytes(p) == 0     # BiCGSTAB(2) is built for the FP64 solve
    p.precision = hosc.HOSC_FP64
    p.solver = 2
    assert hosc.hosc_workspace_bytes(p) == 0


def test_c_client_links_and_calls_host_entry_points(libpath, tmp_path):
    """A plain C program includes the header, links the library and calls the entry points that
    need no device (defaults, validation, workspace sizing, error strings): the boundary is usable
    from C without Python or the CUDA toolkit."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "hosc.h"
int main(void) {
  hosc_params p;
  if (hosc_default_params(&p, 21, 1e3, 1.0, 0.75) != HOSC_OK) return 1;
  if (p.N != 21 || p.Ly != 1.0 || p.solver != 0) return 2;
  size_t b = hosc_workspace_bytes(&p);
  if (b == 0) return 3;
  p.solver = 1;
  if (hosc_workspace_bytes(&p) <= b) return 4;     /* BiCGSTAB(2) vectors */
  p.N = 3;
  if (hosc_workspace_bytes(&p) != 0) return 5;      /* invalid: N < 5 */
  if (hosc_default_params(NULL, 21, 1e3, 1.0, 1.0) != HOSC_EINVAL) return 6;
  if (strlen(hosc_strerror(HOSC_ENOCONV)) == 0) return 7;
  printf("ok %zu\n", b);
  return 0;
}
""")
    exe = tmp_path / "client"
    libdir = os.path.dirname(libpath)
    lib = os.path.basename(libpath)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    os.path.join(libdir, lib), "-Wl,-rpath," + libdir], check=True,
                   capture_output=True, timeout=120)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert out.stdout.startswith("ok ")
