"""The C-ABI library builds, loads without a GPU, and exports every function
include/msc.h declares (no compute calls: this runs on CPU-only machines)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "msc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(msc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1102_2143_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("msc_create", "msc_destroy", "msc_op_staggered", "msc_op_bsr", "msc_solve",
                 "msc_op_apply", "msc_staggered_export_bsr", "msc_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    import paper_1102_2143_gb300 as msc
    assert set(declared_functions()) == set(msc.SIGNATURES)
    lib = msc.load()
    # host-only calls (no device work)
    assert lib.msc_strerror(0).decode() == "ok"
    assert "positive definite" in lib.msc_strerror(4).decode()
    p = msc.msc_params_default()
    assert p.tol == 1e-10 and p.reliable_every == 50 and p.precision == msc.MSC_MIXED


def test_header_compiles_as_c_and_links(lib_path, tmp_path):
    """A plain C99 program includes include/msc.h, links libmsc.so and calls
    the entry points that need no GPU (defaults, error strings) and the
    argument checks that return before any device work."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "msc.h"
int main(void) {
    msc_params p;
    msc_params_default(&p);
    if (p.tol != 1e-10 || p.max_iter != 100000 || p.precision != MSC_MIXED ||
        p.reliable_every != 50 || p.freeze_converged != 1 || p.refine != 4) return 1;
    if (strcmp(msc_strerror(MSC_OK), "ok") != 0) return 2;
    if (strlen(msc_strerror(MSC_ERR_BREAKDOWN)) == 0) return 3;
    if (msc_solve(NULL, NULL, NULL, 1, NULL, 1, &p, NULL, NULL) != MSC_ERR_ARG) return 4;
    if (msc_solve_nonherm(NULL, NULL, NULL, 1, NULL, 1, &p, NULL, NULL) != MSC_ERR_ARG) return 5;
    if (msc_op_destroy(NULL) != MSC_ERR_ARG) return 6;
    puts("abi ok");
    return 0;
}
''')
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib_path)
    cmd = [gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
           "-L", libdir, "-lmsc", "-Wl,-rpath," + libdir, "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and "abi ok" in out.stdout, (out.returncode, out.stderr)
