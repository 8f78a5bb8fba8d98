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
