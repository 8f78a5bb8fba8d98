"""The oracle and the CUDA library are independent: neither imports, links
or includes the other, and the input generators hold no solver arithmetic
and import neither. Checked on the source text."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1102_2143_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _imports(path):
    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.add(node.module.split(".")[0])
    return out


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_library_python_never_imports_the_oracle():
    for f in _files(LIB, (".py",)):
        assert "oracle" not in _imports(f), f


def test_oracle_never_imports_the_library():
    for f in _files(ORACLE, (".py",)):
        assert "paper_1102_2143_gb300" not in _imports(f), f


def test_native_sources_share_no_headers():
    for f in _files(os.path.join(LIB, "csrc"), (".cu", ".cuh", ".h")):
        for inc in re.findall(r'#include\s+"([^"]+)"', open(f).read()):
            assert "oracle" not in inc, (f, inc)
    for f in _files(ORACLE, (".c", ".h")):
        for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', open(f).read()):
            assert "msc" not in inc and "cuda" not in inc, (f, inc)


def test_inputs_import_neither_side():
    imps = _imports(os.path.join(LIB, "inputs.py"))
    assert "oracle" not in imps and "torch" not in imps
    assert not any(i.startswith("paper_1102_2143_gb300") for i in imps)
