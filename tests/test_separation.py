"""The oracle and the CUDA path share no code, and the product path cannot
reach the oracle: checked on the sources (imports and includes) and on the
built library (its dynamic dependencies and exported symbols)."""
import ast
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1412_6238_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _py_imports(path):
    tree = ast.parse(open(path, encoding="utf-8").read(), path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            out.add(node.module.split(".")[0])
    return out


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_never_imports_the_oracle():
    for f in _files(PKG, (".py",)):
        assert "oracle" not in _py_imports(f), f


def test_cuda_sources_include_nothing_of_the_oracle():
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', re.M)
    for f in _files(PKG, (".cu", ".cuh", ".h")):
        for name in inc.findall(open(f, encoding="utf-8").read()):
            assert "oracle" not in name, (f, name)


def test_oracle_includes_nothing_of_the_cuda_path():
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', re.M)
    ours = {os.path.basename(f) for f in _files(PKG, (".cu", ".cuh", ".h"))} | {"lbe.h"}
    for f in _files(ORACLE, (".c", ".h")):
        for name in inc.findall(open(f, encoding="utf-8").read()):
            assert os.path.basename(name) not in ours, (f, name)
    for f in _files(ORACLE, (".py",)):
        assert "paper_1412_6238_gb300" not in _py_imports(f), f


def test_library_does_not_link_the_oracle():
    """liblbe.so (built here from source) needs no oracle library and
    exports none of the oracle's entry points."""
    from paper_1412_6238_gb300 import build as _b
    lib = _b.build()
    try:
        dyn = subprocess.run(["readelf", "-d", lib], capture_output=True, text=True, check=True)
        syms = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                              check=True)
    except (OSError, subprocess.CalledProcessError) as e:
        pytest.skip("binutils not available: %s" % e)
    assert "oracle" not in dyn.stdout
    exported = {ln.split()[-1] for ln in syms.stdout.splitlines() if ln.strip()}
    assert not any(s.startswith("orc_") for s in exported)
    oracle_src = open(os.path.join(ORACLE, "lbe_oracle.c"), encoding="utf-8").read()
    oracle_api = set(re.findall(r"^\w[\w\s\*]*?\b(orc_\w+)\s*\(", oracle_src, re.M))
    assert oracle_api and not (oracle_api & exported)
