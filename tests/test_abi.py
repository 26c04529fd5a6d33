"""CPU-side checks of the C ABI: the library loads and exports every declared entry point."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "symnmf.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(symnmf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared()
    for must in ["symnmf_create", "symnmf_lai_sketch", "symnmf_hals_sweep", "symnmf_lvs_sample",
                 "symnmf_lvs_update", "symnmf_residual", "symnmf_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g

    g.build()
    import paper_2402_08134_gb300 as S

    lib = S.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (symnmf_[a-z0-9_]+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    # the binding covers the same names
    assert set(declared()) <= set(S.EXPORTED)


def test_import_fails_loudly_without_library(tmp_path):
    # a copy of the package without the .so must refuse to import
    import shutil
    import sys

    pkg = tmp_path / "paper_2402_08134_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_2402_08134_gb300"), pkg,
                    ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__"))
    code = "import paper_2402_08134_gb300"
    r = subprocess.run([sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode != 0 and "not built" in r.stderr
