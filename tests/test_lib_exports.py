"""The C-ABI library builds, loads and exports every function include/tbgf.h declares.

CPU only: nothing here launches GPU work.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;",
                             text, flags=re.M):
            names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1402_7285_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = set(_declared_functions())
    for required in ("tb_build_bsr", "tb_build_csr", "shifted_cocg_solve", "gf_reduce_ldos_dm",
                     "tb_bsr_spmm", "tb_ctx_create", "tb_ctx_destroy", "tb_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1402_7285_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib.SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.tb_status_string.restype = ctypes.c_char_p
    assert lib.tb_status_string(0) == b"ok"
    assert b"argument" in lib.tb_status_string(-1)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1402_7285_gb300 import _lib
    monkeypatch.setattr(_lib, "_LIB", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()
