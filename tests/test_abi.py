"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/irk_gb300.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "irk_gb300.h")


def declared_symbols():
    src = open(HEADER).read()
    return re.findall(r"IRK_API\s+[\w\s\*]*?\b(irk_\w+)\s*\(", src)


def test_header_declares_the_boundary():
    syms = set(declared_symbols())
    for need in ("irk_setup", "irk_update_values", "irk_factor", "irk_solve", "irk_destroy",
                 "irk_strerror", "irk_apply_operator", "irk_apply_precond"):
        assert need in syms


def test_library_exports_every_declared_symbol():
    import shutil
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1701_07181_gb300 import build, irk
    path = build.build()
    lib = ctypes.CDLL(path)
    for sym in declared_symbols():
        assert hasattr(lib, sym), sym
    assert sorted(declared_symbols()) == sorted(irk.EXPORTS)
    # a call that needs no GPU: the status strings
    lib.irk_strerror.restype = ctypes.c_char_p
    assert lib.irk_strerror(-3).decode().startswith("singular")


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    from paper_1701_07181_gb300 import irk
    monkeypatch.setattr(irk, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(irk, "_lib", None)
    with pytest.raises(RuntimeError):
        irk.load()
