"""CPU checks of the boundary: the CUDA library builds, loads without a GPU and
exports every entry point include/asm.h declares (no compute calls here)."""
import ctypes as ct
import os
import re

import pytest

from paper_1912_01379_gb300 import asm, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(asm_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["asm_setup", "asm_workspace_bytes", "asm_sample", "asm_average", "asm_chain_state",
              "asm_status", "asm_destroy", "asm_error_string"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ct.CDLL(build.build())
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(asm.EXPORTS) <= set(_declared())


def test_error_strings_without_gpu():
    L = asm.load()
    for code in range(0, -10, -1):
        assert L.asm_error_string(code)
    assert b"unknown" in L.asm_error_string(-99)
    # argument checks that touch no device memory
    assert L.asm_setup(None, None) == -7
    assert L.asm_workspace_bytes(None, 4, 0) == 0
    assert L.asm_sample(None, 4, 0, 1, 0, 0, 0, None, 0, None) == -7
