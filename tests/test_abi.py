"""The C ABI library loads and exports every entry point include/mpt.h declares (CPU only,
no compute calls)."""
import os
import re

import pytest

from paper_2604_22228_gb300 import _ffi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^MPT_API\s+[\w\s\*]*?\b(mpt_\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _ffi.load()


def test_header_declares_functions():
    names = declared_functions()
    assert len(names) >= 19 and len(set(names)) == len(names)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) == set(_ffi.SIGNATURES)


def test_only_abi_symbols_are_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _ffi.LIB_PATH], capture_output=True, text=True).stdout
    text_syms = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert text_syms and all(s.startswith("mpt_") for s in text_syms), text_syms


def test_version_and_error_string(lib):
    assert lib.mpt_version().decode().startswith("mpt ")
    assert isinstance(lib.mpt_last_error(), bytes)
