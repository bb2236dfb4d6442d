"""CPU-only checks of the boundary: the library loads, exports every entry
point that include/brahms.h declares, and the binding knows each of them.
No compute call is made (there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(brahms_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__  # noqa: F401
    from paper_2609_08384_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_header():
    import paper_2609_08384_gb300 as br
    assert _declared() <= set(br.SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.brahms_status_string.restype = ctypes.c_char_p
    assert lib.brahms_status_string(5) == b"BRAHMS_E_NONFINITE"
    lib.brahms_workspace_size.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_size_t)]
    b = ctypes.c_size_t()
    assert lib.brahms_workspace_size(256, 256, 512, 3, ctypes.byref(b)) == 0
    assert b.value >= 3 * 256 * 256 * 512 * 8
    assert lib.brahms_workspace_size(100, 256, 512, 3, ctypes.byref(b)) == 2  # E_SIZE
    assert lib.brahms_workspace_size(256, 256, 512, 4, ctypes.byref(b)) == 1  # E_ARG
