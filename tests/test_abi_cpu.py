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


CTX_CALLS = ["brahms_set_fields", "brahms_set_dk_profile", "brahms_propagate", "brahms_get_fields", "brahms_energy",
             "brahms_sync", "brahms_transform", "brahms_set_dk_map", "brahms_diagnostics", "brahms_heat_accumulate",
             "brahms_heat_set", "brahms_thermal_map", "brahms_get_z", "brahms_timing", "brahms_set_option",
             "brahms_adjoint_forward", "brahms_adjoint_backward", "brahms_shg_efficiency_weights",
             "brahms_set_dk_map_z", "brahms_heat_accumulate_segment"]


def test_null_context_is_an_argument_error_without_gpu(lib):
    """Every entry point that takes a context returns BRAHMS_E_ARG for a NULL
    context before any device work (so it is safe without a GPU)."""
    import paper_2609_08384_gb300 as br
    for name in CTX_CALLS:
        restype, argtypes = br.SIGNATURES[name]
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = restype, argtypes
        args = [None]
        for t in argtypes[1:]:
            args.append(0.0 if t is ctypes.c_double else (0 if t in (ctypes.c_int, ctypes.c_longlong) else None))
        assert fn(*args) == 1, name
    fn = lib.brahms_get_option
    fn.restype, fn.argtypes = ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]
    assert fn(None, 1) == -1
    fn = lib.brahms_launch_count
    fn.restype, fn.argtypes = ctypes.c_longlong, [ctypes.c_void_p]
    assert fn(None) == 0


def test_allocation_failure_hook_without_gpu(lib):
    """brahms_fail_next_allocations: the next allocations report E_OOM before
    the CUDA allocator is called (so this runs without a GPU), each failure is
    consumed once, and a negative count is an argument error."""
    import paper_2609_08384_gb300 as br
    for name in ("brahms_fail_next_allocations", "brahms_pending_allocation_failures", "brahms_batch_create",
                 "brahms_batch_set_timeout"):
        restype, argtypes = br.SIGNATURES[name]
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = restype, argtypes
    assert lib.brahms_fail_next_allocations(-1) == 1
    assert lib.brahms_fail_next_allocations(2) == 0
    assert lib.brahms_pending_allocation_failures() == 2
    out = ctypes.c_void_p()
    assert lib.brahms_batch_create(ctypes.byref(out), None) == 4  # its pinned status word
    assert not out.value
    assert lib.brahms_pending_allocation_failures() == 1
    assert lib.brahms_fail_next_allocations(0) == 0
    assert lib.brahms_pending_allocation_failures() == 0
    assert lib.brahms_batch_set_timeout(None, 1.0) == 1
