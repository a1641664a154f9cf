"""Host-side checks of the C ABI that need no GPU: the library exports every
entry point declared in include/boris.h, and argument validation fails with
BORIS_ERR_INVALID_ARG before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "boris.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|size_t|const char\*)\s+(boris_\w+)\s*\(", src, re.M)))


def load():
    from paper_2008_02478_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libboris.so not built")
    return binding


def test_header_lists_the_binding_exports():
    from paper_2008_02478_gb300 import binding
    assert declared() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol():
    b = load()
    L = b.lib()
    for name in declared():
        assert hasattr(L, name), name


def test_invalid_arguments_rejected_without_device_work():
    b = load()
    L = b.lib()
    h = ctypes.c_void_p()
    assert L.boris_demag_plan(0, 4, 4, 1e-9, 1e-9, 1e-9, 0, None, ctypes.byref(h)) == -1
    assert b"mesh" in L.boris_last_error()
    assert L.boris_demag_plan(4, 4, 4, -1e-9, 1e-9, 1e-9, 0, None, ctypes.byref(h)) == -1
    assert L.boris_demag_plan(4, 4, 4, 1e-9, 1e-9, 1e-9, 0x80, None, ctypes.byref(h)) == -1
    assert L.boris_demag_plan(4, 4, 4, 1e-9, 1e-9, 1e-9, 0, None, None) == -1
    assert L.boris_demag_plan(5000, 4, 4, 1e-9, 1e-9, 1e-9, 0, None, ctypes.byref(h)) == -4
    assert L.boris_demag_apply(None, None, None) == -1
    assert L.boris_llg_step(None, None, None, None) == -1
    L.boris_plan_destroy(None)
