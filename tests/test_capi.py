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


def test_plan_flags_and_null_handles_rejected_without_device_work():
    """Tensor-core flags: FP16 and BF16 together, or with FP64, are refused;
    every entry point refuses a NULL plan; multi-mesh and Oersted plans check
    their geometry first."""
    b = load()
    L = b.lib()
    h = ctypes.c_void_p()
    F64, FP16, BF16 = 0x1, 0x2, 0x4
    assert L.boris_demag_plan(32, 32, 20, 1e-9, 1e-9, 1e-9, FP16 | BF16, None, ctypes.byref(h)) == -1
    assert L.boris_demag_plan(32, 32, 20, 1e-9, 1e-9, 1e-9, FP16 | F64, None, ctypes.byref(h)) == -1
    assert b"FP32" in L.boris_last_error()
    images = (ctypes.c_int * 3)(0, 2000, 0)
    assert L.boris_demag_plan_pbc(8, 8, 2, 1e-9, 1e-9, 1e-9, images, 0, None, ctypes.byref(h)) == -1
    assert L.boris_oersted_plan(0, 8, 2, 1e-9, 1e-9, 1e-9, None, ctypes.byref(h)) == -1
    assert L.boris_oersted_plan(8, 5000, 2, 1e-9, 1e-9, 1e-9, None, ctypes.byref(h)) == -4
    nxyz = (ctypes.c_int * 6)(8, 8, 2, 8, 8, 1)
    hxyz = (ctypes.c_double * 6)(1e-9, 1e-9, 1e-9, 2e-9, 1e-9, 1e-9)  # in-plane sizes differ
    org = (ctypes.c_double * 6)(0, 0, 0, 0, 0, 3e-9)
    assert L.boris_multimesh_plan(0, nxyz, hxyz, org, 0, None, ctypes.byref(h)) == -1
    assert L.boris_multimesh_plan(2, nxyz, hxyz, org, F64, None, ctypes.byref(h)) == -1
    assert L.boris_multimesh_plan(2, nxyz, hxyz, org, 0, None, ctypes.byref(h)) == -1
    assert b"in-plane" in L.boris_last_error()
    out4 = (ctypes.c_int * 4)()
    for call in (lambda: L.boris_demag_apply_noalloc(None, None, None),
                 lambda: L.boris_demag_adjoint(None, None, None),
                 lambda: L.boris_oersted_apply(None, None, None),
                 lambda: L.boris_thermal_set_step(None, 5),
                 lambda: L.boris_set_field_terms(None, None),
                 lambda: L.boris_sync_status(None),
                 lambda: L.boris_plan_schedule(None, out4),
                 lambda: L.boris_plan_multimesh_info(None, out4),
                 lambda: L.boris_profile_enable(None, 1)):
        assert call() == -1
    assert L.boris_plan_device_bytes(None) == 0
