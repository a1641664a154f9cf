"""The allocation-free demag entry point (boris_demag_apply_noalloc).

Some callers cannot allocate device memory while they run (their allocator is
locked, or allocation is forbidden on their hot path); this entry point keeps
its spectral workspace in a fixed array inside the library instead.  Here it
is called through the C ABI and compared with boris_demag_apply on two calls
in a row (the second call reuses the array the first one left filled), under
each y-z schedule that writes the array differently, on a tensor-core plan
(where it runs the FP32 z stage), and a mesh too large for the array and an
Oersted plan are rejected before any kernel runs.  This file runs last."""
import ctypes

import numpy as np
import pytest

from paper_2008_02478_gb300 import inputs
from tests.gpu_util import max_rel, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _noalloc(L, plan, M, H):
    return L.boris_demag_apply_noalloc(plan._h, ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(H.data_ptr()))


# (BORIS_YZ_KIND or None for the autotuner's choice, BORIS_YZ_TMA for kind 2):
# kind 1 keeps only the x half spectrum in the array; kind 2 (split schedule)
# also the padded y-z spectrum at its offset, with all three split kernels
@pytest.mark.parametrize("kind,tma", [(None, None), (1, None), (2, 0), (2, 3)])
def test_noalloc_matches_apply_on_two_calls(kind, tma, monkeypatch):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import BorisError, Plan, lib
    n, h = (48, 40, 6), (2e-9, 2e-9, 3e-9)
    if kind is not None:
        monkeypatch.setenv("BORIS_YZ_KIND", str(kind))
    if tma is not None:
        monkeypatch.setenv("BORIS_YZ_TMA", str(tma))
    try:
        plan = Plan(*n, *h)
    except BorisError as e:
        assert e.code == -4
        pytest.skip("schedule does not fit this mesh")
    if kind is not None:
        assert plan.schedule()[0] == kind
    L = lib()
    for seed in (11, 12):
        M = to_dev(torch, 7e5 * inputs.random_unit(*n, seed=seed))
        ref = plan.apply(M).cpu().numpy()
        H = torch.empty_like(M)
        rc = _noalloc(L, plan, M, H)
        assert rc == 0, L.boris_last_error()
        torch.cuda.synchronize()
        got = H.cpu().numpy()
        assert rel_l2(got, ref) < 1e-5 and max_rel(got, ref) < 1e-5


def test_noalloc_on_tensor_core_plan_runs_fp32_stage():
    """On an FP16 tensor-core plan (pz = 64) the entry point runs the FP32 z
    stage: its field agrees with an FP32 plan's boris_demag_apply."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan, lib
    n, h = (40, 64, 20), (2e-9, 2e-9, 2e-9)
    tc = Plan(*n, *h, tc="fp16")
    assert tc.padded()[2] == 64
    f32 = Plan(*n, *h)
    L = lib()
    for seed in (21, 22):
        M = to_dev(torch, 8e5 * inputs.random_unit(*n, seed=seed))
        ref = f32.apply(M).cpu().numpy()
        H = torch.empty_like(M)
        rc = _noalloc(L, tc, M, H)
        assert rc == 0, L.boris_last_error()
        torch.cuda.synchronize()
        got = H.cpu().numpy()
        assert rel_l2(got, ref) < 1e-5 and max_rel(got, ref) < 1e-5


def test_noalloc_rejects_meshes_beyond_its_array():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan, lib
    n = (256, 256, 32)  # spectrum 257 * 3 * 32 * 256 * 8 bytes > 32 MiB
    plan = Plan(*n, 4e-9, 4e-9, 4e-9)
    M = torch.zeros((3, n[2], n[1], n[0]), dtype=torch.float32, device="cuda")
    H = torch.empty_like(M)
    L = lib()
    rc = _noalloc(L, plan, M, H)
    assert rc == -4
    assert b"bytes" in L.boris_last_error()


def test_noalloc_rejects_oersted_plans():
    """An Oersted plan's spectrum is the curl kernel (4 values per point), not
    the 6-component demag tensor the z stage reads: the call is refused before
    any kernel runs, and the output buffer is left untouched."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import OerstedPlan, lib
    n = (32, 40, 4)
    plan = OerstedPlan(*n, 2e-9, 2e-9, 2e-9)
    J = torch.ones((3, n[2], n[1], n[0]), dtype=torch.float32, device="cuda")
    H = torch.full_like(J, 7.0)
    L = lib()
    rc = _noalloc(L, plan, J, H)
    assert rc == -1
    assert b"demag plans" in L.boris_last_error()
    torch.cuda.synchronize()
    assert bool((H == 7.0).all())
