"""The allocation-free demag entry point (boris_demag_apply_noalloc).

Some callers cannot allocate device memory while they run (their allocator is
locked, or allocation is forbidden on their hot path); this entry point keeps
its spectral workspace in a fixed array inside the library instead.  Here it
is called through the C ABI and compared with boris_demag_apply on two calls
in a row (the second call reuses the array the first one left filled), and a
mesh too large for the array is rejected.  This file runs last."""
import ctypes

import numpy as np
import pytest

from paper_2008_02478_gb300 import inputs
from tests.gpu_util import rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def test_noalloc_matches_apply_on_two_calls():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan, lib
    n, h = (48, 40, 6), (2e-9, 2e-9, 3e-9)
    plan = Plan(*n, *h)
    L = lib()
    for seed in (11, 12):
        M = to_dev(torch, 7e5 * inputs.random_unit(*n, seed=seed))
        ref = plan.apply(M)
        H = torch.empty_like(M)
        rc = L.boris_demag_apply_noalloc(plan._h, ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(H.data_ptr()))
        assert rc == 0, L.boris_last_error()
        torch.cuda.synchronize()
        assert rel_l2(H.cpu().numpy(), ref.cpu().numpy()) < 1e-5


def test_noalloc_rejects_meshes_beyond_its_array():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan, lib
    n = (256, 256, 32)  # spectrum 257 * 3 * 32 * 256 * 8 bytes > 32 MiB
    plan = Plan(*n, 4e-9, 4e-9, 4e-9)
    M = torch.zeros((3, n[2], n[1], n[0]), dtype=torch.float32, device="cuda")
    H = torch.empty_like(M)
    L = lib()
    rc = L.boris_demag_apply_noalloc(plan._h, ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(H.data_ptr()))
    assert rc == -4
    assert b"32 MiB" in L.boris_last_error() or b"bytes" in L.boris_last_error()
