"""Out-of-bounds writes without a sanitizer: every field handed to the library
is a view into a larger buffer whose 4 KB guard bands on both sides hold a
sentinel value; after the call both bands must be unchanged.  This covers the
demag application (every transform length class, ragged sizes, the 2D mode,
both tensor-core forms), the adjoint, RK4 and RKF45 steps in place, the
multi-mesh plan and the Oersted field."""
import math

import numpy as np
import pytest

from paper_2008_02478_gb300 import inputs
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

PAD = 1024  # floats on each side (4 KB: keeps the view 16-byte aligned)
SENTINEL = 1234.5678


def guarded(torch, shape, fill=None, dtype=None):
    dtype = dtype or torch.float32
    n = int(np.prod(shape))
    buf = torch.full((n + 2 * PAD,), SENTINEL, dtype=dtype, device="cuda")
    view = buf[PAD:PAD + n].view(*shape)
    if fill is not None:
        view.copy_(torch.as_tensor(fill, dtype=dtype).reshape(shape))
    return buf, view


def bands_intact(torch, buf):
    torch.cuda.synchronize()
    head, tail = buf[:PAD].cpu().numpy(), buf[-PAD:].cpu().numpy()
    s = np.float32(SENTINEL) if buf.dtype == torch.float32 else SENTINEL
    return bool(np.all(head == s) and np.all(tail == s))


MESHES = [
    ((37, 29, 5), 3e-9),     # ragged, general lengths
    ((24, 16, 1), 2e-9),     # 2D mode
    ((300, 40, 3), 4e-9),    # x length 1024
    ((130, 70, 6), 4e-9),    # lengths 512 / 256
    ((20, 700, 2), 4e-9),    # y length 2048
]


@pytest.mark.parametrize("n,h", MESHES)
def test_demag_adjoint_and_steps_stay_in_bounds(n, h):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import RKF45, LLGParams, Plan
    m0 = inputs.random_unit(*n, seed=7)
    plan = Plan(*n, h, h, h)
    bm, M = guarded(torch, plan.field_shape, 8e5 * m0)
    bh, H = guarded(torch, plan.field_shape)
    plan.apply(M, H)
    assert bands_intact(torch, bm) and bands_intact(torch, bh)
    assert math.isfinite(float(H.abs().max()))
    bg, G = guarded(torch, plan.field_shape)
    plan.adjoint(H, G)
    assert bands_intact(torch, bh) and bands_intact(torch, bg)
    bs, m = guarded(torch, plan.field_shape, m0)
    prm = LLGParams(Ms=8e5, A=1.3e-11, alpha=0.1)
    plan.llg_step(m, prm, 1e-13)
    assert bands_intact(torch, bs)
    prm45 = LLGParams(Ms=8e5, A=1.3e-11, alpha=0.1, method=RKF45, tol=1e-5, dt_min=1e-16, dt_max=1e-12)
    plan.llg_step(m, prm45, 1e-13)
    assert bands_intact(torch, bs)


@pytest.mark.parametrize("tc", ["fp16", "bf16"])
def test_tensor_core_stage_stays_in_bounds(tc, monkeypatch):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    n, h = (40, 72, 21), 4e-9
    for form in ("tcgen05", "mma.sync"):
        if form == "mma.sync":
            monkeypatch.setenv("BORIS_TC_MMASYNC", "1")
        plan = Plan(*n, h, h, h, tc=tc)
        monkeypatch.delenv("BORIS_TC_MMASYNC", raising=False)
        bm, M = guarded(torch, plan.field_shape, 8e5 * inputs.random_unit(*n, seed=8))
        bh, H = guarded(torch, plan.field_shape)
        plan.apply(M, H)
        assert bands_intact(torch, bm) and bands_intact(torch, bh)


def test_multimesh_and_oersted_stay_in_bounds():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import LLGParams, MultiPlan, OerstedPlan
    layers = [(40, 30, 3), (24, 20, 2)]
    cells, origins = inputs.stack_geometry(layers, [2e-9, 3e-9], [1e-9], 4e-9)
    mp = MultiPlan(layers, cells, origins)
    m0 = np.concatenate([inputs.random_unit(*l, seed=9 + i).reshape(-1) for i, l in enumerate(layers)])
    bm, M = guarded(torch, mp.field_shape, 8e5 * m0)
    bh, H = guarded(torch, mp.field_shape)
    mp.apply(M, H)
    assert bands_intact(torch, bm) and bands_intact(torch, bh)
    bs, m = guarded(torch, mp.field_shape, m0)
    mp.llg_step(m, LLGParams(Ms=8e5, A=1.3e-11, alpha=0.1), 5e-14)
    assert bands_intact(torch, bs)
    n, h = (30, 40, 4), 3e-9
    op = OerstedPlan(*n, h, h, h)
    bj, J = guarded(torch, op.field_shape, 1e11 * inputs.random_unit(*n, seed=10))
    bo, Ho = guarded(torch, op.field_shape)
    op.apply(J, Ho)
    assert bands_intact(torch, bj) and bands_intact(torch, bo)
