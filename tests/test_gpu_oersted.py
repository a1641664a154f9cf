"""GPU parity of the Oersted field (Table 1: H = sum K(r - r0) J, with the
cell-averaged kernel derived in the oracle) against the oracle's direct sum,
and of an RK4 step that takes an Oersted field as an additive field map.
Tolerance 1e-5 relative L2 (FP32 field), 2e-4 on the RK4 increment."""
import numpy as np
import pytest

import oracle
from oracle import llg
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import assert_close, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    ((20, 40, 1), (2e-9, 2e-9, 3e-9)),      # single layer: pointwise multiply
    ((16, 36, 3), (2e-9, 1.5e-9, 1e-9)),    # pz = 8
    ((12, 40, 5), (1e-9, 2e-9, 2e-9)),      # pz = 16, ragged z
    ((10, 64, 17), (2e-9, 2e-9, 2e-9)),     # pz = 64
    ((300, 34, 4), (3e-9, 3e-9, 3e-9)),     # length-1024 x passes
]


def current(n, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    J = rng.normal(size=(3, nz, ny, nx)) * 1e11
    return J


@pytest.mark.parametrize("n,h", CASES)
def test_oersted_matches_direct_sum(n, h):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import OerstedPlan
    J = current(n, 61)
    ref = oracle.oersted_direct(J, oracle.oersted_table(*n, *h))
    plan = OerstedPlan(*n, *h)
    H = plan.apply(to_dev(torch, J)).cpu().numpy()
    plan.sync_status()
    assert_close(H, ref, 1e-5)


def test_oersted_field_drives_the_llg_step():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import FieldTerms, LLGParams, OerstedPlan, Plan
    n, h = (16, 36, 3), (2e-9, 2e-9, 2e-9)
    J = np.zeros((3, n[2], n[1], n[0]))
    J[0] = 2e12  # a uniform current along x
    op = OerstedPlan(*n, *h)
    Hoe = op.apply(to_dev(torch, J))
    Hoe_np = Hoe.cpu().numpy().astype(np.float64)
    m0 = inputs.random_unit(*n, seed=62).astype(np.float32).astype(np.float64)
    prm_o = llg.Params(cell=h, Ms=8e5, A=1.3e-11, alpha=0.1)
    dplan = oracle.DemagPlan(*n, *h)
    demag_plus = lambda M: dplan.apply(M) + Hoe_np
    dt = 2e-14
    ref = llg.rk4_step(m0, dt, prm_o, demag_plus)
    plan = Plan(*n, *h)
    plan.set_field_terms(FieldTerms(H_add=Hoe))
    m = torch.tensor(m0, dtype=torch.float32, device="cuda")
    plan.llg_step(m, LLGParams(Ms=8e5, A=1.3e-11, alpha=0.1), dt)
    got = m.cpu().numpy().astype(np.float64)
    assert np.abs(ref - m0).max() > 1e-3
    assert_close(got - m0, ref - m0, 2e-4)
    # the Oersted field counts with the Zeeman energy
    E = plan.energy_terms(m, LLGParams(Ms=8e5, A=1.3e-11, alpha=0.1))
    mm = m.cpu().numpy().astype(np.float64)
    V = h[0] * h[1] * h[2]
    Ez = -llg.MU0 * 8e5 * V * float((mm * Hoe_np).sum())
    assert E[3] == pytest.approx(Ez, rel=1e-5)


def test_oersted_plan_checks():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import BorisError, OerstedPlan, lib
    with pytest.raises(BorisError) as e:
        OerstedPlan(16, 40, 2, 1e-9, 1e-9, 1e-9)  # nz = 2 is not provided
    assert e.value.code == -4
    p = OerstedPlan(16, 40, 1, 1e-9, 1e-9, 1e-9)
    import ctypes
    M = torch.zeros((3, 1, 40, 16), dtype=torch.float32, device="cuda")
    H = torch.empty_like(M)
    rc = lib().boris_demag_apply(p._h, ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(H.data_ptr()))
    assert rc == -1
