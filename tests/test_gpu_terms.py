"""GPU parity of the further effective-field terms (Table 1 cubic and
second-order uniaxial anisotropy, bulk and interfacial DMI with the
non-homogeneous Neumann boundary condition; Eq. 5 surface exchange between
the layers of a multi-mesh plan) against the FP64 oracle, through the C ABI.

Tolerances: the RK4 increment m1 - m0 within 2e-4 relative L2 (FP32 state of
order 1, increments of order 1e-2); exchange, anisotropy and DMI energies
within 1e-6 relative (FP64 sums over the same FP32 state, with the FP32 plan's
parameters 1/h^2, A, D, K rounded to FP32: about 6e-8 each); the demag energy
within 1e-5 (FP32 field)."""
import numpy as np
import pytest

import oracle
from oracle import llg
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import assert_close, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

N, CELL = (19, 13, 5), (1.5e-9, 2e-9, 1.2e-9)
BASE = dict(Ms=8e5, A=1.3e-11, alpha=0.1, Ku=2e4, easy=(0.3, 0.0, 0.954), Hext=(2e4, -1e4, 5e4))
TERMS = {
    "cubic": dict(Kc1=4.5e4, Kc2=-1.5e4, cubic_e1=(0.8, 0.6, 0.0), cubic_e2=(-0.6, 0.8, 0.0)),
    "k2": dict(K2=3e4),
    "bulk": dict(dmi="bulk", D=2.5e-3),
    "interfacial": dict(dmi="interfacial", D=3e-3),
    "all": dict(K2=1e4, Kc1=-2e4, Kc2=1e4, cubic_e1=(0.0, 0.6, 0.8), cubic_e2=(1.0, 0.0, 0.0), dmi="interfacial",
                D=2e-3),
}


def state():
    m = inputs.random_unit(*N, seed=31)
    # smooth it a little so that exchange and DMI fields stay moderate
    m = m + 0.5 * np.roll(m, 1, axis=3) + 0.5 * np.roll(m, 1, axis=2)
    m = m / np.linalg.norm(m, axis=0)
    return m.astype(np.float32).astype(np.float64)


def oracle_params(extra):
    e = np.array(BASE["easy"])
    return llg.Params(cell=CELL, Ms=BASE["Ms"], A=BASE["A"], alpha=BASE["alpha"], Ku=BASE["Ku"],
                      easy=tuple(e / np.linalg.norm(e)), Hext=BASE["Hext"], **extra)


def gpu_objects(extra):
    from paper_2008_02478_gb300.binding import FieldTerms, LLGParams, Plan
    plan = Plan(*N, *CELL)
    plan.set_field_terms(FieldTerms(**extra))
    e = np.array(BASE["easy"])
    prm = LLGParams(Ms=BASE["Ms"], A=BASE["A"], alpha=BASE["alpha"], Ku=BASE["Ku"], easy=tuple(e / np.linalg.norm(e)),
                    Hext=BASE["Hext"])
    return plan, prm


@pytest.mark.parametrize("name", list(TERMS))
def test_rk4_step_with_terms_matches_oracle(name):
    torch = torch_cuda()
    m0 = state()
    prm_o = oracle_params(TERMS[name])
    demag = oracle.DemagPlan(*N, *CELL).apply
    dt = 2e-14
    ref = llg.rk4_step(m0, dt, prm_o, demag)
    plan, prm = gpu_objects(TERMS[name])
    m = torch.tensor(m0, dtype=torch.float32, device="cuda")
    plan.llg_step(m, prm, dt)
    got = m.cpu().numpy().astype(np.float64)
    d_ref = ref - m0
    assert np.abs(d_ref).max() > 1e-3  # the step moves the state
    assert_close(got - m0, d_ref, 2e-4)


@pytest.mark.parametrize("name", list(TERMS))
def test_energies_with_terms_match_oracle(name):
    torch = torch_cuda()
    m0 = state()
    prm_o = oracle_params(TERMS[name])
    demag = oracle.DemagPlan(*N, *CELL).apply
    ref = llg.energies_terms(m0, prm_o, demag)
    plan, prm = gpu_objects(TERMS[name])
    got = plan.energy_terms(torch.tensor(m0, dtype=torch.float32, device="cuda"), prm)
    assert got[0] == pytest.approx(ref[0], rel=1e-5)
    for i in (1, 2, 3, 4):
        assert got[i] == pytest.approx(ref[i], rel=1e-6, abs=1e-30)
    if TERMS[name].get("dmi", "none") != "none":
        assert abs(ref[4]) > 0


def test_rkf45_and_graph_with_terms():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import RKF45
    m0 = state()
    extra = TERMS["all"]
    prm_o = oracle_params(extra)
    demag = oracle.DemagPlan(*N, *CELL).apply
    # one RKF45 trial that is accepted
    plan, prm = gpu_objects(extra)
    prm.method, prm.tol = RKF45, 1e-3
    m = torch.tensor(m0, dtype=torch.float32, device="cuda")
    dt_next = plan.llg_step(m, prm, 1e-14)
    ref, err = llg.rkf45_step(m0, 1e-14, prm_o, demag)
    assert err <= 1e-3
    assert_close(m.cpu().numpy() - m0, ref - m0, 2e-4)
    assert dt_next == pytest.approx(llg.rkf45_next_dt(1e-14, err, 1e-3, prm.dt_min, prm.dt_max), rel=1e-3)
    # graph replay equals separate steps, and a change of terms re-captures
    plan2, prm2 = gpu_objects(extra)
    a = torch.tensor(m0, dtype=torch.float32, device="cuda")
    b = a.clone()
    for _ in range(3):
        plan2.llg_step(a, prm2, 1e-14)
    plan2.llg_run_graph(b, prm2, 1e-14, 3)
    torch.cuda.synchronize()
    assert_close(b.cpu().numpy(), a.cpu().numpy(), 1e-7, 1e-7 * 10)
    from paper_2008_02478_gb300.binding import FieldTerms
    plan2.set_field_terms(FieldTerms())
    c = torch.tensor(m0, dtype=torch.float32, device="cuda")
    d = c.clone()
    plan2.llg_run_graph(c, prm2, 1e-14, 2)
    for _ in range(2):
        plan2.llg_step(d, prm2, 1e-14)
    torch.cuda.synchronize()
    assert_close(c.cpu().numpy(), d.cpu().numpy(), 1e-7, 1e-7 * 10)


def test_terms_argument_checks():
    torch_cuda()
    from paper_2008_02478_gb300.binding import BorisError, FieldTerms, LLGParams, Plan
    plan = Plan(*N, *CELL)
    with pytest.raises(BorisError) as e:
        plan.set_field_terms(FieldTerms(Kc1=1e4, cubic_e1=(1, 0, 0), cubic_e2=(1, 1, 0)))
    assert e.value.code == -1
    with pytest.raises(BorisError) as e:
        plan.set_field_terms(FieldTerms(J1=1e-3))  # surface exchange needs a multi-mesh plan
    assert e.value.code == -1
    with pytest.raises(BorisError) as e:
        plan.set_field_terms(FieldTerms(D=float("nan"), dmi="bulk"))
    assert e.value.code == -1
    plan.set_field_terms(FieldTerms(dmi="bulk", D=1e-3))
    import torch
    m = torch.tensor(state(), dtype=torch.float32, device="cuda")
    with pytest.raises(BorisError) as e:  # the adjoint covers the base terms only
        plan.llg_step_backward(m, LLGParams(), 1e-14, torch.zeros_like(m))
    assert e.value.code == -1
    with pytest.raises(BorisError) as e:  # DMI needs A > 0
        plan.llg_step(m, LLGParams(A=0.0), 1e-14)
    assert e.value.code == -1
    plan.set_field_terms(None)
    plan.llg_step(m, LLGParams(), 1e-14)
