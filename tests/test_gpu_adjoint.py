"""GPU adjoint of the RK4 LLG step and the checkpointed trajectory gradient,
against the FP64 oracle's discrete adjoint and central finite differences
(8 x 8 x 2 sub-problem of the 256 x 256 x 8 differentiation film: 3 nm cells,
smooth-noise Ms in [6e5, 1e6] A/m and Ku in [0, 5e5] J/m^3).  Tolerances:
FP64 plan vs oracle 1e-9; FP32 plan vs oracle 1e-3 (relative L2)."""
import numpy as np
import pytest

import oracle
from oracle import llg
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import assert_close, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

N, H = (8, 8, 2), (3e-9, 3e-9, 3e-9)


def sub_problem():
    Ms = inputs.smooth_noise(*N, 2.0, 6e5, 1e6, 5)
    Ku = inputs.smooth_noise(*N, 2.0, 0.0, 5e5, 6)
    prm = llg.Params(cell=H, Ms=Ms, A=1.3e-11, alpha=0.02, Ku=Ku, easy=(0.0, 0.0, 1.0), Hext=(0.0, 0.0, 0.0))
    m0 = inputs.smooth_texture(*N, 1.5, 5)
    target = inputs.smooth_texture(*N, 1.5, 3)
    return prm, m0, target


def oracle_grad(prm, m0, target, nsteps, dt):
    dem = oracle.DemagPlan(*N, *H)
    traj = [m0]
    for _ in range(nsteps):
        traj.append(llg.rk4_step(traj[-1], dt, prm, dem.apply))
    g = 2 * (traj[-1] - target)
    gMs = np.zeros(m0.shape[1:])
    gKu = np.zeros(m0.shape[1:])
    for s in range(nsteps - 1, -1, -1):
        g, a, b = llg.rk4_step_vjp(traj[s], dt, prm, dem.apply, g)
        gMs += a
        gKu += b
    return np.sum((traj[-1] - target) ** 2), g, gMs, gKu


@pytest.mark.parametrize("fp64", [True, False])
def test_step_backward_matches_oracle(fp64):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import LLGParams, Plan
    prm, m0, target = sub_problem()
    dt = 1e-13
    dem = oracle.DemagPlan(*N, *H)
    gout = inputs.random_unit(*N, seed=9)
    ref_gm, ref_gMs, ref_gKu = llg.rk4_step_vjp(m0, dt, prm, dem.apply, gout)
    plan = Plan(*N, *H, fp64=fp64)
    p = LLGParams(A=prm.A, alpha=prm.alpha, gamma=prm.gamma, easy=prm.easy, Hext=prm.Hext,
                  Ms_map=to_dev(torch, prm.Ms, fp64), Ku_map=to_dev(torch, prm.Ku, fp64))
    gMs = torch.zeros(N[::-1], dtype=plan.dtype, device="cuda")
    gKu = torch.zeros_like(gMs)
    gm = plan.llg_step_backward(to_dev(torch, m0, fp64), p, dt, to_dev(torch, gout, fp64), None, gMs, gKu)
    tol = 1e-9 if fp64 else 1e-3
    assert_close(gm.cpu().numpy(), ref_gm, tol)
    assert_close(gMs.cpu().numpy(), ref_gMs, tol)
    assert_close(gKu.cpu().numpy(), ref_gKu, tol)


def test_checkpointed_trajectory_gradient():
    torch = torch_cuda()
    from paper_2008_02478_gb300.autograd import trajectory
    from paper_2008_02478_gb300.binding import LLGParams, Plan
    prm, m0, target = sub_problem()
    nsteps, dt = 12, 1e-13
    L_ref, gm_ref, gMs_ref, gKu_ref = oracle_grad(prm, m0, target, nsteps, dt)
    for fp64, tol in ((True, 1e-9), (False, 1e-3)):
        plan = Plan(*N, *H, fp64=fp64)
        base = LLGParams(A=prm.A, alpha=prm.alpha, gamma=prm.gamma, easy=prm.easy, Hext=prm.Hext)
        Ms = to_dev(torch, prm.Ms, fp64).requires_grad_(True)
        Ku = to_dev(torch, prm.Ku, fp64).requires_grad_(True)
        m = to_dev(torch, m0, fp64).requires_grad_(True)
        out = trajectory(m, Ms, Ku, plan, base, nsteps, dt, ckpt=5)  # ragged last segment
        L = ((out - to_dev(torch, target, fp64)) ** 2).sum()
        L.backward()
        assert abs(float(L) - L_ref) < (1e-9 if fp64 else 1e-4) * L_ref
        assert_close(Ms.grad.cpu().numpy(), gMs_ref, tol)
        assert_close(Ku.grad.cpu().numpy(), gKu_ref, tol)
        assert_close(m.grad.cpu().numpy(), gm_ref, tol)


def test_trajectory_gradient_vs_central_differences():
    """FP64 plan: dL/dMs and dL/dKu at a few cells against central differences
    of the GPU forward (relative perturbation 1e-6 of the map's scale)."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.autograd import trajectory
    from paper_2008_02478_gb300.binding import LLGParams, Plan
    prm, m0, target = sub_problem()
    nsteps, dt = 6, 1e-13
    plan = Plan(*N, *H, fp64=True)
    base = LLGParams(A=prm.A, alpha=prm.alpha, gamma=prm.gamma, easy=prm.easy, Hext=prm.Hext)
    tgt = to_dev(torch, target, True)
    m0d = to_dev(torch, m0, True)

    def loss(Ms, Ku):
        with torch.no_grad():
            return float(((trajectory(m0d, Ms, Ku, plan, base, nsteps, dt, 50) - tgt) ** 2).sum())
    Ms = to_dev(torch, prm.Ms, True).requires_grad_(True)
    Ku = to_dev(torch, prm.Ku, True).requires_grad_(True)
    L = ((trajectory(m0d, Ms, Ku, plan, base, nsteps, dt, 50) - tgt) ** 2).sum()
    L.backward()
    r = inputs.rng(2)
    for _ in range(3):
        idx = tuple(int(r.integers(0, s)) for s in Ms.shape)
        for which, T, G in (("Ms", Ms, Ms.grad), ("Ku", Ku, Ku.grad)):
            eps = 1e-6 * float(T.max())
            tp, tm = T.detach().clone(), T.detach().clone()
            tp[idx] += eps
            tm[idx] -= eps
            fd = (loss(tp, Ku.detach()) - loss(tm, Ku.detach())) / (2 * eps) if which == "Ms" else \
                 (loss(Ms.detach(), tp) - loss(Ms.detach(), tm)) / (2 * eps)
            g = float(G[idx])
            assert abs(fd - g) <= 1e-5 * float(G.abs().max()) + 1e-5 * abs(fd), (which, fd, g)


# meshes where the backward step runs the production kernels: length-1024 x
# passes with the four-cells-per-thread stage (300 x 64 x 3), length-1024 y
# passes of the split y-z schedule (64 x 300 x 4), and pz = 64 with a ragged
# nz (48 x 40 x 17), where the residue-split z stage is a candidate
BIG = [((300, 64, 3), (3e-9, 3e-9, 3e-9)), ((64, 300, 4), (3e-9, 3e-9, 3e-9)), ((48, 40, 17), (3e-9, 3e-9, 3e-9))]


@pytest.mark.parametrize("n,h", BIG)
@pytest.mark.parametrize("fp64", [False, True])
def test_step_backward_matches_oracle_on_production_kernels(n, h, fp64):
    """g_m, g_Ms and g_Ku of one RK4 step against the oracle's discrete adjoint
    on meshes that take the length-1024 warp transforms, the split y-z
    schedule and the quad stage kernel."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import LLGParams, Plan
    Ms = inputs.smooth_noise(*n, 2.0, 6e5, 1e6, 15)
    Ku = inputs.smooth_noise(*n, 2.0, 0.0, 5e5, 16)
    prm = llg.Params(cell=h, Ms=Ms, A=1.3e-11, alpha=0.02, Ku=Ku, easy=(0.0, 0.0, 1.0), Hext=(0.0, 0.0, 2e4))
    m0 = inputs.smooth_texture(*n, 1.5, 17)
    gout = inputs.random_unit(*n, seed=18)
    dt = 1e-13
    ref_gm, ref_gMs, ref_gKu = llg.rk4_step_vjp(m0, dt, prm, oracle.DemagPlan(*n, *h).apply, gout)
    plan = Plan(*n, *h, fp64=fp64)
    p = LLGParams(A=prm.A, alpha=prm.alpha, gamma=prm.gamma, easy=prm.easy, Hext=prm.Hext,
                  Ms_map=to_dev(torch, Ms, fp64), Ku_map=to_dev(torch, Ku, fp64))
    gMs = torch.zeros(n[::-1], dtype=plan.dtype, device="cuda")
    gKu = torch.zeros_like(gMs)
    gm = plan.llg_step_backward(to_dev(torch, m0, fp64), p, dt, to_dev(torch, gout, fp64), None, gMs, gKu)
    tol = 1e-9 if fp64 else 1e-3
    assert_close(gm.cpu().numpy(), ref_gm, tol)
    assert_close(gMs.cpu().numpy(), ref_gMs, tol)
    assert_close(gKu.cpu().numpy(), ref_gKu, tol)
