"""GPU parity of the fused LLG step (Eq. 1; Table 1 fields; RK4 and RKF45 of
Section 2) and the FP64 energies against the oracle, through the C ABI.
Tolerance on m after 10 RK4 steps: relative L2 1e-5 (FP32)."""
import numpy as np
import pytest

import oracle
from oracle import llg
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import assert_close, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _problem(n, h, per_cell, seed, Hext=(1e4, -2e4, 3e4)):
    nx, ny, nz = n
    if per_cell:
        Ms = inputs.smooth_noise(nx, ny, nz, 2.0, 6e5, 1e6, seed)
        Ku = inputs.smooth_noise(nx, ny, nz, 2.0, 0.0, 5e5, seed + 1)
    else:
        Ms, Ku = 8e5, 1e5
    prm = llg.Params(cell=h, Ms=Ms, A=1.3e-11, alpha=0.02, Ku=Ku, easy=(0.0, 0.6, 0.8), Hext=Hext)
    m0 = inputs.random_unit(nx, ny, nz, seed)
    return prm, m0


def _gpu_params(torch, prm, fp64=False):
    from paper_2008_02478_gb300.binding import LLGParams
    g = LLGParams(A=prm.A, alpha=prm.alpha, gamma=prm.gamma, easy=prm.easy, Hext=prm.Hext)
    if np.ndim(prm.Ms):
        g.Ms_map = to_dev(torch, prm.Ms, fp64)
    else:
        g.Ms = float(prm.Ms)
    if np.ndim(prm.Ku):
        g.Ku_map = to_dev(torch, prm.Ku, fp64)
    else:
        g.Ku = float(prm.Ku)
    return g


@pytest.mark.parametrize("n,h,per_cell", [
    ((32, 32, 4), (5e-9, 5e-9, 5e-9), False),   # small cubic-cell mesh, 10 RK4 steps
    ((20, 13, 3), (3e-9, 3e-9, 3e-9), True),    # per-cell Ms and Ku maps, ragged
    ((24, 16, 1), (2e-9, 2e-9, 3e-9), False),   # 2D mode
    ((21, 10, 2), (3e-9, 2e-9, 4e-9), True),    # nx % 4 != 0: one cell per thread in FP32
])
@pytest.mark.parametrize("fp64", [False, True])
def test_rk4_steps_match_oracle(n, h, per_cell, fp64):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    prm, m0 = _problem(n, h, per_cell, seed=1)
    dt, steps = 1e-13, 10
    dem = oracle.DemagPlan(*n, *h)
    ref = m0.copy()
    for _ in range(steps):
        ref = llg.rk4_step(ref, dt, prm, dem.apply)
    plan = Plan(*n, *h, fp64=fp64)
    m = to_dev(torch, m0, fp64)
    gp = _gpu_params(torch, prm, fp64)
    for _ in range(steps):
        plan.llg_step(m, gp, dt)
    assert_close(m.cpu().numpy(), ref, 1e-10 if fp64 else 1e-5)


@pytest.mark.parametrize("fp64", [False, True])
def test_rkf45_step_matches_oracle(fp64):
    """One accepted RKF45 step (tol large enough to accept the first trial):
    the 4th-order state and the controller's next step against the oracle."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan, RKF45
    n, h = (24, 12, 2), (2e-9, 2e-9, 3e-9)
    prm, m0 = _problem(n, h, False, seed=3)
    dem = oracle.DemagPlan(*n, *h)
    dt = 5e-14
    ref, err_ref = llg.rkf45_step(m0, dt, prm, dem.apply)
    plan = Plan(*n, *h, fp64=fp64)
    m = to_dev(torch, m0, fp64)
    gp = _gpu_params(torch, prm, fp64)
    gp.method, gp.tol, gp.dt_min, gp.dt_max = RKF45, 1.0, 1e-16, 1e-12
    nxt = plan.llg_step(m, gp, dt)
    assert_close(m.cpu().numpy(), ref, 1e-10 if fp64 else 1e-5)
    assert nxt == pytest.approx(llg.rkf45_next_dt(dt, err_ref, 1.0, 1e-16, 1e-12), rel=1e-5 if fp64 else 1e-3)


def _oracle_rkf45_run(m, dt, nsteps, prm, demag, tol, dt_min, dt_max):
    """The oracle's adaptive RKF45 (Section 2 evaluator; controller of the
    stated reading): accepted states, the accepted steps and the next step."""
    t, dts, trials = 0.0, [], 0
    for _ in range(nsteps):
        for _attempt in range(16):
            m_new, err = llg.rkf45_step(m, dt, prm, demag)
            trials += 1
            hn = llg.rkf45_next_dt(dt, err, tol, dt_min, dt_max)
            if err <= tol or dt <= dt_min:
                m, t = m_new, t + dt
                dts.append(dt)
                dt = hn
                break
            dt = hn
        else:
            raise AssertionError("oracle controller ran out of trials")
    return m, dt, t, dts, trials


@pytest.mark.parametrize("fp64", [False, True])
def test_rkf45_frozen_controller_matches_oracle(fp64):
    """Parity with the controller frozen: the GPU steps with the oracle's
    accepted step sequence (every trial accepted), 8 steps."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan, RKF45
    n, h = (24, 12, 2), (3e-9, 3e-9, 3e-9)
    prm, m0 = _problem(n, h, True, seed=5)
    dem = oracle.DemagPlan(*n, *h)
    ref, _, _, dts, _ = _oracle_rkf45_run(m0, 1e-13, 8, prm, dem.apply, 1e-6, 1e-16, 1e-12)
    plan = Plan(*n, *h, fp64=fp64)
    m = to_dev(torch, m0, fp64)
    gp = _gpu_params(torch, prm, fp64)
    gp.method, gp.tol, gp.dt_min, gp.dt_max = RKF45, 1e30, 1e-16, 1e-12
    for dt in dts:
        plan.llg_step(m, gp, dt)
    assert_close(m.cpu().numpy(), ref, 1e-10 if fp64 else 1e-5)


def test_rkf45_device_controller_matches_oracle():
    """Adaptive RKF45 with rejected trials (the first step is far too long):
    the device controller's accept/reject decisions, step sizes, simulated
    time and final state equal the oracle's (FP64 plan, one host
    synchronisation for all steps)."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan, RKF45
    n, h = (24, 12, 2), (3e-9, 3e-9, 3e-9)
    prm, m0 = _problem(n, h, False, seed=6)
    dem = oracle.DemagPlan(*n, *h)
    tol, dmin, dmax, dt0, nsteps = 1e-5, 1e-16, 1e-12, 3e-12, 6
    ref, dt_ref, t_ref, dts, trials = _oracle_rkf45_run(m0, dt0, nsteps, prm, dem.apply, tol, dmin, dmax)
    assert trials > nsteps  # the test exercises rejections
    plan = Plan(*n, *h, fp64=True)
    m = to_dev(torch, m0, True)
    gp = _gpu_params(torch, prm, True)
    gp.method, gp.tol, gp.dt_min, gp.dt_max = RKF45, tol, dmin, dmax
    dt = dt0
    for _ in range(nsteps):
        dt = plan.llg_step(m, gp, dt)
    assert dt == pytest.approx(dt_ref, rel=1e-8)
    assert_close(m.cpu().numpy(), ref, 1e-10)


def test_rkf45_run_equals_single_steps():
    """boris_llg_run_rkf45 (all steps enqueued, one synchronisation) takes the
    same decisions as step-by-step calls: identical state, step and time."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan, RKF45
    n, h = (40, 24, 3), (3e-9, 3e-9, 3e-9)
    prm, m0 = _problem(n, h, True, seed=7)
    plan = Plan(*n, *h)
    gp = _gpu_params(torch, prm)
    gp.method, gp.tol, gp.dt_min, gp.dt_max = RKF45, 1e-5, 1e-16, 1e-12
    a, b = to_dev(torch, m0), to_dev(torch, m0)
    dt_a = 2e-12
    for _ in range(5):
        dt_a = plan.llg_step(a, gp, dt_a)
    dt_b, t_b = plan.llg_run_rkf45(b, gp, 2e-12, 5)
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    assert dt_a == dt_b and t_b > 0
    assert plan.sync_status() == 0


def test_rkf45_rejects_then_accepts():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan, RKF45
    n, h = (16, 16, 1), (2e-9, 2e-9, 3e-9)
    prm, m0 = _problem(n, h, False, seed=4)
    plan = Plan(*n, *h)
    m = to_dev(torch, m0)
    gp = _gpu_params(torch, prm)
    gp.method, gp.tol, gp.dt_min, gp.dt_max = RKF45, 1e-7, 1e-18, 1e-12
    dt = 1e-12
    nxt = plan.llg_step(m, gp, dt)  # too large: rejected, retried smaller
    assert nxt < dt
    nrm = torch.sqrt((m * m).sum(0))
    assert float((nrm - 1).abs().max()) < 1e-6


@pytest.mark.parametrize("per_cell", [False, True])
def test_energies_match_oracle(per_cell):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    n, h = (20, 18, 4), (3e-9, 3e-9, 3e-9)
    prm, m0 = _problem(n, h, per_cell, seed=5)
    ref = llg.energies(m0, prm, oracle.DemagPlan(*n, *h).apply)
    plan = Plan(*n, *h)
    E = plan.energy(to_dev(torch, m0), _gpu_params(torch, prm))
    for e, r in zip(E, ref):
        assert abs(e - r) <= 1e-5 * max(abs(v) for v in ref), (E, ref)


@pytest.mark.parametrize("n", [(32, 32, 4), (256, 64, 1)])
def test_graph_replay_equals_step_calls(n):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import LLGParams, Plan
    h = (2e-9, 2e-9, 3e-9)
    m0 = inputs.random_unit(*n, seed=8)
    # one plan for both routes: two plans may autotune different y-z schedules
    p = Plan(*n, *h)
    prm = LLGParams(Ms=8e5, A=1.3e-11, alpha=0.02, Hext=(0.0, 1e4, 2e4))
    a = to_dev(torch, m0)
    b = to_dev(torch, m0)
    for _ in range(5):
        p.llg_step(a, prm, 1e-13)
    p.llg_run_graph(b, prm, 1e-13, 2)
    p.llg_run_graph(b, prm, 1e-13, 3)  # reuses the captured graph
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_host_buffer_steps_equal_device_steps():
    """boris_llg_run_host (pinned host state copied in, steps, copied back) takes
    the same kernels as the device-resident steps: bit-identical states."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import LLGParams, Plan
    n, h = (48, 20, 3), (3e-9, 3e-9, 3e-9)
    m0 = inputs.random_unit(*n, seed=9)
    p = Plan(*n, *h)
    prm = LLGParams(Ms=8e5, A=1.3e-11, alpha=0.02, Hext=(2e4, 0.0, 1e4))
    a = to_dev(torch, m0)
    for _ in range(4):
        p.llg_step(a, prm, 1e-13)
    host = torch.tensor(m0, dtype=torch.float32).pin_memory()
    p.llg_run_host(host, prm, 1e-13, 1)
    p.llg_run_host(host, prm, 1e-13, 3)  # reuses the captured graph
    torch.cuda.synchronize()
    assert torch.equal(a.cpu(), host)
    p.llg_run_host(host, prm, 1e-13, 0)  # copies in and out only
    assert torch.equal(a.cpu(), host)


# Meshes of 257..512 cells along x (transform length 1024) can run the
# inverse x transform and the RK4 stage as one kernel in FP32; the ragged cases
# leave a partial group of 8 rows at the top of each plane.
@pytest.mark.parametrize("n,per_cell", [
    ((300, 20, 3), True),    # per-cell maps, ny % 8 = 4
    ((512, 13, 2), False),   # full 512-cell rows, ny % 8 = 5
    ((257, 8, 1), True),     # shortest row of the 1024-point transform, 2D mode
])
def test_fused_inverse_x_rk4_matches_oracle(n, per_cell, monkeypatch):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    monkeypatch.setenv("BORIS_FUSE_STAGE", "1")
    h = (3e-9, 3e-9, 3e-9)
    prm, m0 = _problem(n, h, per_cell, seed=11)
    dt, steps = 1e-13, 3
    dem = oracle.DemagPlan(*n, *h)
    ref = m0.copy()
    for _ in range(steps):
        ref = llg.rk4_step(ref, dt, prm, dem.apply)
    plan = Plan(*n, *h)
    assert plan.padded()[0] == 1024
    m = to_dev(torch, m0)
    gp = _gpu_params(torch, prm)
    plan.profile(True)
    for _ in range(steps):
        plan.llg_step(m, gp, dt)
    kern, _ = plan.profile_read()
    assert kern["x_c2r_rk4"][1] == 4 * steps and kern["llg_stage"][1] == 0
    assert_close(m.cpu().numpy(), ref, 1e-5)


def test_fused_and_separate_stage_agree(monkeypatch):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    n, h = (400, 64, 4), (4e-9, 4e-9, 4e-9)
    prm, m0 = _problem(n, h, True, seed=12)
    monkeypatch.setenv("BORIS_FUSE_STAGE", "1")
    fused = Plan(*n, *h)
    monkeypatch.setenv("BORIS_FUSE_STAGE", "0")
    sep = Plan(*n, *h)
    gp = _gpu_params(torch, prm)
    a, b = to_dev(torch, m0), to_dev(torch, m0)
    sep.profile(True)
    for _ in range(4):
        fused.llg_step(a, gp, 1e-13)
        sep.llg_step(b, gp, 1e-13)
    kern, _ = sep.profile_read()
    assert kern["x_c2r_rk4"][1] == 0 and kern["llg_stage"][1] == 16
    assert_close(a.cpu().numpy(), b.cpu().numpy(), 1e-6, 1e-6 * 10)
