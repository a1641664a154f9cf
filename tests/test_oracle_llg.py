"""Pins for the oracle's LLG step (Eq. 1; Table 1 fields; RK4/RKF45 of Section 2)
and its discrete adjoint.  Closed forms: macrospin precession and damping, the
discrete exchange spin-wave dispersion, energy balance dE/dt, convergence order,
and central finite differences for the adjoint."""
import math

import numpy as np
import pytest

import oracle
from oracle import llg
from paper_2008_02478_gb300 import inputs

MU0 = llg.MU0


def no_demag(M):
    return np.zeros_like(M)


def test_gamma_value():
    # gamma = mu0 g muB / hbar with the electron g-factor (Eq. 1, g_rel = 1)
    assert abs(llg.GAMMA_DEFAULT - 2.2127615e5) < 1.0


def test_macrospin_precession_and_damping():
    # one cubic cell: its self demag field (-M/3) is parallel to m, so only the
    # applied field along z exerts torque.  Closed form:
    # tan(theta/2) = tan(theta0/2) exp(-alpha g' H t), phi = phi0 + g' H t
    h = 5e-9
    prm = llg.Params(cell=(h, h, h), Ms=8e5, A=1.3e-11, alpha=0.1, Hext=(0.0, 0.0, 2e5))
    plan = oracle.DemagPlan(1, 1, 1, h, h, h)
    th0, ph0 = 1.0, 0.3
    m = np.array([math.sin(th0) * math.cos(ph0), math.sin(th0) * math.sin(ph0), math.cos(th0)]).reshape(3, 1, 1, 1)
    dt, nsteps = 2e-14, 500
    for _ in range(nsteps):
        m = llg.rk4_step(m, dt, prm, plan.apply)
    t = dt * nsteps
    gp = prm.gamma / (1 + prm.alpha ** 2)
    H = 2e5
    th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-prm.alpha * gp * H * t))
    ph = ph0 + gp * H * t
    exact = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    assert np.abs(m[:, 0, 0, 0] - exact).max() < 1e-9


def test_anisotropy_precession_rate():
    # alpha = 0, single cell, easy axis z: H_an = (2Ku/(mu0 Ms)) m_z z, so m
    # precesses at g' (2Ku/(mu0 Ms)) cos(theta) about z at constant theta
    h = 4e-9
    Ms, Ku = 6e5, 3e5
    prm = llg.Params(cell=(h, h, h), Ms=Ms, A=0.0, alpha=0.0, Ku=Ku, easy=(0, 0, 1))
    plan = oracle.DemagPlan(1, 1, 1, h, h, h)
    th0 = 0.4
    m = np.array([math.sin(th0), 0.0, math.cos(th0)]).reshape(3, 1, 1, 1)
    dt, nsteps = 1e-14, 300
    for _ in range(nsteps):
        m = llg.rk4_step(m, dt, prm, plan.apply)
    w = prm.gamma * 2 * Ku / (MU0 * Ms) * math.cos(th0)
    ph = math.atan2(m[1, 0, 0, 0], m[0, 0, 0, 0])
    assert abs(ph - w * dt * nsteps) < 1e-9
    assert abs(m[2, 0, 0, 0] - math.cos(th0)) < 1e-12


@pytest.mark.parametrize("mode", [0, 3, 10])
def test_discrete_spin_wave_dispersion(mode):
    # exchange + Zeeman, alpha = 0, chain along x with Neumann ends: the mode
    # cos(k (i + 1/2) h), k = pi n/(N h), precesses at
    # w = gamma [H0 + (2A/(mu0 Ms)) (2 - 2 cos(k h))/h^2]   (Section 2, Fig. 3 form)
    N, h, Ms, A, H0, eps = 48, 2e-9, 8e5, 1.3e-11, 1e5, 1e-4
    prm = llg.Params(cell=(h, 1e-9, 1e-9), Ms=Ms, A=A, alpha=0.0, Hext=(0, 0, H0))
    k = math.pi * mode / (N * h)
    u = eps * np.cos(k * (np.arange(N) + 0.5) * h)
    m = np.zeros((3, 1, 1, N))
    m[0, 0, 0] = u
    m[2, 0, 0] = np.sqrt(1 - u * u)
    w = prm.gamma * (H0 + 2 * A / (MU0 * Ms) * (2 - 2 * math.cos(k * h)) / h ** 2)
    T = 1.0 / w
    nsteps = 400
    dt = T / nsteps
    for _ in range(nsteps):
        m = llg.rk4_step(m, dt, prm, no_demag)
    z = (m[0, 0, 0] + 1j * m[1, 0, 0]) @ u / (u @ u)
    assert abs(np.angle(z) - 1.0) < 1e-6
    assert abs(abs(z) - 1.0) < 1e-6


def small_problem(alpha=0.02, seed=11, n=(6, 5, 2), per_cell=True):
    nx, ny, nz = n
    h = (3e-9, 3e-9, 3e-9)
    Ms = inputs.smooth_noise(nx, ny, nz, 2.0, 6e5, 1e6, seed) if per_cell else 8e5
    Ku = inputs.smooth_noise(nx, ny, nz, 2.0, 0.0, 5e5, seed + 1) if per_cell else 1e5
    prm = llg.Params(cell=h, Ms=Ms, A=1.3e-11, alpha=alpha, Ku=Ku, easy=(0.0, 0.0, 1.0),
                     Hext=(1e4, -2e4, 3e4))
    plan = oracle.DemagPlan(nx, ny, nz, *h)
    m0 = inputs.smooth_texture(nx, ny, nz, 1.5, seed + 2)
    return prm, plan, m0


def test_energy_conserved_without_damping():
    prm, plan, m0 = small_problem(alpha=0.0)
    drift = []
    for dt in (4e-14, 2e-14):
        m = m0.copy()
        E0 = sum(llg.energies(m, prm, plan.apply))
        for _ in range(int(round(4e-13 / dt))):
            m = llg.rk4_step(m, dt, prm, plan.apply)
        drift.append(abs(sum(llg.energies(m, prm, plan.apply)) - E0) / abs(E0))
    assert drift[0] < 1e-6
    assert drift[0] / drift[1] > 10.0  # fourth order


def test_energy_dissipation_rate():
    # dE/dt = -mu0 V sum Ms (alpha gamma/(1+alpha^2)) |m x H|^2
    prm, plan, m0 = small_problem(alpha=0.3)
    Ms, _ = prm.maps(m0.shape[1:])
    V = np.prod(prm.cell)
    H = llg.effective_field(m0, prm, plan.apply)
    mxH = llg.cross(m0, H)
    rate = -MU0 * V * np.sum(Ms * prm.alpha * prm.gamma / (1 + prm.alpha ** 2) * llg.dot(mxH, mxH))
    dt = 1e-15
    Ep = sum(llg.energies(llg.rk4_step(m0, dt, prm, plan.apply), prm, plan.apply))
    Em = sum(llg.energies(llg.rk4_step(m0, -dt, prm, plan.apply), prm, plan.apply))
    assert abs((Ep - Em) / (2 * dt) - rate) < 1e-6 * abs(rate)


def test_energy_closed_forms():
    nx, h = 16, 2e-9
    Ms, A, Ku, k = 7e5, 1.1e-11, 2e5, 0.3e9
    V = h ** 3
    prm = llg.Params(cell=(h, h, h), Ms=Ms, A=A, Ku=Ku, easy=(1.0, 0.0, 0.0), Hext=(0.0, 5e4, 0.0))
    x = (np.arange(nx) + 0.5) * h
    m = np.zeros((3, 1, 1, nx))
    m[0, 0, 0], m[1, 0, 0] = np.cos(k * x), np.sin(k * x)
    Ed, Eex, Ean, Ez = llg.energies(m, prm, no_demag)
    assert abs(Eex - A * V * (nx - 1) * (2 - 2 * math.cos(k * h)) / h ** 2) < 1e-12 * abs(Eex)
    assert abs(Ean - V * Ku * np.sum(np.sin(k * x) ** 2)) < 1e-12 * abs(Ean)
    assert abs(Ez + MU0 * V * Ms * 5e4 * np.sum(np.sin(k * x))) < 1e-12 * abs(Ez)
    # uniformly magnetised cube: E_d = mu0 V Ms^2 / 6
    plan = oracle.DemagPlan(1, 1, 1, h, h, h)
    Ed1 = llg.energies(inputs.uniform(1, 1, 1, (1, 1, 0)), llg.Params(cell=(h, h, h), Ms=Ms), plan.apply)[0]
    assert abs(Ed1 - MU0 * V * Ms ** 2 / 6) < 1e-12 * Ed1


def test_rk4_fourth_order_convergence():
    prm, plan, m0 = small_problem(alpha=0.05)
    T = 4e-13

    def run(dt):
        m = m0.copy()
        for _ in range(int(round(T / dt))):
            m = llg.rk4_step(m, dt, prm, plan.apply)
        return m
    ref = run(T / 64)
    e1 = np.abs(run(T / 4) - ref).max()
    e2 = np.abs(run(T / 8) - ref).max()
    assert 12.0 < e1 / e2 < 20.0


def test_norm_drift_fifth_order():
    prm, plan, m0 = small_problem(alpha=0.05)
    d = []
    for dt in (1e-13, 5e-14):
        v = llg.rk4_step(m0, dt, prm, plan.apply, normalize=False)
        d.append(np.abs(np.sqrt(llg.dot(v, v)) - 1).max())
    assert d[0] / d[1] > 20.0


def test_rkf45_orders():
    prm, plan, m0 = small_problem(alpha=0.05)
    errs, diffs = [], []
    for dt in (1e-13, 5e-14):
        m4, err = llg.rkf45_step(m0, dt, prm, plan.apply)
        errs.append(err)
        diffs.append(np.abs(m4 - llg.rk4_step(m0, dt, prm, plan.apply)).max())
    assert 20.0 < errs[0] / errs[1] < 45.0   # embedded estimate is O(dt^5)
    assert diffs[0] / diffs[1] > 20.0        # both 4th order: agree to O(dt^5)


def test_rkf45_controller():
    assert llg.rkf45_next_dt(1e-13, 0.0, 1e-5, 1e-16, 1e-12) == 2e-13
    assert llg.rkf45_next_dt(1e-13, 1e-2, 1e-5, 1e-16, 1e-12) == pytest.approx(2e-14)
    assert llg.rkf45_next_dt(1e-13, 1e-5, 1e-5, 1e-16, 1e-12) == pytest.approx(0.9e-13)
    assert llg.rkf45_next_dt(8e-13, 1e-9, 1e-5, 1e-16, 1e-12) == 1e-12


def loss_and_grad(m0, prm, plan, target, nsteps, dt):
    traj = [m0]
    for _ in range(nsteps):
        traj.append(llg.rk4_step(traj[-1], dt, prm, plan.apply))
    L = np.sum((traj[-1] - target) ** 2)
    g = 2 * (traj[-1] - target)
    gMs = np.zeros(m0.shape[1:])
    gKu = np.zeros(m0.shape[1:])
    for s in range(nsteps - 1, -1, -1):
        g, a, b = llg.rk4_step_vjp(traj[s], dt, prm, plan.apply, g)
        gMs += a
        gKu += b
    return L, g, gMs, gKu


def test_rk4_adjoint_vs_central_differences():
    # 8x8x2 sub-problem with per-cell Ms and Ku maps
    prm, plan, m0 = small_problem(alpha=0.02, n=(8, 8, 2))
    target = inputs.smooth_texture(8, 8, 2, 1.5, 99)
    nsteps, dt = 3, 1e-13
    L, gm, gMs, gKu = loss_and_grad(m0, prm, plan, target, nsteps, dt)
    Ms0, Ku0 = np.array(prm.Ms), np.array(prm.Ku)

    def L_of(Ms=None, Ku=None, m=None):
        p = llg.Params(cell=prm.cell, Ms=Ms0 if Ms is None else Ms, A=prm.A, alpha=prm.alpha,
                       Ku=Ku0 if Ku is None else Ku, easy=prm.easy, Hext=prm.Hext)
        x = m0 if m is None else m
        for _ in range(nsteps):
            x = llg.rk4_step(x, dt, p, plan.apply)
        return np.sum((x - target) ** 2)
    r = inputs.rng(5)
    for _ in range(4):
        idx = tuple(r.integers(0, s) for s in Ms0.shape)
        for name, base, g in (("Ms", Ms0, gMs), ("Ku", Ku0, gKu)):
            eps = 1e-6 * base.max()
            p, q = base.copy(), base.copy()
            p[idx] += eps
            q[idx] -= eps
            fd = (L_of(**{name: p}) - L_of(**{name: q})) / (2 * eps)
            assert abs(fd - g[idx]) <= 1e-6 * np.abs(g).max() + 1e-6 * abs(fd), (name, fd, g[idx])
    d = inputs.random_unit(8, 8, 2, seed=3)
    eps = 1e-6
    fd = (L_of(m=m0 + eps * d) - L_of(m=m0 - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(gm * d)) < 1e-6 * abs(fd)
