"""Stochastic thermal field of the LLG equation ("augmented by thermal
fluctuations", Section 1 with its Ref. [7]; the field's statistics follow the
fluctuation-dissipation form of Eq. 17), FP64 numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Brown's thermal field enters H_eff of the LLG equation as an uncorrelated
Gaussian field with zero mean; over a time step dt each component of each
cell of volume V has standard deviation

    sigma = sqrt(2 alpha k_B T / (gamma mu0 Ms V dt))       (gamma in m/(A s)).

(Eq. 17 states the LLB form, where the field enters the damping torque only
and carries a factor 1/alpha_perp; the fluctuation-dissipation balance is
the same.  Which placement and magnitude are right is pinned by the
Boltzmann distribution of a macrospin, see tests/test_oracle_thermal.py.)
The field is drawn once per step and held through the step's Runge-Kutta
stages.

Random numbers: the counter-based generator Philox4x32-10 (Salmon, Moraes,
Dror and Shaw, SC'11), written here from its published definition: ten
rounds of (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)) with M0 = 0xD2511F53, M1 = 0xCD9E8D57, the
key bumped by (0x9E3779B9, 0xBB67AE85) between rounds.  Cell i at step s
uses the counter (i, s mod 2^32, s div 2^32, 0) and the key (seed mod 2^32,
seed div 2^32); its four words give uniforms u_j = (x_j + 1/2) 2^-32 and,
by the Box-Muller transform, the field components
    g_x = sqrt(-2 ln u0) cos(2 pi u1), g_y = sqrt(-2 ln u0) sin(2 pi u1),
    g_z = sqrt(-2 ln u2) cos(2 pi u3).
"""
from __future__ import annotations

import numpy as np

MU0 = 4e-7 * np.pi
KB = 1.380649e-23  # J/K

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 on uint64 arrays holding 32-bit words."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & np.uint64(_MASK) for v in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & _MASK)
    k1 = np.uint64(int(k1) & _MASK)
    m0, m1, mask = np.uint64(M0), np.uint64(M1), np.uint64(_MASK)
    for r in range(10):
        p0 = c0 * m0  # < 2^64: exact in uint64
        p1 = c2 * m1
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r < 9:
            k0 = (k0 + np.uint64(W0)) & mask
            k1 = (k1 + np.uint64(W1)) & mask
    return c0, c1, c2, c3


def gaussians(ncell, step, seed):
    """Standard normal field g[3][ncell] of step `step` (Box-Muller on Philox words)."""
    i = np.arange(ncell, dtype=np.uint64)
    s = int(step)
    x0, x1, x2, x3 = philox4x32_10(i, s & _MASK, (s >> 32) & _MASK, 0, seed & _MASK, (seed >> 32) & _MASK)
    u = [(x.astype(np.float64) + 0.5) * 2.0 ** -32 for x in (x0, x1, x2, x3)]
    ra = np.sqrt(-2.0 * np.log(u[0]))
    rb = np.sqrt(-2.0 * np.log(u[2]))
    return np.stack([ra * np.cos(2 * np.pi * u[1]), ra * np.sin(2 * np.pi * u[1]), rb * np.cos(2 * np.pi * u[3])])


def sigma(alpha, gamma, Ms, V, dt, T):
    """Per-component standard deviation of the thermal field over one step (A/m)."""
    return np.sqrt(2.0 * alpha * KB * T / (gamma * MU0 * Ms * V * dt))


def thermal_field(shape, step, seed, alpha, gamma, Ms, V, dt, T):
    """Thermal field [3][nz][ny][nx] for step `step`; Ms scalar or [nz][ny][nx]."""
    n = int(np.prod(shape))
    g = gaussians(n, step, seed).reshape((3,) + tuple(shape))
    return sigma(alpha, gamma, np.asarray(Ms, dtype=np.float64), V, dt, T) * g


def rk4_step_thermal(m, dt, prm, demag, step, seed, T):
    """One RK4 step with the thermal field of `step` held through the stages
    (``prm`` an llg.Params; the field is added to H_eff)."""
    from . import llg
    Ms, _ = prm.maps(m.shape[1:])
    V = prm.cell[0] * prm.cell[1] * prm.cell[2]
    Hth = thermal_field(m.shape[1:], step, seed, prm.alpha, prm.gamma, Ms, V, dt, T)
    f = lambda x: llg.llg_rhs(x, llg.effective_field(x, prm, demag) + Hth, prm)
    k1 = f(m)
    k2 = f(m + 0.5 * dt * k1)
    k3 = f(m + 0.5 * dt * k2)
    k4 = f(m + dt * k3)
    return llg.normalise(m + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4))
