"""FP64 LLG oracle: effective field, right-hand side, RK4/RKF45 steps, energies,
and the discrete adjoint of one RK4 step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain numpy, every field
SoA [3][nz][ny][nx].

Paper references (arXiv 2008.02478):
  * Eq. 1 (Section 2): Gilbert form of the LLG equation.  For |m| = 1 it is
    equivalent to the Landau-Lifshitz form used here,
        dm/dt = -gamma/(1+alpha^2) [ m x H + alpha m x (m x H) ].
  * Table 1: exchange H = (2A/(mu0 Ms)) lap(m) with homogeneous Neumann
    boundaries; uniaxial anisotropy H = (2K1/(mu0 Ms)) (m.e) e (K2 = 0);
    demagnetising field H = -sum N(r - r0) M(r).
  * Section 2: RK4 (4 field evaluations per step, Section 7) and RKF45 (4th
    order solution with embedded 5th order error estimate).
Readings where the paper is silent: the exchange stencil is the 7-point
second difference with a mirrored ghost cell (the missing neighbour equals the
cell itself); m is renormalised after every complete step, not between
stages; the RKF45 error is max over cells of |m5 - m4| and the 4th-order
solution is propagated.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MU0 = 4e-7 * math.pi
MU_B = 9.2740100783e-24  # J/T
HBAR = 1.054571817e-34  # J s
G_E = 2.00231930436256  # electron g-factor
#: gamma = mu0 * g * muB / hbar (Eq. 1 with g_rel = 1), m/(A s)
GAMMA_DEFAULT = MU0 * G_E * MU_B / HBAR


@dataclass
class Params:
    """Material and drive parameters; Ms and Ku may be scalars or per-cell maps."""
    cell: tuple  # (dx, dy, dz) in m
    Ms: object = 8e5
    A: float = 1.3e-11
    alpha: float = 0.02
    gamma: float = GAMMA_DEFAULT
    Ku: object = 0.0
    easy: tuple = (0.0, 0.0, 1.0)
    Hext: tuple = (0.0, 0.0, 0.0)
    # further Table 1 terms (oracle/terms.py): second-order uniaxial K2,
    # cubic K1/K2 with axes e1, e2 (e3 = e1 x e2), bulk or interfacial DMI
    K2: float = 0.0
    Kc1: float = 0.0
    Kc2: float = 0.0
    cubic_e1: tuple = (1.0, 0.0, 0.0)
    cubic_e2: tuple = (0.0, 1.0, 0.0)
    dmi: str = "none"
    D: float = 0.0
    # periodic axes (x, y, z): exchange and DMI neighbours wrap around; the
    # demagnetising kernel of such a mesh sums the periodic images
    pbc: tuple = (False, False, False)

    def has_extra(self):
        return self.K2 != 0.0 or self.Kc1 != 0.0 or self.Kc2 != 0.0 or (self.dmi != "none" and self.D != 0.0)

    def maps(self, shape):
        """Ms and Ku as arrays of the mesh shape [nz][ny][nx]."""
        Ms = np.broadcast_to(np.asarray(self.Ms, dtype=np.float64), shape)
        Ku = np.broadcast_to(np.asarray(self.Ku, dtype=np.float64), shape)
        return Ms, Ku


def cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1],
                     a[2] * b[0] - a[0] * b[2],
                     a[0] * b[1] - a[1] * b[0]])


def dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def laplacian(m, cell, pbc=(False, False, False)):
    """sum over axes and existing neighbours j of (m_j - m_i)/h^2 (Neumann);
    along a periodic axis (pbc[axis]) the neighbours wrap around the mesh."""
    out = np.zeros_like(m)
    # axis order in the array: 1 = z, 2 = y, 3 = x
    for ax, h, per in ((3, cell[0], pbc[0]), (2, cell[1], pbc[1]), (1, cell[2], pbc[2])):
        n = m.shape[ax]
        if per:
            out += (np.roll(m, 1, axis=ax) + np.roll(m, -1, axis=ax) - 2.0 * m) / (h * h)
            continue
        if n == 1:
            continue
        d = np.diff(m, axis=ax) / (h * h)  # m[i+1] - m[i]
        lo = [slice(None)] * 4
        hi = [slice(None)] * 4
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        out[tuple(lo)] += d   # cell i gains (m[i+1] - m[i])
        out[tuple(hi)] -= d   # cell i+1 gains (m[i] - m[i+1])
    return out


def exchange_field(m, prm: Params, Ms):
    c = 2.0 * prm.A / (MU0 * Ms)
    return c[None] * laplacian(m, prm.cell, prm.pbc)


def anisotropy_field(m, prm: Params, Ms, Ku):
    e = np.asarray(prm.easy, dtype=np.float64).reshape(3, 1, 1, 1)
    me = dot(m, e)
    return (2.0 * Ku / (MU0 * Ms) * me)[None] * e


def effective_field(m, prm: Params, demag, parts: bool = False):
    """H = H_d(Ms m) + H_ex + H_an + H_ext (+ the further terms of
    ``oracle/terms.py`` when set).  ``demag`` maps M -> H_d.  With parts,
    returns (Hd, Hex, Han, Hz) or, with further terms set, (Hd, Hex, Han, Hz,
    Hdmi) where Han includes the cubic and K2 terms and Hex uses the DMI
    boundary condition."""
    Ms, Ku = prm.maps(m.shape[1:])
    Hd = demag(Ms[None] * m)
    Han = anisotropy_field(m, prm, Ms, Ku)
    Hz = np.asarray(prm.Hext, dtype=np.float64).reshape(3, 1, 1, 1) * np.ones_like(m)
    if not prm.has_extra():
        Hex = exchange_field(m, prm, Ms)
        if parts:
            return Hd, Hex, Han, Hz
        return Hd + Hex + Han + Hz
    from . import terms
    Hex = terms.exchange_field(m, prm.cell, prm.A, Ms, prm.D, prm.dmi, prm.pbc)
    Hdmi = terms.dmi_field(m, prm.cell, prm.A, prm.D, prm.dmi, Ms, prm.pbc)
    Han = Han + terms.uniaxial_k2_field(m, prm.easy, prm.K2, Ms) \
        + terms.cubic_field(m, prm.cubic_e1, prm.cubic_e2, prm.Kc1, prm.Kc2, Ms)
    if parts:
        return Hd, Hex, Han, Hz, Hdmi
    return Hd + Hex + Han + Hz + Hdmi


def llg_rhs(m, H, prm: Params):
    gp = prm.gamma / (1.0 + prm.alpha ** 2)
    mxH = cross(m, H)
    return -gp * (mxH + prm.alpha * cross(m, mxH))


def normalise(v):
    return v / np.sqrt(dot(v, v))[None]


def rk4_step(m, dt, prm: Params, demag, normalize: bool = True):
    """Classical RK4 with one full field evaluation per stage."""
    f = lambda x: llg_rhs(x, effective_field(x, prm, demag), prm)
    k1 = f(m)
    k2 = f(m + 0.5 * dt * k1)
    k3 = f(m + 0.5 * dt * k2)
    k4 = f(m + dt * k3)
    v = m + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return normalise(v) if normalize else v


# Runge-Kutta-Fehlberg 4(5) tableau (Fehlberg 1969)
RKF_C = (0.0, 1.0 / 4, 3.0 / 8, 12.0 / 13, 1.0, 1.0 / 2)
RKF_A = (
    (),
    (1.0 / 4,),
    (3.0 / 32, 9.0 / 32),
    (1932.0 / 2197, -7200.0 / 2197, 7296.0 / 2197),
    (439.0 / 216, -8.0, 3680.0 / 513, -845.0 / 4104),
    (-8.0 / 27, 2.0, -3544.0 / 2565, 1859.0 / 4104, -11.0 / 40),
)
RKF_B4 = (25.0 / 216, 0.0, 1408.0 / 2565, 2197.0 / 4104, -1.0 / 5, 0.0)
RKF_B5 = (16.0 / 135, 0.0, 6656.0 / 12825, 28561.0 / 56430, -9.0 / 50, 2.0 / 55)


def rkf45_step(m, dt, prm: Params, demag):
    """One RKF45 trial step: returns (normalised 4th-order m, err = max |m5 - m4|)."""
    f = lambda x: llg_rhs(x, effective_field(x, prm, demag), prm)
    ks = []
    for s in range(6):
        x = m.copy()
        for j, a in enumerate(RKF_A[s]):
            x = x + dt * a * ks[j]
        ks.append(f(x))
    m4 = m + dt * sum(b * k for b, k in zip(RKF_B4, ks))
    m5 = m + dt * sum(b * k for b, k in zip(RKF_B5, ks))
    err = float(np.max(np.sqrt(dot(m5 - m4, m5 - m4))))
    return normalise(m4), err


def rkf45_next_dt(dt, err, tol, dt_min, dt_max):
    """Step-size controller: dt * clip(0.9 (tol/err)^(1/5), 0.2, 2) within bounds."""
    fac = 2.0 if err == 0.0 else min(2.0, max(0.2, 0.9 * (tol / err) ** 0.2))
    return min(dt_max, max(dt_min, dt * fac))


def energies(m, prm: Params, demag):
    """(E_demag, E_exchange, E_anisotropy, E_Zeeman) in J."""
    return energies_terms(m, prm, demag)[:4]


def energies_terms(m, prm: Params, demag):
    """(E_demag, E_exchange, E_anisotropy, E_Zeeman, E_DMI) in J; the
    anisotropy energy sums the uniaxial (K1, K2) and cubic densities of
    Table 1, exchange and DMI are -(mu0 Ms V/2) sum m.H of their fields."""
    Ms, Ku = prm.maps(m.shape[1:])
    V = prm.cell[0] * prm.cell[1] * prm.cell[2]
    f = effective_field(m, prm, demag, parts=True)
    Hd, Hex, Hz = f[0], f[1], f[3]
    e = np.asarray(prm.easy, dtype=np.float64).reshape(3, 1, 1, 1)
    Ed = -0.5 * MU0 * V * np.sum(Ms * dot(m, Hd))
    Eex = -0.5 * MU0 * V * np.sum(Ms * dot(m, Hex))
    Ean = V * np.sum(Ku * (1.0 - dot(m, e) ** 2))
    Ez = -MU0 * V * np.sum(Ms * dot(m, Hz))
    Edmi = 0.0
    if prm.has_extra():
        from . import terms
        Ean += V * np.sum(terms.uniaxial_k2_energy_density(m, prm.easy, prm.K2)
                          + terms.cubic_energy_density(m, prm.cubic_e1, prm.cubic_e2, prm.Kc1, prm.Kc2))
        Edmi = -0.5 * MU0 * V * np.sum(Ms * dot(m, f[4]))
    return Ed, Eex, Ean, Ez, Edmi


# --------------------------------------------------------------------------
# Discrete adjoint of one RK4 step (the paper has none; it serves the gradient checks)
# --------------------------------------------------------------------------
def _field_vjp(m, gH, prm: Params, demag):
    """Given gH = dL/dH, return (dL/dm, dL/dMs, dL/dKu) through H(m; Ms, Ku)
    (the base terms: demag, exchange, uniaxial K1, applied field).

    The demagnetising operator M -> -N*M is self-adjoint (N_ij = N_ji and
    N(-r) = N(r)), so its transpose is the operator itself."""
    assert not prm.has_extra(), "the adjoint covers the base field terms"
    Ms, Ku = prm.maps(m.shape[1:])
    e = np.asarray(prm.easy, dtype=np.float64).reshape(3, 1, 1, 1)
    DgH = demag(gH)
    gm = Ms[None] * DgH
    gMs = dot(m, DgH)
    c = 2.0 * prm.A / (MU0 * Ms)
    gm = gm + laplacian(c[None] * gH, prm.cell)
    gMs = gMs - (c / Ms) * dot(gH, laplacian(m, prm.cell))
    me, ge = dot(m, e), dot(gH, e)
    gm = gm + (2.0 * Ku / (MU0 * Ms) * ge)[None] * e
    gKu = 2.0 / (MU0 * Ms) * me * ge
    gMs = gMs - 2.0 * Ku / (MU0 * Ms ** 2) * me * ge
    return gm, gMs, gKu


def _rhs_vjp(m, gk, prm: Params, demag):
    """VJP of k = f(m, H(m)) = -g' [m x H + alpha m x (m x H)]."""
    gp = prm.gamma / (1.0 + prm.alpha ** 2)
    H = effective_field(m, prm, demag)
    a = cross(m, H)
    gA = -gp * gk
    gB = -gp * prm.alpha * gk
    # b = m x a :  d/dm = a x gB,  d/da = gB x m
    gm = cross(a, gB)
    ga = gA + cross(gB, m)
    # a = m x H :  d/dm = H x ga,  d/dH = ga x m
    gm = gm + cross(H, ga)
    gH = cross(ga, m)
    gmf, gMs, gKu = _field_vjp(m, gH, prm, demag)
    return gm + gmf, gMs, gKu


def rk4_step_vjp(m, dt, prm: Params, demag, g_out):
    """Gradient of <g_out, rk4_step(m)> with respect to m, Ms and Ku."""
    f = lambda x: llg_rhs(x, effective_field(x, prm, demag), prm)
    m1 = m
    k1 = f(m1)
    m2 = m + 0.5 * dt * k1
    k2 = f(m2)
    m3 = m + 0.5 * dt * k2
    k3 = f(m3)
    m4 = m + dt * k3
    k4 = f(m4)
    v = m + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    nv = np.sqrt(dot(v, v))
    mo = v / nv[None]
    gv = (g_out - mo * dot(mo, g_out)[None]) / nv[None]
    gm = gv.copy()
    gk = [dt / 6.0 * gv, dt / 3.0 * gv, dt / 3.0 * gv, dt / 6.0 * gv]
    shape = m.shape[1:]
    gMs = np.zeros(shape)
    gKu = np.zeros(shape)
    stages = [m1, m2, m3, m4]
    back = [None, 0.5 * dt, 0.5 * dt, dt]  # m_s = m + back[s] * k_{s-1}
    for s in (3, 2, 1, 0):
        gms, a, b = _rhs_vjp(stages[s], gk[s], prm, demag)
        gMs += a
        gKu += b
        gm += gms
        if s > 0:
            gk[s - 1] = gk[s - 1] + back[s] * gms
    return gm, gMs, gKu
