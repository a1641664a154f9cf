"""Further effective-field terms of Table 1 and the surface exchange of Eq. 5,
FP64 numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Fields are SoA
[3][nz][ny][nx]; every field follows H = -(1/(mu0 Ms)) d(eps)/dm from the
energy density eps printed beside it in Table 1 (Appendix A).

  * Uniaxial anisotropy, second order (Table 1):
        eps = K1 (1 - (m.e)^2) + K2 (1 - (m.e)^2)^2
        H   = (2 K1/(mu0 Ms)) (m.e) e + (4 K2/(mu0 Ms)) (1 - (m.e)^2) (m.e) e
  * Cubic anisotropy (Table 1), a = m.e1, b = m.e2, c = m.e3, e3 = e1 x e2:
        eps = K1 (a^2 b^2 + a^2 c^2 + b^2 c^2) + K2 a^2 b^2 c^2
  * Bulk DMI (Table 1): eps = D m.(curl m), H = -(2D/(mu0 Ms)) curl m, with the
    non-homogeneous Neumann boundary condition dm/dn = (D/2A) n x m.
  * Interfacial DMI (Table 1): eps = -D m.((div m) z - grad m_z),
    H = (2D/(mu0 Ms)) ((div m) z - grad m_z), boundary dm/dn = (D/2A)(z x n) x m.
  * Surface exchange between two layers (Eq. 5):
        eps = -(J1/Delta) m_i.m_j - (J2/Delta) (m_i.m_j)^2
        H_i = (J1/(mu0 Ms Delta)) m_j + (2 J2/(mu0 Ms Delta)) (m_i.m_j) m_j

Readings where the paper gives the continuum form only:
  * first derivatives are central differences (m_+ - m_-)/(2h) per axis;
  * a neighbour outside the mesh is the ghost value m + h dm/dn, with dm/dn
    from the boundary condition at the cell itself (n the outward normal);
    the same ghosts enter the exchange Laplacian, so with D = 0 (or no DMI)
    the exchange is the homogeneous-Neumann stencil of ``llg.laplacian``;
  * the DMI and exchange energies are -(mu0 Ms V/2) sum m.H of their fields;
  * Delta of Eq. 5 is the z size of the interface cell that receives the
    field (the layer thickness when the layer is one cell thick).
"""
from __future__ import annotations

import numpy as np

MU0 = 4e-7 * np.pi

#: boundary-condition kinds of the DMI terms
DMI_KINDS = ("none", "bulk", "interfacial")


def _cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------------------
# anisotropy
# ---------------------------------------------------------------------------
def uniaxial_k2_energy_density(m, e, K2):
    me = _dot(m, np.asarray(e, dtype=np.float64).reshape(3, *([1] * (m.ndim - 1))))
    return K2 * (1.0 - me ** 2) ** 2


def uniaxial_k2_field(m, e, K2, Ms):
    e = np.asarray(e, dtype=np.float64).reshape(3, *([1] * (m.ndim - 1)))
    me = _dot(m, e)
    return (4.0 * K2 / (MU0 * Ms) * (1.0 - me ** 2) * me)[None] * e


def cubic_axes(e1, e2):
    e1 = _unit(e1)
    e2 = _unit(e2)
    return e1, e2, np.cross(e1, e2)


def cubic_energy_density(m, e1, e2, K1, K2):
    a1, a2, a3 = cubic_axes(e1, e2)
    sh = (3,) + (1,) * (m.ndim - 1)
    a, b, c = (_dot(m, ax.reshape(sh)) for ax in (a1, a2, a3))
    return K1 * (a * a * b * b + a * a * c * c + b * b * c * c) + K2 * a * a * b * b * c * c


def cubic_field(m, e1, e2, K1, K2, Ms):
    a1, a2, a3 = cubic_axes(e1, e2)
    sh = (3,) + (1,) * (m.ndim - 1)
    E1, E2, E3 = (ax.reshape(sh) for ax in (a1, a2, a3))
    a, b, c = _dot(m, E1), _dot(m, E2), _dot(m, E3)
    f1 = -2.0 * K1 / (MU0 * Ms)
    f2 = -2.0 * K2 / (MU0 * Ms)
    H = (f1 * a * (b * b + c * c))[None] * E1 + (f1 * b * (a * a + c * c))[None] * E2 \
        + (f1 * c * (a * a + b * b))[None] * E3
    H = H + (f2 * a * b * b * c * c)[None] * E1 + (f2 * a * a * b * c * c)[None] * E2 \
        + (f2 * a * a * b * b * c)[None] * E3
    return H


# ---------------------------------------------------------------------------
# exchange with the DMI boundary condition, and DMI
# ---------------------------------------------------------------------------
_ZHAT = np.array([0.0, 0.0, 1.0])


def _bc_vector(kind, n):
    """u with dm/dn = (D/2A) u x m on a face with outward normal n."""
    n = np.asarray(n, dtype=np.float64)
    if kind == "bulk":
        return n
    if kind == "interfacial":
        return np.cross(_ZHAT, n)
    return np.zeros(3)


def padded(m, cell, A=0.0, D=0.0, kind="none", pbc=(False, False, False)):
    """m with one ghost layer on each face (array axes 1 = z, 2 = y, 3 = x).
    Ghost = m_face + h (D/2A) u x m_face (u from the boundary condition);
    with no DMI the ghost equals the face cell; along a periodic axis it is
    the cell on the opposite face (the neighbour across the period).  Edge
    and corner entries of the padded array are never read."""
    nz, ny, nx = m.shape[1:]
    p = np.zeros((3, nz + 2, ny + 2, nx + 2))
    p[:, 1:-1, 1:-1, 1:-1] = m
    k = 0.0 if (kind == "none" or D == 0.0) else D / (2.0 * A)
    # (array axis, cell size, unit vector of the axis)
    axes = ((3, cell[0], np.array([1.0, 0, 0])), (2, cell[1], np.array([0, 1.0, 0])), (1, cell[2], np.array([0, 0, 1.0])))
    for ax, h, e in axes:
        per = pbc[3 - ax]
        for side, sgn in ((0, -1.0), (-1, 1.0)):
            face = [slice(None), slice(1, -1), slice(1, -1), slice(1, -1)]
            ghost = list(face)
            face[ax] = slice(1, 2) if side == 0 else slice(-2, -1)
            ghost[ax] = slice(0, 1) if side == 0 else slice(-1, None)
            if per:
                far = list(face)
                far[ax] = slice(-2, -1) if side == 0 else slice(1, 2)
                p[tuple(ghost)] = p[tuple(far)]
                continue
            mf = p[tuple(face)]
            u = _bc_vector(kind, sgn * e).reshape(3, 1, 1, 1)
            p[tuple(ghost)] = mf + h * k * _cross(np.broadcast_to(u, mf.shape), mf)
    return p


def _shift(p, ax, d):
    """Neighbour values m(cell + d along array axis ax) from the padded array."""
    s = [slice(None), slice(1, -1), slice(1, -1), slice(1, -1)]
    n = p.shape[ax]
    s[ax] = slice(1 + d, n - 1 + d)
    return p[tuple(s)]


def exchange_field(m, cell, A, Ms, D=0.0, kind="none", pbc=(False, False, False)):
    """(2A/(mu0 Ms)) sum over axes (m_+ + m_- - 2m)/h^2 with boundary ghosts."""
    p = padded(m, cell, A, D, kind, pbc)
    lap = np.zeros_like(m)
    for ax, h in ((3, cell[0]), (2, cell[1]), (1, cell[2])):
        lap += (_shift(p, ax, 1) + _shift(p, ax, -1) - 2.0 * m) / (h * h)
    return (2.0 * A / (MU0 * Ms))[None] * lap if np.ndim(Ms) else 2.0 * A / (MU0 * Ms) * lap


def gradients(m, cell, A, D, kind, pbc=(False, False, False)):
    """d m / d(x, y, z): central differences with boundary ghosts, [axis][comp]..."""
    p = padded(m, cell, A, D, kind, pbc)
    out = []
    for ax, h in ((3, cell[0]), (2, cell[1]), (1, cell[2])):
        out.append((_shift(p, ax, 1) - _shift(p, ax, -1)) / (2.0 * h))
    return out  # out[a][c] = d m_c / d x_a


def dmi_field(m, cell, A, D, kind, Ms, pbc=(False, False, False)):
    if kind == "none" or D == 0.0:
        return np.zeros_like(m)
    dx, dy, dz = gradients(m, cell, A, D, kind, pbc)
    c = 2.0 * D / (MU0 * Ms)
    if kind == "bulk":
        curl = np.stack([dy[2] - dz[1], dz[0] - dx[2], dx[1] - dy[0]])
        return -c * curl
    if kind == "interfacial":
        return c * np.stack([-dx[2], -dy[2], dx[0] + dy[1]])
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# surface exchange (Eq. 5)
# ---------------------------------------------------------------------------
def surface_exchange_field(mi, mj, J1, J2, Ms, delta):
    c = 1.0 / (MU0 * Ms * delta)
    return c * (J1 * mj + 2.0 * J2 * _dot(mi, mj)[None] * mj) if np.ndim(mi) > 1 else \
        c * (J1 * mj + 2.0 * J2 * np.dot(mi, mj) * mj)


def surface_exchange_energy_density(mi, mj, J1, J2, delta):
    d = _dot(mi, mj) if np.ndim(mi) > 1 else np.dot(mi, mj)
    return -(J1 / delta) * d - (J2 / delta) * d * d
