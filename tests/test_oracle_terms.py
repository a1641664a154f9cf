"""Pins of the oracle's further field terms (``oracle/terms.py``): Table 1
cubic and second-order uniaxial anisotropy, bulk and interfacial DMI with
their non-homogeneous Neumann boundary conditions, and the surface exchange of
Eq. 5.  Each pin is fixed by something other than the field formula itself:
the energy density printed beside it (field = -(1/(mu0 Ms)) d eps/dm), closed
forms for spin spirals, the chirality and convergence of the bulk-DMI helix
with its boundary condition, an embedding of every boundary ghost in a larger
mesh, and closed-form two-macrospin dynamics."""
import numpy as np
import pytest

from oracle import llg
from oracle import terms as T

MU0 = 4e-7 * np.pi
pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def rot_axes(seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q[:, 0], q[:, 1]


def random_unit(shape, seed):
    v = np.random.default_rng(seed).normal(size=(3,) + shape)
    return v / np.linalg.norm(v, axis=0)


def fd_gradient(eps, m, h=1e-6):
    """d eps / dm by central differences in each Cartesian component."""
    g = np.zeros_like(m)
    for c in range(3):
        d = np.zeros_like(m)
        d[c] = h
        g[c] = (eps(m + d) - eps(m - d)) / (2 * h)
    return g


# --------------------------------------------------------------------------- anisotropy
@pytest.mark.parametrize("K1,K2", [(4.5e4, 0.0), (-2e4, 1.5e4), (0.0, 3e4)])
def test_cubic_field_is_minus_energy_gradient(K1, K2):
    e1, e2 = rot_axes(3)
    m = random_unit((5,), 1)
    Ms = 7e5
    H = T.cubic_field(m, e1, e2, K1, K2, Ms)
    g = fd_gradient(lambda x: T.cubic_energy_density(x, e1, e2, K1, K2), m)
    assert np.allclose(H, -g / (MU0 * Ms), rtol=1e-7, atol=1e-9 * np.abs(H).max())


def test_uniaxial_k2_field_is_minus_energy_gradient():
    e = np.array([0.3, -0.5, 0.8])
    e /= np.linalg.norm(e)
    m = random_unit((6,), 2)
    Ms, K2 = 9e5, 2.2e4
    H = T.uniaxial_k2_field(m, e, K2, Ms)
    g = fd_gradient(lambda x: T.uniaxial_k2_energy_density(x, e, K2), m)
    assert np.allclose(H, -g / (MU0 * Ms), rtol=1e-7, atol=1e-9 * np.abs(H).max())
    # torque-free along the axis and perpendicular to it
    for v in (e, -e, np.cross(e, [1.0, 0, 0]) / np.linalg.norm(np.cross(e, [1.0, 0, 0]))):
        assert np.linalg.norm(np.cross(v, T.uniaxial_k2_field(v, e, K2, Ms))) < 1e-9


def test_cubic_extrema_on_axes_and_diagonals():
    """K1 > 0: the cube axes are minima (eps = 0) and the body diagonals
    maxima (eps = K1/3 + K2/27); both are torque-free.  K1 < 0 swaps them."""
    e1, e2 = rot_axes(5)
    e3 = np.cross(e1, e2)
    Ms = 8e5
    for K1, K2 in ((5e4, 0.0), (5e4, 2e4), (-5e4, 0.0)):
        for v in (e1, -e2, e3):
            assert abs(T.cubic_energy_density(v, e1, e2, K1, K2)) < 1e-9
            assert np.linalg.norm(np.cross(v, T.cubic_field(v, e1, e2, K1, K2, Ms))) < 1e-9
        d = (e1 + e2 + e3) / np.sqrt(3)
        assert T.cubic_energy_density(d, e1, e2, K1, K2) == pytest.approx(K1 / 3 + K2 / 27, rel=1e-12)
        assert np.linalg.norm(np.cross(d, T.cubic_field(d, e1, e2, K1, K2, Ms))) < 1e-9 * abs(K1) / (MU0 * Ms)
        # a nearby direction: axes are minima for K1 > 0, maxima for K1 < 0
        w = (e1 + 0.05 * e2) / np.linalg.norm(e1 + 0.05 * e2)
        assert (T.cubic_energy_density(w, e1, e2, K1, K2) > 0) == (K1 > 0)


# --------------------------------------------------------------------------- DMI
def spiral(N, h, q, axis, kind):
    """Spin spiral along `axis` (0 = x, 1 = y, 2 = z) on a 1D chain: a cycloid
    (rotation in the plane of the axis and z) for interfacial DMI, a helix
    (rotation in the plane normal to the axis) for bulk DMI."""
    shape = [1, 1, 1]
    shape[2 - axis] = N
    s = (np.arange(N) + 0.5) * h
    m = np.zeros((3,) + tuple(shape))
    a, b = np.sin(q * s).reshape(shape), np.cos(q * s).reshape(shape)
    if kind == "interfacial":
        m[axis] = a
        m[2] = b
    else:
        u, v = [(1, 2), (2, 0), (0, 1)][axis]
        m[u] = a
        m[v] = b
    return m


@pytest.mark.parametrize("kind,axis", [("interfacial", 0), ("interfacial", 1), ("bulk", 0), ("bulk", 1), ("bulk", 2)])
def test_dmi_spiral_interior_closed_form(kind, axis):
    """Away from the ends, central differences of a spiral of wave number q
    give derivative factor sin(qh)/h, and the DMI field is parallel to m:
    interfacial cycloid H = +(2D/(mu0 Ms)) (sin qh/h) m; bulk helix
    H = -(2D/(mu0 Ms)) (sin qh/h) m (curl m = q m for these helices).  The
    chain is one cell wide across the spiral, so its side faces would add
    boundary terms; a very large A makes the boundary slope D/2A vanish and
    leaves the chain's own differences."""
    N, h, q, D, Ms = 24, 0.7e-9, 2.1e8, 2.5e-3, 9e5
    m = spiral(N, h, q, axis, kind)
    H = T.dmi_field(m, (h, h, h), 1e30, D, kind, Ms)
    c = 2 * D / (MU0 * Ms) * np.sin(q * h) / h
    sign = 1.0 if kind == "interfacial" else -1.0
    inner = [slice(None)] + [slice(None)] * 3
    inner[3 - axis] = slice(1, N - 1)
    assert np.allclose(H[tuple(inner)], sign * c * m[tuple(inner)], rtol=1e-10, atol=1e-6 * c)


def test_bulk_dmi_helix_boundary_condition_chirality_and_order():
    """A chain with exchange and bulk DMI: the continuum helix of wave number
    -D/(2A) meets dm/dn = (D/2A) n x m exactly, so its discrete torque is
    zero inside and vanishes at first order at the ends; the opposite
    chirality violates the boundary condition and its end torque grows as
    1/h."""
    A, D, Ms, L = 1.3e-11, 3e-3, 8e5, 40e-9
    q = D / (2 * A)
    ends_ok, ends_bad = [], []
    for N in (16, 32, 64):
        h = L / N
        for qq, store in ((-q, ends_ok), (q, ends_bad)):
            m = spiral(N, h, qq, 0, "bulk")
            H = T.exchange_field(m, (h, h, h), A, Ms, D, "bulk") + T.dmi_field(m, (h, h, h), A, D, "bulk", Ms)
            t = np.linalg.norm(np.cross(m[:, 0, 0].T, H[:, 0, 0].T), axis=1) / (2 * A / (MU0 * Ms) * q * q)
            assert t[1:-1].max() < 1e-9 if qq < 0 else True
            store.append(max(t[0], t[-1]))
    assert ends_ok[0] < 0.2 and ends_ok[1] / ends_ok[0] == pytest.approx(0.5, abs=0.05)
    assert ends_ok[2] / ends_ok[1] == pytest.approx(0.5, abs=0.05)
    assert ends_bad[2] / ends_bad[1] == pytest.approx(2.0, abs=0.1) and ends_bad[0] > 5


# outward normal -> u with dm/dn = (D/2A) u x m, worked out by hand from
# Table 1: bulk u = n; interfacial u = z x n (z x x = y, z x y = -x, z x z = 0)
U_BY_HAND = {
    "bulk": {(1, 0, 0): (1, 0, 0), (-1, 0, 0): (-1, 0, 0), (0, 1, 0): (0, 1, 0), (0, -1, 0): (0, -1, 0),
             (0, 0, 1): (0, 0, 1), (0, 0, -1): (0, 0, -1)},
    "interfacial": {(1, 0, 0): (0, 1, 0), (-1, 0, 0): (0, -1, 0), (0, 1, 0): (-1, 0, 0), (0, -1, 0): (1, 0, 0),
                    (0, 0, 1): (0, 0, 0), (0, 0, -1): (0, 0, 0)},
}


@pytest.mark.parametrize("kind", ["bulk", "interfacial"])
def test_dmi_boundary_ghosts_by_embedding(kind):
    """The field of every face cell equals the field of the same cell inside a
    mesh one cell larger on that face, whose extra layer holds the ghost
    m + h (D/2A) u x m with u taken from the hand-derived table; this pins
    the orientation of every face's boundary condition."""
    A, D, Ms = 1.1e-11, 2.7e-3, 7.5e5
    cell = (0.8e-9, 1.1e-9, 0.9e-9)
    n = (5, 4, 3)  # nx, ny, nz
    m = random_unit((n[2], n[1], n[0]), 11)
    k = D / (2 * A)
    H = T.exchange_field(m, cell, A, Ms, D, kind) + T.dmi_field(m, cell, A, D, kind, Ms)
    for ax in range(3):  # 0 = x, 1 = y, 2 = z
        for sgn in (-1, 1):
            nrm = [0, 0, 0]
            nrm[ax] = sgn
            u = np.array(U_BY_HAND[kind][tuple(nrm)], dtype=float)
            arr_ax = 3 - ax
            face = [slice(None)] * 4
            face[arr_ax] = slice(0, 1) if sgn < 0 else slice(-1, None)
            mf = m[tuple(face)]
            ghost = mf + cell[ax] * k * np.cross(u, mf, axis=0)
            big = np.concatenate([ghost, m] if sgn < 0 else [m, ghost], axis=arr_ax)
            Hb = T.exchange_field(big, cell, A, Ms, D, kind) + T.dmi_field(big, cell, A, D, kind, Ms)
            inner = [slice(None)] * 4
            inner[arr_ax] = slice(1, 2) if sgn < 0 else slice(-2, -1)
            # in the larger mesh the face cell is interior along this axis; its
            # field depends on the ghost only through the axis neighbours
            assert np.allclose(Hb[tuple(inner)], H[tuple(face)], rtol=1e-12, atol=1e-9 * np.abs(H).max())


def test_exchange_without_dmi_is_the_neumann_laplacian():
    m = random_unit((3, 4, 5), 4)
    cell = (1e-9, 1.3e-9, 0.7e-9)
    prm = llg.Params(cell=cell, A=1.2e-11)
    ref = llg.exchange_field(m, prm, np.full(m.shape[1:], 8e5))
    assert np.allclose(T.exchange_field(m, cell, 1.2e-11, 8e5), ref, rtol=1e-13, atol=1e-12 * np.abs(ref).max())


# --------------------------------------------------------------------------- surface exchange
def test_surface_exchange_field_is_minus_energy_gradient():
    mi, mj = random_unit((7,), 6), random_unit((7,), 7)
    J1, J2, Ms, delta = -1e-3, 3e-4, 1.1e6, 2e-9
    H = T.surface_exchange_field(mi, mj, J1, J2, Ms, delta)
    g = fd_gradient(lambda x: T.surface_exchange_energy_density(x, mj, J1, J2, delta), mi)
    assert np.allclose(H, -g / (MU0 * Ms), rtol=1e-7, atol=1e-9 * np.abs(H).max())


def test_two_macrospins_precess_about_their_sum():
    """Two moments of equal Ms Delta coupled by J1 only, no damping: their sum
    S is conserved and each precesses about S at omega = gamma J1 |S|/(mu0 Ms
    Delta) (in the sense of -m x H)."""
    J1, Ms, delta, g = 1e-3, 8e5, 2e-9, llg.GAMMA_DEFAULT
    mi0 = np.array([1.0, 0.0, 0.2])
    mj0 = np.array([0.3, 1.0, -0.1])
    mi0 /= np.linalg.norm(mi0)
    mj0 /= np.linalg.norm(mj0)
    S = mi0 + mj0

    def rhs(y):
        a, b = y[:3], y[3:]
        Ha = T.surface_exchange_field(a, b, J1, 0.0, Ms, delta)
        Hb = T.surface_exchange_field(b, a, J1, 0.0, Ms, delta)
        return np.concatenate([-g * np.cross(a, Ha), -g * np.cross(b, Hb)])

    w = g * J1 * np.linalg.norm(S) / (MU0 * Ms * delta)
    t_end = 0.7 * 2 * np.pi / w
    nstep = 4000
    dt = t_end / nstep
    y = np.concatenate([mi0, mj0])
    for _ in range(nstep):
        k1 = rhs(y)
        k2 = rhs(y + 0.5 * dt * k1)
        k3 = rhs(y + 0.5 * dt * k2)
        k4 = rhs(y + dt * k3)
        y = y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    assert np.allclose(y[:3] + y[3:], S, atol=1e-10)
    # closed form: rotation of mi0 about s = S/|S| by angle -w t (dm/dt = -w s x m... sign from -m x H)
    s = S / np.linalg.norm(S)
    th = w * t_end
    par = s * np.dot(s, mi0)
    perp = mi0 - par
    expect = par + perp * np.cos(th) + np.cross(s, perp) * np.sin(th)
    assert np.allclose(y[:3], expect, atol=1e-8)


def test_dmi_energy_decreases_for_the_favoured_chirality():
    """Through llg.energies_terms on a one-cell-wide chain: the helix of the
    favoured chirality has the lower DMI energy.  The chain's side faces add
    the same -D^2/(2A) per unit volume to both chiralities (their boundary
    slopes give curl m an extra -(D/2A) m), so the sum of the two energies is
    -2 (D^2/2A) V N and their difference 2 D (sin qh/h) V N (interior closed
    form, ends aside)."""
    from oracle.llg import Params, energies_terms
    N, h, D, A = 40, 0.5e-9, 3e-3, 1.3e-11
    q = D / (2 * A)
    zero = lambda M: np.zeros_like(M)
    prm = Params(cell=(h, h, h), A=A, dmi="bulk", D=D)
    e_good = energies_terms(spiral(N, h, -q, 0, "bulk"), prm, zero)[4]
    e_bad = energies_terms(spiral(N, h, q, 0, "bulk"), prm, zero)[4]
    V = h ** 3
    assert e_good < e_bad
    assert e_good + e_bad == pytest.approx(-2 * D * D / (2 * A) * V * N, rel=1e-9)
    assert e_bad - e_good == pytest.approx(2 * D * np.sin(q * h) / h * V * N, rel=0.1)
