"""Pins of the oracle's Oersted kernel (Table 1: H = sum K(r - r0) J; its
Ref. [63] is not in the paper): for a uniform current density J in a source
cell the target-cell average of the Biot-Savart field is J x g(D), with
g = -(1/(4 pi V)) grad P and N_ij = d_i g_j.  The oracle builds g_k by
integrating N_kk along axis k; these pins fix it by other means:

  * the cross derivatives d_x g_y and d_y g_x reproduce Newell's off-diagonal
    N_xy (a different closed form, not the integrand);
  * g is odd in its own axis: the integral from 0 to the far zone cancels
    (g_k(0, Y, Z) = 0) without that being imposed;
  * a tensor-product Gauss-Legendre quadrature of the Biot-Savart kernel
    u/|u|^3 over both cells, for separated cells;
  * continuity at the switch to the far-field form, and the point-current
    limit (V/4 pi) D/|D|^3 far away;
  * the direct sum for a long straight wire against the Biot-Savart field of
    a finite line current (H = I (cos t1 - cos t2)/(4 pi rho)).
"""
import numpy as np
import pytest

import oracle

H = (1.0e-9, 1.3e-9, 0.8e-9)


def gl_nodes(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


@pytest.mark.parametrize("D", [(1.5e-9, 0.4e-9, 0.3e-9), (0.7e-9, 2.1e-9, -0.9e-9), (3.3e-9, 1.2e-9, 2.0e-9),
                               (0.2e-9, 0.3e-9, 0.1e-9)])
def test_cross_derivatives_give_newell_off_diagonals(D):
    """Central differences with step 1e-12 m (h/1000): rounding noise of g
    (about 1e-10 relative) and the step's truncation error stay near 1e-7 of
    the tensor's scale; tolerance 1e-5."""
    d = 1e-12
    X, Y, Z = D
    gxy = (oracle.oersted_g(X + d, Y, Z, *H)[1] - oracle.oersted_g(X - d, Y, Z, *H)[1]) / (2 * d)
    gyx = (oracle.oersted_g(X, Y + d, Z, *H)[0] - oracle.oersted_g(X, Y - d, Z, *H)[0]) / (2 * d)
    gzx = (oracle.oersted_g(X, Y, Z + d, *H)[0] - oracle.oersted_g(X, Y, Z - d, *H)[0]) / (2 * d)
    N = oracle.newell_exact(X, Y, Z, *H)
    scale = np.abs(N).max()
    gyy = (oracle.oersted_g(X, Y + d, Z, *H)[1] - oracle.oersted_g(X, Y - d, Z, *H)[1]) / (2 * d)
    assert abs(gxy - N[3]) < 1e-5 * scale
    assert abs(gyx - N[3]) < 1e-5 * scale
    assert abs(gzx - N[4]) < 1e-5 * scale
    assert abs(gyy - N[1]) < 1e-5 * scale


def test_odd_in_own_axis():
    for Y, Z in ((0.0, 0.0), (1.3e-9, 0.0), (2.6e-9, 1.6e-9), (0.4e-9, 5e-9)):
        g = oracle.oersted_g(0.0, Y, Z, *H)
        ref = np.abs(oracle.oersted_g(H[0], Y + H[1], Z + H[2], *H)).max()
        assert abs(g[0]) < 1e-8 * ref
    g = oracle.oersted_g(2e-9, -1.3e-9, 0.0, *H)
    assert abs(g[2]) < 1e-8 * np.abs(g).max()
    gm = oracle.oersted_g(-2e-9, 1.3e-9, 0.8e-9, *H)
    gp = oracle.oersted_g(2e-9, 1.3e-9, 0.8e-9, *H)
    assert gm[0] == pytest.approx(-gp[0], rel=1e-12) and gm[1] == pytest.approx(gp[1], rel=1e-12)


@pytest.mark.parametrize("D", [(2.0e-9, 0.0, 0.0), (2.0e-9, 1.3e-9, 0.0), (1.0e-9, 2.6e-9, 1.6e-9),
                               (3.0e-9, -1.3e-9, 0.8e-9)])
def test_against_biot_savart_quadrature(D):
    """g = (1/(4 pi V)) int_target int_source u/|u|^3, u = r - r', for cells
    that do not touch along the separating axis."""
    x, w = gl_nodes(12)
    hx, hy, hz = H
    # points in a cell: centre + h/2 * node
    px, py, pz = np.meshgrid(x * hx / 2, x * hy / 2, x * hz / 2, indexing="ij")
    W = (np.einsum("i,j,k->ijk", w, w, w) * (hx * hy * hz) / 8).ravel()
    P = np.stack([px.ravel(), py.ravel(), pz.ravel()], axis=1)
    acc = np.zeros(3)
    for t in range(len(W)):
        u = (np.array(D) + P[t])[None, :] - P
        r3 = np.linalg.norm(u, axis=1) ** 3
        acc += W[t] * (W[:, None] * u / r3[:, None]).sum(axis=0)
    V = hx * hy * hz
    ref = acc / (4 * np.pi * V)
    g = oracle.oersted_g(*D, *H)
    assert np.allclose(g, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_far_zone_continuity_and_point_limit():
    hmax = max(H)
    for direction in (np.array([1.0, 0.3, 0.2]), np.array([0.2, -1.0, 0.5])):
        u = direction / np.linalg.norm(direction)
        inside = oracle.oersted_g(*(u * 39.9 * hmax), *H)
        outside = oracle.oersted_g(*(u * 40.1 * hmax), *H)
        # g falls as 1/r^2: compare after scaling to the same radius
        assert np.allclose(inside * 39.9 ** 2, outside * 40.1 ** 2, rtol=2e-3)
    D = np.array([300e-9, 120e-9, -80e-9])
    V = H[0] * H[1] * H[2]
    point = V / (4 * np.pi) * D / np.linalg.norm(D) ** 3
    assert np.allclose(oracle.oersted_g(*D, *H), point, rtol=1e-5)


def test_long_wire_matches_line_current():
    """A wire of 81 cells along x (cross-section one cell) carrying J_x: the
    field at a cell 6 cells away in y, opposite the middle, against the
    Biot-Savart field of a line current of the same length (the finite
    cross-section changes it at order (h/rho)^2)."""
    nx, ny, nz = 81, 7, 1
    h = (1e-9, 1e-9, 1e-9)
    G = oracle.oersted_table(nx, ny, nz, *h)
    J = np.zeros((3, nz, ny, nx))
    J[0, 0, 0, :] = 1e11  # A/m^2
    Hf = oracle.oersted_direct(J, G)
    I = 1e11 * h[1] * h[2]
    rho = 6 * h[1]
    half = nx * h[0] / 2
    c = half / np.hypot(half, rho)
    Hline = I / (4 * np.pi * rho) * 2 * c
    got = Hf[:, 0, 6, nx // 2]
    # J along +x, target at +y: H = J x g points along +z... J x (y) = +z
    assert got[2] == pytest.approx(Hline, rel=0.01)
    assert abs(got[0]) < 1e-6 * abs(got[2]) and abs(got[1]) < 1e-6 * abs(got[2])
