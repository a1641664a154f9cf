"""Pins for the oracle's Newell tensor (Table 1 "Demagnetizing Field", Ref. [50]).

The Newell closed form is checked against things that do not use it:
analytic self-demagnetising factors, a Gauss-Legendre quadrature of the
point-dipole kernel averaged over the two cells, the prism identity, and the
thin-film limit."""
import math

import numpy as np
import pytest

import oracle


def quad_tensor(R, h, npts=14):
    """-(1/(4 pi V)) int int d_i d_j (1/|R + u - u'|) du du' by tensor-product
    Gauss-Legendre: per axis the difference w = u - u' has weight (h - |w|) on
    [-h, h]; each half interval gets its own rule (the weight has a kink at 0)."""
    xg, wg = np.polynomial.legendre.leggauss(npts)
    axes = []
    for k in range(3):
        hk = h[k]
        # [0, h] and [-h, 0]
        t = 0.5 * hk * (xg + 1.0)
        wt = 0.5 * hk * wg * (hk - t)
        pts = np.concatenate([t, -t])
        wts = np.concatenate([wt, wt])
        axes.append((pts, wts))
    X = R[0] + axes[0][0][:, None, None]
    Y = R[1] + axes[1][0][None, :, None]
    Z = R[2] + axes[2][0][None, None, :]
    W = axes[0][1][:, None, None] * axes[1][1][None, :, None] * axes[2][1][None, None, :]
    r2 = X * X + Y * Y + Z * Z
    r5 = r2 * r2 * np.sqrt(r2)
    comps = [(X, X), (Y, Y), (Z, Z), (X, Y), (X, Z), (Y, Z)]
    V = h[0] * h[1] * h[2]
    out = []
    for c, (a, b) in enumerate(comps):
        D = 3.0 * a * b / r5
        if c < 3:
            D = D - 1.0 / (r2 * np.sqrt(r2))
        out.append(-(W * D).sum() / (4.0 * math.pi * V))
    return np.array(out)


def test_self_factors_cube():
    v = oracle.newell_exact(0, 0, 0, 1e-9, 1e-9, 1e-9)
    assert np.allclose(v[:3], 1.0 / 3.0, rtol=0, atol=1e-14)
    assert np.allclose(v[3:], 0.0, atol=1e-15)


@pytest.mark.parametrize("h", [(1.0, 2.0, 3.0), (5.0, 5.0, 1.0), (1.95, 1.95, 3.0), (4.0, 0.5, 2.0)])
def test_self_trace_is_one(h):
    v = oracle.newell_exact(0, 0, 0, *h)
    assert abs(v[:3].sum() - 1.0) < 1e-13
    assert np.all(v[:3] > 0)
    assert np.allclose(v[3:], 0.0, atol=1e-15)


def test_self_factors_prolate_ordering():
    # the longest axis has the smallest demagnetising factor
    v = oracle.newell_exact(0, 0, 0, 3.0, 1.0, 2.0)
    assert v[0] < v[2] < v[1]


def test_square_plate_analytic_limit():
    # a 1 x 1 x t plate: N_zz -> 1 - (2/pi) * t * (ln(1/t) + ...) ; check monotone -> 1
    prev = 0.0
    for t in (0.5, 0.1, 0.01, 0.001):
        nzz = oracle.newell_exact(0, 0, 0, 1.0, 1.0, t)[2]
        assert nzz > prev
        prev = nzz
    assert 1.0 - prev < 0.006


@pytest.mark.parametrize("R,h", [
    ((3.0, 0.0, 0.0), (1.0, 1.0, 1.0)),
    ((2.0, 3.0, 1.0), (1.0, 1.0, 1.0)),
    ((4.0, -2.0, 3.0), (1.0, 2.0, 0.5)),
    ((-3.0, 1.0, -5.0), (1.5, 1.0, 2.0)),
    ((0.0, 6.0, 4.0), (2.0, 2.0, 2.0)),
])
def test_exact_vs_quadrature(R, h):
    ex = oracle.newell_exact(*R, *h)
    q = quad_tensor(np.array(R, float), h)
    scale = np.abs(q).max()
    # FP64 cancellation in the 27-point second differences grows like (r/h)^6
    tol = max(1e-12, 1e-15 * (np.linalg.norm(R) / min(h)) ** 6)
    assert np.abs(ex - q).max() / scale < tol, (ex, q)


@pytest.mark.parametrize("R,h", [
    ((40.0, 0.0, 0.0), (1.0, 1.0, 1.0)),
    ((30.0, 25.0, 7.0), (1.0, 1.0, 1.0)),
    ((60.0, -50.0, 3.0), (1.95, 1.95, 3.0)),
    ((0.0, 90.0, 40.0), (2.0, 1.0, 3.0)),
])
def test_asymptotic_vs_quadrature(R, h):
    a = oracle.newell_asymptotic(*R, *h)
    q = quad_tensor(np.array(R, float), h, npts=8)
    scale = np.abs(q).max()
    hr = max(h) / np.linalg.norm(R)
    # truncation is fourth order in h/r (the h^2 term is kept)
    assert np.abs(a - q).max() / scale < 10.0 * hr ** 4, (a, q)


def test_asymptotic_second_order_term_matters():
    # for a non-cubic cell the h^2 correction is needed: dropping it is caught
    R, h = (20.0, 10.0, 5.0), (1.0, 1.0, 4.0)
    q = quad_tensor(np.array(R), h, npts=8)
    a = oracle.newell_asymptotic(*R, *h)
    x = np.array(R)
    r = np.linalg.norm(x)
    V = np.prod(h)
    dip = np.array([-(V / (4 * math.pi)) * (3 * x[i] * x[j] - (r * r if i == j else 0)) / r ** 5
                    for i, j in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]])
    err_a = np.abs(a - q).max()
    err_d = np.abs(dip - q).max()
    assert err_a < 0.05 * err_d


def test_parity_and_permutation_symmetry():
    X, Y, Z, h = 2.0, 3.0, 1.0, (1.0, 1.5, 0.7)
    base = oracle.newell_exact(X, Y, Z, *h)
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                v = oracle.newell_exact(sx * X, sy * Y, sz * Z, *h)
                expect = base * np.array([1, 1, 1, sx * sy, sx * sz, sy * sz])
                assert np.abs(v - expect).max() < 1e-12 * np.abs(base).max()
    # swapping the roles of x and y swaps xx<->yy and xz<->yz
    w = oracle.newell_exact(Y, X, Z, h[1], h[0], h[2])
    assert np.abs(w[[1, 0, 2, 3, 5, 4]] - base).max() < 1e-12 * np.abs(base).max()


def prism_average(nx, ny, nz, h, rs):
    T = oracle.tensor_table(nx, ny, nz, *h, rs=rs)
    # mean over targets of sum over sources of N(r_i - r_j): each displacement
    # (i,j,k) occurs (nx-|i|)(ny-|j|)(nz-|k|) times
    tot = np.zeros(6)
    for c in range(6):
        for k in range(-nz + 1, nz):
            for j in range(-ny + 1, ny):
                wj = ny - abs(j)
                wk = nz - abs(k)
                row = T[c, abs(k), abs(j)]
                i = np.arange(-nx + 1, nx)
                w = (nx - np.abs(i)) * wj * wk
                sgn = np.ones_like(i, dtype=float)
                if c == 3:
                    sgn = np.sign(i + 0.0) * (1 if j >= 0 else -1)
                    sgn[i == 0] = 1
                    sgn = np.where(i < 0, -1.0, 1.0) * (1 if j >= 0 else -1)
                elif c == 4:
                    sgn = np.where(i < 0, -1.0, 1.0) * (1 if k >= 0 else -1)
                elif c == 5:
                    sgn = np.ones_like(i, dtype=float) * (1 if j >= 0 else -1) * (1 if k >= 0 else -1)
                tot[c] += (w * sgn * row[np.abs(i)]).sum()
    return tot / (nx * ny * nz)


@pytest.mark.parametrize("n,h", [((4, 3, 2), (1.0, 1.0, 1.0)), ((5, 4, 3), (1.0, 2.0, 0.5)), ((6, 1, 2), (2.0, 1.0, 1.0))])
def test_prism_identity_exact(n, h):
    avg = prism_average(*n, h, rs=1e9)
    whole = oracle.newell_exact(0, 0, 0, n[0] * h[0], n[1] * h[1], n[2] * h[2])
    assert np.abs(avg - whole).max() < 1e-12, (avg, whole)


def test_prism_identity_with_far_field_switch():
    n, h = (96, 80, 2), (1.0, 1.0, 1.0)
    avg = prism_average(*n, h, rs=40.0)
    whole = oracle.newell_exact(0, 0, 0, n[0], n[1], n[2])
    assert np.abs(avg - whole).max() < 2e-6, (avg, whole)


def aharoni_dz(a, b, c):
    """Demagnetising factor along c of a uniformly magnetised 2a x 2b x 2c
    prism (A. Aharoni, J. Appl. Phys. 83, 3432 (1998)) - an independent closed
    form for the self term of the Newell tensor of one cell."""
    r = math.sqrt(a * a + b * b + c * c)
    ab, bc, ac = math.hypot(a, b), math.hypot(b, c), math.hypot(a, c)
    s = (b * b - c * c) / (2 * b * c) * math.log((r - a) / (r + a))
    s += (a * a - c * c) / (2 * a * c) * math.log((r - b) / (r + b))
    s += b / (2 * c) * math.log((ab + a) / (ab - a))
    s += a / (2 * c) * math.log((ab + b) / (ab - b))
    s += c / (2 * a) * math.log((bc - b) / (bc + b))
    s += c / (2 * b) * math.log((ac - a) / (ac + a))
    s += 2 * math.atan(a * b / (c * r))
    s += (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
    s += (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
    s += c / (a * b) * (ac + bc)
    s -= (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c)
    return s / math.pi


@pytest.mark.parametrize("L", [(1, 1, 1), (2, 1, 1), (3, 2, 1), (1, 1, 0.01), (5, 7, 11), (4.0, 4.0, 3.0)])
def test_self_term_vs_aharoni(L):
    v = oracle.newell_exact(0, 0, 0, *L)
    assert abs(v[2] - aharoni_dz(L[0] / 2, L[1] / 2, L[2] / 2)) < 1e-13
    # and the x factor from the permuted prism
    assert abs(v[0] - aharoni_dz(L[1] / 2, L[2] / 2, L[0] / 2)) < 1e-13


def test_thin_film_limit():
    # a wide thin film: N_zz of the whole prism tends to 1, in-plane factors to 0
    prev = 0.0
    for L in (20.0, 200.0, 2000.0, 20000.0):
        whole = oracle.newell_exact(0, 0, 0, L, L, 1.0)
        assert whole[2] > prev
        prev = whole[2]
        assert abs(whole[2] - aharoni_dz(L / 2, L / 2, 0.5)) < 1e-11
    assert 1.0 - prev < 5e-4 and whole[0] < 3e-4


def test_table_switch_continuity():
    # exact and asymptotic forms agree near the switch radius
    for R in [(40.0, 0, 0), (28.0, 28.0, 3.0), (39.0, 5.0, 10.0)]:
        e = oracle.newell_exact(*R, 1.0, 1.0, 1.0)
        a = oracle.newell_asymptotic(*R, 1.0, 1.0, 1.0)
        assert np.abs(e - a).max() / np.abs(e).max() < 2e-5
