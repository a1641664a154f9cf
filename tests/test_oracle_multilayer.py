"""Pins for the oracle's multi-mesh demag (Eq. 4): the inter-mesh tensor for
cells of unequal z size against its equal-size reduction, reciprocity, source
splitting and quadrature; the stacked direct sum against the single-mesh one."""
import math

import numpy as np
import pytest

import oracle
from oracle import multilayer as ml
from paper_2008_02478_gb300 import inputs


def quad_pair(R, hx, hy, a, b, npts=12):
    """-(1/(4 pi V_t)) int int d_i d_j (1/|R + u - u'|), boxes (hx, hy, a) and
    (hx, hy, b): per axis the difference of two uniform points has the
    trapezoidal weight (box convolution), integrated piecewise by Gauss-Legendre."""
    xg, wg = np.polynomial.legendre.leggauss(npts)

    def axis(p, q):
        # density of w = u - v, u ~ U(-p/2, p/2), v ~ U(-q/2, q/2), times p q
        s, d = 0.5 * (p + q), 0.5 * abs(p - q)
        knots = [-s, -d, d, s] if d > 0 else [-s, 0.0, s]
        pts, wts = [], []
        for lo, hi in zip(knots[:-1], knots[1:]):
            t = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
            w = 0.5 * (hi - lo) * wg
            dens = np.minimum(np.minimum(t + s, s - t), min(p, q))
            pts.append(t)
            wts.append(w * dens)
        return np.concatenate(pts), np.concatenate(wts)
    (px, wx), (py, wy), (pz, wz) = axis(hx, hx), axis(hy, hy), axis(a, b)
    X = R[0] + px[:, None, None]
    Y = R[1] + py[None, :, None]
    Z = R[2] + pz[None, None, :]
    W = wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
    r2 = X * X + Y * Y + Z * Z
    r3 = r2 * np.sqrt(r2)
    r5 = r3 * r2
    out = []
    for c, (u, v) in enumerate([(X, X), (Y, Y), (Z, Z), (X, Y), (X, Z), (Y, Z)]):
        D = 3 * u * v / r5 - (1.0 / r3 if c < 3 else 0.0)
        out.append(-(W * D).sum() / (4 * math.pi * hx * hy * a))
    return np.array(out)


@pytest.mark.parametrize("R", [(0, 0, 0), (1.0, 2.0, 0.5), (3.0, -1.0, 4.0), (10.0, 7.0, -3.0)])
def test_equal_thickness_reduces_to_newell(R):
    for h in [(1.0, 1.0, 1.0), (2.0, 1.5, 0.7)]:
        assert np.allclose(ml.pair_exact(*R, h[0], h[1], h[2], h[2]), oracle.newell_exact(*R, *h), rtol=1e-11,
                           atol=1e-14 * 1)


@pytest.mark.parametrize("R,hx,hy,a,b", [
    ((4.0, 1.0, 3.0), 1.0, 1.0, 2.0, 0.5),
    ((0.0, 3.0, 5.0), 1.0, 2.0, 3.0, 1.0),
    ((6.0, -2.0, -4.0), 1.5, 1.0, 1.0, 2.5),
    ((3.0, 3.0, 0.0), 1.0, 1.0, 0.5, 2.0),
])
def test_pair_vs_quadrature(R, hx, hy, a, b):
    ex = ml.pair_exact(*R, hx, hy, a, b)
    q = quad_pair(np.array(R, float), hx, hy, a, b)
    hmin = min(hx, hy, a, b)
    tol = max(1e-11, 1e-15 * (np.linalg.norm(R) / hmin) ** 6)
    assert np.abs(ex - q).max() / np.abs(q).max() < tol, (ex, q)


@pytest.mark.parametrize("R,a,b", [((50.0, 20.0, 10.0), 2.0, 5.0), ((0.0, 80.0, -40.0), 3.0, 1.0)])
def test_pair_asymptotic_vs_quadrature(R, a, b):
    asy = ml.pair_asymptotic(*R, 1.0, 1.0, a, b)
    q = quad_pair(np.array(R, float), 1.0, 1.0, a, b, npts=8)
    hr = max(a, b) / np.linalg.norm(R)
    assert np.abs(asy - q).max() / np.abs(q).max() < 20 * hr ** 4


@pytest.mark.parametrize("R", [(1.0, 2.0, 3.0), (0.0, 0.0, 2.5), (5.0, -3.0, -1.0)])
def test_reciprocity(R):
    a, b = 2.0, 0.75
    # V_t N_ts(r) = V_s N_st(-r), and each component is even under r -> -r
    lhs = a * ml.pair_exact(*R, 1.0, 1.0, a, b)
    rhs = b * ml.pair_exact(*R, 1.0, 1.0, b, a)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()


@pytest.mark.parametrize("R", [(0.0, 0.0, 3.0), (2.0, 1.0, -2.5), (4.0, 4.0, 0.0)])
def test_source_splitting(R):
    # a source box of height 2h is two boxes of height h at z -+ h/2
    a, h = 1.5, 1.0
    whole = ml.pair_exact(*R, 1.0, 1.0, a, 2 * h)
    parts = ml.pair_exact(R[0], R[1], R[2] + 0.5 * h, 1.0, 1.0, a, h) + \
        ml.pair_exact(R[0], R[1], R[2] - 0.5 * h, 1.0, 1.0, a, h)
    assert np.abs(whole - parts).max() < 1e-11 * np.abs(whole).max()


def test_stack_of_equal_layers_equals_single_mesh():
    # three 6 x 5 layers of equal thickness stacked without gaps = one 6 x 5 x 4 mesh
    h = (2e-9, 2e-9, 1.5e-9)
    stack = ml.centred_stack([(6, 5, 1), (6, 5, 2), (6, 5, 1)], [h[2]] * 3, [0.0, 0.0], h[0], h[1])
    M = inputs.random_unit(6, 5, 4, seed=3)
    layers = [M[:, 0:1], M[:, 1:3], M[:, 3:4]]
    Mc = np.concatenate([l.reshape(-1) for l in layers])
    H = ml.direct(stack, Mc)
    T = oracle.tensor_table(6, 5, 4, *h)
    ref = oracle.demag_direct(M, T)
    refc = np.concatenate([ref[:, 0:1].reshape(-1), ref[:, 1:3].reshape(-1), ref[:, 3:4].reshape(-1)])
    assert np.abs(H - refc).max() < 1e-12 * np.abs(refc).max()


def test_centred_offsets_and_positions():
    s = ml.centred_stack([(8, 8, 2), (4, 6, 1)], [2e-9, 3e-9], [1e-9], 1e-9)
    assert s.ox == [0, 2] and s.oy == [0, 1]
    assert s.zb[1] == pytest.approx(2 * 2e-9 + 1e-9)


def test_input_stack_geometry_matches_the_oracle_layout():
    """bench.py and the profiling entry lay the six-layer stack out with
    inputs.stack_geometry (the product side may not import the oracle); it must
    give the oracle's centred stack: same cell sizes, offsets and z bases."""
    from paper_2008_02478_gb300 import inputs
    d = inputs.MULTILAYER
    st = ml.centred_stack(d["layers"], d["hz"], d["gaps"], d["hxy"])
    cells, origins = inputs.stack_geometry(d["layers"], d["hz"], d["gaps"], d["hxy"])
    assert cells == [(st.hx, st.hy, h) for h in st.hz]
    for (x, y, z), ox, oy, zb in zip(origins, st.ox, st.oy, st.zb):
        assert x == ox * st.hx and y == oy * st.hy and z == zb
