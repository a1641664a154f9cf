"""Pins for the oracle's demagnetising field (Table 1; Section 7 convolution
theorem with zero padding to twice the mesh size)."""
import numpy as np
import pytest

import oracle
from paper_2008_02478_gb300 import inputs


@pytest.mark.parametrize("n", [1, 2, 8, 64, 400, 768, 7, 13, 12, 30])
def test_fft1d_matches_library(n):
    x = inputs.rng(n).standard_normal(n) + 1j * inputs.rng(n + 1).standard_normal(n)
    assert np.abs(oracle.fft1d(x, -1) - np.fft.fft(x)).max() < 1e-12 * max(1, n)
    assert np.abs(oracle.fft1d(x, +1) - np.fft.ifft(x) * n).max() < 1e-12 * max(1, n)


def test_fft3d_matches_library():
    a = inputs.rng(3).standard_normal((6, 10, 8)) + 0j
    assert np.abs(oracle.fft3d(a, -1) - np.fft.fftn(a)).max() < 1e-11


@pytest.mark.parametrize("n,h", [
    ((32, 32, 4), (5e-9, 5e-9, 5e-9)),   # the small cubic-cell mesh
    ((7, 5, 3), (1e-9, 2e-9, 1.5e-9)),   # ragged, non-power-of-two
    ((12, 9, 1), (2e-9, 2e-9, 3e-9)),    # 2D mode (nz = 1)
    ((1, 6, 5), (1e-9, 1e-9, 1e-9)),     # degenerate x
    ((1, 1, 1), (1e-9, 1e-9, 1e-9)),     # single cell
])
def test_fft_convolution_equals_direct_sum(n, h):
    nx, ny, nz = n
    M = 8e5 * inputs.random_unit(nx, ny, nz, seed=1)
    plan = oracle.DemagPlan(nx, ny, nz, *h)
    Hf = plan.apply(M)
    Hd = oracle.demag_direct(M, plan.table)
    err = np.linalg.norm(Hf - Hd) / np.linalg.norm(Hd)
    assert err < 1e-12, err


def test_direct_sum_at_samples_matches_full():
    nx, ny, nz = 9, 7, 3
    M = inputs.random_unit(nx, ny, nz, seed=4)
    T = oracle.tensor_table(nx, ny, nz, 1.0, 1.0, 1.0)
    H = oracle.demag_direct(M, T)
    cells = np.array([0, 5, 17, nx * ny * nz - 1])
    Hs = oracle.demag_direct_at(M, T, cells)
    assert np.allclose(Hs, H.reshape(3, -1)[:, cells].T, rtol=0, atol=1e-14)


def test_kernel_spectrum_is_real():
    plan = oracle.DemagPlan(8, 6, 4, 1.0, 1.5, 2.0)
    K = plan.spectrum()
    assert np.abs(K.imag).max() <= 1e-13 * np.abs(K.real).max()


def test_padding_is_twice_the_mesh():
    assert oracle.DemagPlan(8, 5, 1, 1, 1, 1).padded_dims() == (16, 10, 1)


def test_uniform_cube_single_cell():
    M = np.zeros((3, 1, 1, 1))
    M[:, 0, 0, 0] = (3.0, -1.0, 2.0)
    H = oracle.DemagPlan(1, 1, 1, 2e-9, 2e-9, 2e-9).apply(M)
    assert np.allclose(H[:, 0, 0, 0], -M[:, 0, 0, 0] / 3.0, rtol=1e-14, atol=0)


def test_uniform_prism_mean_field():
    # mean field of a uniformly magnetised prism = -N_prism M (prism identity)
    nx, ny, nz, h = 10, 6, 3, (1.0, 1.0, 2.0)
    M = inputs.uniform(nx, ny, nz, (0.2, -0.5, 1.0))
    H = oracle.DemagPlan(nx, ny, nz, *h, rs=1e9).apply(M)
    Np = oracle.newell_exact(0, 0, 0, nx * h[0], ny * h[1], nz * h[2])
    N = np.array([[Np[0], Np[3], Np[4]], [Np[3], Np[1], Np[5]], [Np[4], Np[5], Np[2]]])
    assert np.allclose(H.reshape(3, -1).mean(axis=1), -N @ M[:, 0, 0, 0], rtol=1e-11, atol=1e-14)


def test_demag_is_self_adjoint():
    nx, ny, nz = 11, 6, 3
    plan = oracle.DemagPlan(nx, ny, nz, 1e-9, 1.2e-9, 0.8e-9)
    a = inputs.random_unit(nx, ny, nz, seed=7)
    b = inputs.random_unit(nx, ny, nz, seed=8)
    lhs = np.sum(b * plan.apply(a))
    rhs = np.sum(plan.apply(b) * a)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # and it is negative semi-definite: the magnetostatic energy is >= 0
    assert np.sum(a * plan.apply(a)) < 0
