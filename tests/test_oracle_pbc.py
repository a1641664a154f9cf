"""Pins of the oracle's periodic boundary conditions (multiple-images method,
Section 4; periodic neighbours of the exchange and DMI stencils).

  * The image-summed kernel reproduces, to rounding, the field of an
    explicitly tiled mesh (2K + 1 copies of the magnetisation along each
    periodic axis) at the cells of the central copy, computed with the plain
    (already pinned) Newell table and direct sum.
  * The convolution-theorem demag with the image-summed table equals the
    direct sum with it.
  * A uniformly magnetised periodic thin film tends to the infinite-film
    factors N_zz -> 1, N_xx, N_yy -> 0 as the number of images grows.
  * On a periodic mesh a spin spiral of wave number 2 pi n / L is an exact
    eigenvector of the discrete exchange (factor 2 (cos kh - 1)/h^2) and, for
    interfacial DMI, of the central-difference DMI operator (sin kh / h), at
    every cell: no boundary remains.
"""
import numpy as np
import pytest

import oracle
from oracle import llg
from oracle import terms as T

MU0 = 4e-7 * np.pi


def random_unit(shape, seed):
    v = np.random.default_rng(seed).normal(size=(3,) + shape)
    return v / np.linalg.norm(v, axis=0)


@pytest.mark.parametrize("images", [(2, 0, 0), (1, 2, 0), (1, 1, 1)])
def test_image_sum_equals_tiled_mesh(images):
    nx, ny, nz = 5, 4, 2
    cell = (2e-9, 3e-9, 1.5e-9)
    kx, ky, kz = images
    M = 6e5 * random_unit((nz, ny, nx), 1)
    Tp = oracle.tensor_table_pbc(nx, ny, nz, *cell, images)
    H = oracle.demag_direct(M, Tp)
    # explicit tiling with the plain tensor
    Mt = np.tile(M, (1, 2 * kz + 1, 2 * ky + 1, 2 * kx + 1))
    _, NZ, NY, NX = Mt.shape
    Tt = oracle.tensor_table(NX, NY, NZ, *cell)
    Ht = oracle.demag_direct(Mt, Tt)
    centre = Ht[:, kz * nz:(kz + 1) * nz, ky * ny:(ky + 1) * ny, kx * nx:(kx + 1) * nx]
    assert np.allclose(H, centre, rtol=1e-11, atol=1e-11 * np.abs(centre).max())


def test_fft_with_image_table_equals_direct_sum():
    """Tolerance 1e-11: the image sums make the table's far entries (next to
    the neighbouring image) as large as its near ones, so the transforms'
    FP64 rounding relative to the field is a few times that of the plain
    kernel (1e-12 there)."""
    nx, ny, nz = 8, 6, 3
    cell = (2e-9, 2e-9, 3e-9)
    M = 8e5 * random_unit((nz, ny, nx), 2)
    Tp = oracle.tensor_table_pbc(nx, ny, nz, *cell, (3, 2, 0))
    H_direct = oracle.demag_direct(M, Tp)
    H_fft = oracle.DemagPlan(nx, ny, nz, *cell, table=Tp).apply(M)
    assert np.linalg.norm(H_fft - H_direct) / np.linalg.norm(H_direct) < 1e-11


def test_periodic_film_tends_to_infinite_film_factors():
    nx, ny, nz = 8, 8, 1
    cell = (4e-9, 4e-9, 2e-9)
    M = np.zeros((3, nz, ny, nx))
    M[2] = 1.0
    dev = []
    for K in (1, 4, 16):
        Tp = oracle.tensor_table_pbc(nx, ny, nz, *cell, (K, K, 0))
        H = oracle.demag_direct(M, Tp)
        Nzz = -H[2].mean()
        dev.append(1.0 - Nzz)
        Mx = np.zeros_like(M)
        Mx[0] = 1.0
        assert -oracle.demag_direct(Mx, Tp)[0].mean() < dev[-1]  # in-plane factor below the deficit
    assert dev[0] > dev[1] > dev[2] > 0
    assert dev[2] < 0.02


def test_periodic_exchange_and_interfacial_dmi_spiral_is_exact_everywhere():
    N, h, A, D, Ms = 24, 0.6e-9, 1.3e-11, 2.5e-3, 8e5
    k = 2 * np.pi * 3 / (N * h)
    x = (np.arange(N) + 0.5) * h
    m = np.zeros((3, 1, 1, N))
    m[0, 0, 0] = np.sin(k * x)
    m[2, 0, 0] = np.cos(k * x)
    cell = (h, h, h)
    pbc = (True, True, False)
    Hex = T.exchange_field(m, cell, A, Ms, D, "interfacial", pbc)
    Hd = T.dmi_field(m, cell, A, D, "interfacial", Ms, pbc)
    cex = 2 * A / (MU0 * Ms) * 2 * (np.cos(k * h) - 1) / (h * h)
    cd = 2 * D / (MU0 * Ms) * np.sin(k * h) / h
    assert np.allclose(Hex, cex * m, rtol=1e-10, atol=1e-9 * abs(cex))
    assert np.allclose(Hd, cd * m, rtol=1e-10, atol=1e-9 * abs(cd))
    # the base Laplacian of llg with the same periodic axes agrees
    prm = llg.Params(cell=cell, A=A, pbc=pbc)
    assert np.allclose(llg.exchange_field(m, prm, np.full(m.shape[1:], Ms)), cex * m, rtol=1e-10,
                       atol=1e-9 * abs(cex))
