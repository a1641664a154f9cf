"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
comparisons.  Generators only: no step of the demag or LLG arithmetic lives here.

Every generator is deterministic in its seed (numpy PCG64) and returns FP64
numpy arrays in the SoA layout [3][nz][ny][nx] (vector fields) or [nz][ny][nx]
(scalar maps).  The shapes and value ranges stand in for the paper's workloads
(thin films, Voronoi grains, multilayer stacks): the generators below state
each recipe.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_unit(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """Independent unit vectors, uniform on the sphere (normalised N(0, I3))."""
    g = rng(seed).standard_normal((3, nz, ny, nx))
    return g / np.sqrt((g * g).sum(axis=0, keepdims=True))


def uniform(nx: int, ny: int, nz: int, direction) -> np.ndarray:
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.broadcast_to(d.reshape(3, 1, 1, 1), (3, nz, ny, nx)).copy()


def voronoi_columnar(nx: int, ny: int, nz: int, cell, grain: float, seed: int) -> np.ndarray:
    """Columnar (in-plane) Voronoi grains, each uniformly magnetised along a
    random direction.  round(Lx*Ly/grain^2) seeds, uniform in the film area;
    each cell takes the nearest seed to its centre (ties: lowest index)."""
    r = rng(seed)
    Lx, Ly = nx * cell[0], ny * cell[1]
    ns = max(1, int(round(Lx * Ly / (grain * grain))))
    sx = r.uniform(0.0, Lx, ns)
    sy = r.uniform(0.0, Ly, ns)
    d = r.standard_normal((ns, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    cx = (np.arange(nx) + 0.5) * cell[0]
    cy = (np.arange(ny) + 0.5) * cell[1]
    owner = np.empty((ny, nx), dtype=np.int64)
    # chunked nearest-seed search (argmin keeps the lowest index on ties)
    for j0 in range(0, ny, 16):
        yy = cy[j0:j0 + 16]
        dx2 = (cx[None, :, None] - sx[None, None, :]) ** 2
        dy2 = (yy[:, None, None] - sy[None, None, :]) ** 2
        owner[j0:j0 + 16] = np.argmin(dx2 + dy2, axis=2)
    m2 = d[owner]  # [ny][nx][3]
    m = np.broadcast_to(np.moveaxis(m2, 2, 0)[:, None], (3, nz, ny, nx)).copy()
    return m


def smooth_noise(nx: int, ny: int, nz: int, sigma: float, lo: float, hi: float, seed: int) -> np.ndarray:
    """White noise smoothed by a periodic Gaussian of std ``sigma`` cells (in x
    and y; columns are uniform through z), mapped affinely onto [lo, hi]."""
    w = rng(seed).standard_normal((ny, nx))
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    filt = np.exp(-2.0 * (math.pi * sigma) ** 2 * (kx * kx + ky * ky))
    s = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    s = (s - s.min()) / max(s.max() - s.min(), 1e-300)
    return np.broadcast_to((lo + (hi - lo) * s)[None], (nz, ny, nx)).copy()


def smooth_texture(nx: int, ny: int, nz: int, sigma: float, seed: int) -> np.ndarray:
    """Unit vector field from three smoothed noise components."""
    comps = [smooth_noise(nx, ny, nz, sigma, -1.0, 1.0, seed * 7 + c) for c in range(3)]
    v = np.stack(comps)
    return v / np.sqrt((v * v).sum(axis=0, keepdims=True))


# ---------------------------------------------------------------------------
# Workload descriptions
# ---------------------------------------------------------------------------
#: (nx, ny, nz) and cell size (m) of the single-mesh workloads
SMALL_CUBE_MESH = dict(n=(32, 32, 4), cell=(5e-9, 5e-9, 5e-9), seed=1)
FILM_SP4_MESH = dict(n=(256, 64, 1), cell=(1.953125e-9, 1.953125e-9, 3e-9), seed=2)
LARGE_FILM_MESH = dict(n=(512, 512, 32), cell=(4e-9, 4e-9, 4e-9), seed=3)
GRAD_FILM_MESH = dict(n=(256, 256, 8), cell=(3e-9, 3e-9, 3e-9), seed=5)

#: six stacked layers: (nx, ny, nz), z cell size (m), Ms (A/m); in-plane cell 4 nm,
#: gaps between consecutive layers (m); layers laterally centred
def stack_geometry(layers, hz, gaps, hxy):
    """Cell sizes and lower-corner origins (m) of layers laterally centred on
    the largest one (integer cell offsets) and stacked bottom-up with the given
    gaps between consecutive layers: the layout of the six-layer stack below."""
    NX = max(l[0] for l in layers)
    NY = max(l[1] for l in layers)
    cells, origins, z = [], [], 0.0
    for i, l in enumerate(layers):
        cells.append((hxy, hxy, hz[i]))
        origins.append((((NX - l[0]) // 2) * hxy, ((NY - l[1]) // 2) * hxy, z))
        z += l[2] * hz[i] + (gaps[i] if i < len(gaps) else 0.0)
    return cells, origins


MULTILAYER = dict(
    layers=[(512, 512, 8), (256, 256, 4), (384, 128, 2), (128, 128, 16), (512, 64, 1), (200, 200, 3)],
    hz=[2e-9, 5e-9, 3e-9, 4e-9, 2e-9, 3e-9],
    Ms=[8e5, 1.4e6, 4e5, 1e6, 6e5, 1.2e6],
    gaps=[1e-9, 10e-9, 2e-9, 5e-9, 3e-9],
    hxy=4e-9,
    seed=4,
)
