"""Pins of the oracle's thermal field (``oracle/thermal.py``).

  * Statistical mechanics: an ensemble of independent macrospins (no exchange,
    no demag) in a field H at temperature T relaxes to the Boltzmann
    distribution, whose mean projection is the Langevin function
    <m.h> = coth(xi) - 1/xi, xi = mu0 Ms V H / (k_B T).  This fixes the
    magnitude of the field (a factor 2 in sigma^2 moves xi by 2) and its
    placement in the LLG equation.
  * The generator: Philox is a bijection of the counter for a fixed key
    (distinct counters give distinct words), its uniforms are flat and its
    Box-Muller normals have unit variance and no correlation between
    components, cells, steps or seeds.
"""
import numpy as np
import pytest

from oracle import llg
from oracle import thermal as th


def test_philox_words_are_distinct_and_uniform():
    n = 1 << 16
    i = np.arange(n, dtype=np.uint64)
    w = th.philox4x32_10(i, 7, 0, 0, 12345, 678)
    words = np.stack(w).astype(np.uint64)
    # bijection: the 128-bit outputs of distinct counters differ
    key = (words[0] << np.uint64(32)) | words[1]
    assert len(np.unique(key)) == n
    u = (words.astype(np.float64) + 0.5) / 2.0 ** 32
    hist, _ = np.histogram(u.ravel(), bins=64, range=(0, 1))
    expected = u.size / 64
    chi2 = float(((hist - expected) ** 2 / expected).sum())
    assert chi2 < 120  # 63 degrees of freedom: p ~ 1e-5 at 120


def test_gaussians_moments_and_independence():
    g = th.gaussians(1 << 16, step=3, seed=99)
    assert abs(g.mean()) < 0.01
    assert g.var() == pytest.approx(1.0, abs=0.01)
    c = np.corrcoef(g)
    assert np.abs(c - np.eye(3)).max() < 0.02
    g2 = th.gaussians(1 << 16, step=4, seed=99)
    g3 = th.gaussians(1 << 16, step=3, seed=100)
    for other in (g2, g3):
        assert abs(np.corrcoef(g[0], other[0])[0, 1]) < 0.02
    # kurtosis of a normal
    assert np.mean(g ** 4) == pytest.approx(3.0, abs=0.1)


def test_macrospin_ensemble_reaches_the_langevin_function():
    """4096 independent cubic cells (A = 0, no demag), Ms = 8e5 A/m, mu0 H =
    0.1 T along z, T = 300 K, V chosen for xi = 2: after equilibration the
    ensemble-and-time average of m_z is L(2) = coth 2 - 1/2 = 0.5373."""
    T, Ms, B = 300.0, 8e5, 0.1
    H = B / llg.MU0
    xi = 2.0
    V = xi * th.KB * T / (llg.MU0 * Ms * H)
    h = V ** (1.0 / 3.0)
    n = 4096
    prm = llg.Params(cell=(h, h, h), Ms=Ms, A=0.0, alpha=0.5, Hext=(0.0, 0.0, H))
    zero = lambda M: np.zeros_like(M)
    rng = np.random.default_rng(0)
    m = rng.normal(size=(3, 1, 1, n))
    m /= np.linalg.norm(m, axis=0)
    dt = 1e-12
    acc, cnt = 0.0, 0
    for s in range(1400):
        m = th.rk4_step_thermal(m, dt, prm, zero, step=s, seed=2024, T=T)
        if s >= 400:
            acc += m[2].mean()
            cnt += 1
    mz = acc / cnt
    L = 1.0 / np.tanh(xi) - 1.0 / xi
    assert mz == pytest.approx(L, abs=0.02)
