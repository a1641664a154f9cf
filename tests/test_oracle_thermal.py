"""Pins of the oracle's thermal field (``oracle/thermal.py``).

  * Statistical mechanics: an ensemble of independent macrospins (no exchange,
    no demag) in a field H at temperature T relaxes to the Boltzmann
    distribution, whose mean projection is the Langevin function
    <m.h> = coth(xi) - 1/xi, xi = mu0 Ms V H / (k_B T).  This fixes the
    magnitude of the field (a factor 2 in sigma^2 moves xi by 2) and its
    placement in the LLG equation.
  * The generator: the published known-answer vectors of Philox4x32-10
    (tests/golden/philox4x32_10_kat.txt, with their source) fix its rounds,
    multipliers, key schedule and word order bit for bit; beyond that, Philox
    is a bijection of the counter for a fixed key
    (distinct counters give distinct words), its uniforms are flat and its
    Box-Muller normals have unit variance and no correlation between
    components, cells, steps or seeds.
"""
import os

import numpy as np
import pytest

from oracle import llg
from oracle import thermal as th

KAT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")


def kat_vectors():
    """(counter words, key words, output words) of each published vector."""
    rows = []
    for line in open(KAT):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answer_vectors():
    rows = kat_vectors()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = th.philox4x32_10(*[np.array([c], dtype=np.uint64) for c in ctr], *key)
        assert [int(g[0]) for g in got] == want, (ctr, key)


def test_philox_known_answers_catch_plausible_mistakes():
    """Each of these slips (swapped output words, nine rounds, a wrong Weyl
    constant) changes every known-answer output, so the vectors above are a
    real pin of the round function."""
    ctr, key, want = kat_vectors()[2]

    def run(rounds=10, w0=th.W0, swap=False):
        c0, c1, c2, c3 = (np.uint64(x) for x in ctr)
        k0, k1 = np.uint64(key[0]), np.uint64(key[1])
        mask = np.uint64(0xFFFFFFFF)
        for r in range(rounds):
            p0, p1 = c0 * np.uint64(th.M0), c2 * np.uint64(th.M1)
            hi0, lo0, hi1, lo1 = p0 >> np.uint64(32), p0 & mask, p1 >> np.uint64(32), p1 & mask
            if swap:
                c0, c1, c2, c3 = hi0 ^ c1 ^ k0, lo0, hi1 ^ c3 ^ k1, lo1
            else:
                c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            k0, k1 = (k0 + np.uint64(w0)) & mask, (k1 + np.uint64(th.W1)) & mask
        return [int(c0), int(c1), int(c2), int(c3)]

    assert run() == want
    for bad in (run(rounds=9), run(w0=th.W0 + 2), run(swap=True)):
        assert all(b != w for b, w in zip(bad, want))


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
