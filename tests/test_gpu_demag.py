"""GPU parity of the demagnetising field H = -N * M (Table 1; Section 7) against
the FP64 oracle, through the C ABI.  Tolerances: relative L2 error 1e-5 for
FP32, 1e-9 for the FP64 plan (the two sides evaluate the Newell tensor with
different asinh/atan implementations; its near-field cancellation bounds the
agreement)."""
import os

import numpy as np
import pytest

import oracle
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import assert_close, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    ((32, 32, 4), (5e-9, 5e-9, 5e-9)),      # small cubic-cell mesh
    ((7, 5, 3), (1e-9, 2e-9, 1.5e-9)),      # ragged, anisotropic cells
    ((12, 9, 1), (2e-9, 2e-9, 3e-9)),       # 2D mode
    ((1, 6, 5), (1e-9, 1e-9, 1e-9)),        # degenerate x
    ((1, 1, 1), (2e-9, 2e-9, 2e-9)),        # single cell
    ((9, 1, 1), (1e-9, 1e-9, 1e-9)),        # chain
    ((50, 37, 6), (3e-9, 3e-9, 2e-9)),      # several tiles + ragged tails
    ((64, 48, 16), (4e-9, 4e-9, 4e-9)),
    ((256, 64, 1), (1.953125e-9, 1.953125e-9, 3e-9)),  # SP4-shaped film
    ((300, 280, 3), (3e-9, 3e-9, 3e-9)),    # length-1024 x and y transforms, ragged rows
    ((512, 300, 2), (4e-9, 4e-9, 4e-9)),    # full 512-cell rows
    ((40, 301, 3), (3e-9, 3e-9, 3e-9)),     # odd ny on the length-1024 y passes (one line per warp)
    ((280, 30, 3), (3e-9, 2e-9, 2e-9)),     # length-1024 x pass, ragged 16-row blocks
    ((300, 17, 2), (3e-9, 3e-9, 3e-9)),     # odd ny: the x inverse pass without tensor copies
    ((600, 21, 2), (3e-9, 3e-9, 3e-9)),     # length-2048 x passes, ragged 8-row blocks
    ((1024, 9, 1), (2e-9, 2e-9, 3e-9)),     # full 1024-cell rows, 2D mode
    ((601, 6, 3), (2e-9, 3e-9, 2e-9)),      # odd row length on the length-2048 x passes
    ((24, 700, 3), (3e-9, 2e-9, 2e-9)),     # length-2048 y passes
    ((520, 530, 2), (4e-9, 4e-9, 4e-9)),    # both in-plane axes of length 2048
    ((200, 45, 2), (3e-9, 3e-9, 3e-9)),     # length-512 x passes (two packed lines per warp), ragged 32-row blocks
    ((131, 7, 3), (2e-9, 3e-9, 2e-9)),      # shortest row of the length-512 passes, odd lengths
    ((40, 250, 3), (3e-9, 2e-9, 2e-9)),     # length-512 y passes
    ((100, 70, 3), (3e-9, 3e-9, 3e-9)),     # length-256 x and y passes (four lines per warp), ragged 64-row blocks
    ((128, 5, 2), (2e-9, 2e-9, 3e-9)),      # full 128-cell rows on the length-256 passes
    ((65, 9, 1), (2e-9, 3e-9, 2e-9)),       # shortest row of the length-256 passes, 2D mode
    ((1100, 9, 2), (2e-9, 2e-9, 3e-9)),     # length-4096 x passes, ragged 4-row blocks
    ((2048, 4, 1), (2e-9, 2e-9, 2e-9)),     # full 2048-cell rows, 2D mode
    ((1301, 6, 2), (2e-9, 3e-9, 2e-9)),     # odd row length on the length-4096 x passes
    ((10, 1500, 2), (3e-9, 2e-9, 2e-9)),    # length-4096 y passes
]


@pytest.mark.parametrize("n,h", CASES)
@pytest.mark.parametrize("fp64", [False, True])
def test_demag_matches_oracle(n, h, fp64):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    nx, ny, nz = n
    M = 8e5 * inputs.random_unit(nx, ny, nz, seed=1)
    ref = oracle.DemagPlan(nx, ny, nz, *h).apply(M)
    plan = Plan(nx, ny, nz, *h, fp64=fp64)
    H = plan.apply(to_dev(torch, M, fp64)).cpu().numpy()
    assert_close(H, ref, 1e-9 if fp64 else 1e-5)


SCHEDULE_MESHES = [
    ((40, 64, 5), (2e-9, 2e-9, 3e-9)),    # pz = 16
    ((24, 32, 17), (2e-9, 2e-9, 2e-9)),   # pz = 64, ragged nz
    ((30, 16, 3), (1e-9, 2e-9, 3e-9)),    # pz = 8 > 2 nz
    ((20, 48, 2), (2e-9, 2e-9, 2e-9)),    # pz = 4, ny not a power of two
    ((64, 40, 1), (2e-9, 2e-9, 3e-9)),    # 2D mode
    ((18, 33, 9), (2e-9, 1e-9, 2e-9)),    # pz = 32, ragged nz and ny
    ((12, 40, 3), (3e-9, 2e-9, 1e-9)),    # pz = 8, py = 128
    ((24, 20, 32), (2e-9, 2e-9, 2e-9)),   # pz = 64, nz = 32 filling the z tile (no cropped rows)
    ((12, 600, 4), (2e-9, 2e-9, 2e-9)),   # py = 2048: the length-2048 y passes of the split schedule
    ((6, 1300, 3), (2e-9, 2e-9, 2e-9)),   # py = 4096: the length-4096 y passes of the split schedule
    ((10, 170, 5), (2e-9, 2e-9, 2e-9)),   # py = 512: the length-512 y passes, odd number of lines
    ((8, 100, 3), (2e-9, 2e-9, 2e-9)),    # py = 256: the length-256 y passes, 9 lines (a partial warp)
]
# (kind, CTAs per cluster or per SM, threads | "tma1"/"tma2" for the bulk-copy z
# convolution | "tma3" for the residue-split z convolution)
SCHEDULES = [(0, 1, None), (0, 2, None), (0, 4, None), (0, 8, None), (0, 16, None),
             (1, 1, 384), (1, 1, 768), (1, 8, 384), (1, 8, 768), (1, 16, 384), (1, 16, 768), (2, 2, None), (2, 3, None),
             (2, 3, "tma1"), (2, 2, "tma2"), (2, 4, "tma3"), (2, 3, "tma3")]


@pytest.mark.parametrize("n,h", SCHEDULE_MESHES)
@pytest.mark.parametrize("kind,C,NT", SCHEDULES)
def test_every_yz_schedule_matches_oracle(n, h, kind, C, NT, monkeypatch):
    """Each schedule of the fused y-z pass (shared-memory or register z stage,
    1 to 16 CTAs per cluster) that fits the mesh gives the same field."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import BorisError, Plan
    nx, ny, nz = n
    M = 6e5 * inputs.random_unit(nx, ny, nz, seed=2)
    ref = oracle.DemagPlan(nx, ny, nz, *h).apply(M)
    monkeypatch.setenv("BORIS_YZ_KIND", str(kind))
    monkeypatch.setenv("BORIS_YZ_CLUSTER", str(C))
    if kind == 2:
        monkeypatch.setenv("BORIS_YZ_TMA", NT[3:] if NT else "0")
    elif NT:
        monkeypatch.setenv("BORIS_YZ_THREADS", str(NT))
    elif kind == 0:
        monkeypatch.setenv("BORIS_YZ_QC", "7")  # ragged z-stage chunks
    try:
        plan = Plan(nx, ny, nz, *h)
    except BorisError as e:
        assert e.code == -4  # this schedule does not fit this mesh
        pytest.skip("schedule does not fit")
    assert plan.schedule()[:2] == (kind, C)
    if kind == 2:
        assert plan.schedule()[2] == (int(NT[3:]) if NT else 0)
    H = plan.apply(to_dev(torch, M)).cpu().numpy()
    plan.sync_status()
    assert_close(H, ref, 1e-5)


def test_uniform_prism_mean_field_gpu():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    nx, ny, nz, h = 24, 16, 4, (1e-9, 1e-9, 2e-9)
    M = 1e6 * inputs.uniform(nx, ny, nz, (0.3, -0.4, 1.0))
    H = Plan(nx, ny, nz, *h).apply(to_dev(torch, M)).cpu().numpy().astype(np.float64)
    Np = oracle.newell_exact(0, 0, 0, nx * h[0], ny * h[1], nz * h[2])
    N = np.array([[Np[0], Np[3], Np[4]], [Np[3], Np[1], Np[5]], [Np[4], Np[5], Np[2]]])
    # the switch to the far-field form perturbs the prism identity at ~1e-7
    assert np.allclose(H.reshape(3, -1).mean(axis=1), -N @ M[:, 0, 0, 0], rtol=2e-6, atol=1e-2)


def test_adjoint_dot_product():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    nx, ny, nz, h = 33, 20, 6, (2e-9, 2e-9, 2e-9)
    plan = Plan(nx, ny, nz, *h, fp64=True)
    a = to_dev(torch, inputs.random_unit(nx, ny, nz, 3), True)
    b = to_dev(torch, inputs.random_unit(nx, ny, nz, 4), True)
    lhs = float((b * plan.apply(a)).sum())
    rhs = float((plan.apply(b) * a).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    p32 = Plan(nx, ny, nz, *h)
    g = p32.adjoint(b.float())
    assert rel_l2(g.cpu().numpy(), p32.apply(b.float()).cpu().numpy()) == 0.0


def test_large_film_sampled_direct_sum():
    """512 x 512 x 32 cells of 4 nm with 2621 columnar Voronoi grains: 24 random
    target cells against the oracle's O(N) direct sum at each of them."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    n, cell, seed = inputs.LARGE_FILM_MESH["n"], inputs.LARGE_FILM_MESH["cell"], inputs.LARGE_FILM_MESH["seed"]
    nx, ny, nz = n
    M = 8e5 * inputs.voronoi_columnar(nx, ny, nz, cell, 40e-9, seed)
    plan = Plan(nx, ny, nz, *cell)
    H = plan.apply(to_dev(torch, M)).cpu().numpy().reshape(3, -1)
    T = oracle.tensor_table(nx, ny, nz, *cell)
    cells = inputs.rng(7).integers(0, nx * ny * nz, 24)
    ref = oracle.demag_direct_at(M, T, cells)
    assert_close(H[:, cells].T, ref, 1e-5)
