"""Mixed-precision variant: the zero-padded z transforms on the tensor cores
with FP16 or BF16 operands, per-column scaling and FP32 accumulation, against
the FP64 oracle.  Tolerance: relative L2 error of H_d <= 1e-2.  Both forms of
the stage are covered: tcgen05 products with tensor-memory accumulators (the
default wherever py >= 64) and the mma.sync form (BORIS_TC_MMASYNC=1, and the
only form for py < 64)."""
import numpy as np
import pytest

import oracle
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import assert_close, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    ((48, 40, 32), (4e-9, 4e-9, 4e-9)),    # pz = 64 with nz = 32
    ((37, 29, 20), (3e-9, 3e-9, 2e-9)),    # ragged: nz = 20 still pads to 64, ragged column tiles
    ((64, 300, 17), (4e-9, 4e-9, 4e-9)),   # length-1024 y transforms; several tiles per persistent CTA
    ((40, 700, 24), (4e-9, 4e-9, 4e-9)),   # py = 2048 (y passes built from the warp transform)
    ((24, 1100, 18), (4e-9, 4e-9, 4e-9)),  # py = 4096
]
FORMS = {"tcgen05": 5, "mma.sync": 4}


def tc_plan(monkeypatch, form, *args, **kw):
    """Plan with the tensor-core z stage in the given form; "tcgen05" keeps the
    FP32 spectrum (BORIS_TC_STORE16=0), "store16" the 16-bit one (BF16, or FP16
    scaled by a power of two from max |M|)."""
    from paper_2008_02478_gb300.binding import Plan
    if form == "mma.sync":
        monkeypatch.setenv("BORIS_TC_MMASYNC", "1")
    else:
        monkeypatch.delenv("BORIS_TC_MMASYNC", raising=False)
    monkeypatch.setenv("BORIS_TC_STORE16", "1" if form == "store16" else "0")
    plan = Plan(*args, **kw)
    monkeypatch.delenv("BORIS_TC_MMASYNC", raising=False)
    monkeypatch.delenv("BORIS_TC_STORE16", raising=False)
    return plan


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("n,h", CASES)
@pytest.mark.parametrize("tc", ["fp16", "bf16"])
def test_tensor_core_z_stage_matches_oracle(n, h, tc, form, monkeypatch):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    nx, ny, nz = n
    M = 8e5 * inputs.voronoi_columnar(nx, ny, nz, h, 20e-9, seed=3)
    ref = oracle.DemagPlan(nx, ny, nz, *h).apply(M)
    plan = tc_plan(monkeypatch, form, nx, ny, nz, *h, tc=tc)
    assert plan.schedule()[2] == FORMS[form]
    H = plan.apply(to_dev(torch, M)).cpu().numpy()
    err, _ = assert_close(H, ref, 1e-2)
    # and it is genuinely the reduced-precision path (not bit-equal to FP32)
    H32 = Plan(nx, ny, nz, *h).apply(to_dev(torch, M)).cpu().numpy()
    assert_close(H32, ref, 1e-5)
    assert err > rel_l2(H32, ref)


@pytest.mark.parametrize("form", list(FORMS))
def test_tensor_core_random_magnetisation(form, monkeypatch):
    torch = torch_cuda()
    n, h = (32, 24, 32), (5e-9, 5e-9, 5e-9)
    M = 8e5 * inputs.random_unit(*n, seed=1)
    ref = oracle.DemagPlan(*n, *h).apply(M)
    for tc in ("fp16", "bf16"):
        H = tc_plan(monkeypatch, form, *n, *h, tc=tc).apply(to_dev(torch, M)).cpu().numpy()
        assert_close(H, ref, 1e-2)


def test_tcgen05_and_mma_sync_forms_agree(monkeypatch):
    """The two forms round the same products to 16 bits under different column
    scales (a power of two against the exact maximum), so they agree to within
    one unit roundoff of the operand format (2^-11 FP16, 2^-8 BF16)."""
    torch = torch_cuda()
    n, h = (96, 80, 24), (3e-9, 3e-9, 3e-9)
    M = to_dev(torch, 8e5 * inputs.voronoi_columnar(*n, h, 20e-9, seed=7))
    for tc in ("fp16", "bf16"):
        a = tc_plan(monkeypatch, "tcgen05", *n, *h, tc=tc).apply(M).cpu().numpy()
        b = tc_plan(monkeypatch, "mma.sync", *n, *h, tc=tc).apply(M).cpu().numpy()
        tol = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}[tc]
        assert_close(a, b, tol, 8 * tol)


def test_tcgen05_stage_repeats_and_checks_status(monkeypatch):
    """Persistent CTAs over many tiles, applied twice: identical results, and
    no bounded wait gave up."""
    torch = torch_cuda()
    n, h = (160, 256, 32), (4e-9, 4e-9, 4e-9)
    plan = tc_plan(monkeypatch, "tcgen05", *n, *h, tc="fp16")
    M = to_dev(torch, 8e5 * inputs.random_unit(*n, seed=9))
    a = plan.apply(M).cpu().numpy()
    b = plan.apply(M).cpu().numpy()
    assert np.array_equal(a, b)
    assert plan.sync_status() == 0
    # sampled cells against the oracle's direct sum
    Mh = M.cpu().numpy().astype(np.float64)
    T = oracle.tensor_table(*n, *h)
    cells = inputs.rng(11).integers(0, n[0] * n[1] * n[2], 12)
    ref = oracle.demag_direct_at(Mh, T, cells)
    got = a.reshape(3, -1)[:, cells].T
    assert_close(got, ref, 1e-2)


def test_tensor_core_rejects_unsupported_depth():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import BorisError, Plan
    with pytest.raises(BorisError) as e:
        Plan(32, 32, 8, 1e-9, 1e-9, 1e-9, tc="fp16")
    assert e.value.code == -4


_FILM = {}


def _large_film_reference():
    """512 x 512 x 32 film of 4 nm cells with 2621 columnar Voronoi grains,
    and the oracle's O(N) direct sums at 24 sampled cells (cached)."""
    if not _FILM:
        n, cell, seed = inputs.LARGE_FILM_MESH["n"], inputs.LARGE_FILM_MESH["cell"], inputs.LARGE_FILM_MESH["seed"]
        M = 8e5 * inputs.voronoi_columnar(*n, cell, 40e-9, seed)
        T = oracle.tensor_table(*n, *cell)
        cells = inputs.rng(13).integers(0, n[0] * n[1] * n[2], 24)
        _FILM.update(n=n, cell=cell, M=M, cells=cells, ref=oracle.demag_direct_at(M, T, cells))
    return _FILM


@pytest.mark.parametrize("tc", ["fp16", "bf16"])
def test_large_film_tensor_core_stage_sampled_direct_sum(tc, monkeypatch):
    """The configuration the benchmark times: the tcgen05 z stage on the
    512 x 512 x 32 film, against the oracle's direct sum at sampled cells."""
    torch = torch_cuda()
    f = _large_film_reference()
    plan = tc_plan(monkeypatch, "tcgen05", *f["n"], *f["cell"], tc=tc)
    assert plan.schedule()[2] == FORMS["tcgen05"]
    H = plan.apply(to_dev(torch, f["M"])).cpu().numpy().reshape(3, -1)
    assert plan.sync_status() == 0
    assert_close(H[:, f["cells"]].T, f["ref"], 1e-2)


# meshes for the 16-bit-storage z stage: length-1024 x and y passes (257 <= nx, ny <= 512), pz = 64
STORE16 = [
    ((64, 300, 17), (4e-9, 4e-9, 4e-9)),    # ragged nz, partial 128-column tiles of ny
    ((48, 512, 32), (3e-9, 3e-9, 3e-9)),    # full z tile and full y lines
    ((130, 400, 24), (3e-9, 2e-9, 3e-9)),   # anisotropic cells, odd nx
    ((40, 301, 20), (3e-9, 3e-9, 3e-9)),    # odd ny: the one-line-per-warp y passes
]


@pytest.mark.parametrize("tc", ["fp16", "bf16"])
@pytest.mark.parametrize("n,h", STORE16)
def test_16bit_storage_stage_matches_oracle(n, h, tc, monkeypatch):
    """Tensor-core plans store the padded y-z spectrum in 16 bits (BF16, or
    FP16 scaled by a power of two from max |M|) and run the tcgen05 z stage
    with the data as the 128-row operand: H_d against the FP64 oracle (bound
    1e-2 on both norms), twice in a row (the persistent CTAs leave no state
    behind), with no bounded wait giving up."""
    torch = torch_cuda()
    M = 8e5 * inputs.voronoi_columnar(*n, h, 20e-9, seed=5)
    ref = oracle.DemagPlan(*n, *h).apply(M)
    plan = tc_plan(monkeypatch, "store16", *n, *h, tc=tc)
    assert plan.schedule()[2] == 6
    Md = to_dev(torch, M)
    a = plan.apply(Md).cpu().numpy()
    b = plan.apply(Md).cpu().numpy()
    assert plan.sync_status() == 0
    assert np.array_equal(a, b)
    err, _ = assert_close(a, ref, 1e-2)
    # it is the reduced-precision path, not an FP32 one
    H32 = __import__("paper_2008_02478_gb300.binding", fromlist=["Plan"]).Plan(*n, *h).apply(Md).cpu().numpy()
    assert err > 10 * rel_l2(H32, ref)


@pytest.mark.parametrize("tc", ["bf16", "fp16"])
def test_persistent_y_passes_match_one_line_per_warp(tc, monkeypatch):
    """The persistent 16-bit y passes (each warp walks many lines and stages
    the next line's input by asynchronous copies while it transforms the
    current one) give bit for bit the results of the one-line-per-warp grid:
    the same arithmetic in the same order."""
    torch = torch_cuda()
    n, h = (72, 400, 20), (3e-9, 3e-9, 3e-9)
    Md = to_dev(torch, 8e5 * inputs.voronoi_columnar(*n, h, 20e-9, seed=8))
    out = []
    for yp in ("0", "1"):
        monkeypatch.setenv("BORIS_Y_PERSIST", yp)
        plan = tc_plan(monkeypatch, "store16", *n, *h, tc=tc)
        assert plan.schedule()[2] == 6
        out.append(plan.apply(Md).cpu().numpy())
        assert plan.sync_status() == 0
        plan.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("tc", ["fp16", "bf16"])
def test_16bit_storage_stage_on_large_film(tc, monkeypatch):
    """The 512 x 512 x 32 film with the 16-bit-storage stage against the
    oracle's direct sums at sampled cells."""
    torch = torch_cuda()
    f = _large_film_reference()
    plan = tc_plan(monkeypatch, "store16", *f["n"], *f["cell"], tc=tc)
    assert plan.schedule()[2] == 6
    H = plan.apply(to_dev(torch, f["M"])).cpu().numpy().reshape(3, -1)
    assert plan.sync_status() == 0
    assert_close(H[:, f["cells"]].T, f["ref"], 1e-2)


@pytest.mark.parametrize("tc", ["fp16", "bf16"])
def test_16bit_storage_rk4_step_matches_oracle(tc, monkeypatch):
    """One RK4 step of a 16-bit-storage plan (four evaluations through the
    stage, the FP16 scale taken from Ms m) against the FP64 oracle: the change
    of m within 1e-2."""
    torch = torch_cuda()
    from oracle import llg
    from paper_2008_02478_gb300.binding import LLGParams
    n, h = (64, 300, 17), (4e-9, 4e-9, 4e-9)
    m0 = inputs.voronoi_columnar(*n, h, 20e-9, seed=6)
    prm = llg.Params(cell=h, Ms=8e5, A=1.3e-11, alpha=0.02, Hext=(0.0, 0.0, 8e4))
    ref = llg.rk4_step(m0, 1e-13, prm, oracle.DemagPlan(*n, *h).apply)
    plan = tc_plan(monkeypatch, "store16", *n, *h, tc=tc)
    m = to_dev(torch, m0)
    plan.llg_step(m, LLGParams(Ms=8e5, A=1.3e-11, alpha=0.02, Hext=(0.0, 0.0, 8e4)), 1e-13)
    assert_close(m.cpu().numpy() - m0, ref - m0, 1e-2)


@pytest.mark.parametrize("scale", [1e-6, 1.0, 1e7])
def test_fp16_storage_scale_follows_the_magnetisation(scale, monkeypatch):
    """The FP16 spectrum's power-of-two scale comes from max |M| of each
    evaluation: magnetisations 1e-6, 1 and 1e7 times the film's give fields
    scaled alike, each within the FP16 bound of the oracle (no overflow of
    the large one, no underflow of the small one), and an FP16 error below
    the BF16 one."""
    torch = torch_cuda()
    n, h = (64, 300, 17), (4e-9, 4e-9, 4e-9)
    M = 8e5 * scale * inputs.voronoi_columnar(*n, h, 20e-9, seed=8)
    ref = oracle.DemagPlan(*n, *h).apply(M)
    H16 = tc_plan(monkeypatch, "store16", *n, *h, tc="fp16").apply(to_dev(torch, M)).cpu().numpy()
    Hb = tc_plan(monkeypatch, "store16", *n, *h, tc="bf16").apply(to_dev(torch, M)).cpu().numpy()
    assert np.isfinite(H16).all()
    e16, _ = assert_close(H16, ref, 1e-3)
    eb, _ = assert_close(Hb, ref, 1e-2)
    assert e16 < eb


@pytest.mark.parametrize("n,h", [((64, 300, 17), (4e-9, 4e-9, 4e-9)),     # x length 128: separate maximum
                                 ((300, 260, 20), (4e-9, 4e-9, 4e-9))])   # x length 1024: maximum in the x pass
def test_fp16_storage_rk4_step_with_ms_map(n, h, monkeypatch):
    """An FP16-storage plan stepping a film whose Ms map spans 1e4 to 1e6 A/m:
    the spectrum's scale comes from max |Ms m| over the map (found by the x
    pass, or by the separate reduction where the x pass is not the
    length-1024 one); one RK4 step against the FP64 oracle, the change of m
    within 1e-2."""
    torch = torch_cuda()
    from oracle import llg
    from paper_2008_02478_gb300.binding import LLGParams
    # (down to 1e3 A/m the exchange field of the weakest cells turns m by order 1
    # in one 0.1 ps step, where the step itself, not the demag field, sets the
    # FP32 / FP64 difference)
    Ms = inputs.smooth_noise(*n, 3.0, 1e4, 1e6, 31)
    m0 = inputs.voronoi_columnar(*n, h, 20e-9, seed=32)
    prm = llg.Params(cell=h, Ms=Ms, A=1.3e-11, alpha=0.02, Hext=(0.0, 0.0, 8e4))
    ref = llg.rk4_step(m0, 1e-13, prm, oracle.DemagPlan(*n, *h).apply)
    plan = tc_plan(monkeypatch, "store16", *n, *h, tc="fp16")
    assert plan.schedule()[2] == 6
    m = to_dev(torch, m0)
    gp = LLGParams(A=prm.A, alpha=prm.alpha, Hext=prm.Hext)
    gp.Ms_map = to_dev(torch, Ms)
    plan.llg_step(m, gp, 1e-13)
    assert plan.sync_status() == 0
    assert_close(m.cpu().numpy() - m0, ref - m0, 1e-2)
