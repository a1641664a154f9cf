"""GPU parity of periodic boundary conditions (multiple-images method,
Section 4): the image-summed demag kernel against the oracle's FFT plan with
its image-summed table, and RK4 steps with wrapping exchange (and DMI)
neighbours against the oracle.  Tolerances as for the open meshes: 1e-5
relative L2 for FP32 fields, 1e-9 for the FP64 plan; the RK4 increment within
2e-4."""
import numpy as np
import pytest

import oracle
from oracle import llg
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import assert_close, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    ((16, 12, 3), (2e-9, 2.5e-9, 2e-9), (4, 3, 0)),
    ((9, 7, 2), (1e-9, 1.5e-9, 2e-9), (2, 0, 1)),
    ((300, 20, 2), (3e-9, 3e-9, 3e-9), (2, 2, 0)),   # length-1024 x pass
    ((32, 32, 1), (4e-9, 4e-9, 2e-9), (6, 6, 0)),    # periodic thin film
]


@pytest.mark.parametrize("n,h,images", CASES)
@pytest.mark.parametrize("fp64", [False, True])
def test_pbc_demag_matches_oracle(n, h, images, fp64):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    M = 7e5 * inputs.random_unit(*n, seed=41)
    table = oracle.tensor_table_pbc(*n, *h, images)
    ref = oracle.DemagPlan(*n, *h, table=table).apply(M)
    plan = Plan(*n, *h, fp64=fp64, images=images)
    H = plan.apply(to_dev(torch, M, fp64)).cpu().numpy()
    assert_close(H, ref, (1e-9 if fp64 else 1e-5))


@pytest.mark.parametrize("n,images,dmi", [((16, 12, 3), (3, 2, 0), None), ((15, 12, 3), (2, 2, 0), None),
                                          ((16, 10, 2), (3, 3, 0), "interfacial"), ((13, 9, 4), (1, 2, 1), "bulk")])
def test_pbc_rk4_step_matches_oracle(n, images, dmi):
    """Quad stage kernel (nx % 4 == 0), the one-cell kernel, and the DMI
    path, each with wrapping neighbours along the periodic axes."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import FieldTerms, LLGParams, Plan
    h = (2e-9, 2e-9, 2e-9)
    m0 = inputs.random_unit(*n, seed=43)
    m0 = m0 + 0.6 * np.roll(m0, 1, axis=3)
    m0 = (m0 / np.linalg.norm(m0, axis=0)).astype(np.float32).astype(np.float64)
    pbc = tuple(k > 0 for k in images)
    extra = dict(dmi=dmi, D=2e-3) if dmi else {}
    prm_o = llg.Params(cell=h, Ms=8e5, A=1.3e-11, alpha=0.1, Hext=(1e4, 0.0, 3e4), pbc=pbc, **extra)
    demag = oracle.DemagPlan(*n, *h, table=oracle.tensor_table_pbc(*n, *h, images)).apply
    dt = 3e-14
    ref = llg.rk4_step(m0, dt, prm_o, demag)
    plan = Plan(*n, *h, images=images)
    if dmi:
        plan.set_field_terms(FieldTerms(dmi=dmi, D=2e-3))
    m = torch.tensor(m0, dtype=torch.float32, device="cuda")
    plan.llg_step(m, LLGParams(Ms=8e5, A=1.3e-11, alpha=0.1, Hext=(1e4, 0.0, 3e4)), dt)
    got = m.cpu().numpy().astype(np.float64)
    assert np.abs(ref - m0).max() > 1e-3
    assert_close(got - m0, ref - m0, 2e-4)


def test_pbc_argument_checks():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import BorisError, LLGParams, Plan
    with pytest.raises(BorisError) as e:
        Plan(8, 8, 2, 1e-9, 1e-9, 1e-9, images=(-1, 0, 0))
    assert e.value.code == -1
    plan = Plan(8, 8, 2, 1e-9, 1e-9, 1e-9, images=(2, 2, 0))
    m = torch.tensor(inputs.random_unit(8, 8, 2, seed=1), dtype=torch.float32, device="cuda")
    with pytest.raises(BorisError) as e:  # the adjoint serves open meshes
        plan.llg_step_backward(m, LLGParams(), 1e-14, torch.zeros_like(m))
    assert e.value.code == -1
