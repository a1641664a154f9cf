"""Mixed-precision variant: the zero-padded z transforms on the tensor cores
with FP16 or BF16 operands, per-column scaling and FP32 accumulation, against
the FP64 oracle.  Tolerance: relative L2 error of H_d <= 1e-2."""
import numpy as np
import pytest

import oracle
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    ((48, 40, 32), (4e-9, 4e-9, 4e-9)),    # pz = 64 with nz = 32
    ((37, 29, 20), (3e-9, 3e-9, 2e-9)),    # ragged: nz = 20 still pads to 64, ragged column tiles
    ((64, 300, 17), (4e-9, 4e-9, 4e-9)),   # length-1024 y transforms
]


@pytest.mark.parametrize("n,h", CASES)
@pytest.mark.parametrize("tc", ["fp16", "bf16"])
def test_tensor_core_z_stage_matches_oracle(n, h, tc):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    nx, ny, nz = n
    M = 8e5 * inputs.voronoi_columnar(nx, ny, nz, h, 20e-9, seed=3)
    ref = oracle.DemagPlan(nx, ny, nz, *h).apply(M)
    plan = Plan(nx, ny, nz, *h, tc=tc)
    H = plan.apply(to_dev(torch, M)).cpu().numpy()
    err = rel_l2(H, ref)
    assert err < 1e-2, err
    # and it is genuinely the reduced-precision path (not bit-equal to FP32)
    H32 = Plan(nx, ny, nz, *h).apply(to_dev(torch, M)).cpu().numpy()
    assert rel_l2(H32, ref) < 1e-5
    assert err > rel_l2(H32, ref)


def test_tensor_core_random_magnetisation():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import Plan
    n, h = (32, 24, 32), (5e-9, 5e-9, 5e-9)
    M = 8e5 * inputs.random_unit(*n, seed=1)
    ref = oracle.DemagPlan(*n, *h).apply(M)
    for tc in ("fp16", "bf16"):
        H = Plan(*n, *h, tc=tc).apply(to_dev(torch, M)).cpu().numpy()
        assert rel_l2(H, ref) < 1e-2


def test_tensor_core_rejects_unsupported_depth():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import BorisError, Plan
    with pytest.raises(BorisError) as e:
        Plan(32, 32, 8, 1e-9, 1e-9, 1e-9, tc="fp16")
    assert e.value.code == -4
