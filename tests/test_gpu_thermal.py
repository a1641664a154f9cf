"""GPU parity of the stochastic thermal field against the oracle: the same
counter-based generator (Philox4x32-10, Box-Muller) on both sides gives the
same field for the same (seed, step, cell), so an RK4 step at T > 0 is
compared like a deterministic one (increment within 2e-4 relative L2 in
FP32, 1e-9 in FP64); the step counter advances once per RK4 step, also
inside CUDA-graph replays."""
import numpy as np
import pytest

import oracle
from oracle import llg
from oracle import thermal as th
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import assert_close, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

N, CELL = (20, 12, 3), (2e-9, 2e-9, 2e-9)
T, SEED, ALPHA = 300.0, 0x1234567890ABCDEF, 0.1


def setup(fp64=False):
    from paper_2008_02478_gb300.binding import FieldTerms, LLGParams, Plan
    plan = Plan(*N, *CELL, fp64=fp64)
    plan.set_field_terms(FieldTerms(temperature=T, seed=SEED))
    prm = LLGParams(Ms=8e5, A=1.3e-11, alpha=ALPHA, Hext=(0.0, 0.0, 5e4))
    prm_o = llg.Params(cell=CELL, Ms=8e5, A=1.3e-11, alpha=ALPHA, Hext=(0.0, 0.0, 5e4))
    return plan, prm, prm_o


@pytest.mark.parametrize("fp64", [False, True])
def test_thermal_rk4_steps_match_oracle(fp64):
    torch = torch_cuda()
    m0 = inputs.random_unit(*N, seed=51)
    m0 = m0 + 0.8 * np.roll(m0, 1, axis=3)
    m0 = (m0 / np.linalg.norm(m0, axis=0)).astype(np.float32).astype(np.float64)
    plan, prm, prm_o = setup(fp64)
    demag = oracle.DemagPlan(*N, *CELL).apply
    dt = 1e-14
    plan.thermal_set_step(5)
    m = torch.tensor(m0, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
    ref = m0
    for s in (5, 6):
        prev = ref
        ref = th.rk4_step_thermal(ref, dt, prm_o, demag, step=s, seed=SEED, T=T)
        mprev = m.cpu().numpy().astype(np.float64)
        plan.llg_step(m, prm, dt)
        got = m.cpu().numpy().astype(np.float64)
        assert np.abs(ref - prev).max() > 1e-3
        assert_close(got - mprev, ref - prev, (1e-9 if fp64 else 2e-4))
    # without the thermal field the same step is clearly different
    det = llg.rk4_step(m0, dt, prm_o, demag)
    first = th.rk4_step_thermal(m0, dt, prm_o, demag, step=5, seed=SEED, T=T)
    assert rel_l2(det - m0, first - m0) > 0.1


def test_thermal_graph_replay_advances_the_counter():
    torch = torch_cuda()
    m0 = inputs.random_unit(*N, seed=52)
    plan, prm, _ = setup()
    a = torch.tensor(m0, dtype=torch.float32, device="cuda")
    b = a.clone()
    plan.thermal_set_step(100)
    for _ in range(4):
        plan.llg_step(a, prm, 1e-14)
    plan.thermal_set_step(100)
    plan.llg_run_graph(b, prm, 1e-14, 4)
    torch.cuda.synchronize()
    assert_close(b.cpu().numpy(), a.cpu().numpy(), 1e-7, 1e-7 * 10)
    # a replay from a different counter draws different fields
    c = torch.tensor(m0, dtype=torch.float32, device="cuda")
    plan.thermal_set_step(200)
    plan.llg_run_graph(c, prm, 1e-14, 4)
    torch.cuda.synchronize()
    assert rel_l2(c.cpu().numpy(), a.cpu().numpy()) > 1e-3


def test_thermal_argument_checks():
    torch_cuda()
    from paper_2008_02478_gb300.binding import RKF45, BorisError, FieldTerms, LLGParams, Plan
    plan = Plan(*N, *CELL)
    with pytest.raises(BorisError) as e:
        plan.set_field_terms(FieldTerms(temperature=-1.0))
    assert e.value.code == -1
    plan.set_field_terms(FieldTerms(temperature=300.0))
    import torch
    m = torch.tensor(inputs.random_unit(*N, seed=1), dtype=torch.float32, device="cuda")
    with pytest.raises(BorisError) as e:  # adaptive steps do not take the thermal field
        plan.llg_step(m, LLGParams(method=RKF45), 1e-14)
    assert e.value.code == -1


def test_checkpoint_resume_continues_the_thermal_sequence(tmp_path):
    """Four RK4 steps, a checkpoint, three more: a fresh plan resumed from the
    checkpoint (counter set back to step 4) ends where the uninterrupted run
    ends; resumed with the counter left at 0 it draws other fields and does
    not."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import FieldTerms
    from paper_2008_02478_gb300.state import load_state, resume, save_state
    m0 = inputs.random_unit(*N, seed=53)
    dt = 1e-14
    plan, prm, _ = setup()
    a = torch.tensor(m0, dtype=torch.float32, device="cuda")
    for _ in range(4):
        plan.llg_step(a, prm, dt)
    path = tmp_path / "run.npz"
    save_state(path, a, t=4 * dt, dt=dt, step=4, seed=SEED, temperature=T)
    for _ in range(3):
        plan.llg_step(a, prm, dt)
    s = load_state(path)
    plan2, _, _ = setup()
    plan2.set_field_terms(FieldTerms(temperature=s["temperature"], seed=s["seed"]))
    b = resume(plan2, s)
    assert s["step"] == 4 and abs(s["t"] - 4 * dt) < 1e-30
    for _ in range(3):
        plan2.llg_step(b, prm, s["dt"])
    assert_close(b.cpu().numpy(), a.cpu().numpy(), 1e-6, 1e-6 * 10)
    plan3, _, _ = setup()
    c = torch.tensor(s["m"], device="cuda")  # counter left at 0
    for _ in range(3):
        plan3.llg_step(c, prm, s["dt"])
    assert rel_l2(c.cpu().numpy(), a.cpu().numpy()) > 1e-4


def test_device_philox_matches_known_answers_and_oracle_bit_for_bit():
    """The stage kernels' Philox4x32-10 (through boris_philox4x32_10) gives the
    published known-answer outputs and the oracle's words on random counters
    and keys, bit for bit."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import philox4x32_10
    from oracle import thermal as th
    from tests.test_oracle_thermal import kat_vectors
    rows = kat_vectors()
    rng = np.random.default_rng(31)
    rand = rng.integers(0, 2 ** 32, size=(512, 6), dtype=np.uint64)
    ctr = np.concatenate([np.array([r[0] for r in rows], dtype=np.uint64), rand[:, :4]])
    key = np.concatenate([np.array([r[1] for r in rows], dtype=np.uint64), rand[:, 4:]])
    as_i32 = lambda a: torch.tensor(a.astype(np.uint32).view(np.int32), device="cuda")
    out = philox4x32_10(as_i32(ctr), as_i32(key)).cpu().numpy().view(np.uint32).astype(np.uint64)
    for i, (_, _, want) in enumerate(rows):
        assert [int(x) for x in out[i]] == want
    ref = np.stack([np.concatenate([np.stack(th.philox4x32_10(c[0:1], c[1:2], c[2:3], c[3:4], k[0], k[1]))[:, 0]])
                    for c, k in zip(ctr, key)])
    assert np.array_equal(out, ref)
