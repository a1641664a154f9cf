"""Bounded device-side waits: the bulk-copy, residue-split and tcgen05 z stages (both the
FP32-spectrum one and the 16-bit-storage one with its producer warp) wait on mbarriers
with a time limit.  Through a test hook the first wait of every CTA expects
16 bytes that never arrive; the kernel must give up after its limit, latch
BORIS_ERR_TIMEOUT in the plan's status word (read by boris_sync_status) and
leave the context usable.  No GPU fault is involved: the wait simply runs
out."""
import numpy as np
import pytest

import oracle
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import assert_close, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

N, H = (24, 40, 9), (2e-9, 2e-9, 2e-9)


@pytest.mark.parametrize("variant", ["1", "3"])  # bulk-copy pipeline, residue-split z convolution
def test_wait_that_runs_out_reports_timeout_and_context_survives(variant, monkeypatch):
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import BorisError, Plan
    M = 7e5 * inputs.random_unit(*N, seed=21)
    monkeypatch.setenv("BORIS_YZ_KIND", "2")
    monkeypatch.setenv("BORIS_YZ_TMA", variant)
    monkeypatch.setenv("BORIS_TEST_WAIT_TIMEOUT", "1")
    bad = Plan(*N, *H)
    assert bad.schedule()[0] == 2 and bad.schedule()[2] == int(variant)
    bad.apply(to_dev(torch, M))
    with pytest.raises(BorisError) as ei:
        bad.sync_status()
    assert ei.value.code == -5
    bad.sync_status()  # the status word was cleared by the read
    bad.close()
    monkeypatch.delenv("BORIS_TEST_WAIT_TIMEOUT")
    good = Plan(*N, *H)
    Hd = good.apply(to_dev(torch, M))
    good.sync_status()
    ref = oracle.DemagPlan(*N, *H).apply(M)
    assert_close(Hd.cpu().numpy(), ref, 1e-5)


def test_tcgen05_stage_wait_that_runs_out(monkeypatch):
    """The tensor-core z stage (tcgen05) gives up the same way: it latches the
    timeout, lets its other copies land, frees its tensor memory and returns;
    a following plan (which allocates tensor memory again) is correct."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import BorisError, Plan
    n, h = (24, 40, 20), (2e-9, 2e-9, 2e-9)
    M = 7e5 * inputs.random_unit(*n, seed=22)
    monkeypatch.setenv("BORIS_TEST_WAIT_TIMEOUT", "1")
    bad = Plan(*n, *h, tc="fp16")
    assert bad.schedule()[2] == 5
    bad.apply(to_dev(torch, M))
    with pytest.raises(BorisError) as ei:
        bad.sync_status()
    assert ei.value.code == -5
    bad.sync_status()
    bad.close()
    monkeypatch.delenv("BORIS_TEST_WAIT_TIMEOUT")
    good = Plan(*n, *h, tc="fp16")
    Hd = good.apply(to_dev(torch, M))
    good.sync_status()
    ref = oracle.DemagPlan(*n, *h).apply(M)
    assert_close(Hd.cpu().numpy(), ref, 1e-2)


@pytest.mark.parametrize("tc", ["bf16", "fp16"])
def test_16bit_storage_stage_wait_that_runs_out(tc, monkeypatch):
    """The 16-bit-storage z stage: the producer warp's first data copy never
    completes, so it and the sixteen compute warps (waiting for products that
    are never issued) give up after the limit; the CTA latches the timeout,
    lets its kernel-row copy land, frees its tensor memory and returns, and a
    following plan is correct."""
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import BorisError, Plan
    n, h = (64, 300, 17), (4e-9, 4e-9, 4e-9)
    M = 7e5 * inputs.voronoi_columnar(*n, h, 20e-9, seed=23)
    monkeypatch.setenv("BORIS_TEST_WAIT_TIMEOUT", "1")
    bad = Plan(*n, *h, tc=tc)
    assert bad.schedule()[2] == 6
    bad.apply(to_dev(torch, M))
    with pytest.raises(BorisError) as ei:
        bad.sync_status()
    assert ei.value.code == -5
    bad.sync_status()
    bad.close()
    monkeypatch.delenv("BORIS_TEST_WAIT_TIMEOUT")
    good = Plan(*n, *h, tc=tc)
    Hd = good.apply(to_dev(torch, M))
    good.sync_status()
    ref = oracle.DemagPlan(*n, *h).apply(M)
    assert_close(Hd.cpu().numpy(), ref, 1e-2)
