"""Multi-GPU runs are replicas: one independent simulation per GPU and no
collective on the data path.  bench.py times them with a barrier on both sides
and takes the maximum over ranks; the whole-job rate divides all ranks' work by
that time.  Here that host logic (bench.Replicas, bench.whole_job_rate) runs
as two gloo ranks on CPU processes, and the reference arm's other ranks are
checked to exit without work."""
import argparse
import json
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, seconds, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    ranks = bench.Replicas(world, "gloo", "cpu")
    ranks.barrier()
    t = ranks.max(seconds[rank])
    rate = bench.whole_job_rate(world, 1000.0, t)
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"t": t, "rate": rate}, f)
    ranks.close()


def test_two_gloo_ranks_time_the_slowest_replica(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    seconds = [0.5, 2.0]
    mp.spawn(_rank, args=(2, _free_port(), seconds, str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        with open(tmp_path / ("rank%d.json" % rank)) as f:
            d = json.load(f)
        assert d["t"] == 2.0  # every rank sees the slowest rank's time
        assert d["rate"] == 2 * 1000.0 / 2.0  # both ranks' work over that time


def test_single_rank_needs_no_process_group():
    pytest.importorskip("torch")
    import bench
    ranks = bench.Replicas(1, "gloo", "cpu")
    assert ranks.dist is None
    ranks.barrier()
    assert ranks.max(1.25) == 1.25
    ranks.close()
    assert bench.whole_job_rate(1, 10.0, 2.0) == 5.0


def test_reference_arm_other_ranks_exit_without_work(capsys):
    import bench
    args = argparse.Namespace(steps=3, warmup=3, gpus=2)
    assert bench.run_reference(args, 1) == 0
    assert capsys.readouterr().out == ""
