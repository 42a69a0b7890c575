"""Host logic of the N > 1 benchmark path (independent replicas, one per rank):
barriers around the timed region, the slowest rank's time, and the whole-job
rate.  Two gloo ranks on the CPU stand in for two GPUs."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # rank r "took" 100 + 10 r ms for the timed region and 5 - r for a second figure
        ms, other = bench.max_over_ranks([100.0 + 10.0 * rank, 5.0 - rank], world, torch.device("cpu"))
        value = bench.replica_rate(world, 20, ms)
        bench.barrier(world)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms": ms, "other": other, "value": value}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replicas_take_slowest_rank(tmp_path, world):
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    slow = 100.0 + 10.0 * (world - 1)
    for r in range(world):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["ms"] == slow and got["other"] == 5.0
        # all ranks' steps over the slowest rank's time
        assert got["value"] == pytest.approx(world * 20 / (slow / 1e3))


def test_single_rank_is_identity():
    assert bench.max_over_ranks([3.5, 7], 1, None) == [3.5, 7.0]
    assert bench.replica_rate(1, 40, 2000.0) == pytest.approx(20.0)
    bench.barrier(1)  # no process group needed


def test_reference_arm_other_ranks_do_no_work(capsys):
    class Args:
        workload = "fd2d_n4096"
        steps = warmup = 1

    assert bench.run_reference(Args(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""
