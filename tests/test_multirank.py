"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2):
each rank times its own replica; the job rate uses the slowest rank's time
and the units of all ranks; only rank 0 runs the reference arm."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.reduce_max(1.5 + rank, "cpu")          # rank times 1.5 s and 2.5 s
    out[rank] = (t, bench.job_rate(1000, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    assert res[0][1] == pytest.approx(2 * 1000 / 2.5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(bench.parse_args(["--impl", "reference", "--gpus", "2"])) is None


def test_single_rank_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.25, "cpu") == 3.25
    assert bench.job_rate(100, 1, 2.0) == 50.0
