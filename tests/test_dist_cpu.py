"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): each rank is an independent
replica; only the units (summed) and the time (max over ranks) are combined.  The reference arm
runs on rank 0 alone."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, ms = bench.reduce_timing(1000.0 * (rank + 1), 10.0 * (rank + 1), device="cpu")
    out[rank] = (units, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_timing_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert res[0] == res[1] == (3000.0, 20.0)


def test_reference_arm_idle_on_nonzero_rank(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        workload = "shell128"; steps = 1; warmup = 0; gpus = 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""


def test_single_rank_reduce_is_identity():
    import bench
    assert bench.reduce_timing(5.0, 7.0, device="cpu") == (5.0, 7.0)
