"""The multi-GPU form of bench.py: one independent replica per rank, a barrier
around the timed region and the max over ranks of the elapsed time. The exchange
itself needs no GPU: two gloo ranks on the CPU run the same helpers."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # bench.py's own exchange: barrier, then the max over ranks of each rank's time
        bench.barrier(world)
        elapsed = bench.allreduce_max(1.5 + rank, world)
        # weak scaling: value = world * units per replica / max time
        units = 198147 * 256
        value = world * units / elapsed
        out[rank] = (elapsed, value)
    finally:
        dist.destroy_process_group()


def test_two_rank_max_time_and_weak_value():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 2.5
    assert out[0][1] == pytest.approx(2 * 198147 * 256 / 2.5)


def test_bench_reference_arm_is_rank0_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
