"""The multi-rank (replica) logic of bench.py on CPU with two gloo ranks: every rank
gets the slowest rank's time, the whole-job value counts all ranks' units, and the
reference arm prints on rank 0 only."""

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank
    slowest = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    out[rank] = (slowest, bench.replicas_value(world, 1000, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_value():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.5, None, None) == 7.5
    assert bench.replicas_value(1, 500, 250.0) == pytest.approx(2000.0)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(_args(bench))
    assert buf.getvalue() == ""


def _args(bench):
    old = sys.argv
    sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
    try:
        return bench.parse()
    finally:
        sys.argv = old
