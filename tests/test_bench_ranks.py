"""The multi-rank aggregation of bench.py (one process per GPU, replicas of the problem)
run as two gloo ranks on the CPU: the time is the maximum over ranks and the rate counts
every rank's units."""
import importlib.util
import os
import socket
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _bench():
    spec = importlib.util.spec_from_file_location("bench_ranks_under_test", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    sys.modules["bench_ranks_under_test"] = mod
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        ms = 10.0 + 5.0 * rank          # rank 1 is the slower one
        t = b.max_over_ranks(ms, "cpu")
        out[rank] = (t, b.whole_job_rate(1.0, world, t / 1e3))
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    t, rate = res[0]
    assert t == 15.0
    assert rate == pytest.approx(2 / 0.015)


def test_single_process_is_unchanged():
    b = _bench()
    assert b.max_over_ranks(12.5, "cpu") == 12.5
    assert b.whole_job_rate(1.0, 1, 0.032) == pytest.approx(31.25)
