"""The multi-rank host logic of bench.py on CPU: two gloo ranks (replicas) take the slowest rank's
time as the job's and report the whole job's rate; the reference arm runs on rank 0 only."""
import importlib.util
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        ranks = bench.Ranks(world, dist, "cpu")
        ranks.barrier()
        ms = ranks.max(10.0 * (rank + 1))           # rank 0: 10 ms, rank 1: 20 ms
        rate = ranks.rate(5, ms)                      # 5 steps per rank
        out[rank] = (ms, rate)
        ranks.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == 20.0
        assert abs(rate - world * 5 / 20e-3) < 1e-9  # 500 steps/s for the job


def test_single_rank_needs_no_process_group():
    bench = _bench()
    ranks = bench.Ranks()
    ranks.barrier()
    assert ranks.max(12.5) == 12.5 and ranks.rate(10, 12.5) == 800.0


def test_reference_arm_runs_on_rank_zero_only():
    bench = _bench()
    saved = sys.argv
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2"]
    try:
        args = bench.parse()
    finally:
        sys.argv = saved
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.reference_main(args, rank=1) is None
    assert buf.getvalue() == ""
