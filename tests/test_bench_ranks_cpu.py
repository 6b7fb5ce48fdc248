"""The replica (N > 1) path of bench.py on the CPU: two gloo ranks on
127.0.0.1 reduce their timings to the maximum and their units to the sum,
and the oracle arm prints from rank 0 only."""
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


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, units = bench.job_totals(1.0 + rank, [10.0 * (rank + 1), 2.0], world, "cpu")
        q.put((rank, t, units))
    finally:
        dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, units in got:
        assert t == 2.0                    # slowest rank's time
        assert units == [30.0, 4.0]        # units of both ranks


def test_job_totals_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(3.5, [1, 2], 1, "cpu") == (3.5, [1.0, 2.0])


def test_reference_arm_prints_on_rank0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(steps=1, warmup=0, cpu_seconds=1.0)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""


def test_products_per_mode():
    """H.v products of a blocked solve: double-float columns stop at their own
    convergence, the multi-column modes run every column to the last one."""
    sys.path.insert(0, ROOT)
    import bench
    it = [5294, 4647, 5288, 4651]
    assert bench.products(it, "df") == sum(it)
    for prec in ("fp64", "mixed", "fp32"):
        assert bench.products(it, prec) == 4 * 5294
