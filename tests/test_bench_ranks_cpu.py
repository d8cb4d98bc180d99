"""The multi-rank reduction of bench.py on two gloo ranks (CPU).

Under torchrun every rank runs its own problem instance; the bench line reports the slowest
rank's time and the units all ranks processed.  Two processes with different times and
different unit counts check the MAX and the SUM, and one process checks the pass-through.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as td
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.reduce_over_ranks(100.0 + 50.0 * rank, (1000 + 7 * rank, 2.5 * (rank + 1)), td, "cpu")
    out.put((rank, ms, units))
    td.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units in res:
        assert ms == 150.0                        # the slower rank's time
        assert units == [2007.0, 7.5]             # both ranks' units


def test_reduce_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(12.5, (3, 4.5), None, "cpu") == (12.5, [3.0, 4.5])
