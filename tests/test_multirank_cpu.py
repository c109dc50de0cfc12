"""The N > 1 path of bench.py, with two gloo ranks on the CPU.

Each rank solves its own shard (workload seed = rank) with no data-path
collective; the job's time is the slowest rank's and its work the sum of the
shards.  Checked here: the shards differ between ranks and are reproducible,
and the whole-job reduction returns the maximum time and the total cells.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.timeout(120) if hasattr(pytest.mark, "timeout") else []

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    from paper_2303_02898_gb300 import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shard = workloads.solve_targets(64, seed=rank)
        ms, cells = bench.whole_job(dist, 10.0 + 5.0 * rank, 64 + rank, torch.device("cpu"))
        q.put((rank, ms, cells, np.asarray(shard.v)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_whole_job_and_shards():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    out = sorted(q.get() for _ in range(2))
    for rank, ms, cells, _ in out:
        assert ms == 15.0 and cells == 64 + 65
    v0, v1 = out[0][3], out[1][3]
    assert not np.allclose(v0, v1)
    sys.path.insert(0, ROOT)
    from paper_2303_02898_gb300 import workloads
    assert np.array_equal(v0, np.asarray(workloads.solve_targets(64, seed=0).v))


def test_single_process_whole_job_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(None, 12.5, 100, None) == (12.5, 100)
