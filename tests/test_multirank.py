"""World-size-2 gloo run of bench.py's multi-rank host logic (CPU only):
per-rank workloads, max-over-ranks timing and the whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2601_16791_gb300 import workloads as W
    w = W.make(bench.WORKLOAD, seed=bench.rank_seed(rank), nsmall=50)
    t_local = 10.0 + rank                       # rank 1 is the slow one
    t_max = bench.reduce_max(t_local, "cpu")
    rate = bench.whole_job_rate(w.n, 7, world, t_max)
    out[rank] = (t_max, rate, float(w.xv_helio[0, 5]), w.n)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    world = 2
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (t0, r0, x0, n0), (t1, r1, x1, n1) = out[0], out[1]
    assert t0 == t1 == 11.0                      # max over ranks
    assert r0 == r1 == 2 * n0 * 7 / 11.0         # units of all ranks / slowest time
    assert n0 == n1 and x0 != x1                 # same size, independent disks
