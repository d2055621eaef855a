"""Host logic of bench.py's multi-GPU path (one rank per GPU, walkers sharded,
timings reduced with MAX) on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from paper_2501_08261_gb300 import workloads
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = bench.max_over_ranks(torch, dist, [10.0 + rank, 5.0 * (ws - rank), 7.0])
    th = workloads.prior_draws(4, 17280, 5.0, seed=bench.walker_seed(rank))
    got = [None] * ws
    dist.all_gather_object(got, th[:, 0].tolist())
    dist.barrier()
    if rank == 0:
        out.put((ms, got, bench.job_throughput(256, ws, 10, ms[0])))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_distinct_walkers():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ms, masses, value = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ms == [11.0, 10.0, 7.0]
    assert masses[0] != masses[1]                       # each rank its own walkers
    assert value == pytest.approx(256 * 2 * 10 / 11e-3)
