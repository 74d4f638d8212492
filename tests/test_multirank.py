"""Multi-process path of bench.py (replicas: one independent fit per rank, no
data-path collective) on CPU with the gloo backend, world size 2: process
group set-up from the launcher's environment, the barrier, the max-over-ranks
timing and the sum-over-ranks throughput."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup(None)
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    ms = 10.0 + 5.0 * rank            # this rank's time for the same work
    work = 1000.0 * (rank + 1)        # this rank's units
    out.put((rank, bench.max_over_ranks(w, ms), bench.sum_over_ranks(w, work)))
    dist.destroy_process_group()


def test_two_ranks_gloo_max_time_and_summed_work():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 3000.0), (1, 15.0, 3000.0)]
