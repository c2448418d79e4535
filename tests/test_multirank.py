"""Host side of the multi-rank bench path on CPU: two gloo ranks (spawned
processes, rendezvous on 127.0.0.1) run bench.py's rank setup, barrier and
max-over-ranks reduction, and the whole-job rate is the weak-scaling sum."""

import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, q):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    bench.barrier(w)
    ms = 1.0 + 2.0 * r                                  # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, w)
    q.put((r, w, local, ms_max, bench.whole_job_rate(1000, w, ms_max)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_max_and_weak_scaling_rate():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for r, (rank, w, local, ms_max, rate) in enumerate(got):
        assert (rank, w, local) == (r, world, r)
        assert ms_max == 3.0                            # the max over ranks, on every rank
        assert abs(rate - 2 * 1000 / 3e-3) < 1e-6       # both ranks' units over the slowest time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.whole_job_rate(10, 1, 1.0) == 10 / 1e-3
