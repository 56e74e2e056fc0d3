"""The multi-GPU path of bench.py is replicas: one process per GPU, each
running the whole workload, with a barrier around the timed region and the
maximum time over ranks.  Its host logic runs here on CPU as two gloo ranks
(127.0.0.1 rendezvous)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    dist, r, w = bench.dist_setup()
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    bench.barrier(dist)
    # each rank's step time; the job's is the slowest rank's
    ms = bench.max_over_ranks(dist, 10.0 + rank)
    out.put((rank, ms, w * 1e3 / ms))
    # the reference arm: rank 0 alone works, the others return at once
    class A:
        workload, steps, warmup = "small", 1, 0
    if rank != 0:
        bench.run_reference(A, dist, rank, world)
    bench.barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_time_as_one_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks report the max over ranks, and value = world x 1e3 / ms
    assert [r[1] for r in res] == [11.0, 11.0]
    assert res[0][2] == pytest.approx(2 * 1e3 / 11.0)
