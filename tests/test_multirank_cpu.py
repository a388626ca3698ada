"""The benchmark's multi-rank logic on CPU ranks (gloo, world size 2).

Under torchrun every rank runs an independent problem (seed 1 + rank) with no
collective on the data path; the only collectives are the barrier around the
timed region and the max of the ranks' times.  These tests run that logic in
two spawned processes on the gloo backend: dist_setup picks gloo without a
GPU, max_over_ranks returns the slowest rank's time on every rank, the
reference arm runs on rank 0 only, and the whole-job value divides all ranks'
work by the slowest rank's time.
"""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    t_max = bench.max_over_ranks(1.0 + rank, w)  # rank 1 is the slower one
    ref = bench.run_reference(None, w, r) if r != 0 else "rank0"
    out.put((rank, t_max, ref, bench.whole_job_value(1000, 3, w, t_max)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, ref, value in got:
        assert t_max == 2.0                       # the slowest rank's time on both ranks
        assert value == pytest.approx(1000 * 3 * 2 / 2.0)
        if rank == 1:
            assert ref is None                    # the reference arm runs on rank 0 only


def test_whole_job_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.whole_job_value(5, 4, 1, 2.0) == 10.0
    assert bench.max_over_ranks(3.5, 1) == 3.5
