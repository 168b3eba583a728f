"""The multi-GPU path of bench.py is replicas only: each rank solves its
own copy of the workload, and the process group carries only the barriers
and the max-over-ranks step time.  That host logic runs here on CPU with
two gloo ranks."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    ws, r, local = bench.dist_setup("gloo")
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier(ws)
    # a rank's step time; the job's time is the slowest rank's
    out[rank] = bench.max_over_ranks(0.25 + 0.5 * rank, ws)
    bench.barrier(ws)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step_time():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert dict(out) == {0: 0.75, 1: 0.75}


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    os.environ.pop("WORLD_SIZE", None)
    assert bench.dist_setup("gloo")[0] == 1
    assert bench.max_over_ranks(1.5, 1) == 1.5
