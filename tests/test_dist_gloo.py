"""Multi-rank path of the benchmark on CPU (gloo, world size 2): ranks filter independent
image streams and only the elapsed time is reduced (max over ranks); the reference arm
runs on rank 0 alone."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks(1.5 + rank, torch.device("cpu"), world)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_image_seed(rank))
    out = io.StringIO()

    class A:
        steps, warmup = 1, 0
    if rank == 1:                       # non-zero ranks of the reference arm print nothing
        with redirect_stdout(out):
            bench.run_reference(A)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, seeds, out.getvalue()))


def test_two_rank_reduction_and_independent_streams():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, seeds, printed in res:
        assert got == 2.5                           # max over ranks
        assert seeds == [1, 2]                      # distinct per-rank image streams
        assert printed == ""
