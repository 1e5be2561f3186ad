"""The benchmark's multi-process (replicas) host logic on CPU: two gloo ranks, each with its
own mixture (seed = rank), the timing maxed over ranks and the whole-job rate counting every
rank's units. No GPU and no collective on the data path."""
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
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rate, ms = bench.job_throughput(100.0 * (rank + 1), world, 10, 3, dist)
    spec = bench.spec_for(rank)
    out.put((rank, rate, ms, spec.seed, spec.J))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_timing_and_per_rank_mixtures():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms, seed, J in res:
        assert ms == 200.0                                   # the slower rank's time
        assert abs(rate - world * 10 * 3 / 0.2) < 1e-9       # every rank's units over that time
        assert seed == rank
    assert res[0][4] == res[1][4]                            # same workload shape on every rank
