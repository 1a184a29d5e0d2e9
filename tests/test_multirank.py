"""The multi-rank path of the benchmark on CPU (gloo, world size 2): ranks run disjoint
walks (weak scaling) and the job's throughput is the units of all ranks over the
slowest rank's time.  No GPU needed."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    wl, specs = bench.rank_specs(8, rank)
    local_ms = 100.0 * (rank + 1)                 # rank 1 is the slow one
    units = len(specs) * specs[0].N * 3
    value, ms_max = bench.aggregate(local_ms, units, world, dist)
    out.put((rank, [s.seed for s in specs], value, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_disjoint_walks_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    [p.start() for p in procs]
    res = sorted(q.get(timeout=120) for _ in procs)
    [p.join(timeout=60) for p in procs]
    assert all(p.exitcode == 0 for p in procs)
    (r0, seeds0, v0, t0), (r1, seeds1, v1, t1) = res
    assert not set(seeds0) & set(seeds1) and len(seeds0) == len(seeds1) == 8
    assert t0 == t1 == 200.0                                   # max over ranks
    assert v0 == v1 == pytest.approx(2 * 8 * 6912 * 3 / 0.2)   # all ranks' units / slowest time
