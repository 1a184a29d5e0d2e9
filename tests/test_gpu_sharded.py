"""Single-walk k-sharding on the GPU: ranks emulated in one process as separate contexts
on one GPU (no kernel of one rank waits on another's: the exchanges are host-side sums
between the steps).  Every rank must follow the oracle step by step, and the sharded walk
must make the same decisions as the same walk run unsharded."""
import numpy as np
import pytest

import psl_workloads as W
from helpers import compare_final_state, compare_traces, have_gpu, oracle_walk, same_decisions

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def P():
    from paper_2107_09801_gb300 import build
    build.build()
    import paper_2107_09801_gb300 as P
    return P


def _run_sharded(P, spec, world, init_seq=None):
    from paper_2107_09801_gb300.sharded import ShardedWalk, run_together
    ctxs = [P.Context(arena_bytes=2 * P.psl_walk_bytes(spec.L, spec.n_lmt, spec.budget) + (64 << 20), max_walks=2)
            for _ in range(world)]
    try:
        walks = [ShardedWalk(c, r, world, None, L=spec.L, seed=spec.seed, alpha1=spec.alpha1, alpha2=spec.alpha2,
                             budget=spec.budget, n_lmt=spec.n_lmt, ls_lmt=spec.ls_lmt, flip_lmt=spec.flip_lmt,
                             topk=spec.topk, init_seq=init_seq, trace_cap=spec.budget) for r, c in enumerate(ctxs)]
        assert run_together(walks) == spec.budget
        out = [(c.trace(w.wid, spec.budget), c.export_state(w.wid)) for c, w in zip(ctxs, walks)]
        ks = [c.shard_layout(w.wid)[0] for c, w in zip(ctxs, walks)]
        with pytest.raises(P.PslError):
            ctxs[0].step(1)   # a sharded walk is stepped only through the shard calls
        return out, ks
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("L,world", [(65535, 2), (65535, 4), (20000, 3)])
def test_sharded_walk_matches_oracle(P, L, world):
    spec = W.WalkSpec(L=L, seed=L + world, alpha1=4, alpha2=13, budget=6, ls_lmt=2, flip_lmt=10)
    res, ks = _run_sharded(P, spec, world)
    w = oracle_walk(spec)
    otr = w.run(spec.budget)
    assert len(set(ks)) == 1 and ks[0] % world == 0
    for r, (tr, st) in enumerate(res):
        compare_traces(tr, otr, f"rank {r}/{world} L={L}")
        compare_final_state(st, w, f"rank {r}")
    # the same walk unsharded
    with P.Context(arena_bytes=2 * P.psl_walk_bytes(L, spec.n_lmt, spec.budget) + (64 << 20), max_walks=2) as ctx:
        wid = ctx.submit_ex(L, spec.seed, spec.alpha1, spec.alpha2, spec.budget, ls_lmt=spec.ls_lmt,
                            flip_lmt=spec.flip_lmt, trace_cap=spec.budget)
        ctx.run()
        assert same_decisions(res[0][0], ctx.trace(wid, spec.budget))


def test_sharded_walk_with_candidate_overflow(P):
    """All-ones start, alpha = 1: thousands of tied candidates, so the re-check words include
    the whole-range slots past the first 64 candidates."""
    spec = W.WalkSpec(L=40000, seed=5, alpha1=1, alpha2=2, budget=4, ls_lmt=1, flip_lmt=3)
    s0 = np.ones(spec.L, dtype=np.int8)
    res, _ = _run_sharded(P, spec, 2, init_seq=s0)
    w = oracle_walk(spec, s0=s0)
    otr = w.run(spec.budget)
    for r, (tr, st) in enumerate(res):
        assert int(tr["ncand"].max()) > 64
        compare_traces(tr, otr, f"rank {r}")
        compare_final_state(st, w)


def test_shard_argument_errors(P):
    with P.Context(arena_bytes=1 << 28, max_walks=4) as ctx:
        for bad in [dict(shard_rank=2, shard_count=2), dict(L=900, shard_rank=0, shard_count=2),
                    dict(shard_rank=0, shard_count=17)]:
            kw = dict(L=65535, shard_rank=0, shard_count=2)
            kw.update(bad)
            with pytest.raises(P.PslError):
                ctx.submit_ex(kw["L"], 1, 4, 13, 5, shard_rank=kw["shard_rank"], shard_count=kw["shard_count"])
        wid = ctx.submit_ex(1023, 1, 4, 13, 5)
        with pytest.raises(P.PslError):
            ctx.shard_layout(wid)                 # not a sharded walk
        with pytest.raises(P.PslError):
            ctx.submit_ex(65535, 1, 4, 13, 5, shard_rank=0, shard_count=2)   # needs a context of its own


def _shard_rank(rank, world, port, q, spec_kw):
    import os
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2107_09801_gb300 as P
    from paper_2107_09801_gb300.sharded import ShardedWalk, torch_exchange
    L, budget = spec_kw["L"], spec_kw["budget"]
    with P.Context(arena_bytes=2 * P.psl_walk_bytes(L, 6912, budget) + (64 << 20), max_walks=2) as ctx:
        walk = ShardedWalk(ctx, rank, world, torch_exchange(), trace_cap=budget, **spec_kw)
        n = walk.run()
        tr = ctx.trace(walk.wid, budget)
        st = ctx.export_state(walk.wid)
    q.put((rank, n, tr.tobytes(), st["C"].tobytes(), st["pivot"].tobytes()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_exchange_through_gloo(P):
    """Two processes, each a rank with its own context on the GPU, exchanging the partial
    arrays through a gloo all-reduce on host tensors (no kernel waits on the other process:
    the exchange happens between launches)."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    spec_kw = dict(L=20011, seed=77, alpha1=4, alpha2=11, budget=5, ls_lmt=2, flip_lmt=6)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q, spec_kw)) for r in range(2)]
    [p.start() for p in procs]
    res = sorted(q.get(timeout=600) for _ in procs)
    [p.join(timeout=120) for p in procs]
    assert all(p.exitcode == 0 for p in procs)
    spec = W.WalkSpec(**spec_kw)
    w = oracle_walk(spec)
    otr = w.run(spec.budget)
    for rank, n, tr, C, piv in res:
        assert n == spec.budget
        compare_traces(np.frombuffer(tr, dtype=P.TRACE_DTYPE), otr, f"process {rank}")
        assert np.array_equal(np.frombuffer(C, dtype=np.int32), w.C)
        assert np.array_equal(np.frombuffer(piv, dtype=np.int8), w.s)
