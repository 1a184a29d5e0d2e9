"""The exchange of single-walk k-sharding on CPU (gloo, world size 2), without a GPU: each
rank produces zero-filled arrays of its own k-chunks (partial FP32 scores, exact re-check
words), and after the sums over ranks every rank holds the full arrays, exactly -- the
property that makes selection and decision identical on every rank.  A fake context stands
in for the library."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

KS, N, WORDS, STEPS = 6, 37, 5 * 12, 3


def full_arrays(step):
    rng = np.random.Generator(np.random.PCG64(step))
    parts = (rng.standard_normal((KS, N)) * 10.0 ** rng.integers(-30, 30, (KS, N))).astype(np.float32)
    parts[0, :3] = [np.float32(1e-40), np.float32(3.4e38), np.float32(-7.0)]     # subnormal, near max, negative
    words = rng.integers(0, 2**32, WORDS, dtype=np.uint64).astype(np.uint32)
    words[:4] = [0xFFFFFFFF, 0x80000000, 0, 1]
    return parts, words


class FakeShardCtx:
    """The shard_* calls of a context, for a walk whose k-chunk c (score rows) and re-check
    word w belong to rank c % world and (w // 12) % world."""

    def __init__(self, rank, world):
        self.rank, self.world, self.step = rank, world, 0
        self.got_parts, self.got_words = [], []

    def submit_ex(self, *a, shard_rank=0, shard_count=0, **kw):
        assert (shard_rank, shard_count) == (self.rank, self.world)
        return 0

    def shard_score(self, wid):
        parts, _ = full_arrays(self.step)
        mine = np.zeros_like(parts)
        own = [c for c in range(KS) if c % self.world == self.rank]
        mine[own] = parts[own]
        return mine

    def shard_select(self, wid, parts):
        self.got_parts.append(parts.copy())
        _, words = full_arrays(self.step)
        mine = np.zeros_like(words)
        own = (np.arange(WORDS) // 12) % self.world == self.rank
        mine[own] = words[own]
        return mine

    def shard_decide(self, wid, words):
        self.got_words.append(words.copy())
        self.step += 1
        from paper_2107_09801_gb300.binding import PSL_DONE, PSL_RUNNING
        return PSL_DONE if self.step == STEPS else PSL_RUNNING


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2107_09801_gb300.sharded import ShardedWalk, torch_exchange
    ctx = FakeShardCtx(rank, world)
    walk = ShardedWalk(ctx, rank, world, torch_exchange(), L=65535, seed=1)
    n = walk.run()
    q.put((rank, n, [p.tobytes() for p in ctx.got_parts], [w.tobytes() for w in ctx.got_words]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_gives_every_rank_the_full_arrays(world):
    pytest.importorskip("torch.distributed")
    mpc = mp.get_context("spawn")
    q = mpc.Queue()
    port = _free_port()
    procs = [mpc.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    [p.start() for p in procs]
    res = sorted(q.get(timeout=180) for _ in procs)
    [p.join(timeout=60) for p in procs]
    assert all(p.exitcode == 0 for p in procs)
    for rank, n, parts, words in res:
        assert n == STEPS
        for step in range(STEPS):
            want_p, want_w = full_arrays(step)
            got_p = np.frombuffer(parts[step], dtype=np.float32).reshape(KS, N)
            got_w = np.frombuffer(words[step], dtype=np.uint32)
            assert np.array_equal(got_p.view(np.uint32), want_p.view(np.uint32)), (rank, step)   # bit for bit
            assert np.array_equal(got_w, want_w), (rank, step)
