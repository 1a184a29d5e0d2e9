"""Single-walk k-sharding: one walk of Algorithm 1 split over several ranks by shift k.

Sec. 3 evaluates the neighbourhood in parallel; Eq. 4's fitness is a sum over k, so the
score of every neighbour is a sum of per-k-chunk partial scores.  Each rank (one context,
typically one GPU) keeps the walk's whole state, scores and re-checks only its own
k-chunks, and the ranks exchange two zero-filled arrays per step:

  parts = rank's partial FP32 scores [ksplit, N], other ranks' chunks zero
  rc    = rank's exact re-check words of the candidates, other ranks' chunks zero

Every entry of either array is non-zero on at most one rank, so their sum over ranks
(an all-reduce) is exact; selection, the exact decision and the O(L) update then run on
identical inputs on every rank, and the trajectory equals the walk's unsharded one.
Argument marshalling and the exchange only: every step of the path runs in libpsl.so.
"""
from __future__ import annotations

from typing import Callable

import numpy as np

from .binding import PSL_DONE, PSL_RUNNING, Context

Exchange = Callable[[np.ndarray], np.ndarray]


def torch_exchange(group=None, device=None) -> Exchange:
    """Sum over the ranks of a torch.distributed group (gloo on host tensors, or NCCL with
    `device`).  uint32 words travel as int64: one non-zero term per entry, so no carry."""
    import torch
    import torch.distributed as dist

    def ex(a: np.ndarray) -> np.ndarray:
        dt = a.dtype
        t = torch.from_numpy(np.ascontiguousarray(a.astype(np.int64) if dt == np.uint32 else a))
        if device is not None:
            t = t.to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out = t.cpu().numpy()
        return out.astype(np.uint32) if dt == np.uint32 else out

    return ex


class ShardedWalk:
    """One rank's share of a sharded walk.  All ranks call step() together."""

    def __init__(self, ctx: Context, rank: int, world: int, exchange: Exchange, *, L: int, seed: int,
                 alpha1: int = 4, alpha2: int = 13, budget: int = 2000, **walk_kw):
        self.ctx, self.exchange = ctx, exchange
        self.wid = ctx.submit_ex(L, seed, alpha1, alpha2, budget, shard_rank=rank, shard_count=world, **walk_kw)

    def step(self) -> int:
        """One step of Algorithm 1; returns the walk state (PSL_RUNNING or PSL_DONE)."""
        parts = self.exchange(self.ctx.shard_score(self.wid))
        rc = self.exchange(self.ctx.shard_select(self.wid, parts))
        return self.ctx.shard_decide(self.wid, rc)

    def run(self, max_moves: int | None = None) -> int:
        n = 0
        state = PSL_RUNNING
        while state == PSL_RUNNING and (max_moves is None or n < max_moves):
            state = self.step()
            n += 1
        return n


def step_together(walks: list[ShardedWalk]) -> list[int]:
    """One step of every rank of a sharded walk held in this process (ranks emulated in one
    process, e.g. several contexts on one GPU): the exchanges are plain sums."""
    parts = [w.ctx.shard_score(w.wid) for w in walks]
    total = np.sum(parts, axis=0, dtype=np.float32)
    rcs = [w.ctx.shard_select(w.wid, total) for w in walks]
    rc = np.sum([r.astype(np.uint64) for r in rcs], axis=0).astype(np.uint32)
    return [w.ctx.shard_decide(w.wid, rc) for w in walks]


def run_together(walks: list[ShardedWalk]) -> int:
    """Steps the in-process ranks until the walk reaches its budget; returns the steps run."""
    n = 0
    while True:
        states = step_together(walks)
        n += 1
        assert len(set(states)) == 1, states  # every rank decides the same
        if states[0] != PSL_RUNNING:
            return n if states[0] == PSL_DONE else -n
