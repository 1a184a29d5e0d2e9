"""Restart-from-best rounds (Sec. 4.2 of the paper): after a round of independent walks,
the best sequence found (lowest PSL; the first walk of the round on ties) becomes the
start sequence of every walk of the next round."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .binding import Context


@dataclass
class RoundResult:
    round: int
    psl_best: int
    walk: int               # index of the walk (within the round) that found it
    sequence: np.ndarray    # +-1 values


def restart_rounds(ctx: Context, L: int, walks_per_round: int, rounds: int, budget: int, alpha1: int = 4,
                   alpha2: int = 13, seed0: int = 0, start: np.ndarray | None = None, **walk_kw) -> list[RoundResult]:
    """Runs `rounds` rounds of `walks_per_round` walks; walk i of round r has seed
    seed0 + r * walks_per_round + i.  Round 0 starts from Rand(L, SEED) (or from `start`)."""
    history = []
    for r in range(rounds):
        ids = [ctx.submit_ex(L, seed0 + r * walks_per_round + i, alpha1, alpha2, budget, init_seq=start, **walk_kw)
               for i in range(walks_per_round)]
        ctx.run()
        found = [ctx.best(w) for w in ids]
        for w in ids:
            ctx.release(w)
        i_best = min(range(walks_per_round), key=lambda i: (found[i][0], i))
        start = found[i_best][1]
        history.append(RoundResult(r, found[i_best][0], i_best, start.copy()))
    return history
