"""Control-parameter studies of Sec. 4.1 of the paper at a chosen scale: the two-phase
fitness exponents (alpha1/alpha2 pairs, Table "alpha") and the phase-switch trigger
LS_lmt against the perturbation size FLIP_lmt (Table "par").  Each run is one walk with a
budget of sequence evaluations (NSE, Table "speed": one evaluated neighbour is one
NSE), so a run gets ceil(NSE / N) moves with N = min(N_lmt, L).  Run r of every setting
starts from the same seed r, so the settings are compared on paired starts.  All runs
of a study go to the GPU as one batch of walks with per-walk parameters."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .binding import PSL_DONE, Context


def moves_for_nse(nse: int, L: int, n_lmt: int = 6912) -> int:
    """Moves of a run limited to `nse` sequence evaluations: each move evaluates N = min(N_lmt, L)."""
    return max(1, -(-int(nse) // min(int(n_lmt), int(L))))


@dataclass(frozen=True)
class Setting:
    alpha1: int
    alpha2: int
    ls_lmt: int
    flip_lmt: int


@dataclass
class SettingResult:
    setting: Setting
    psl_best: list          # per run, run r has seed seed0 + r

    @property
    def mean(self) -> float:
        return float(np.mean(self.psl_best))

    @property
    def std(self) -> float:
        return float(np.std(self.psl_best, ddof=1)) if len(self.psl_best) > 1 else 0.0


def run_settings(ctx: Context, L: int, settings, runs: int, nse: int, n_lmt: int = 6912,
                 seed0: int = 0) -> list[SettingResult]:
    """Runs `runs` walks of length L for every setting, each limited to `nse` sequence
    evaluations, and returns their best PSL values."""
    budget = moves_for_nse(nse, L, n_lmt)
    ids = []
    for st in settings:
        ids.append([ctx.submit_ex(L, seed0 + r, st.alpha1, st.alpha2, budget, n_lmt=n_lmt, ls_lmt=st.ls_lmt,
                                  flip_lmt=st.flip_lmt) for r in range(runs)])
    ctx.run()
    out = []
    for st, row in zip(settings, ids):
        psl = []
        for w in row:
            if ctx.poll(w)["state"] != PSL_DONE:
                raise RuntimeError(f"walk {w} of setting {st} did not finish")
            psl.append(int(ctx.best(w)[0]))
            ctx.release(w)
        out.append(SettingResult(st, psl))
    return out


def alpha_pairs(ctx: Context, L: int, runs: int, nse: int, pairs=((4, 13), (4, 4), (13, 13)), ls_lmt: int = 2000,
                flip_lmt: int = 10, **kw) -> list[SettingResult]:
    """Table "alpha": the two-phase pair against a single exponent used in both phases."""
    return run_settings(ctx, L, [Setting(a1, a2, ls_lmt, flip_lmt) for a1, a2 in pairs], runs, nse, **kw)


def ls_flip_grid(ctx: Context, L: int, runs: int, nse: int, ls_values=(4000, 2000, 1000, 500, 250),
                 flip_values=(20, 10, 5, 2, 1), alpha1: int = 4, alpha2: int = 13, **kw) -> list[SettingResult]:
    """Table "par": every (LS_lmt, FLIP_lmt) pair at alpha1/alpha2."""
    return run_settings(ctx, L, [Setting(alpha1, alpha2, ls, fl) for fl in flip_values for ls in ls_values],
                        runs, nse, **kw)
