"""Shared helpers of the GPU tests: run walks through the C-ABI and through the oracle,
and compare them record by record."""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle as O

FLAG_MASK = O.IMPROVED | O.WORSE | O.SWITCH | O.PSL_BEST
INT_MAX = 2**31 - 1


def have_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


def limbs32_to_int(limbs) -> int:
    v = 0
    for i, w in enumerate(limbs):
        v |= int(w) << (32 * i)
    if v >> 383:
        v -= 1 << 384
    return v


def oracle_walk(spec, s0=None):
    p = O.WalkParams(L=spec.L, seed=spec.seed, alpha1=spec.alpha1, alpha2=spec.alpha2, n_lmt=spec.n_lmt,
                     ls_lmt=spec.ls_lmt, flip_lmt=spec.flip_lmt)
    return O.Walk(p, s0=s0)


def submit_spec(ctx, spec, trace=True, init_seq=None):
    return ctx.submit_ex(spec.L, spec.seed, spec.alpha1, spec.alpha2, spec.budget, n_lmt=spec.n_lmt,
                         ls_lmt=spec.ls_lmt, flip_lmt=spec.flip_lmt, topk=spec.topk, init_seq=init_seq,
                         trace_cap=spec.budget if trace else 0)


def compare_traces(gpu_tr, orc_tr, label=""):
    """Step-by-step equality of a GPU trace and an oracle trace."""
    assert len(gpu_tr) == len(orc_tr), (label, len(gpu_tr), len(orc_tr))
    prev_best = None
    for t, (g, o) in enumerate(zip(gpu_tr, orc_tr)):
        where = f"{label} step {t}"
        assert g["start"] == o["start"], where
        assert g["kstar"] == o["kstar"], (where, g["kstar"], o["kstar"], g["ncand"])
        assert g["alpha"] == o["alpha"], where
        assert limbs32_to_int(g["value_exact"]) == O.limbs_to_int(o["value_exact"]), where
        assert g["value_step"] == o["value_step"], where
        assert g["unimproved"] == o["unimproved"], where
        assert g["psl"] == o["psl"], (where, g["psl"], o["psl"])
        assert g["psl_best"] == o["psl_best"], (where, g["psl_best"], o["psl_best"])
        assert (g["flags"] & FLAG_MASK) == (o["flags"] & FLAG_MASK), (where, g["flags"], o["flags"])
        assert g["nflip"] == o["nflip"], where
        if g["win_psl"] != INT_MAX:
            assert g["win_psl"] == o["win_psl"] and g["win_psl_j"] == o["win_psl_j"], where
        elif prev_best is not None:
            # the GPU skips neighbour PSLs only when none can beat psl_best
            assert o["win_psl"] >= prev_best, where
        prev_best = o["psl_best"]


def compare_final_state(st, w: O.Walk, label=""):
    assert np.array_equal(st["pivot"], w.s), label
    assert np.array_equal(st["local_best"], w.local_best), label
    assert np.array_equal(st["sol_best"], w.sol_best), label
    assert np.array_equal(st["C"], w.C), label
    assert st["F"] == w.F, label
    assert st["value_local"] == w.value_local, label
    assert st["alpha"] == w.alpha and st["unimproved"] == w.unimproved, label
    assert st["psl"] == w.psl and st["psl_best"] == w.psl_best, label
    assert st["rng_ctr"] == w.rng_ctr, label


def fft_autocorr(s: np.ndarray) -> np.ndarray:
    L = len(s)
    M = 1 << (2 * L - 1).bit_length()
    S = np.fft.rfft(s.astype(np.float64), M)
    return np.rint(np.fft.irfft(np.abs(S) ** 2, M)[:L]).astype(np.int64)


def parallel_eval(s, C, alpha, js, workers=None):
    """Oracle F and PSL of the neighbours js, split over host threads (ctypes drops the GIL)."""
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    js = np.asarray(js, dtype=np.uint32)
    parts = [p for p in np.array_split(js, workers) if len(p)]
    with ThreadPoolExecutor(len(parts)) as ex:
        res = list(ex.map(lambda p: O.eval_neighbours(s, C, alpha, p), parts))
    vals = [v for r in res for v in r[0]]
    psls = np.concatenate([r[1] for r in res])
    return vals, psls


DECISION_FIELDS = ("step", "start", "kstar", "alpha", "unimproved", "psl", "psl_best", "win_psl", "win_psl_j",
                   "flags", "nflip", "value_step", "value_exact")


def same_decisions(a, b) -> bool:
    """Equality of two GPU traces on every decision field (FP32 filter scores, the bound
    and the candidate count may differ between launch configurations)."""
    return len(a) == len(b) and all(np.array_equal(a[f], b[f]) for f in DECISION_FIELDS)


def fp32_error_ratios(trace, F0=None):
    """|FP32 score of the chosen move - its exact Delta F| / bound B, both in the step's
    table units 2^(alpha * scale_e), for every step whose previous exact F is known (the
    first step needs F0; steps right after a phase switch are skipped)."""
    import math
    out = []
    prev = F0
    for r in trace:
        v = limbs32_to_int(r["value_exact"])
        if prev is not None:
            exact = math.ldexp(float(v - prev), -int(r["alpha"]) * int(r["scale_e"]))
            out.append(abs(float(r["score_kstar"]) - exact) / float(r["bound"]))
        prev = None if (r["flags"] & O.SWITCH) else v
    return out
