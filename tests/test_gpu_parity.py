"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Bar: bit-exact C_k, PSL, chosen moves, psl_best / solution_best and exact F;
the FP64 value of F equals the correctly rounded exact value (so it is within
1e-12 of the oracle's FP64 value by construction)."""
import numpy as np
import pytest

import oracle as O
import psl_workloads as W
from helpers import (compare_final_state, compare_traces, fft_autocorr, have_gpu, limbs32_to_int, oracle_walk,
                     parallel_eval, same_decisions, submit_spec)

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]

ARENA = 6 << 30


@pytest.fixture(scope="module")
def P():
    from paper_2107_09801_gb300 import build
    build.build()
    import paper_2107_09801_gb300 as P
    return P


def run_gpu(P, specs, form="batched", init_seqs=None, **ctx_kw):
    with P.Context(form=form, arena_bytes=ctx_kw.pop("arena_bytes", ARENA), max_walks=max(8, len(specs)),
                   **ctx_kw) as ctx:
        ids = [submit_spec(ctx, s, init_seq=None if init_seqs is None else init_seqs[i]) for i, s in enumerate(specs)]
        ctx.run()
        out = []
        for i, s in zip(ids, specs):
            assert ctx.poll(i)["state"] == P.PSL_DONE
            out.append((ctx.trace(i, s.budget), ctx.export_state(i), ctx.poll(i), ctx.best(i)))
        return out


# ------------------------------------------------------------------------------------------------
# a0: autocorrelation
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 3, 13, 31, 32, 33, 63, 64, 65, 1000, 4095])
def test_autocorr_matches_oracle(P, L):
    seqs = np.stack([W.random_pm1(L, 100 * L + r) for r in range(3)])
    with P.Context(arena_bytes=1 << 24, max_walks=8) as ctx:
        C = ctx.autocorr(seqs)
    for r in range(3):
        assert np.array_equal(C[r], O.autocorr(seqs[r]))


@pytest.mark.parametrize("L", [131071, 1048575])
def test_autocorr_full_size_matches_fft(P, L):
    s = W.random_pm1(L, L)
    with P.Context(arena_bytes=1 << 26, max_walks=8) as ctx:
        C = ctx.autocorr(s)[0]
    assert np.array_equal(C.astype(np.int64), fft_autocorr(s))


# ------------------------------------------------------------------------------------------------
# whole trajectories: a1..a6 through the C-ABI, step by step against the oracle
# ------------------------------------------------------------------------------------------------
SMALL = W.small_specs(seed=7, count=10)


@pytest.mark.parametrize("form", ["batched", "plain"])
def test_trajectories_match_oracle(P, form):
    res = run_gpu(P, SMALL, form=form)
    for spec, (tr, st, pl, best) in zip(SMALL, res):
        w = oracle_walk(spec)
        otr = w.run(spec.budget)
        label = f"{form} L={spec.L} seed={spec.seed} a={spec.alpha1}/{spec.alpha2} N={spec.N} ls={spec.ls_lmt}"
        compare_traces(tr, otr, label)
        compare_final_state(st, w, label)
        assert best[0] == w.psl_best and np.array_equal(best[1], w.sol_best)
        assert pl["F"] == float(w.F) and pl["moves"] == spec.budget
        assert pl["flip_evals"] == spec.budget * spec.N


def test_phase_switches_are_exercised(P):
    specs = [W.WalkSpec(L=L, seed=3 + L, alpha1=3, alpha2=11, n_lmt=nl, ls_lmt=2, flip_lmt=fl, budget=150)
             for L, nl, fl in ((31, 31, 4), (127, 40, 10), (255, 6912, 7), (500, 100, 10))]
    res = run_gpu(P, specs)
    for spec, (tr, st, pl, _) in zip(specs, res):
        w = oracle_walk(spec)
        otr = w.run(spec.budget)
        compare_traces(tr, otr, f"L={spec.L}")
        compare_final_state(st, w)
        assert pl["switches"] >= 3


@pytest.mark.parametrize("L", [2, 3, 4, 5, 7])
def test_tiny_lengths(P, L):
    specs = [W.WalkSpec(L=L, seed=s, alpha1=1 + s % 5, alpha2=16, n_lmt=L, ls_lmt=1, flip_lmt=1 + s % L, budget=30)
             for s in range(3)]
    res = run_gpu(P, specs)
    for spec, (tr, st, _, _) in zip(specs, res):
        w = oracle_walk(spec)
        compare_traces(tr, w.run(spec.budget), f"L={L}")
        compare_final_state(st, w)


def test_explicit_start_sequence(P, golden):
    (row,) = golden("barker13.txt")
    barker = np.array([1 if ch == "+" else -1 for ch in row], dtype=np.int8)
    rnd = W.random_pm1(700, 1)
    specs = [W.WalkSpec(L=13, seed=5, n_lmt=13, ls_lmt=3, budget=40),
             W.WalkSpec(L=700, seed=9, n_lmt=250, ls_lmt=20, budget=60)]
    res = run_gpu(P, specs, init_seqs=[barker, rnd])
    for spec, s0, (tr, st, _, best) in zip(specs, (barker, rnd), res):
        w = oracle_walk(spec, s0=s0)
        compare_traces(tr, w.run(spec.budget))
        compare_final_state(st, w)
    assert res[0][3][0] == 1   # Barker-13 stays the best solution (PSL 1)


def test_plain_form_matches_paper_window(P):
    """L = 1023 with the full neighbourhood (N = L), seed 1, alpha 4/13, 2000 moves."""
    spec = W.plain_small().walks[0]
    w = oracle_walk(spec)
    otr = w.run(spec.budget)
    for form in ("batched", "plain"):
        (tr, st, pl, _), = run_gpu(P, [spec], form=form)
        compare_traces(tr, otr, form)
        compare_final_state(st, w, form)


def test_graph_capture_matches_launches(P):
    specs = W.small_specs(seed=11, count=6)
    a = run_gpu(P, specs, steps_per_graph=0)
    b = run_gpu(P, specs, steps_per_graph=8)
    for (ta, sa, _, _), (tb, sb, _, _) in zip(a, b):
        assert ta.tobytes() == tb.tobytes()
        assert np.array_equal(sa["C"], sb["C"])


# ------------------------------------------------------------------------------------------------
# batching: the same walk alone and in a mix gives the same result
# ------------------------------------------------------------------------------------------------
def test_batch_composition_invariance(P):
    specs = W.small_specs(seed=3, count=8, L_choices=(31, 255, 1023, 4095))
    mixed = run_gpu(P, specs)
    for spec, (tr, st, _, _) in zip(specs, mixed):
        (tr1, st1, _, _), = run_gpu(P, [spec])     # alone, its k range is split over more blocks
        assert same_decisions(tr, tr1)
        assert np.array_equal(st["C"], st1["C"]) and np.array_equal(st["pivot"], st1["pivot"])


def test_fused_step_tail_matches_separate_kernels(P):
    """Short walks alone run selection, re-check, decision and update as one kernel; with one
    long walk in the batch they run as four.  Both follow the oracle step by step."""
    specs = [W.WalkSpec(L=L, seed=60 + r, alpha1=1 + r % 5, alpha2=6 + r % 8, budget=40, n_lmt=nl, ls_lmt=3,
                        flip_lmt=4, topk=1 + r % 3)
             for r, (L, nl) in enumerate([(255, 255), (1023, 1023), (2047, 700), (8192, 2048), (31, 31), (700, 6912)])]
    long = W.WalkSpec(L=10000, seed=9, budget=40, ls_lmt=3)
    with P.Context(arena_bytes=ARENA, max_walks=16, steps_per_graph=8) as ctx:
        ids = [submit_spec(ctx, s) for s in specs]
        ctx.profile(1)
        ctx.run()
        assert ctx.profile_read()["tail"][0] > 0
        fused = [(ctx.trace(i, s.budget), ctx.export_state(i)) for i, s in zip(ids, specs)]
    with P.Context(arena_bytes=ARENA, max_walks=16, steps_per_graph=8) as ctx:
        ids = [submit_spec(ctx, s) for s in specs + [long]]
        ctx.profile(1)
        ctx.run()
        assert ctx.profile_read()["tail"][0] == 0
        sep = [(ctx.trace(i, s.budget), ctx.export_state(i)) for i, s in zip(ids, specs + [long])]
    for s, (tf, sf), (ts, ss) in zip(specs, fused, sep):
        w = oracle_walk(s)
        compare_traces(tf, w.run(s.budget), f"fused L={s.L}")
        compare_final_state(sf, w)
        assert same_decisions(tf, ts)
        assert np.array_equal(sf["C"], ss["C"])
    w = oracle_walk(long)
    compare_traces(sep[-1][0], w.run(long.budget), "long")


def test_resizing_sm_share_mid_run_keeps_results(P):
    """The SM count a context's kernels are sized for changes which blocks score which k
    range, never a decision: resize between steps and compare with the oracle."""
    specs = W.small_specs(seed=21, count=6, L_choices=(255, 1023, 4095)) + [W.WalkSpec(L=40000, seed=9, budget=6,
                                                                                          ls_lmt=4)]
    with P.Context(arena_bytes=ARENA, max_walks=16, steps_per_graph=4) as ctx:
        ids = [submit_spec(ctx, s) for s in specs]
        for sms in (7, 0, 33, 152, 1, 0):
            assert ctx.set_max_sms(sms) >= 1
            ctx.step(3)
        ctx.run()
        for i, s in zip(ids, specs):
            w = oracle_walk(s)
            compare_traces(ctx.trace(i, s.budget), w.run(s.budget), f"L={s.L}")
            compare_final_state(ctx.export_state(i), w)
        with pytest.raises(P.PslError):
            ctx.set_max_sms(-1)


def test_continuous_admission_matches_alone(P):
    """Walks submitted while others are on the GPU, admitted as memory frees up."""
    specs = [W.WalkSpec(L=L, seed=100 + r, alpha1=2 + r % 4, alpha2=9 + r % 5, budget=20 + 7 * r, ls_lmt=5)
             for r, L in enumerate([1023, 4095, 255, 16383, 511, 2047, 8191, 127])]
    big = max(P.psl_walk_bytes(s.L, s.n_lmt, s.budget) for s in specs)
    with P.Context(arena_bytes=3 * big, max_walks=4) as ctx:   # room for about three walks at once
        ids, pending, results = {}, list(specs), {}
        while pending or len(results) < len(ids):
            if pending:
                s = pending.pop(0)
                ids[submit_spec(ctx, s)] = s
            ctx.step(5)
            for i, s in list(ids.items()):
                if i not in results and ctx.poll(i)["state"] == P.PSL_DONE:
                    results[i] = (ctx.trace(i, s.budget), ctx.export_state(i))
                    ctx.release(i)
        assert len(results) == len(specs)
    for i, s in ids.items():
        w = oracle_walk(s)
        compare_traces(results[i][0], w.run(s.budget), f"L={s.L}")
        compare_final_state(results[i][1], w)


# ------------------------------------------------------------------------------------------------
# full sizes, in the launch configuration the benchmark times: every walk's final state
# recomputed from scratch, and the last decision of some walks over their whole window
# ------------------------------------------------------------------------------------------------
def _check_walk_state(ctx, wid, st=None):
    """C_k of the pivot by the FFT route (Eq. 2), PSL (Eq. 3), exact F (Eq. 4) and the best
    sequence's PSL recomputed from scratch; returns the exported state."""
    st = st if st is not None else ctx.export_state(wid)
    C = fft_autocorr(st["pivot"])
    assert np.array_equal(st["C"].astype(np.int64), C), wid
    assert st["psl"] == int(np.abs(C[1:]).max()), wid
    Fx, _, _ = O.fitness(st["C"], st["alpha"])
    assert st["F"] == Fx, wid
    psl_b, sol = ctx.best(wid)
    assert psl_b == st["psl_best"] and np.array_equal(sol, st["sol_best"]), wid
    assert int(np.abs(fft_autocorr(sol)[1:]).max()) == psl_b, wid
    return st


def _check_full_size(P, wl, steps, n_check, every_walk=True):
    specs = list(wl.walks)
    with P.Context(arena_bytes=int(1.3 * sum(P.psl_walk_bytes(s.L, s.n_lmt, steps) for s in specs)) + (1 << 28),
                   max_walks=len(specs)) as ctx:
        ids = [submit_spec(ctx, W.with_budget(s, steps)) for s in specs]
        # state before the last step, for the decision check
        ctx.step(steps - 1)
        pre = {}
        rng = np.random.Generator(np.random.PCG64(1))
        check = sorted(rng.choice(len(specs), size=n_check, replace=False).tolist())
        for q in check:
            pre[q] = ctx.export_state(ids[q])
        ctx.step(1)
        for q in check:
            spec, wid = specs[q], ids[q]
            tr = ctx.trace(wid, steps)
            assert len(tr) == steps and ctx.poll(wid)["state"] == P.PSL_DONE
            _check_walk_state(ctx, wid)
            # the last decision over the whole window: k* minimises the exact F (first in scan
            # order), and the window's first minimum PSL is the one the GPU reports
            p = pre[q]
            last = tr[-1]
            L, N = spec.L, spec.N
            assert last["start"] == p["start"]
            js = [(p["start"] + i) % L for i in range(1, N + 1)]
            vals, psls = parallel_eval(p["pivot"], p["C"], p["alpha"], js)
            best = min(range(N), key=lambda n: (vals[n], n))
            assert int(last["kstar"]) == js[best], (q, int(last["kstar"]), js[best])
            assert limbs32_to_int(last["value_exact"]) == vals[best]
            pmin = int(psls.min())
            if last["win_psl"] != 2**31 - 1:
                assert last["win_psl"] == pmin and last["win_psl_j"] == js[int(np.argmin(psls))]
            else:
                assert pmin >= p["psl_best"]   # skipped only when no neighbour can beat psl_best
            assert last["psl_best"] == min(p["psl_best"], pmin)
        if every_walk:
            # every walk of the batch: its whole state after the run, from scratch
            for q, wid in enumerate(ids):
                st = _check_walk_state(ctx, wid)
                assert st["moves"] == steps and ctx.poll(wid)["state"] == P.PSL_DONE, q


def test_full_size_L16383_x4096(P):
    _check_full_size(P, W.batch_16383(), steps=2, n_check=3)


def test_full_size_L131071_x1024(P):
    _check_full_size(P, W.batch_131071(), steps=2, n_check=2)


def test_full_size_L1048575_x148(P):
    _check_full_size(P, W.batch_1048575(), steps=2, n_check=1)


# whole budgets of the workloads on a few walks (phase switches included): the final pivot's
# C, PSL and exact F, the best sequence, and the last decision against the oracle
def test_full_budget_L16383_x8(P):
    _check_full_size(P, W.batch_16383(walks=8), steps=10_000, n_check=3)


def test_full_budget_L131071_x2(P):
    _check_full_size(P, W.batch_131071(walks=2), steps=2000, n_check=2)


def test_full_budget_L1048575_x1(P):
    _check_full_size(P, W.batch_1048575(walks=1), steps=200, n_check=1)


# ------------------------------------------------------------------------------------------------
# many exact ties: more certified candidates than one re-check pass holds (the overflow path)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("form", ["batched", "plain"])
def test_candidate_overflow_matches_oracle(P, form):
    """From the all-ones sequence with alpha = 1 almost every neighbour of the first window
    has the same exact F (the flip changes every C_k = L - k by the same amount), so the
    certified set far exceeds 64 candidates; later steps and a phase switch to alpha = 4
    follow.  L = 40000 spreads each re-check over three k-chunks."""
    specs = [W.WalkSpec(L=255, seed=1, alpha1=1, alpha2=4, n_lmt=255, ls_lmt=3, flip_lmt=5, budget=25),
             W.WalkSpec(L=1023, seed=2, alpha1=1, alpha2=1, n_lmt=1023, ls_lmt=2000, budget=12),
             W.WalkSpec(L=40000, seed=3, alpha1=1, alpha2=2, n_lmt=6912, ls_lmt=1, flip_lmt=3, budget=5)]
    inits = [np.ones(s.L, dtype=np.int8) for s in specs]
    res = run_gpu(P, specs, form=form, init_seqs=inits)
    for spec, s0, (tr, st, _, _) in zip(specs, inits, res):
        assert int(tr["ncand"].max()) > 64, (spec.L, tr["ncand"])
        w = oracle_walk(spec, s0=s0)
        compare_traces(tr, w.run(spec.budget), f"{form} L={spec.L}")
        compare_final_state(st, w)


# ------------------------------------------------------------------------------------------------
# error behaviour of the boundary
# ------------------------------------------------------------------------------------------------
def test_argument_errors(P):
    with P.Context(arena_bytes=1 << 22, max_walks=2) as ctx:
        for bad in [dict(L=1), dict(L=1 << 20), dict(alpha1=0), dict(alpha2=17), dict(budget=0)]:
            kw = dict(L=100, seed=1, alpha1=4, alpha2=13, budget=10)
            kw.update(bad)
            with pytest.raises(P.PslError) as e:
                ctx.submit_ex(kw["L"], kw["seed"], kw["alpha1"], kw["alpha2"], kw["budget"])
            assert e.value.code == -1
        with pytest.raises(P.PslError) as e:
            ctx.submit(100, 1, 4.5, 13, 10)
        assert e.value.code == -1
        with pytest.raises(P.PslError) as e:
            ctx.submit(1048575, 1, 4, 13, 10)      # needs far more than the 4 MB arena
        assert e.value.code == -2
        with pytest.raises(P.PslError) as e:
            ctx.poll(12345)
        assert e.value.code == -3
        wid = ctx.submit(100, 1, 4, 13, 10)
        with pytest.raises(P.PslError) as e:
            ctx.best(wid)                            # still queued
        assert e.value.code == -4
        ctx.run()
        assert ctx.poll(wid)["state"] == P.PSL_DONE
        ctx.release(wid)
        with pytest.raises(P.PslError):
            ctx.poll(wid)


# ------------------------------------------------------------------------------------------------
# configurations of the neighbourhood kernel and the autotuner leave every decision unchanged
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("threads,tile_sb", [(128, 16), (128, 32), (256, 16), (512, 16), (512, 32), (448, 16),
                                             (896, 32)])
def test_hot_kernel_configurations_match_oracle(P, threads, tile_sb):
    specs = W.small_specs(seed=21, count=6, L_choices=(63, 1000, 2047, 4095))
    res = run_gpu(P, specs, hot_threads=threads, hot_tile_sb=tile_sb)
    for spec, (tr, st, _, _) in zip(specs, res):
        w = oracle_walk(spec)
        compare_traces(tr, w.run(spec.budget), f"{threads}/{tile_sb} L={spec.L}")
        compare_final_state(st, w)


@pytest.mark.parametrize("threads,tile_sb", [(512, 32), (448, 16), (896, 32)])
def test_hot_kernel_configurations_long_walks(P, threads, tile_sb):
    """Walks of L >= 4096 (the long-walk kernel variants), alone (k range split over blocks)
    and in a batch, in the regular and the producer / consumer forms."""
    specs = [W.WalkSpec(L=L, seed=80 + L, alpha1=a1, alpha2=a2, budget=b, n_lmt=nl, ls_lmt=2, flip_lmt=5)
             for L, a1, a2, b, nl in ((4096, 4, 13, 12, 6912), (9001, 3, 10, 10, 900), (20011, 4, 13, 8, 6912),
                                      (70001, 2, 11, 4, 6912))]
    for group in (specs, specs[-1:]):
        res = run_gpu(P, group, hot_threads=threads, hot_tile_sb=tile_sb)
        for spec, (tr, st, _, _) in zip(group, res):
            w = oracle_walk(spec)
            compare_traces(tr, w.run(spec.budget), f"{threads}/{tile_sb} L={spec.L}")
            compare_final_state(st, w)


def test_autotune_keeps_results(P, tmp_path):
    specs = W.small_specs(seed=5, count=5, L_choices=(1023, 4095, 8191))
    with P.Context(arena_bytes=ARENA, max_walks=8) as ctx:
        ids = [submit_spec(ctx, s) for s in specs]
        ctx.step(3)
        t, sb = ctx.autotune(reps=2, cache=str(tmp_path / "tune.json"))
        assert (t, sb) in [(a, b) for a in (128, 256, 512) for b in (16, 32)]
        assert ctx.autotune(cache=str(tmp_path / "tune.json")) == (t, sb)   # cached choice
        ctx.run()
        got = [(ctx.trace(i, s.budget), ctx.export_state(i)) for i, s in zip(ids, specs)]
    for spec, (tr, st) in zip(specs, got):
        w = oracle_walk(spec)
        compare_traces(tr, w.run(spec.budget), f"L={spec.L}")
        compare_final_state(st, w)


def test_single_long_walk_k_split(P):
    """One long walk alone is split over k-chunks; it must still follow the oracle."""
    spec = W.WalkSpec(L=65535, seed=3, alpha1=4, alpha2=13, budget=3, ls_lmt=1, flip_lmt=10)
    (tr, st, _, _), = run_gpu(P, [spec])
    w = oracle_walk(spec)
    compare_traces(tr, w.run(spec.budget), "L=65535 alone")
    compare_final_state(st, w)


# ------------------------------------------------------------------------------------------------
# failure path: a bounded device wait that runs out ends one walk, not the context
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("hot", [(256, 32), (896, 32), (448, 16)])
def test_bounded_wait_timeout_marks_only_that_walk(P, hot):
    specs = [W.WalkSpec(L=L, seed=40 + r, alpha1=3, alpha2=9, budget=12, ls_lmt=4)
             for r, L in enumerate([1023, 2047, 4095, 5000])]
    with P.Context(arena_bytes=ARENA, max_walks=8, hot_threads=hot[0], hot_tile_sb=hot[1]) as ctx:
        ids = [submit_spec(ctx, s) for s in specs]
        ctx.step(2)
        ctx.inject_stall(ids[1])
        ctx.run()
        st = [ctx.poll(i) for i in ids]
        assert st[1]["state"] == P.PSL_ERROR and st[1]["error"] == -5       # PSL_ETIMEOUT
        assert st[1]["moves"] == 2
        for k in (0, 2, 3):
            assert st[k]["state"] == P.PSL_DONE
            w = oracle_walk(specs[k])
            compare_traces(ctx.trace(ids[k], specs[k].budget), w.run(specs[k].budget), f"L={specs[k].L}")
        # the context stays usable
        extra = W.WalkSpec(L=511, seed=99, budget=10)
        wid = submit_spec(ctx, extra)
        ctx.run()
        assert ctx.poll(wid)["state"] == P.PSL_DONE
        compare_traces(ctx.trace(wid, extra.budget), oracle_walk(extra).run(extra.budget), "after timeout")


# ------------------------------------------------------------------------------------------------
# serving: requests arriving over time, served by length class on separate streams
# ------------------------------------------------------------------------------------------------
def test_serving_by_length_class_matches_oracle(P):
    from paper_2107_09801_gb300.serving import serve_classes
    trace = [W.Request(0.002 * r, W.WalkSpec(L=L, seed=500 + r, alpha1=2 + r % 4, alpha2=8 + r % 5,
                                               budget=8 + 3 * (r % 5), ls_lmt=3, n_lmt=300))
             for r, L in enumerate([127, 20000, 1023, 8191, 150000, 255, 40000, 4095, 511, 131071])]
    res = serve_classes(trace, arena_bytes=2 << 30, keep_sequences=True)
    assert res.errors == 0 and len(res.latencies_s) == len(trace)
    for r, req in enumerate(trace):
        w = oracle_walk(req.spec)
        w.run(req.spec.budget)
        psl, seq = res.psl_best[r]
        assert psl == w.psl_best and np.array_equal(seq, w.sol_best), r


# ------------------------------------------------------------------------------------------------
# precision: the FP32 score of every chosen move stays within the rigorous bound of its exact ΔF
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("form", ["batched", "plain"])
def test_fp32_scores_within_bound(P, form):
    from helpers import fp32_error_ratios
    specs = W.small_specs(seed=13, count=8, L_choices=(255, 1023, 4095, 16383)) + \
        [W.WalkSpec(L=65535, seed=7, alpha1=4, alpha2=13, budget=6), W.WalkSpec(L=131071, seed=8, alpha1=13,
                                                                                  alpha2=4, budget=4)]
    res = run_gpu(P, specs, form=form)
    ratios = []
    for spec, (tr, st, _, _) in zip(specs, res):
        F0 = O.fitness(O.autocorr(O.init_seq(spec.L, spec.seed)), spec.alpha1)[0]
        r = fp32_error_ratios(tr, F0)
        assert all(np.isfinite(r)), spec
        ratios += r
    assert len(ratios) > 100
    assert max(ratios) <= 1.0, max(ratios)
    print(f"{form}: max |FP32 score - exact| / bound over {len(ratios)} moves = {max(ratios):.3e}")


def test_plain_and_batched_agree_at_full_size(P):
    spec = W.WalkSpec(L=131071, seed=3, budget=3)
    (tb, sb, _, _), = run_gpu(P, [spec], form="batched")
    (tp, sp, _, _), = run_gpu(P, [spec], form="plain")
    assert same_decisions(tb, tp)
    assert np.array_equal(sb["C"], sp["C"]) and np.array_equal(sb["pivot"], sp["pivot"])


# ------------------------------------------------------------------------------------------------
# restart-from-best rounds: each round restarts every walk from the previous round's best
# ------------------------------------------------------------------------------------------------
def test_restart_rounds_match_oracle(P):
    from paper_2107_09801_gb300.rounds import restart_rounds
    L, n, rounds, budget = 255, 3, 3, 40
    with P.Context(arena_bytes=1 << 26, max_walks=8) as ctx:
        hist = restart_rounds(ctx, L, n, rounds, budget, alpha1=4, alpha2=13, seed0=100, ls_lmt=5)
    start = None
    for r in range(rounds):
        found = []
        for i in range(n):
            spec = W.WalkSpec(L=L, seed=100 + r * n + i, alpha1=4, alpha2=13, budget=budget, ls_lmt=5)
            w = oracle_walk(spec, s0=start)
            w.run(budget)
            found.append((w.psl_best, w.sol_best.copy()))
        i_best = min(range(n), key=lambda i: (found[i][0], i))
        start = found[i_best][1]
        assert hist[r].psl_best == found[i_best][0] and hist[r].walk == i_best
        assert np.array_equal(hist[r].sequence, start)
    assert hist[-1].psl_best <= hist[0].psl_best


# ------------------------------------------------------------------------------------------------
# control-parameter studies (alpha pairs, LS_lmt x FLIP_lmt) at a tiny scale: every run's best
# PSL and best sequence equal the oracle's walk with the same parameters
# ------------------------------------------------------------------------------------------------
def test_parameter_studies_match_oracle(P):
    from paper_2107_09801_gb300.ablation import alpha_pairs, ls_flip_grid, moves_for_nse
    L, runs, nse = 255, 2, 255 * 24
    with P.Context(arena_bytes=ARENA, max_walks=64, steps_per_graph=4) as ctx:
        res = alpha_pairs(ctx, L, runs, nse, ls_lmt=4, flip_lmt=3) + \
            ls_flip_grid(ctx, L, runs, nse, ls_values=(8, 2), flip_values=(5, 1), seed0=40)
    budget = moves_for_nse(nse, L)
    assert budget == 24 and len(res) == 3 + 4
    for i, r in enumerate(res):
        st = r.setting
        seed0 = 0 if i < 3 else 40
        for k, got in enumerate(r.psl_best):
            w = oracle_walk(W.WalkSpec(L=L, seed=seed0 + k, alpha1=st.alpha1, alpha2=st.alpha2, budget=budget,
                                       ls_lmt=st.ls_lmt, flip_lmt=st.flip_lmt))
            w.run(budget)
            assert got == w.psl_best, (st, k)


# ------------------------------------------------------------------------------------------------
# one objective (alpha1 == alpha2): the lowest-F pivot; alpha = 2 is the merit-factor energy
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("form", ["batched", "plain"])
def test_lowest_fitness_pivot_matches_oracle(P, form):
    specs = [W.WalkSpec(L=L, seed=70 + r, alpha1=a, alpha2=a, budget=b, ls_lmt=ls, flip_lmt=5)
             for r, (L, a, b, ls) in enumerate([(31, 2, 60, 3), (255, 2, 50, 4), (1023, 2, 30, 1000),
                                                 (4095, 3, 12, 2), (127, 5, 40, 5), (2000, 2, 16, 3)])]
    other = W.WalkSpec(L=255, seed=5, alpha1=2, alpha2=4, budget=10)
    with P.Context(form=form, arena_bytes=ARENA, max_walks=16, steps_per_graph=4) as ctx:
        ids = [submit_spec(ctx, s) for s in specs]
        oid = submit_spec(ctx, other)
        ctx.run()
        for i, s in zip(ids, specs):
            w = oracle_walk(s)
            compare_traces(ctx.trace(i, s.budget), w.run(s.budget), f"L={s.L}")
            F_best, seq = ctx.best_fitness(i)
            assert F_best == w.F_best, (s, F_best, w.F_best)
            assert np.array_equal(seq, w.fbest_seq), s
        with pytest.raises(P.PslError):
            ctx.best_fitness(oid)


@pytest.mark.parametrize("tables", [False, True])
def test_merit_factor_workload_sampled_walks(P, tables):
    """The alpha = 2 workload at full size (L=1023, full neighbourhood, 4096 walks), by the
    closed form and by the tables: every walk's lowest energy equals sum C_k^2 of its
    sequence, and sampled walks follow the oracle."""
    specs = W.labs_1023(4096, budget=12).walks
    with P.Context(arena_bytes=ARENA, max_walks=len(specs), steps_per_graph=4, alpha2_tables=tables) as ctx:
        ids = [submit_spec(ctx, s, trace=False) for s in specs]
        assert ctx.hot_variant().startswith("k_hot_batched" if tables else "k_hot_alpha2")
        ctx.run()
        got = [ctx.best_fitness(i) for i in ids]
        for E, seq in got[::97]:
            c = np.correlate(seq.astype(np.int64), seq.astype(np.int64), "full")[len(seq):]
            assert E == int(np.dot(c, c))
        for r in (0, 1, 2047, 4095):
            w = oracle_walk(specs[r])
            w.run(specs[r].budget)
            assert got[r][0] == w.F_best and np.array_equal(got[r][1], w.fbest_seq), r


# ------------------------------------------------------------------------------------------------
# alpha = 2: the closed-form score (bit planes of C) against the oracle, in every block size,
# and the subset-sum tables on the same walks
# ------------------------------------------------------------------------------------------------
def alpha2_specs():
    # lengths around the word boundaries of the planes, windows shorter than L, the largest
    # length the closed form takes; phase switches every few steps
    shapes = [(2, 2, 3), (3, 3, 4), (13, 13, 10), (33, 33, 12), (64, 64, 12), (100, 50, 15), (1023, 1023, 20),
              (2047, 700, 12), (4095, 4095, 8)]
    return [W.WalkSpec(L=L, seed=300 + r, alpha1=2, alpha2=2, n_lmt=n, ls_lmt=3, flip_lmt=3, budget=b)
            for r, (L, n, b) in enumerate(shapes)]


_ALPHA2_ORACLE = {}


def alpha2_oracle(q, spec):
    """The oracle's walk of alpha2_specs()[q] after its budget (run once per module)."""
    if q not in _ALPHA2_ORACLE:
        w = oracle_walk(spec)
        _ALPHA2_ORACLE[q] = (w, w.run(spec.budget))
    return _ALPHA2_ORACLE[q]


@pytest.mark.parametrize("threads", [128, 256, 448, 512, 896])
def test_alpha2_closed_form_matches_oracle(P, threads):
    specs = alpha2_specs()
    tile = 16 if threads == 448 else 32
    with P.Context(arena_bytes=ARENA, max_walks=16, hot_threads=threads, hot_tile_sb=tile) as ctx:
        ids = [submit_spec(ctx, s) for s in specs]
        assert ctx.hot_variant() == f"k_hot_alpha2<{threads}>"
        ctx.run()
        for q, (i, s) in enumerate(zip(ids, specs)):
            w, otr = alpha2_oracle(q, s)
            compare_traces(ctx.trace(i, s.budget), otr, f"alpha2 {threads} L={s.L}")
            compare_final_state(ctx.export_state(i), w, f"alpha2 {threads} L={s.L}")


def test_alpha2_closed_form_extremes(P):
    """Starts with the widest planes (all ones: |C_k| = L - k, 13 planes at L = 4095) and the
    narrowest (a Barker sequence, |C_k| <= 1); the tables give the same trajectories."""
    barker = np.array([1, 1, 1, 1, 1, -1, -1, 1, 1, -1, 1, -1, 1], dtype=np.int8)
    specs = [W.WalkSpec(L=4095, seed=1, alpha1=2, alpha2=2, n_lmt=4095, ls_lmt=2, flip_lmt=4, budget=6),
             W.WalkSpec(L=2000, seed=2, alpha1=2, alpha2=2, n_lmt=300, ls_lmt=2, flip_lmt=4, budget=6),
             W.WalkSpec(L=13, seed=3, alpha1=2, alpha2=2, n_lmt=13, ls_lmt=2, flip_lmt=2, budget=8)]
    inits = [np.ones(4095, dtype=np.int8), np.ones(2000, dtype=np.int8), barker]
    res = {}
    for tables in (False, True):
        with P.Context(arena_bytes=ARENA, max_walks=8, alpha2_tables=tables) as ctx:
            ids = [submit_spec(ctx, s, init_seq=q) for s, q in zip(specs, inits)]
            name = ctx.hot_variant()
            assert name.startswith("k_hot_batched") if tables else name.startswith("k_hot_alpha2"), name
            ctx.run()
            res[tables] = [ctx.trace(i, s.budget) for i, s in zip(ids, specs)]
    for q, (s, s0) in enumerate(zip(specs, inits)):
        otr = oracle_walk(s, s0=s0).run(s.budget)
        compare_traces(res[False][q], otr, f"closed form L={s.L}")
        compare_traces(res[True][q], otr, f"tables L={s.L}")


def test_alpha2_mixed_batch_uses_tables(P):
    """A batch with any walk outside the closed form's reach (alpha != 2, or L > 4095) is scored
    by the tables throughout, with the same results."""
    specs = alpha2_specs()[4:7] + [W.WalkSpec(L=255, seed=9, alpha1=2, alpha2=5, budget=10),
                                   W.WalkSpec(L=5000, seed=10, alpha1=2, alpha2=2, budget=6)]
    with P.Context(arena_bytes=ARENA, max_walks=16) as ctx:
        ids = [submit_spec(ctx, s) for s in specs]
        assert not ctx.hot_variant().startswith("k_hot_alpha2")
        ctx.run()
        for i, s in zip(ids, specs):
            compare_traces(ctx.trace(i, s.budget), oracle_walk(s).run(s.budget), f"mixed L={s.L}")


# ------------------------------------------------------------------------------------------------
# measurement hooks: events inside captured graphs, counted copies, the pipe microbenchmarks
# ------------------------------------------------------------------------------------------------
def test_graph_profile_and_transfer_counts(P):
    specs = W.small_specs(seed=31, count=4, L_choices=(255, 1023, 4095))
    specs = [W.with_budget(s, 20) for s in specs]
    with P.Context(arena_bytes=ARENA, max_walks=8) as ctx:
        ids = [submit_spec(ctx, s) for s in specs]
        h0, d0 = ctx.transfer_bytes()
        ctx.step(2)
        ctx.profile(2)                   # neighbourhood kernel only, from event nodes of the graph
        ctx.set_steps_per_graph(4)       # captured now: no step runs
        assert ctx.poll(ids[0])["moves"] == 2
        ctx.step(8)
        pr = ctx.profile_read()
        assert pr["hot"][0] == 8 and pr["hot"][1] > 0 and pr["graph"][0] == 2
        assert pr["select"][0] == 0 and pr["apply"][0] == 0
        ctx.profile(1)                   # every kernel: the graph is captured again
        ctx.step(4)
        pr = ctx.profile_read()
        tail = ("select", "recheck", "decide", "apply")
        assert pr["hot"][0] == 4, pr
        if pr["tail"][0]:                # short walks only: the step after the score is one kernel
            assert pr["tail"][0] == 4 and all(pr[k][0] == 0 for k in tail), pr
        else:
            assert all(pr[k][0] == 4 for k in tail), pr
        ctx.profile(0)
        ctx.set_steps_per_graph(0)
        ctx.run()
        h1, d1 = ctx.transfer_bytes()
        assert h1 > h0 and d1 > d0
        psl, seq = ctx.best(ids[0])
        h2, d2 = ctx.transfer_bytes()
        assert h2 == h1 and d2 - d1 == 4 * ((specs[0].L + 31) // 32)
        for i, s in zip(ids, specs):
            w = oracle_walk(s)
            compare_traces(ctx.trace(i, s.budget), w.run(s.budget), f"L={s.L}")
            compare_final_state(ctx.export_state(i), w)


def test_alu_peak_microbenchmark(P):
    import torch
    from paper_2107_09801_gb300 import binding as B
    pk = B.psl_alu_peak(0, torch.cuda.current_stream().cuda_stream)
    assert pk["sm_count"] == torch.cuda.get_device_properties(0).multi_processor_count
    per_clk = {k: pk[k] / (pk["sm_count"] * pk["max_clock_mhz"] * 1e6) for k in ("fadd", "alu", "mix", "lookup", "popc")}
    # lane-ops per SM per clock at the top clock: no pipe can exceed 4 schedulers x 32 lanes
    assert all(0 < v <= 128 * 1.02 for v in per_clk.values()), per_clk
    assert per_clk["fadd"] > 32 and per_clk["mix"] > 32 and per_clk["lookup"] > 4 and per_clk["popc"] > 4, per_clk
    print("lane-ops (lookups) per SM per clock:", per_clk)


def test_best_many_matches_best(P):
    specs = W.small_specs(seed=41, count=7, L_choices=(13, 255, 1000, 4095))
    with P.Context(arena_bytes=ARENA, max_walks=16) as ctx:
        ids = [submit_spec(ctx, s, trace=False) for s in specs]
        ctx.run()
        d0 = ctx.transfer_bytes()[1]
        psl, seqs = ctx.best_many(ids)
        assert ctx.transfer_bytes()[1] - d0 == sum(4 * ((s.L + 31) // 32) for s in specs)
        for q, (i, s) in enumerate(zip(ids, specs)):
            p1, seq1 = ctx.best(i)
            assert psl[q] == p1 and np.array_equal(seqs[q, :s.L], seq1) and not seqs[q, s.L:].any()
            w = oracle_walk(s)
            w.run(s.budget)
            assert psl[q] == w.psl_best and np.array_equal(seqs[q, :s.L], w.sol_best)
        with pytest.raises(P.PslError):
            ctx.best_many(ids + [12345])
