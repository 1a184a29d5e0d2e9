#!/usr/bin/env python
"""Benchmark of the limited-neighbourhood search (arXiv 2107.09801, Algorithm 1).

Metric: flip-evals/s (neighbours scored per second, the paper's NSE/s) at
L = 2^17 - 1 over 1024 independent walks (seeds 0..1023, alpha 4/13,
N_lmt 6912), batched form; the plain form (one walk per launch, one thread per
neighbour, host-side selection) is measured beside it.  One step = one pass of
the whole hot path (score window, select, exact re-check, decide, O(L) update)
for every walk of the batch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import dataclasses
import csv
import hashlib
import re
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import psl_workloads as W  # noqa: E402

METRIC = "flip evals/s at L=2^17−1 (batched vs plain); p50/p99 serving latency"
UNIT = "flip-evals/s"
PAPER_A100_L131071 = 638043  # Table 4 of the paper: one walk on an A100 SXM4 (context only)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--walks", type=int, default=1024)
    ap.add_argument("--workload", default="L131071", choices=["L131071", "L16383", "L1048575", "LABS_L1023"],
                    help="batch timed as the main line (default: the L=2^17-1 batch of the metric)")
    ap.add_argument("--plain-steps", type=int, default=4)
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--alpha2-tables", action="store_true",
                    help="score alpha = 2 batches with the subset-sum tables instead of the closed form")
    ap.add_argument("--other-configs", type=int, default=1, help="also time the L=16383 x 4096 and L=1048575 x 148 batches")
    ap.add_argument("--serving", type=int, default=100,
                    help="requests of the serving trace run at 0.8x the capacity measured by the probe (0: skip)")
    ap.add_argument("--serving-probe", type=int, default=40,
                    help="requests of the saturated probe (arrivals at --serving-rate) that measures the capacity")
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--graph-steps", type=int, default=0,
                    help="steps per CUDA graph launch in the timed region (0: all timed steps, at most 50)")
    ap.add_argument("--serving-study", type=int, default=0,
                    help="run only the serving study on this many requests: the trace at --serving-rate "
                         "(saturated), then at 0.8x the measured capacity; prints its own JSON line")
    ap.add_argument("--serving-study-light", type=int, default=300,
                    help="requests of the 0.8x-capacity leg of the serving study")
    ap.add_argument("--serving-compare", type=int, default=0,
                    help="serving study: also run this many requests at --serving-rate under each SM split "
                         "(fixed, by outstanding work, by live requests)")
    ap.add_argument("--serving-policy", default="balanced", choices=["balanced", "requests", "work"],
                    help="SM split between the serving length classes")
    ap.add_argument("--ablation", action="store_true",
                    help="run only the control-parameter studies (alpha pairs; LS_lmt x FLIP_lmt) at reduced "
                         "scale; prints their own JSON line")
    ap.add_argument("--ablation-L", type=int, default=16383)
    ap.add_argument("--ablation-runs", type=int, default=30)
    ap.add_argument("--ablation-nse", type=float, default=1e9, help="sequence evaluations per run, alpha pairs")
    ap.add_argument("--grid-runs", type=int, default=10)
    ap.add_argument("--grid-nse", type=float, default=2e8, help="sequence evaluations per run, LS x FLIP grid")
    ap.add_argument("--hot-threads", type=int, default=0, help="force the neighbourhood-kernel block size")
    ap.add_argument("--hot-tile", type=int, default=0, help="force the k-tile (super-blocks of 30)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        self.f.close()
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# the oracle on the host cores (reference arm and cpu_baseline)
# ------------------------------------------------------------------------------------------------
class OracleSampler:
    """Times the oracle's neighbour evaluation (exact F and PSL of each neighbour, Eq. 2-4
    through the one-element flip of Sec. 3) on `threads` host threads, each on its own walk
    of length L, over bounded samples of the walk's window."""

    def __init__(self, L: int, n_lmt: int, alpha: int, threads: int | None = None):
        import oracle as O
        self.O, self.L, self.n_lmt, self.alpha = O, L, n_lmt, alpha
        self.threads = threads or os.cpu_count() or 1
        self.walks = [None] * self.threads

        def init(r):
            self.walks[r] = O.Walk(O.WalkParams(L=L, seed=r, alpha1=alpha, alpha2=13, n_lmt=n_lmt))

        ts = [threading.Thread(target=init, args=(r,)) for r in range(self.threads)]
        [t.start() for t in ts]
        [t.join() for t in ts]
        w0 = self.walks[0]
        t0 = time.perf_counter()
        O.eval_neighbours(w0.s, w0.C, alpha, [1, 2])
        self.per = max((time.perf_counter() - t0) / 2, 1e-5)

    def sample_one_core(self, seconds: float):
        """The same work on one host thread (the paper's CPU solver ran on one core)."""
        n_per = int(max(1, min(self.n_lmt, seconds / self.per)))
        w = self.walks[0]
        start = self.O.splitmix64(w.p.seed, w.rng_ctr) % self.L
        t0 = time.perf_counter()
        self.O.eval_neighbours(w.s, w.C, self.alpha, [(start + i) % self.L for i in range(1, n_per + 1)])
        dt = time.perf_counter() - t0
        return n_per / dt, n_per, dt

    def sample(self, seconds: float):
        n_per = int(max(1, min(self.n_lmt, seconds / self.per)))

        def work(r):
            w = self.walks[r]
            start = self.O.splitmix64(w.p.seed, w.rng_ctr) % self.L
            self.O.eval_neighbours(w.s, w.C, self.alpha, [(start + i) % self.L for i in range(1, n_per + 1)])

        ts = [threading.Thread(target=work, args=(r,)) for r in range(self.threads)]
        t0 = time.perf_counter()
        [t.start() for t in ts]
        [t.join() for t in ts]
        dt = time.perf_counter() - t0
        return self.threads * n_per / dt, n_per, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    L, N = 131071, W.N_LMT
    sampler = OracleSampler(L, N, 4)
    # each step: every host thread evaluates a bounded slice of its walk's window
    per_step_s = max(0.5, min(6.0, 150.0 / max(1, args.steps + args.warmup)))
    vals = []
    for s in range(args.warmup + args.steps):
        v, n_per, dt = sampler.sample(per_step_s)
        if s >= args.warmup:
            vals.append((v, dt, n_per))
    value = statistics.median(v for v, _, _ in vals)
    cores = sampler.threads
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.median(d for _, d, _ in vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i384 exact (oracle)",
            "data": "synthetic", "config": {"workload": "L131071_x1024", "L": L, "n_lmt": N, "alpha": "4/13"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step: {cores} threads x {vals[0][2]} window neighbours of their own "
                                       f"L=131071 walk (exact F and PSL each)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def _code_only(src: str) -> str:
    """C++ source without comments and blank lines (string literals here hold no comment
    markers), so that the hash follows the code the counters were measured on."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_source_hash(kernel: str = "k_hot_batched") -> str:
    """Hash of the code of a neighbourhood kernel (its translation unit and device header,
    comments left out)."""
    h = hashlib.sha256()
    tu = "psl_alpha2.cu" if kernel.startswith("k_hot_alpha2") else "psl_hot.cu"
    for fn in (tu, "psl_device.cuh"):
        with open(os.path.join(ROOT, "paper_2107_09801_gb300", "csrc", fn), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


KERNELS_PER_PHASE = {"hot": 1, "select": 1, "recheck": 2, "decide": 1, "apply": 2, "tail": 1}


def kernels_per_step(breakdown: dict) -> int:
    """Kernel launches of one step from a per-phase breakdown of whole steps (a phase's
    launches count its brackets, one per step)."""
    steps = max(breakdown.get("hot", (0, 0.0))[0], 1)
    total = sum(KERNELS_PER_PHASE.get(k, 1) * n for k, (n, _) in breakdown.items() if n)
    return int(round(total / steps))


def plane_steps_per_flip_eval(L: int, psls) -> float:
    """Bit-plane steps (logic op, population count, add) of the alpha = 2 closed form per
    flip-eval, averaged over the neighbour position: P = bitlen(PSL) + 1 planes for each of the
    about (L-1)/32 + 1 forward and backward words, and one step per word of the
    min(j, L-1-j) shifts of the partner-product term."""
    P = float(np.mean([int(p).bit_length() + 1 for p in psls])) if len(psls) else 1.0
    return P * ((L - 1) / 32.0 + 1.0) + (L / 4.0) / 32.0


def stored_counters(kernel: str, workload: str):
    """Per-launch ncu counters of a kernel (DRAM bytes, warp instructions), only if they were
    taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
        rec = d[kernel][workload]
        if rec.get("source_hash") == kernel_source_hash(kernel):
            return rec
    except Exception:
        pass
    return None


WORKLOADS = {"L131071": W.batch_131071, "L16383": W.batch_16383, "L1048575": W.batch_1048575,
             "LABS_L1023": W.labs_1023}


def rank_specs(walks: int, rank: int, workload: str = "L131071"):
    """The walks one rank runs: the workload (by default L=131071) with seeds offset by rank, so
    ranks never share a walk (weak scaling: every rank keeps the same number of walks)."""
    wl = WORKLOADS[workload](walks=walks)
    return wl, [dataclasses.replace(s, seed=s.seed + rank * walks) for s in wl.walks]


def aggregate(local_ms: float, local_units: int, world: int, dist=None, device=None):
    """Whole-job throughput: units summed over ranks / the slowest rank's time."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) / 1000.0), float(t.item())


def fp32_error_stats(traces) -> dict:
    """Worst |FP32 score - exact Delta F| of the chosen moves relative to the rigorous bound B,
    over consecutive traced steps (the exact F before each step is the previous step's)."""
    import math
    worst, worst_rel, n = 0.0, 0.0, 0
    for tr in traces:
        prev = None
        for r in tr:
            v = 0
            for i, w in enumerate(r["value_exact"]):
                v |= int(w) << (32 * i)
            if v >> 383:
                v -= 1 << 384
            if prev is not None:
                exact = math.ldexp(float(v - prev), -int(r["alpha"]) * int(r["scale_e"]))
                err = abs(float(r["score_kstar"]) - exact)
                worst = max(worst, err / float(r["bound"]))
                worst_rel = max(worst_rel, err / max(abs(exact), 1e-300))
                n += 1
            prev = None if (int(r["flags"]) & 4) else v
    return {"moves_checked": n, "max_err_over_bound": worst, "max_rel_err": worst_rel}


def term_counts(L: int) -> dict:
    """Per flip-eval, averaged over the neighbour position j (a window start is uniform):
    nominal terms L-1; live terms (shifts with at least one partner: k <= max(j, L-1-j));
    and the lookups of the neighbourhood kernel's tables (two per 5 two-partner shifts, one
    per 5 one-partner shifts)."""
    j = np.arange(L, dtype=np.float64)
    kin = np.minimum(j, L - 1 - j)
    kout = np.maximum(j, L - 1 - j)
    return {"nominal": float(L - 1), "live": float(kout.mean()),
            "lookups": float((2.0 * kin / 5.0 + (kout - kin) / 5.0).mean())}


def measure_alu_peak(local: int, stream) -> dict:
    """The microbenchmarks of the CUDA-core pipes (psl_alu_peak) with the SM clock sampled
    while they run."""
    from paper_2107_09801_gb300 import binding as B
    clk = ClockSampler(local)
    clk.start()
    pk = B.psl_alu_peak(local, stream.cuda_stream)
    pk["clocks"] = clk.stop()
    return pk


def hot_roofline(walks_x_N: int, L: int, hot_avg_ms: float, peak: dict, mhz_run: float, counters,
                 kernel: str, psls=()) -> dict:
    """Roofline of the neighbourhood kernel: 2 lane-ops per (neighbour, shift) term against the
    measured FP32-add / integer-add / logic-op mix rate, scaled to the clock of the timed region;
    also on live terms, and against the lookup ceiling of the kernel's own inner pattern."""
    tc = term_counts(L)
    mhz_peak = peak["clocks"].get("sm_mhz") or peak["max_clock_mhz"]
    scale = (mhz_run / mhz_peak) if (mhz_run and mhz_peak) else 1.0
    p_mix = peak["mix"] * scale
    p_lookup = peak["lookup"] * scale
    sec = hot_avg_ms / 1000.0
    achieved = walks_x_N * 2 * tc["nominal"] / sec
    achieved_live = walks_x_N * 2 * tc["live"] / sec
    lookups = walks_x_N * tc["lookups"] / sec
    out = {"bound": "alu", "kernel": kernel, "achieved": achieved / 1e12, "peak": p_mix / 1e12,
           "unit": "Tops/s", "frac": achieved / p_mix,
           "peak_basis": f"measured: psl_alu_peak mix microbenchmark (FP32 add, integer add, logic op 1:1:1 on "
                         f"{peak['sm_count']} SMs) {peak['mix'] / 1e12:.2f} Tops/s at {mhz_peak:.0f} MHz, scaled to "
                         f"the timed region's {mhz_run:.0f} MHz",
           "ops_basis": "2 lane-ops per (neighbour, shift) term, (L-1) terms per flip-eval",
           "frac_live_terms": achieved_live / p_mix,
           "live_basis": f"2 lane-ops per term with a partner: {tc['live']:.0f} of {tc['nominal']:.0f} shifts per "
                         "flip-eval on average",
           "lookup_ceiling": {"lookups_per_s_measured": peak["lookup"], "lookups_per_flip_eval": tc["lookups"],
                              "flip_evals_per_s_ceiling": p_lookup / tc["lookups"],
                              "frac": lookups / p_lookup},
           "traffic": None, "issue_frac": None}
    if kernel.startswith("k_hot_alpha2"):
        # the closed form does no table lookups: its own ceiling is the bit-plane step rate
        steps = plane_steps_per_flip_eval(L, psls)
        p_popc = peak["popc"] * scale
        out["lookup_ceiling"] = None
        out["plane_step_ceiling"] = {"plane_steps_per_s_measured": peak["popc"], "plane_steps_per_flip_eval": steps,
                                     "flip_evals_per_s_ceiling": p_popc / steps,
                                     "frac": walks_x_N * steps / sec / p_popc}
    if counters:
        out["traffic"] = counters.get("bytes_per_launch")
        if counters.get("warp_inst_per_launch") and peak.get("sm_count"):
            # 4 schedulers per SM, one warp instruction each per clock
            issue_peak = peak["sm_count"] * 4 * mhz_run * 1e6
            out["issue_frac"] = counters["warp_inst_per_launch"] / sec / issue_peak
    return out


def serving_leg(args, local, sms):
    """Continuous batching at a sustainable rate: a saturated probe of the serving trace measures
    the capacity (requests / wall time), then requests arrive at 0.8x that capacity."""
    import paper_2107_09801_gb300 as P
    from paper_2107_09801_gb300.serving import serve_classes

    def leg(n, rate, offset=0):
        trace = W.serving_trace(n_requests=n + offset, rate_hz=rate)[offset:]
        t0 = trace[0].t_arrival
        trace = [W.Request(r.t_arrival - t0, r.spec) for r in trace]
        arena = min(24 << 30, int(sum(P.psl_walk_bytes(r.spec.L, r.spec.n_lmt, 0) for r in trace) * 1.5) + (256 << 20))
        res = serve_classes(trace, arena, sm_count=sms, ctx_kwargs=dict(device=local),
                            share_policy=args.serving_policy)
        return res, trace

    probe, _ = leg(args.serving_probe, args.serving_rate)
    capacity = args.serving_probe / probe.wall_s
    rate = 0.8 * capacity
    res, trace = leg(args.serving, rate, offset=args.serving_probe)   # requests not seen by the probe
    return dict(res.summary(), rate_hz=rate, capacity_requests_per_s=capacity,
                capacity_basis=f"saturated probe: {args.serving_probe} requests arriving at {args.serving_rate} "
                               f"req/s, completed in {probe.wall_s:.1f} s (p50 {probe.summary()['p50_s']:.2f} s)",
                arrival_span_s=trace[-1].t_arrival,
                trace="Poisson arrivals at 0.8x capacity, m~U{10..20}, budgets ~U{100..10^4}, alpha1~U{2..6}, "
                      "alpha2~U{alpha1+4..13}, request r has seed r",
                classes="L<=2^14, <=2^17, <=2^20: one context, stream and host thread each; SMs split by "
                        f"{args.serving_policy} (8-SM floor per busy class)")


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2107_09801_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    wl, specs = rank_specs(args.walks, rank, args.workload)
    L, N = specs[0].L, specs[0].N
    G = args.graph_steps or min(args.steps, 50)
    K2 = min(args.steps, 10)
    assert args.warmup + args.steps + K2 + 2 <= specs[0].budget and args.warmup >= 1
    need = sum(P.psl_walk_bytes(s.L, s.n_lmt, 0) for s in specs)
    arena = torch.empty(int(need * 1.1) + (64 << 20), dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    peak = measure_alu_peak(local, stream)
    with P.Context(arena_tensor=arena, stream=stream, max_walks=len(specs), device=local,
                   alpha2_tables=args.alpha2_tables) as ctx:
        # the first walks keep a per-step trace so that the FP32 score error can be stated
        n_traced = min(8, len(specs))
        ids = [ctx.submit_ex(s.L, s.seed, s.alpha1, s.alpha2, s.budget, topk=s.topk,
                             trace_cap=args.warmup + args.steps + K2 + 2 if q < n_traced else 0)
               for q, s in enumerate(specs)]
        ctx.step(1)             # admission and initialisation
        if args.hot_threads or args.hot_tile:
            ctx._set_hot(args.hot_threads or 256, args.hot_tile or 32)
            tuned = (args.hot_threads or 256, args.hot_tile or 32)
        else:
            tuned = ctx.autotune(reps=2) if not args.no_autotune else None
        ctx.step(args.warmup - 1)
        # the timed steps run from a CUDA graph of G steps, captured here (no step runs), with
        # event-record nodes around the neighbourhood kernel only
        ctx.profile(2)
        ctx.set_steps_per_graph(G)
        barrier()
        clk = ClockSampler(local)
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(args.steps)
        e1.record(stream)
        barrier()
        clocks = clk.stop()
        prof = ctx.profile_read()
        ctx.profile(0)
        ms = e0.elapsed_time(e1)
        hot_name = ctx.hot_variant()
        psls = [ctx.poll(i)["psl"] for i in ids[:64]]
        # the same steps as plain launches (no graph, no events), for comparison
        ctx.set_steps_per_graph(0)
        barrier()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        ctx.step(K2)
        p1.record(stream)
        barrier()
        ms_plain_launch = p0.elapsed_time(p1)
        # per-kernel breakdown, untimed: every kernel between its own events
        ctx.profile(1)
        ctx.step(2)
        breakdown = ctx.profile_read()
        ctx.profile(0)
        st = [ctx.poll(i) for i in ids[:4]]
        assert all(s["moves"] == args.warmup + args.steps + K2 + 2 for s in st)
        fp32_err = fp32_error_stats([ctx.trace(i, args.warmup + args.steps) for i in ids[:n_traced]])
    flip_evals_rank = len(specs) * N * args.steps
    value, ms_max = aggregate(ms, flip_evals_rank, world, dist, dev)

    # roofline of the dominant kernel (the neighbourhood score), live durations in the timed region
    n_hot, hot_ms = prof.get("hot", (0, 0.0))
    hot_avg_ms = hot_ms / max(n_hot, 1)
    mhz = clocks.get("sm_mhz") or peak["max_clock_mhz"]
    roof = hot_roofline(len(specs) * N, L, hot_avg_ms, peak, mhz, stored_counters(hot_name, wl.name), hot_name,
                        psls)
    roof["hot_launches_timed"] = n_hot
    kernels = {k: {"launches": n, "avg_ms": (ms_ / n if n else 0.0)} for k, (n, ms_) in breakdown.items() if n}
    # kernels per step, from the untimed breakdown (each profiled phase brackets its kernels):
    # the neighbourhood score, then either the fused tail (short walks) or select, the two
    # re-check kernels (histogram / term sums), decide and the two update passes (ordinary
    # moves; initialisation and switches)
    launches = args.steps * kernels_per_step(breakdown)

    # plain form: one walk per launch, one thread per neighbour, host-side selection
    plain = None
    if not args.no_plain and rank == 0:
        with P.Context(form="plain", arena_bytes=P.psl_walk_bytes(L, N, 0) + (16 << 20), stream=stream,
                       max_walks=2, device=local) as pc:
            pid = pc.submit(L, 0, specs[0].alpha1, specs[0].alpha2, 2000)
            pc.step(1)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            pc.step(args.plain_steps)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            plain = {"value": N * args.plain_steps / dt, "walks": 1, "steps": args.plain_steps,
                     "ms_per_step": 1000 * dt / args.plain_steps}

    # end to end through the public API: submit from the host, initialise, run the steps from a
    # CUDA graph, read every walk's status and best sequence back into host memory; the bytes
    # are the library's own count of what it copied
    e2e = None
    if not args.no_e2e:
        barrier()
        t0 = time.perf_counter()
        hot = dict(hot_threads=tuned[0], hot_tile_sb=tuned[1]) if tuned else {}
        with P.Context(arena_tensor=arena, stream=stream, max_walks=len(specs), device=local,
                       steps_per_graph=G, alpha2_tables=args.alpha2_tables, **hot) as ctx:
            ids = [ctx.submit(s.L, s.seed, s.alpha1, s.alpha2, s.budget) for s in specs]
            ctx.step(args.steps)
            psl_best, seqs = ctx.best_many(ids)      # every walk's best sequence, one synchronisation
            h2d, d2h = ctx.transfer_bytes()
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        td = torch.tensor([dt], device=dev)
        if world > 1:
            dist.all_reduce(td, op=dist.ReduceOp.MAX)
        e2e = {"value": world * flip_evals_rank / float(td.item()), "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "bytes_counted": "by the library at each host<->device copy (psl_transfer_bytes)",
               "includes": "submit, walk initialisation, graph capture, steps, status readback, every walk's best "
                           "sequence read back (psl_best_many)"}

    # the small configuration: L = 1023, one walk from seed 1, N = L, 2000 moves, time to budget
    small = None
    if args.other_configs and rank == 0:
        spec1 = W.plain_small().walks[0]
        small = {"workload": W.plain_small().name, "moves": spec1.budget}
        for label, kw in (("plain_s", dict(form="plain")), ("batched_graph_s", dict(steps_per_graph=50))):
            with P.Context(arena_bytes=64 << 20, stream=stream, max_walks=2, device=local, **kw) as c1:
                wid = c1.submit_ex(spec1.L, spec1.seed, spec1.alpha1, spec1.alpha2, spec1.budget, n_lmt=spec1.n_lmt)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                c1.run()
                torch.cuda.synchronize(dev)
                small[label] = time.perf_counter() - t0
                small[label.replace("_s", "_psl_best")] = c1.poll(wid)["psl_best"]

    # the other batch configurations: throughput only (a few timed steps each, from a graph)
    others = None
    if args.other_configs and rank == 0:
        others = {}
        for wl_o, k_o in ((W.batch_16383(), 5), (W.batch_1048575(), 5), (W.labs_1023(), 100)):
            specs_o = list(wl_o.walks)
            need_o = sum(P.psl_walk_bytes(x.L, x.n_lmt, 0) for x in specs_o)
            with P.Context(arena_bytes=int(need_o * 1.1) + (64 << 20), stream=stream, max_walks=len(specs_o),
                           device=local) as oc:
                for x in specs_o:
                    oc.submit_ex(x.L, x.seed, x.alpha1, x.alpha2, x.budget, topk=x.topk)
                torch.cuda.synchronize(dev)
                t_init = time.perf_counter()
                oc.step(1)
                t_init = time.perf_counter() - t_init
                tune_o = oc.autotune(reps=1)
                oc.step(2)
                oc.profile(2)
                oc.set_steps_per_graph(k_o)
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                oc.step(k_o)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                prof_o = oc.profile_read()
                oc.profile(0)
                ms_o = e0.elapsed_time(e1)
                name_o = oc.hot_variant()
                psls_o = [oc.poll(w)["psl"] for w in sorted(oc.L_of)[:64]]
                quality = None
                if specs_o[0].alpha1 == specs_o[0].alpha2 == 2:
                    # merit factor L^2 / (2 E) of every walk's lowest-energy pivot so far
                    ids_o = sorted(oc.L_of)
                    mf = [specs_o[0].L ** 2 / (2.0 * oc.best_fitness(w)[0]) for w in ids_o]
                    quality = {"moves": 3 + k_o, "merit_factor_mean": float(np.mean(mf)),
                               "merit_factor_best": float(np.max(mf))}
            Lo, No = specs_o[0].L, specs_o[0].N
            n_hot, hot_ms_o = prof_o.get("hot", (0, 0.0))
            roof_o = hot_roofline(len(specs_o) * No, Lo, hot_ms_o / max(n_hot, 1), peak, mhz,
                                  stored_counters(name_o, wl_o.name), name_o, psls_o)
            others[wl_o.name] = {"value": len(specs_o) * No * k_o / (ms_o / 1000.0), "unit": UNIT,
                                 "ms_per_step": ms_o / k_o, "steps": k_o, "graph_steps": k_o,
                                 "hot_kernel": {"threads": tune_o[0], "tile_superblocks": tune_o[1], "name": name_o,
                                                "avg_ms": hot_ms_o / max(n_hot, 1)},
                                 "roofline_frac": roof_o["frac"], "roofline_frac_live_terms": roof_o["frac_live_terms"],
                                 "lookup_ceiling_frac": (roof_o["lookup_ceiling"] or {}).get("frac"),
                                 "plane_step_ceiling_frac": (roof_o.get("plane_step_ceiling") or {}).get("frac"),
                                 "issue_frac": roof_o["issue_frac"], "traffic": roof_o["traffic"],
                                 "init_s": t_init, "description": wl_o.description}
            if quality:
                others[wl_o.name]["quality"] = quality

    # serving: Poisson arrivals of walks with L = 2^m - 1, m uniform in 10..20, continuous batching,
    # at 0.8x the capacity a saturated probe measures
    serving = None
    if args.serving > 0 and rank == 0:
        serving = serving_leg(args, local, sms)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32 (exact i384 decisions)",
                "data": "synthetic",
                "config": {"workload": wl.name, "L": L, "walks_per_gpu": len(specs), "n_lmt": N,
                           "alpha": f"{specs[0].alpha1}/{specs[0].alpha2}",
                           "ls_lmt": W.LS_LMT, "flip_lmt": W.FLIP_LMT, "form": "batched",
                           "timed_path": f"CUDA graph of {G} steps per launch, event-record nodes around the "
                                         "neighbourhood kernel only",
                           "hot_kernel": {"threads": tuned[0], "tile_superblocks": tuned[1]} if tuned else "default",
                           "l2": "inputs larger than L2 (walk state %.1f GB per GPU)" % (need / 1e9)},
                "roofline": roof,
                "alu_peak": {k: v for k, v in peak.items()},
                "clocks": clocks, "gpu_launches": launches, "kernels": kernels,
                "plain_launches": {"value": len(specs) * N * K2 / (ms_plain_launch / 1000.0), "steps": K2,
                                   "ms_per_step": ms_plain_launch / K2,
                                   "note": "the same batch and kernels launched one by one (no graph)"},
                "fp32_score_error": fp32_err,
                "plain": plain,
                "batched_over_plain": (value / world) / plain["value"] if plain else None,
                "paper_context": {"A100_one_walk_flip_evals_per_s_L131071": PAPER_A100_L131071},
                "serving": serving,
                "other_configs": others,
                "small_config": small,
                "e2e": e2e}
        if not args.no_cpu_baseline:
            sampler = OracleSampler(L, N, 4)
            v, n_per, dt = sampler.sample(args.cpu_sample_s)
            cores = sampler.threads
            v1, n1, dt1 = sampler.sample_one_core(min(3.0, args.cpu_sample_s))
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"{cores} threads x {n_per} window neighbours of their own L=131071 "
                                              f"walk, exact F and PSL each ({dt:.1f} s)",
                                    "one_core": {"value": v1, "unit": UNIT, "sample": f"1 thread x {n1} window "
                                                 f"neighbours ({dt1:.1f} s)"}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


SHARE_POLICIES = {"work": "proportional to outstanding work", "requests": "proportional to live requests",
                  "balanced": "proportional to sqrt(work x requests)", None: "fixed 12/30/58%"}


def run_serving_study(args):
    """Serving with continuous batching on one GPU: a finite trace of requests at the trace's
    arrival rate, far above capacity, so the queue saturates; the capacity in requests/s
    measured there; then a second trace at 0.8x that capacity, where latency must stay
    bounded (the later half of the requests is compared with the earlier half)."""
    import torch

    import paper_2107_09801_gb300 as P
    from paper_2107_09801_gb300.serving import serve_classes, walk_terms_per_move

    torch.cuda.set_device(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    desc = ("Poisson arrivals, L=2^m-1 with m~U{10..20}, budgets ~U{100..10^4} moves, alpha1~U{2..6}, "
            "alpha2~U{alpha1+4..13}, N_lmt 6912, LS_lmt 2000, FLIP_lmt 10, request r has seed r")

    def leg(n, rate, policy=args.serving_policy):
        trace = W.serving_trace(n_requests=n, rate_hz=rate)
        arena = min(48 << 30, int(sum(P.psl_walk_bytes(r.spec.L, r.spec.n_lmt, 0) for r in trace) * 1.5) + (256 << 20))
        clk = ClockSampler(0)
        clk.start()
        res = serve_classes(trace, arena, sm_count=sms, share_policy=policy)
        clocks = clk.stop()
        terms = sum(r.spec.budget * walk_terms_per_move(r.spec) for r in trace)
        # requests in arrival order (the trace is generated in arrival order)
        lat = [res.latency_of[r] for r in range(len(trace)) if r in res.latency_of]
        half = len(lat) // 2
        return dict(res.summary(), rate_hz=rate, arrival_span_s=trace[-1].t_arrival, terms=terms,
                    terms_per_s=terms / res.wall_s, requests_per_s=n / res.wall_s,
                    shares=SHARE_POLICIES[policy], clocks=clocks,
                    p50_first_half_s=float(np.percentile(lat[:half], 50)) if half else None,
                    p50_second_half_s=float(np.percentile(lat[half:], 50)) if half else None,
                    p99_first_half_s=float(np.percentile(lat[:half], 99)) if half else None,
                    p99_second_half_s=float(np.percentile(lat[half:], 99)) if half else None)

    line = {"metric": "serving time to budget (p50/p99, arrival to result read back)", "impl": "ours",
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "trace": desc,
            "share_policy": args.serving_policy}
    if args.serving_study:
        sat = leg(args.serving_study, args.serving_rate)
        capacity = sat["requests_per_s"]
        line.update(saturated=sat, capacity_requests_per_s=capacity,
                    capacity_basis="requests completed / wall time of the saturated leg (queue never empty "
                                   "until the drain, so this slightly understates the capacity)",
                    at_0_8_capacity=leg(args.serving_study_light, 0.8 * capacity))
    if args.serving_compare:
        # the same saturated requests under each SM split between the length classes
        line["share_policies_saturated"] = {str(p): leg(args.serving_compare, args.serving_rate, policy=p)
                                            for p in (None, "work", "requests", "balanced")}
    print(json.dumps(line), flush=True)
    return 0


def run_ablation(args):
    """The paper's two control-parameter studies (Tables "alpha" and "par": L=65535, 30 runs
    of 10^10 sequence evaluations each) at a scale that fits a few GPU-minutes."""
    import torch

    import paper_2107_09801_gb300 as P
    from paper_2107_09801_gb300.ablation import alpha_pairs, ls_flip_grid, moves_for_nse

    torch.cuda.set_device(0)
    L = args.ablation_L
    line = {"metric": "mean best PSL of independent runs (lower is better)", "impl": "ours", "unit": "PSL",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic (uniform random +-1 starts, run r has seed r)",
            "L": L, "n_lmt": W.N_LMT}
    walks = max(3 * args.ablation_runs, 25 * args.grid_runs)
    with P.Context(arena_bytes=int(walks * P.psl_walk_bytes(L, W.N_LMT, 0) * 1.2) + (64 << 20),
                   max_walks=walks, steps_per_graph=64) as ctx:
        t = time.perf_counter()
        res = alpha_pairs(ctx, L, args.ablation_runs, int(args.ablation_nse))
        line["alpha_pairs"] = {"runs": args.ablation_runs, "nse_per_run": args.ablation_nse,
                               "moves_per_run": moves_for_nse(args.ablation_nse, L), "ls_lmt": 2000, "flip_lmt": 10,
                               "wall_s": time.perf_counter() - t,
                               "mean_psl": {f"{r.setting.alpha1}/{r.setting.alpha2}": r.mean for r in res},
                               "std_psl": {f"{r.setting.alpha1}/{r.setting.alpha2}": r.std for r in res},
                               "psl": {f"{r.setting.alpha1}/{r.setting.alpha2}": r.psl_best for r in res}}
        if args.grid_runs > 0:
            t = time.perf_counter()
            res = ls_flip_grid(ctx, L, args.grid_runs, int(args.grid_nse))
            line["ls_flip_grid"] = {"runs": args.grid_runs, "nse_per_run": args.grid_nse,
                                    "moves_per_run": moves_for_nse(args.grid_nse, L), "alpha": "4/13",
                                    "wall_s": time.perf_counter() - t,
                                    "mean_psl": {f"LS{r.setting.ls_lmt}/FLIP{r.setting.flip_lmt}": r.mean
                                                 for r in res}}
    line["paper_context"] = {"scale": "L=65535, 30 runs, 10^10 NSE per run (A100)",
                             "alpha_table_mean_psl": {"4/13": 212.700, "4/4": 232.833, "13/13": 238.967}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ablation:
        return run_ablation(args)
    if args.serving_study or args.serving_compare:
        return run_serving_study(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
