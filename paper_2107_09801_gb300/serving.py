"""Serving loop: continuous batching of walk requests through the C ABI.

Requests arrive over time (an arrival trace); every request is submitted as soon as it
has arrived, the library admits it into the batch as soon as the device arena has room,
every admitted walk advances together in the batched kernels, and finished walks are
read out and released at once so their memory serves the next request.  Latency is the
time from arrival to the moment the walk's result has been read back.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from .binding import PSL_DONE, PSL_ERROR, Context


@dataclass
class ServeResult:
    latencies_s: list = field(default_factory=list)   # arrival -> result read back, per request
    psl_best: dict = field(default_factory=dict)      # request index -> best PSL
    latency_of: dict = field(default_factory=dict)    # request index -> latency in s
    flip_evals: int = 0
    wall_s: float = 0.0
    errors: int = 0
    max_active: int = 0

    def percentile(self, p: float) -> float:
        return float(np.percentile(np.asarray(self.latencies_s), p)) if self.latencies_s else float("nan")

    def summary(self) -> dict:
        return {"requests": len(self.latencies_s), "p50_s": self.percentile(50), "p99_s": self.percentile(99),
                "mean_s": float(np.mean(self.latencies_s)) if self.latencies_s else float("nan"),
                "flip_evals_per_s": self.flip_evals / self.wall_s if self.wall_s else 0.0,
                "wall_s": self.wall_s, "errors": self.errors, "max_active": self.max_active}


def walk_terms_per_move(spec, n_lmt_default: int = 6912) -> int:
    """(neighbour, shift) terms one move of the walk scores: N x (L - 1), N = min(N_lmt, L)."""
    n_lmt = getattr(spec, "n_lmt", 0) or n_lmt_default
    return min(n_lmt, spec.L) * (spec.L - 1)


class SmShares:
    """Splits the device's SMs between contexts that step side by side (one per length
    class), with a floor for every context that has work, so that a short walk never
    waits for an SM.  The rest of the SMs follow a weight per context:
      - "work": the work it has outstanding, remaining moves x N x (L-1) summed over its
        live walks -- throughput-optimal, every context finishes at about the same time;
      - "requests": the number of live walks it holds -- every request gets an equal slice
        of the GPU (processor sharing over requests), so short requests are not held back
        by the amount of work of long ones;
      - "balanced" (default): the geometric mean of the two weights.  Measured on 200
        saturated requests it keeps most of the throughput of "work" and most of the
        median latency of "requests".
    A context with no work holds no share, which keeps the split work-conserving: once one
    class drains, the others get its SMs.  Thread-safe; a new share is handed out only when
    it differs from the one in use by more than `hysteresis` (resizing recaptures the
    context's CUDA graph)."""

    def __init__(self, sm_count: int, n: int, floor: int = 8, hysteresis: float = 0.15, policy: str = "balanced"):
        if policy not in ("work", "requests", "balanced"):
            raise ValueError(f"unknown share policy {policy!r}")
        self.sm_count, self.floor, self.hysteresis = int(sm_count), int(floor), float(hysteresis)
        self.policy = policy
        self.work = [0] * n
        self.count = [0] * n
        self.in_use = [0] * n
        self._mu = threading.Lock()

    def _target(self, i: int) -> int:
        busy = [c for c, w in enumerate(self.work) if w > 0]
        if self.work[i] <= 0:
            return 0
        if self.policy == "work":
            weight = self.work
        elif self.policy == "requests":
            weight = [max(1, n) for n in self.count]
        else:
            weight = [(w * max(1, n)) ** 0.5 for w, n in zip(self.work, self.count)]
        floor = min(self.floor, self.sm_count // len(busy))
        spare = self.sm_count - floor * len(busy)
        return floor + int(spare * weight[i] / sum(weight[c] for c in busy))

    def update(self, i: int, work: int, count: int = 1) -> int:
        """Records context i's outstanding work and live walks; returns the SM count it should use."""
        with self._mu:
            self.work[i] = int(work)
            self.count[i] = int(count) if work > 0 else 0
            t = self._target(i)
            cur = self.in_use[i]
            if cur == 0 or t == 0 or abs(t - cur) > self.hysteresis * cur:
                self.in_use[i] = t
            return self.in_use[i]


def serve(ctx: Context, trace, steps_per_round: int = 8, keep_sequences: bool = False,
          shares: SmShares | None = None, share_index: int = 0) -> ServeResult:
    """Runs a list of requests (objects with .t_arrival in seconds from the start and .spec,
    a WalkSpec-like object with L, seed, alpha1, alpha2, budget, n_lmt, ls_lmt, flip_lmt,
    topk) through the context and returns per-request latencies.  With `shares`, the
    context reports its outstanding work before every round and is resized to the SM
    count it is given."""
    res = ServeResult()
    order = sorted(range(len(trace)), key=lambda r: trace[r].t_arrival)
    nxt = 0
    live = {}  # walk id -> request index
    left = {}  # walk id -> moves still to go
    sms_now = -1
    t0 = time.perf_counter()
    while nxt < len(order) or live:
        now = time.perf_counter() - t0
        while nxt < len(order) and trace[order[nxt]].t_arrival <= now:
            r = order[nxt]
            s = trace[r].spec
            wid = ctx.submit_ex(s.L, s.seed, s.alpha1, s.alpha2, s.budget, n_lmt=s.n_lmt, ls_lmt=s.ls_lmt,
                                flip_lmt=s.flip_lmt, topk=s.topk)
            live[wid] = r
            left[wid] = s.budget
            nxt += 1
        if shares is not None:
            want = shares.update(share_index, sum(left[w] * walk_terms_per_move(trace[r].spec)
                                                  for w, r in live.items()), len(live))
            if want > 0 and want != sms_now:
                sms_now = ctx.set_max_sms(want)
        if not live:
            # idle until the next arrival
            time.sleep(max(0.0, trace[order[nxt]].t_arrival - (time.perf_counter() - t0)))
            continue
        ctx.step(steps_per_round)
        for wid in list(live):
            st = ctx.poll(wid)
            left[wid] = max(0, trace[live[wid]].spec.budget - int(st["moves"]))
            if st["state"] in (PSL_DONE, PSL_ERROR):
                r = live.pop(wid)
                left.pop(wid)
                if st["state"] == PSL_DONE:
                    psl, seq = ctx.best(wid)
                    res.psl_best[r] = (psl, seq) if keep_sequences else psl
                    res.flip_evals += int(st["flip_evals"])
                else:
                    res.errors += 1
                res.latencies_s.append(time.perf_counter() - t0 - trace[r].t_arrival)
                res.latency_of[r] = res.latencies_s[-1]
                ctx.release(wid)
        res.max_active = max(res.max_active, len(live))
    res.wall_s = time.perf_counter() - t0
    return res


# Length classes of serve_classes: (longest L of the class, share of the SMs, steps per round).
# Short walks are bound by step latency, long ones by the neighbourhood kernel's throughput.
DEFAULT_CLASSES = ((1 << 14, 0.12, 32), (1 << 17, 0.30, 16), (1 << 20, 0.58, 8))


def serve_classes(trace, arena_bytes: int, sm_count: int = 152, classes=DEFAULT_CLASSES, ctx_kwargs=None,
                  steps_per_graph: int = 8, keep_sequences: bool = False, share_policy: str | None = "balanced",
                  share_floor: int = 8) -> ServeResult:
    """Serves the trace with one context per length class, each on its own stream and host
    thread, its persistent kernels launched for its share of the SMs, so that a short walk
    no longer waits for the steps of long walks.  Requests are routed by L; arena bytes are
    split between the classes in proportion to the bytes their requests need.  With
    share_policy ("balanced", "requests" or "work", see SmShares) the SM split follows the
    classes' load; with None it is the fixed share of `classes`."""
    from .binding import psl_walk_bytes
    ctx_kwargs = dict(ctx_kwargs or {})
    parts = [[] for _ in classes]
    index = {id(req): r for r, req in enumerate(trace)}
    for req in trace:
        c = next(i for i, (lmax, _, _) in enumerate(classes) if req.spec.L <= lmax)
        parts[c].append(req)
    need = [sum(psl_walk_bytes(r.spec.L, r.spec.n_lmt, 0) for r in p) for p in parts]
    results = [None] * len(classes)
    errors = []
    shares = SmShares(sm_count, len(classes), floor=share_floor, policy=share_policy) if share_policy else None

    def run(ci):
        try:
            lmax, share, spr = classes[ci]
            nbytes = max(64 << 20, int(arena_bytes * need[ci] / max(1, sum(need))))
            with Context(arena_bytes=nbytes, max_walks=max(8, len(parts[ci])), max_sms=max(1, int(sm_count * share)),
                         steps_per_graph=steps_per_graph, **ctx_kwargs) as ctx:
                results[ci] = serve(ctx, parts[ci], steps_per_round=spr, keep_sequences=keep_sequences,
                                    shares=shares, share_index=ci)
        except Exception as e:  # surfaced to the caller below
            errors.append(e)

    t0 = time.perf_counter()
    ths = [threading.Thread(target=run, args=(ci,)) for ci in range(len(classes)) if parts[ci]]
    [t.start() for t in ths]
    [t.join() for t in ths]
    if errors:
        raise errors[0]
    out = ServeResult(wall_s=time.perf_counter() - t0)
    for ci, r in enumerate(results):
        if r is None:
            continue
        out.latencies_s += r.latencies_s
        for local, v in r.psl_best.items():  # back to indices of the whole trace
            out.psl_best[index[id(parts[ci][local])]] = v
        for local, v in r.latency_of.items():
            out.latency_of[index[id(parts[ci][local])]] = v
        out.flip_evals += r.flip_evals
        out.errors += r.errors
        out.max_active += r.max_active
    return out
