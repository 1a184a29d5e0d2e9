"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds only workload descriptions and seeded generators of inputs
(walk parameters, serving arrival traces, explicit start sequences for tests).
It contains none of the method's arithmetic: the search's own random draws are
made by each implementation from its walk seed.

The paper's workloads are uniform random +-1 starts at L = 2^m - 1
(Sec. 4; the random start of Alg. 1) with N_lmt = 6912,
LS_lmt = 2000, FLIP_lmt = 10, alpha1 = 4 and alpha2 = 13 (m <= 17) or
10 (m = 20) (Sec. 4.1 and Table 3).  There is no dataset: these synthetic
starts are the workload itself.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

N_LMT = 6912     # Sec. 4.1: neighbourhood size = A100 CUDA core count
LS_LMT = 2000    # Sec. 4.1, Table 1
FLIP_LMT = 10    # Sec. 4.1, Table 1


@dataclass(frozen=True)
class WalkSpec:
    """Parameters of one walk of Algorithm 1."""
    L: int
    seed: int
    alpha1: int = 4
    alpha2: int = 13
    budget: int = 2000
    n_lmt: int = N_LMT
    ls_lmt: int = LS_LMT
    flip_lmt: int = FLIP_LMT
    topk: int = 1            # FP32-ranked neighbours re-scored exactly besides the certified set

    @property
    def N(self) -> int:
        return min(self.n_lmt, self.L)


@dataclass(frozen=True)
class Workload:
    name: str
    walks: tuple = field(repr=False)
    description: str = ""

    @property
    def L_values(self):
        return sorted({w.L for w in self.walks})


def plain_small() -> Workload:
    """L = 1023, one walk from seed 1, full neighbourhood (N = L), 2000 moves."""
    return Workload("L1023_full_nbhd_1walk",
                    (WalkSpec(L=1023, seed=1, n_lmt=1023, budget=2000),),
                    "plain method, small: L=1023, seed 1, N=L, alpha 4/13, 2000 moves")


def batch_16383(walks: int = 4096, budget: int = 10_000) -> Workload:
    return Workload(f"L16383_x{walks}",
                    tuple(WalkSpec(L=16383, seed=s, budget=budget, topk=4) for s in range(walks)),
                    "L=16383, seeds 0..walks-1, alpha 4/13, N_lmt 6912, exact re-check of the FP32 top-4")


def batch_131071(walks: int = 1024, budget: int = 2000) -> Workload:
    return Workload(f"L131071_x{walks}",
                    tuple(WalkSpec(L=131071, seed=s, budget=budget) for s in range(walks)),
                    "L=131071, seeds 0..walks-1, alpha 4/13, N_lmt 6912, 2000 moves")


def batch_1048575(walks: int = 148, budget: int = 200) -> Workload:
    return Workload(f"L1048575_x{walks}",
                    tuple(WalkSpec(L=1048575, seed=s, alpha2=10, budget=budget, topk=1) for s in range(walks)),
                    "L=1048575, seeds 0..walks-1, alpha 4/10, N_lmt 6912, 200 moves")


def labs_1023(walks: int = 4096, budget: int = 2000) -> Workload:
    """The merit-factor objective: alpha = 2 in both phases, so F is the energy sum C_k^2
    and MF = L^2 / (2 F); the full neighbourhood (N = L)."""
    return Workload(f"LABS_L1023_x{walks}",
                    tuple(WalkSpec(L=1023, seed=s, alpha1=2, alpha2=2, budget=budget) for s in range(walks)),
                    "L=1023, seeds 0..walks-1, alpha 2/2 (energy of the merit factor), N = L, LS_lmt 2000")


@dataclass(frozen=True)
class Request:
    t_arrival: float
    spec: WalkSpec


def serving_trace(n_requests: int = 1000, rate_hz: float = 200.0, seed: int = 12345,
                  m_range=(10, 20), budget_range=(100, 10_000)) -> list[Request]:
    """Poisson arrivals; L = 2^m - 1 with m uniform in m_range; budgets uniform in
    budget_range; alpha1 uniform in 2..6 and alpha2 uniform in alpha1+4..13;
    request r carries walk seed r."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        budget = int(rng.integers(budget_range[0], budget_range[1] + 1))
        a1 = int(rng.integers(2, 7))
        a2 = int(rng.integers(a1 + 4, 14))
        out.append(Request(t, WalkSpec(L=(1 << m) - 1, seed=r, alpha1=a1, alpha2=a2, budget=budget)))
    return out


def random_pm1(L: int, seed: int) -> np.ndarray:
    """An explicit uniform +-1 sequence for tests (numpy PCG64; not the walk's own RNG)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (1 - 2 * rng.integers(0, 2, size=L)).astype(np.int8)


def small_specs(seed: int = 0, count: int = 8, L_choices=(13, 31, 63, 100, 255, 1023)) -> list[WalkSpec]:
    """Mixed small walks for parity tests: ragged lengths, small LS_lmt so that phase
    switches happen, assorted alpha pairs and window sizes (N < L and N = L)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        L = int(rng.choice(L_choices))
        a1 = int(rng.integers(1, 9))
        a2 = int(rng.integers(a1, 17))
        n_lmt = int(rng.choice([L, max(1, L // 3), 6912, 37]))
        out.append(WalkSpec(L=L, seed=int(rng.integers(0, 2**63)), alpha1=a1, alpha2=a2,
                            budget=int(rng.integers(20, 120)), n_lmt=n_lmt,
                            ls_lmt=int(rng.choice([1, 3, 5, 50])), flip_lmt=int(rng.integers(1, 11)),
                            topk=int(rng.integers(1, 5))))
    return out


def with_budget(spec: WalkSpec, budget: int) -> WalkSpec:
    return replace(spec, budget=budget)
