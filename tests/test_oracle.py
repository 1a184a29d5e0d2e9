"""Pins of the CPU oracle against facts that do not come from the oracle itself:
published test vectors, textbook sequences, closed forms, FFT identities,
symmetries, exhaustive search on tiny inputs, and the rules of Algorithm 1
checked transition by transition.  No GPU needed."""
import math

import numpy as np
import pytest

import oracle as O
import psl_workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# --------------------------------------------------------------------------------------------
# independent routes used by the pins (numpy FFT, Python integers)
# --------------------------------------------------------------------------------------------
def fft_autocorr(s):
    """C_k by the Wiener-Khinchin route: |DFT|^2 of the zero-padded sequence."""
    L = len(s)
    M = 1 << (2 * L - 1).bit_length()
    S = np.fft.rfft(s.astype(np.float64), M)
    r = np.fft.irfft(np.abs(S) ** 2, M)[:L]
    return np.rint(r).astype(np.int64)


def py_fitness(C, alpha):
    return sum(abs(int(c)) ** alpha for c in C[1:])


def barker13(golden):
    (row,) = golden("barker13.txt")
    return np.array([1 if ch == "+" else -1 for ch in row], dtype=np.int8)


# --------------------------------------------------------------------------------------------
# Rand
# --------------------------------------------------------------------------------------------
def test_splitmix64_published_vectors(golden):
    for seed, n, value in golden("splitmix64.txt"):
        assert O.splitmix64(int(seed), int(n)) == int(value)


def test_start_sequence_bit_mapping(golden):
    # draw 0 of seed 0 is published; bit b of it decides s_b (bit 1 -> -1)
    d0 = int([r for r in golden("splitmix64.txt") if r[0] == "0" and r[1] == "0"][0][2])
    d1 = int([r for r in golden("splitmix64.txt") if r[0] == "0" and r[1] == "1"][0][2])
    s = O.init_seq(100, 0)
    want = [(-1 if (d0 >> b) & 1 else 1) for b in range(64)] + [(-1 if (d1 >> b) & 1 else 1) for b in range(36)]
    assert s.tolist() == want


# --------------------------------------------------------------------------------------------
# Eq. (2): autocorrelation
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 3, 7, 13, 64, 255, 1000, 4095])
def test_autocorr_closed_forms(L):
    s = W.random_pm1(L, 1000 + L)
    C = O.autocorr(s)
    assert C[0] == L
    k = np.arange(L)
    assert np.all((C - (L - k)) % 2 == 0)                       # C_k = L-k (mod 2)
    assert C[L - 1] == int(s[0]) * int(s[L - 1])                # single product at k = L-1
    assert int(C[1:].astype(np.int64).sum()) == (int(s.astype(np.int64).sum()) ** 2 - L) // 2


@pytest.mark.parametrize("L", [2, 5, 31, 256, 1023, 4096])
def test_autocorr_matches_fft_route(L):
    s = W.random_pm1(L, L)
    assert np.array_equal(O.autocorr(s).astype(np.int64), fft_autocorr(s))


def test_autocorr_symmetries():
    s = W.random_pm1(777, 5)
    C = O.autocorr(s)
    assert np.array_equal(O.autocorr(-s), C)
    assert np.array_equal(O.autocorr(s[::-1].copy()), C)
    alt = (s * np.where(np.arange(777) % 2 == 0, 1, -1)).astype(np.int8)
    assert np.array_equal(O.autocorr(alt), C * np.where(np.arange(777) % 2 == 0, 1, -1))


# --------------------------------------------------------------------------------------------
# Eq. (3): PSL, and the goal Eq. (5) by exhaustive search
# --------------------------------------------------------------------------------------------
def test_barker13_psl_and_fitness(golden):
    b = barker13(golden)
    C = O.autocorr(b)
    assert O.psl(C) == 1
    for alpha in range(1, 17):
        exact, rounded, naive = O.fitness(C, alpha)
        assert exact == 6 and rounded == 6.0 and naive == 6.0


def test_psl_range_includes_k1():
    # the printed range "1 < k < L" is read as k = 1..L-1: a sequence whose largest sidelobe
    # sits only at k = 1 must report it
    s = np.array([1, 1, 1, 1, 1, 1, -1], dtype=np.int8)   # C = 7, 4, 3, 2, 1, 0, -1
    C = O.autocorr(s)
    assert abs(C[1]) > max(abs(int(c)) for c in C[2:])
    assert O.psl(C) == abs(int(C[1]))
    assert O.psl(O.autocorr(np.ones(9, dtype=np.int8))) == 8


def test_brute_force_min_psl_matches_literature(golden):
    for L, want in golden("min_psl_small.txt"):
        L, want = int(L), int(want)
        if L > 18:
            continue  # 2^(L-1) sequences; the largest cases are covered by test_brute_force_large
        got, seq = O.brute_min_psl(L)
        assert got == want, L
        assert O.psl(O.autocorr(seq)) == got


@pytest.mark.slow
def test_brute_force_large(golden):
    table = {int(a): int(b) for a, b in golden("min_psl_small.txt")}
    for L in (19, 20):
        assert O.brute_min_psl(L)[0] == table[L]


# --------------------------------------------------------------------------------------------
# Eq. (4): fitness
# --------------------------------------------------------------------------------------------
def test_fitness_all_ones_faulhaber():
    sympy = pytest.importorskip("sympy")
    k, n = sympy.symbols("k n", integer=True, positive=True)
    for alpha in range(1, 17):
        closed = sympy.expand(sympy.summation(k ** alpha, (k, 1, n)))    # Faulhaber polynomial
        for L in (2, 5, 100, 2000):
            C = O.autocorr(np.ones(L, dtype=np.int8))                     # C_k = L - k
            exact, rounded, _ = O.fitness(C, alpha)
            want = int(closed.subs(n, L - 1))
            assert exact == want, (alpha, L)
            assert rounded == float(want)                                 # Python rounds ints correctly


@pytest.mark.parametrize("L", [13, 100, 1023, 3000])
def test_fitness_alpha2_parseval(L):
    # sum_{k=-(L-1)}^{L-1} C_k^2 = L^2 + 2 F_2 = (1/M) sum_m |S_m|^4 (Parseval on |S|^2)
    s = W.random_pm1(L, 7 * L)
    M = 1 << (2 * L - 1).bit_length()
    S = np.fft.fft(s.astype(np.float64), M)
    total = float(np.sum(np.abs(S) ** 4) / M)
    exact, _, _ = O.fitness(O.autocorr(s), 2)
    assert abs(L * L + 2 * exact - total) < 1e-6 * total
    assert (L * L + 2 * exact) == round(total)


def test_fitness_symmetries_and_rounding():
    s = W.random_pm1(501, 9)
    for alpha in (1, 4, 10, 13, 16):
        base = O.fitness(O.autocorr(s), alpha)
        assert O.fitness(O.autocorr(-s), alpha) == base
        assert O.fitness(O.autocorr(s[::-1].copy()), alpha) == base
        exact, rounded, naive = base
        assert rounded == float(exact)
        assert abs(naive - rounded) <= 1e-12 * rounded


def test_wide_to_double_is_correctly_rounded():
    rng = np.random.Generator(np.random.PCG64(3))
    cases = [0, 1, -1, 2**53 - 1, 2**53, 2**53 + 1, 2**53 + 3, -(2**53 + 1), 2**300 + 2**247, 2**300 + 2**247 + 1,
             2**300 + 3 * 2**247, 2**339 - 1]
    for _ in range(2000):
        bits = int(rng.integers(1, 340))
        v = int.from_bytes(rng.bytes(48), "little") >> (384 - bits)
        if rng.integers(0, 2):
            v = -v
        cases.append(v)
        # exact ties at the 53-bit boundary, both parities
        if bits > 60:
            top = v >> (bits - 54)
            cases.append(((top | 1) << (bits - 54)))
    for v in cases:
        assert O.wide_to_double(v) == float(v), v


# --------------------------------------------------------------------------------------------
# Sec. 3: one-element flip
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 3, 13, 64, 301])
def test_flip_update_equals_recompute_every_j(L):
    s = W.random_pm1(L, 11 * L)
    C = O.autocorr(s)
    for j in range(L):
        t = s.copy()
        t[j] = -t[j]
        assert np.array_equal(O.flip_autocorr(s, C, j), O.autocorr(t)), j


def test_flip_update_equals_recompute_large():
    L = 4096
    s = W.random_pm1(L, 4)
    C = O.autocorr(s)
    for j in (0, 1, 2047, 2048, 4094, 4095):
        t = s.copy()
        t[j] = -t[j]
        assert np.array_equal(O.flip_autocorr(s, C, j).astype(np.int64), fft_autocorr(t))


# --------------------------------------------------------------------------------------------
# Alg. 1 neighbourhood evaluation without a move (the checker of the full-size GPU checks):
# every neighbour's exact F (Eq. 4) and PSL (Eq. 3) against the flipped sequence rebuilt
# from scratch by the FFT route and scored with Python integers
# --------------------------------------------------------------------------------------------
def _neighbour_psl_plus4(s, C):
    """Positions j whose neighbour has a sidelobe of magnitude PSL + 4 (the largest a single
    flip can reach), found by the flip rule of Sec. 3 written out in numpy."""
    L, P = len(s), int(np.abs(C[1:]).max())
    out = []
    for j in range(L):
        k = np.arange(1, L)
        part = np.where(j + k < L, s[np.minimum(j + k, L - 1)], 0) + np.where(j - k >= 0, s[np.maximum(j - k, 0)], 0)
        if int(np.abs(C[1:] - 2 * int(s[j]) * part).max()) == P + 4:
            out.append(j)
    return out


@pytest.mark.parametrize("L,alpha,sample", [(13, 4, None), (13, 16, None), (300, 1, None), (300, 16, None),
                                            (300, 13, None), (4096, 4, 48), (4096, 16, 24)])
def test_eval_neighbours_against_recompute(L, alpha, sample):
    s = W.random_pm1(L, 7 * L + alpha)
    C = O.autocorr(s)
    js = list(range(L))
    if sample:
        rng = np.random.Generator(np.random.PCG64(L + alpha))
        js = sorted(set(rng.choice(L, size=sample, replace=False).tolist()) | {0, 1, L // 2, L - 2, L - 1})
    plus4 = _neighbour_psl_plus4(s, C) if L <= 300 else []
    if L == 300:
        assert plus4, "no neighbour reaches PSL + 4: the +4 headroom of the power table is not exercised"
        js = sorted(set(js) | set(plus4))
    vals, psls = O.eval_neighbours(s, C, alpha, js)
    for j, v, p in zip(js, vals, psls):
        t = s.copy()
        t[j] = -t[j]
        Cn = fft_autocorr(t)
        assert v == py_fitness(Cn, alpha), (L, alpha, j)
        assert p == int(np.abs(Cn[1:]).max()), (L, alpha, j)
    # the neighbours' order is kept and the pivot itself is untouched
    vals_rev, _ = O.eval_neighbours(s, C, alpha, js[::-1])
    assert vals_rev == vals[::-1]
    assert np.array_equal(O.autocorr(s), C)


# --------------------------------------------------------------------------------------------
# Algorithm 1: one decision against brute force over the window
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("L,n_lmt,alpha", [(13, 13, 4), (31, 10, 13), (63, 63, 1), (63, 5, 2), (100, 40, 16)])
def test_step_decision_brute_force(L, n_lmt, alpha):
    w = O.Walk(O.WalkParams(L=L, seed=2 * L + alpha, alpha1=alpha, alpha2=alpha, n_lmt=n_lmt, ls_lmt=50))
    for _ in range(5):
        s0, psl_best0, ctr0 = w.s.copy(), w.psl_best, w.rng_ctr
        (rec,) = w.run(1)
        start = O.splitmix64(w.p.seed, ctr0) % L        # Rand() % L of Alg. 1 from the published draw
        assert rec["start"] == start
        N = min(n_lmt, L)
        vals, psls = [], []
        for i in range(1, N + 1):
            j = (start + i) % L
            t = s0.copy()
            t[j] = -t[j]
            C = fft_autocorr(t)
            vals.append((py_fitness(C, alpha), j))
            psls.append((int(np.abs(C[1:]).max()), j))
        vmin = min(v for v, _ in vals)
        first = next(j for v, j in vals if v == vmin)    # strict "<" in scan order keeps the first
        assert rec["kstar"] == first
        assert O.limbs_to_int(rec["value_exact"]) == vmin
        pmin = min(p for p, _ in psls)
        assert rec["win_psl"] == pmin and rec["win_psl_j"] == next(j for p, j in psls if p == pmin)
        assert rec["psl_best"] == min(psl_best0, pmin)
        if pmin < psl_best0:                              # solution_best = first improving neighbour
            t = s0.copy()
            jb = next(j for p, j in psls if p == pmin)
            t[jb] = -t[jb]
            assert rec["flags"] & O.PSL_BEST and np.array_equal(w.sol_best, t)
        # the pivot really moved to kstar
        t = s0.copy()
        t[first] = -t[first]
        if not rec["flags"] & O.SWITCH:
            assert np.array_equal(w.s, t)


# --------------------------------------------------------------------------------------------
# Algorithm 1: bookkeeping and phase switch, transition by transition
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("spec", W.small_specs(seed=1, count=6, L_choices=(7, 13, 31, 63, 127)),
                         ids=lambda s: f"L{s.L}")
def test_trajectory_rules(spec):
    p = O.WalkParams(L=spec.L, seed=spec.seed, alpha1=spec.alpha1, alpha2=spec.alpha2, n_lmt=spec.n_lmt,
                     ls_lmt=spec.ls_lmt, flip_lmt=spec.flip_lmt)
    w = O.Walk(p)
    nflip_expect = min(spec.flip_lmt, spec.L)
    psl_best_prev = w.psl_best
    for _ in range(spec.budget):
        vl0, un0, alpha0, lb0 = w.value_local, w.unimproved, w.alpha, w.local_best.copy()
        (r,) = w.run(1)
        v = O.limbs_to_int(r["value_exact"])
        assert r["alpha"] == alpha0
        if v < vl0:
            assert r["flags"] & O.IMPROVED and w.unimproved == 0 and w.value_local == v
            assert np.array_equal(w.local_best, w.s)
        elif v > vl0:
            assert r["flags"] & O.WORSE
            if un0 + 1 > spec.ls_lmt:
                assert r["flags"] & O.SWITCH and w.unimproved == 0
                assert w.alpha == (spec.alpha2 if alpha0 == spec.alpha1 else spec.alpha1)
                assert np.array_equal(w.local_best, lb0)                      # local_best kept
                assert int(np.sum(w.s != lb0)) == nflip_expect == r["nflip"]   # distinct flips
                assert w.value_local == py_fitness(fft_autocorr(w.s), w.alpha)
            else:
                assert not r["flags"] & O.SWITCH and w.unimproved == un0 + 1
        else:
            assert not r["flags"] & (O.IMPROVED | O.WORSE | O.SWITCH)
            assert w.unimproved == un0 and w.value_local == vl0
        # state consistency against independent recomputation
        C = fft_autocorr(w.s)
        assert np.array_equal(w.C.astype(np.int64), C)
        assert w.psl == r["psl"] == int(np.abs(C[1:]).max())
        assert w.F == py_fitness(C, w.alpha)
        assert w.psl_best <= psl_best_prev
        psl_best_prev = w.psl_best
        assert int(np.abs(fft_autocorr(w.sol_best)[1:]).max()) == w.psl_best


@pytest.mark.parametrize("L", [13, 31, 100])
def test_incremental_and_full_modes_agree(L):
    p = O.WalkParams(L=L, seed=L, alpha1=3, alpha2=9, n_lmt=L // 2 + 1, ls_lmt=4, flip_lmt=3)
    a, b = O.Walk(p), O.Walk(p)
    ta = a.run(80, O.MODE_INCREMENTAL)
    tb = b.run(80, O.MODE_FULL)
    assert ta.tobytes() == tb.tobytes()
    c = O.Walk(p)
    tc = c.run(80, O.MODE_CROSSCHECK)
    assert tc.tobytes() == ta.tobytes()


def test_naive_fp64_matches_exact_on_moderate_sizes():
    p = O.WalkParams(L=255, seed=5, alpha1=4, alpha2=13, n_lmt=100, ls_lmt=10, flip_lmt=5)
    w = O.Walk(p)
    tr = w.run(60, O.MODE_NAIVE)
    rel = np.abs(tr["value_naive"] - tr["value_step"]) / tr["value_step"]
    assert rel.max() <= 1e-12
    assert w.near_ties == int(np.sum((tr["flags"] & O.NAIVE_DIFFERS) != 0))


def test_search_quality_loose():
    """Parity unpinned: no worked trajectory is printed in the paper.  Loose check only:
    the search drives PSL well below that of the random start and below sqrt(L)."""
    p = O.WalkParams(L=255, seed=1, alpha1=4, alpha2=13, n_lmt=6912, ls_lmt=20, flip_lmt=10)
    w = O.Walk(p)
    psl0 = w.psl
    w.run(300)
    assert w.psl_best < 0.6 * psl0 and w.psl_best < math.sqrt(255)


# --------------------------------------------------------------------------------------------
# fixed objective (alpha1 == alpha2): the lowest-F pivot; alpha = 2 is the merit-factor energy
# --------------------------------------------------------------------------------------------
def np_energy(s):
    """E = sum_{k>=1} C_k^2 by numpy's full correlation (an independent route to Eq. 2)."""
    c = np.correlate(s.astype(np.int64), s.astype(np.int64), mode="full")[len(s):]
    return int(np.dot(c, c))


@pytest.mark.parametrize("L,alpha", [(31, 2), (63, 2), (100, 2), (45, 3)])
def test_lowest_f_pivot_is_first_minimum_of_visited_pivots(L, alpha):
    """No switch (LS_lmt above the budget): the pivots are the start plus one flip per move,
    so every visited pivot is rebuilt from the move list and scored independently."""
    p = O.WalkParams(L=L, seed=L + alpha, alpha1=alpha, alpha2=alpha, n_lmt=L, ls_lmt=10**6, flip_lmt=3)
    w = O.Walk(p)
    s = w.s.copy()
    tr = w.run(120)
    assert not np.any(tr["flags"] & O.SWITCH)
    pivots = [s.copy()]
    for r in tr:
        s[r["kstar"]] = -s[r["kstar"]]
        pivots.append(s.copy())
    f = [py_fitness(fft_autocorr(q), alpha) for q in pivots]
    if alpha == 2:
        assert f == [np_energy(q) for q in pivots]
    first = int(np.argmin(f))        # numpy: first index of the minimum
    assert w.F_best == f[first]
    assert np.array_equal(w.fbest_seq, pivots[first])


@pytest.mark.parametrize("L", [31, 127])
def test_lowest_energy_with_switches(L):
    p = O.WalkParams(L=L, seed=3 * L, alpha1=2, alpha2=2, n_lmt=L, ls_lmt=3, flip_lmt=4)
    w = O.Walk(p)
    F0 = w.F
    tr = w.run(200)
    assert np.any(tr["flags"] & O.SWITCH)
    assert np.all(tr["alpha"] == 2)
    steps = [O.limbs_to_int(v) for v in tr["value_exact"]]
    assert w.F_best <= min([F0] + steps)              # switch pivots may go lower still
    assert np_energy(w.fbest_seq) == w.F_best


def test_lowest_energy_not_kept_when_phases_differ():
    p = O.WalkParams(L=63, seed=9, alpha1=2, alpha2=5, n_lmt=63, ls_lmt=3, flip_lmt=4)
    w = O.Walk(p)
    s0, F0 = w.s.copy(), w.F
    w.run(60)
    assert w.F_best == F0 and np.array_equal(w.fbest_seq, s0)


def test_barker13_is_a_lowest_energy_start(golden):
    """Barker-13 has energy 6 (merit factor 169/12), the minimum over all 2^13 sequences
    (exhaustive search below); a walk started there never leaves it as its lowest pivot."""
    b = barker13(golden)
    assert np_energy(b) == 6
    best = min(np_energy(np.array([1 if (m >> i) & 1 else -1 for i in range(13)], dtype=np.int8))
               for m in range(1 << 12))   # s_12 = -1 fixed: negation symmetry covers the rest
    assert best == 6
    p = O.WalkParams(L=13, seed=1, alpha1=2, alpha2=2, n_lmt=13, ls_lmt=2, flip_lmt=3)
    w = O.Walk(p, s0=b)
    assert w.F_best == 6
    w.run(50)
    assert w.F_best == 6 and np.array_equal(w.fbest_seq, b)
