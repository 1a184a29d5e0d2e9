"""Host logic of the serving loop: the SM split between length-class contexts."""
import threading

from paper_2107_09801_gb300.serving import SmShares, walk_terms_per_move
import psl_workloads as W


def settle(sh, works, counts=None):
    # every context reports once more after all have reported, as the serving loop does
    counts = counts or [1] * len(works)
    for i, (w, n) in enumerate(zip(works, counts)):
        sh.update(i, w, n)
    return [sh.update(i, w, n) for i, (w, n) in enumerate(zip(works, counts))]


def test_shares_follow_outstanding_work():
    sh = SmShares(152, 3, floor=8, hysteresis=0.0, policy="work")
    got = settle(sh, [1, 10, 89])
    assert sum(got) <= 152 and all(g >= 8 for g in got)
    assert got[0] < got[1] < got[2]
    spare = 152 - 3 * 8
    assert got == [8 + int(spare * w / 100) for w in (1, 10, 89)]


def test_idle_context_holds_no_share_and_the_rest_take_the_gpu():
    sh = SmShares(152, 3, floor=8, hysteresis=0.0, policy="work")
    settle(sh, [5, 5, 5])
    got = settle(sh, [5, 0, 0])
    assert got == [152, 0, 0]


def test_floor_shrinks_when_contexts_outnumber_it():
    sh = SmShares(16, 4, floor=8, hysteresis=0.0)
    got = settle(sh, [1, 1, 1, 1000])
    assert sum(got) <= 16 and min(got) >= 4


def test_hysteresis_keeps_small_changes_out():
    sh = SmShares(152, 2, floor=8, hysteresis=0.15, policy="work")
    a, b = settle(sh, [50, 50])
    assert sh.update(0, 52) == a          # a few percent: no resize
    assert sh.update(0, 500) > a          # large change: resized


def test_concurrent_updates_keep_the_split_within_the_device():
    sh = SmShares(152, 3, floor=8, hysteresis=0.0, policy="work")

    def run(i):
        for t in range(2000):
            sh.update(i, (t * (i + 3)) % 97)

    ths = [threading.Thread(target=run, args=(i,)) for i in range(3)]
    [t.start() for t in ths]
    [t.join() for t in ths]
    got = settle(sh, [3, 0, 40])
    assert sum(got) <= 152 and got[1] == 0


def test_terms_per_move_is_window_times_shifts():
    assert walk_terms_per_move(W.WalkSpec(L=1023, seed=0)) == 1023 * 1022
    assert walk_terms_per_move(W.WalkSpec(L=131071, seed=0)) == 6912 * 131070
    assert walk_terms_per_move(W.WalkSpec(L=131071, seed=0, n_lmt=300)) == 300 * 131070


def test_request_policy_gives_every_live_request_an_equal_slice():
    sh = SmShares(152, 3, floor=8, hysteresis=0.0, policy="requests")
    got = settle(sh, [10**6, 10**9, 10**12], counts=[30, 10, 20])
    spare = 152 - 3 * 8
    assert got == [8 + int(spare * n / 60) for n in (30, 10, 20)]
    assert settle(sh, [0, 10**9, 10**12], counts=[0, 10, 20])[0] == 0


def test_unknown_policy_is_rejected():
    import pytest
    with pytest.raises(ValueError):
        SmShares(152, 3, policy="fair")


def test_balanced_policy_sits_between_work_and_requests():
    works, counts = [10**6, 10**9, 10**12], [30, 10, 20]
    got = {p: settle(SmShares(152, 3, floor=8, hysteresis=0.0, policy=p), works, counts)
           for p in ("work", "requests", "balanced")}
    for c in range(3):
        lo, hi = sorted((got["work"][c], got["requests"][c]))
        assert lo <= got["balanced"][c] <= hi
