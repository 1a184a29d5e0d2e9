"""Host-side arithmetic of bench.py's roofline: term counts, the closed form's plane steps,
the fractions and the source-hash check of the stored ncu counters (no GPU)."""
import json
import os
import shutil

import numpy as np
import pytest

import bench


@pytest.mark.parametrize("L", [2, 3, 13, 1023, 4096])
def test_term_counts_by_enumeration(L):
    tc = bench.term_counts(L)
    assert tc["nominal"] == L - 1
    # a shift k has a partner for neighbour j when j + k <= L - 1 or j - k >= 0
    live = np.mean([sum(1 for k in range(1, L) if j + k <= L - 1 or j - k >= 0) for j in range(L)])
    assert tc["live"] == pytest.approx(live)
    # two lookups per five two-partner shifts, one per five one-partner shifts
    look = np.mean([2 * min(j, L - 1 - j) / 5 + (max(j, L - 1 - j) - min(j, L - 1 - j)) / 5 for j in range(L)])
    assert tc["lookups"] == pytest.approx(look)


def test_plane_steps_per_flip_eval():
    # P = bitlen(PSL) + 1 planes over about (L-1)/32 + 1 words, plus the partner-product words
    assert bench.plane_steps_per_flip_eval(1023, [40]) == pytest.approx(7 * (1022 / 32 + 1) + 1023 / 128)
    assert bench.plane_steps_per_flip_eval(1023, [31, 32]) == pytest.approx(6.5 * (1022 / 32 + 1) + 1023 / 128)


def _peak():
    return {"mix": 40e12, "lookup": 8e12, "popc": 5e12, "sm_count": 152, "max_clock_mhz": 2000,
            "clocks": {"sm_mhz": 2000.0}}


def test_hot_roofline_table_kernel():
    L, wn, ms = 131071, 1024 * 6912, 33.7
    r = bench.hot_roofline(wn, L, ms, _peak(), 2000.0, {"bytes_per_launch": 123, "warp_inst_per_launch": 4.0e10},
                           "k_hot_pc<28,32,8>")
    ach = wn * 2 * (L - 1) / (ms / 1e3)
    assert r["kernel"] == "k_hot_pc<28,32,8>" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(ach / 1e12) and r["frac"] == pytest.approx(ach / 40e12)
    assert r["lookup_ceiling"]["frac"] == pytest.approx(wn * bench.term_counts(L)["lookups"] / (ms / 1e3) / 8e12)
    assert r["traffic"] == 123
    assert r["issue_frac"] == pytest.approx(4.0e10 / (ms / 1e3) / (152 * 4 * 2000e6))
    assert "plane_step_ceiling" not in r


def test_hot_roofline_closed_form_and_clock_scaling():
    L, wn, ms = 1023, 4096 * 1023, 0.28
    r = bench.hot_roofline(wn, L, ms, _peak(), 1000.0, None, "k_hot_alpha2<256>", [40] * 8)
    # the peaks were measured at 2000 MHz, the timed region ran at 1000 MHz: half the denominator
    assert r["peak"] == pytest.approx(20.0)
    assert r["lookup_ceiling"] is None
    steps = bench.plane_steps_per_flip_eval(L, [40])
    pc = r["plane_step_ceiling"]
    assert pc["plane_steps_per_flip_eval"] == pytest.approx(steps)
    assert pc["frac"] == pytest.approx(wn * steps / (ms / 1e3) / 2.5e12)
    assert r["traffic"] is None and r["issue_frac"] is None


def test_stored_counters_only_for_the_current_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2107_09801_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(bench.ROOT, "paper_2107_09801_gb300", "csrc")
    for fn in ("psl_hot.cu", "psl_alpha2.cu", "psl_device.cuh"):
        shutil.copy(os.path.join(src, fn), csrc / fn)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h_tab, h_a2 = bench.kernel_source_hash("k_hot_pc<28,32,8>"), bench.kernel_source_hash("k_hot_alpha2<256>")
    assert h_tab != h_a2  # each kernel is hashed with its own translation unit
    rec = {"k_hot_pc<28,32,8>": {"W": {"source_hash": h_tab, "bytes_per_launch": 1}},
           "k_hot_alpha2<256>": {"W": {"source_hash": "stale", "bytes_per_launch": 2}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.stored_counters("k_hot_pc<28,32,8>", "W")["bytes_per_launch"] == 1
    assert bench.stored_counters("k_hot_alpha2<256>", "W") is None  # taken on another source
    assert bench.stored_counters("k_hot_pc<28,32,8>", "other") is None
    # a comment or a blank line leaves the counters valid; a change to the code does not
    with open(csrc / "psl_hot.cu", "a") as f:
        f.write("\n// a remark\n\n/* another */\n")
    assert bench.stored_counters("k_hot_pc<28,32,8>", "W")["bytes_per_launch"] == 1
    with open(csrc / "psl_hot.cu", "a") as f:
        f.write("static int unused_probe_value;\n")
    assert bench.stored_counters("k_hot_pc<28,32,8>", "W") is None


def test_kernels_per_step():
    # two profiled steps: the general path launches seven kernels a step, the fused tail two
    general = {"hot": (2, 1.0), "select": (2, 0.1), "recheck": (2, 0.1), "decide": (2, 0.1), "apply": (2, 0.1)}
    assert bench.kernels_per_step(general) == 7
    assert bench.kernels_per_step({"hot": (2, 1.0), "tail": (2, 0.1)}) == 2
    assert bench.kernels_per_step({"hot": (2, 1.0)}) == 1
