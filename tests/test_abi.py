"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/psl.h declares.  Only host-side helpers are called: no GPU is needed."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(psl_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpsl():
    from paper_2107_09801_gb300 import build
    path = build.build()
    return ct.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("psl_init", "psl_submit", "psl_step", "psl_poll", "psl_best"):
        assert required in names


def test_every_declared_symbol_is_exported(libpsl):
    missing = [n for n in declared_functions() if not hasattr(libpsl, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2107_09801_gb300 import binding
    assert sorted(binding.EXPORTED) == declared_functions()


def test_host_helpers_without_gpu(libpsl):
    from paper_2107_09801_gb300 import binding as B
    cfg = B.psl_config_default()
    assert (cfg.n_lmt, cfg.ls_lmt, cfg.flip_lmt, cfg.form) == (6912, 2000, 10, B.PSL_FORM_BATCHED)
    assert B.psl_walk_bytes(1, 6912, 0) == 0
    small, big = B.psl_walk_bytes(1023, 6912, 0), B.psl_walk_bytes(131071, 6912, 0)
    assert 0 < small < big
    # C (two copies), the FP32 tables and the near-peak list dominate: 32 bytes per k
    assert 32 * 131071 <= big <= 40 * 131071 + (1 << 20)
    assert B.psl_walk_bytes(1023, 6912, 100) > small


def test_product_path_has_no_oracle_import():
    # the CUDA path and its binding never import the oracle
    pkg = os.path.join(ROOT, "paper_2107_09801_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text and "psl_oracle" not in text, fn
