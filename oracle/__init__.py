"""Plain CPU oracle for the two-phase low-PSL search (arXiv 2107.09801).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library and
its Python binding never import it, and it imports nothing from them.

The arithmetic lives in ``psl_oracle.c`` (plain C, exact 384-bit fitness); this
module only compiles it with gcc, loads it with ctypes and marshals numpy
arrays.  Passages followed: Eq. (1)-(4), the one-element flip of Sec. 3 and
Algorithm 1 of the paper; see the header of ``psl_oracle.c``.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psl_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

WL = 6  # limbs of the exact fitness

IMPROVED, WORSE, SWITCH, PSL_BEST, NAIVE_DIFFERS = 1, 2, 4, 8, 16
MODE_INCREMENTAL, MODE_FULL, MODE_CROSSCHECK, MODE_NAIVE = 0, 1, 2, 4


def build(force: bool = False) -> str:
    """Compile psl_oracle.c into a shared library with gcc (no GPU needed)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fvisibility=hidden",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ct.Structure):
    _fields_ = [("L", ct.c_uint32), ("n_lmt", ct.c_uint32), ("ls_lmt", ct.c_uint32),
                ("flip_lmt", ct.c_uint32), ("alpha1", ct.c_uint32), ("alpha2", ct.c_uint32),
                ("seed", ct.c_uint64)]


class _State(ct.Structure):
    _fields_ = [("s", ct.c_void_p), ("local_best", ct.c_void_p), ("sol_best", ct.c_void_p),
                ("C", ct.c_void_p), ("value_local", ct.c_uint64 * WL), ("F", ct.c_uint64 * WL),
                ("alpha", ct.c_uint32), ("unimproved", ct.c_uint32), ("psl", ct.c_int32),
                ("psl_best", ct.c_int32), ("rng_ctr", ct.c_uint64), ("steps", ct.c_uint64),
                ("near_ties", ct.c_uint64), ("fbest_seq", ct.c_void_p), ("F_best", ct.c_uint64 * WL)]


TRACE_DTYPE = np.dtype([("step", "<u8"), ("start", "<u4"), ("kstar", "<u4"), ("alpha", "<u4"),
                        ("unimproved", "<u4"), ("psl", "<i4"), ("psl_best", "<i4"), ("win_psl", "<i4"),
                        ("win_psl_j", "<u4"), ("flags", "<u4"), ("nflip", "<u4"),
                        ("value_step", "<f8"), ("value_naive", "<f8"), ("value_exact", "<u8", (WL,))])

_lib = None


def lib():
    global _lib
    if _lib is None:
        # PSL_ORACLE_LIB lets the mutation test load a deliberately broken copy of the oracle
        _lib = ct.CDLL(os.environ.get("PSL_ORACLE_LIB") or build())
        L = _lib
        L.orc_splitmix64.restype = ct.c_uint64
        L.orc_splitmix64.argtypes = [ct.c_uint64, ct.c_uint64]
        L.orc_init_seq.argtypes = [ct.c_uint32, ct.c_uint64, ct.c_void_p]
        L.orc_autocorr.argtypes = [ct.c_void_p, ct.c_uint32, ct.c_void_p]
        L.orc_psl.restype = ct.c_int32
        L.orc_psl.argtypes = [ct.c_void_p, ct.c_uint32]
        L.orc_fitness.restype = ct.c_int
        L.orc_fitness.argtypes = [ct.c_void_p, ct.c_uint32, ct.c_uint32, ct.c_void_p,
                                  ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
        L.orc_wide_to_double.restype = ct.c_double
        L.orc_wide_to_double.argtypes = [ct.c_void_p]
        L.orc_flip_autocorr.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_uint32, ct.c_uint32, ct.c_void_p]
        L.orc_brute_min_psl.restype = ct.c_int32
        L.orc_brute_min_psl.argtypes = [ct.c_uint32, ct.c_void_p]
        L.orc_init.restype = ct.c_int
        L.orc_init.argtypes = [ct.POINTER(Params), ct.POINTER(_State)]
        L.orc_run.restype = ct.c_int
        L.orc_run.argtypes = [ct.POINTER(Params), ct.POINTER(_State), ct.c_uint64, ct.c_int, ct.c_void_p]
        L.orc_eval_neighbours.restype = ct.c_int
        L.orc_eval_neighbours.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_uint32, ct.c_uint32, ct.c_void_p,
                                          ct.c_uint32, ct.c_void_p, ct.c_void_p]
        for name in ("orc_sizeof_state", "orc_sizeof_trace", "orc_sizeof_params"):
            getattr(L, name).restype = ct.c_uint32
        assert L.orc_sizeof_state() == ct.sizeof(_State)
        assert L.orc_sizeof_trace() == TRACE_DTYPE.itemsize
        assert L.orc_sizeof_params() == ct.sizeof(Params)
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def limbs_to_int(limbs) -> int:
    """Two's-complement 384-bit limbs -> Python int."""
    v = 0
    for i, w in enumerate(limbs):
        v |= int(w) << (64 * i)
    if v >> (64 * WL - 1):
        v -= 1 << (64 * WL)
    return v


def int_to_limbs(v: int) -> np.ndarray:
    v &= (1 << (64 * WL)) - 1
    return np.array([(v >> (64 * i)) & ((1 << 64) - 1) for i in range(WL)], dtype=np.uint64)


def splitmix64(seed: int, n: int) -> int:
    return int(lib().orc_splitmix64(seed, n))


def init_seq(L: int, seed: int) -> np.ndarray:
    s = np.empty(L, dtype=np.int8)
    lib().orc_init_seq(L, seed, _ptr(s))
    return s


def autocorr(s: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.int8)
    C = np.empty(len(s), dtype=np.int32)
    lib().orc_autocorr(_ptr(s), len(s), _ptr(C))
    return C


def psl(C: np.ndarray) -> int:
    C = np.ascontiguousarray(C, dtype=np.int32)
    return int(lib().orc_psl(_ptr(C), len(C)))


def fitness(C: np.ndarray, alpha: int):
    """(exact int, correctly rounded float, naive ordered FP64 sum) of Eq. (4)."""
    C = np.ascontiguousarray(C, dtype=np.int32)
    limbs = np.zeros(WL, dtype=np.uint64)
    fr, fn = ct.c_double(), ct.c_double()
    rc = lib().orc_fitness(_ptr(C), len(C), alpha, _ptr(limbs), ct.byref(fr), ct.byref(fn))
    assert rc == 0
    return limbs_to_int(limbs), fr.value, fn.value


def wide_to_double(v: int) -> float:
    limbs = int_to_limbs(v)
    return float(lib().orc_wide_to_double(_ptr(limbs)))


def flip_autocorr(s: np.ndarray, C: np.ndarray, j: int) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.int8)
    C = np.ascontiguousarray(C, dtype=np.int32)
    Cn = np.empty_like(C)
    lib().orc_flip_autocorr(_ptr(s), _ptr(C), len(s), j, _ptr(Cn))
    return Cn


def brute_min_psl(L: int):
    seq = np.zeros(max(L, 1), dtype=np.int8)
    v = int(lib().orc_brute_min_psl(L, _ptr(seq)))
    return v, seq[:L].copy()


def eval_neighbours(s: np.ndarray, C: np.ndarray, alpha: int, js) -> tuple[list[int], np.ndarray]:
    """Exact F and PSL of the neighbours s with s_j flipped, for each j in js."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    C = np.ascontiguousarray(C, dtype=np.int32)
    js = np.ascontiguousarray(js, dtype=np.uint32)
    limbs = np.zeros((len(js), WL), dtype=np.uint64)
    psls = np.zeros(len(js), dtype=np.int32)
    rc = lib().orc_eval_neighbours(_ptr(s), _ptr(C), len(s), alpha, _ptr(js), len(js), _ptr(limbs), _ptr(psls))
    assert rc == 0
    return [limbs_to_int(r) for r in limbs], psls


@dataclass
class WalkParams:
    L: int
    seed: int
    alpha1: int = 4
    alpha2: int = 13
    n_lmt: int = 6912
    ls_lmt: int = 2000
    flip_lmt: int = 10

    def c(self) -> Params:
        return Params(self.L, self.n_lmt, self.ls_lmt, self.flip_lmt, self.alpha1, self.alpha2, self.seed)


class Walk:
    """One walk of Algorithm 1, state held in numpy arrays owned by this object."""

    def __init__(self, p: WalkParams, s0: np.ndarray | None = None):
        self.p = p
        L = p.L
        self.s = np.zeros(L, dtype=np.int8)
        self.local_best = np.zeros(L, dtype=np.int8)
        self.sol_best = np.zeros(L, dtype=np.int8)
        self.C = np.zeros(L, dtype=np.int32)
        self.fbest_seq = np.zeros(L, dtype=np.int8)
        self._st = _State(_ptr(self.s), _ptr(self.local_best), _ptr(self.sol_best), _ptr(self.C))
        self._st.fbest_seq = _ptr(self.fbest_seq)
        self._pc = p.c()
        rc = lib().orc_init(ct.byref(self._pc), ct.byref(self._st))
        if rc != 0:
            raise ValueError(f"oracle rejected parameters {p}")
        if s0 is not None:
            self.load_state(s=s0, local_best=s0, sol_best=s0, alpha=p.alpha1, unimproved=0,
                            rng_ctr=(L + 63) // 64, value_local=None)

    # -- state access ---------------------------------------------------------------------------
    @property
    def alpha(self) -> int:
        return int(self._st.alpha)

    @property
    def unimproved(self) -> int:
        return int(self._st.unimproved)

    @property
    def psl(self) -> int:
        return int(self._st.psl)

    @property
    def psl_best(self) -> int:
        return int(self._st.psl_best)

    @property
    def rng_ctr(self) -> int:
        return int(self._st.rng_ctr)

    @property
    def steps(self) -> int:
        return int(self._st.steps)

    @property
    def near_ties(self) -> int:
        return int(self._st.near_ties)

    @property
    def value_local(self) -> int:
        return limbs_to_int(self._st.value_local)

    @property
    def F(self) -> int:
        return limbs_to_int(self._st.F)

    @property
    def F_best(self) -> int:
        """Lowest exact F over the visited pivots (kept only when alpha1 == alpha2)."""
        return limbs_to_int(self._st.F_best)

    def load_state(self, *, s, local_best, sol_best, alpha, unimproved, rng_ctr, value_local=None,
                   psl_best=None, steps=0):
        """Replace the walk state (decision replay from an exported state).  C, PSL and F are
        recomputed here from s by Eq. (2)-(4); value_local defaults to F(s)."""
        self.s[:] = s
        self.local_best[:] = local_best
        self.sol_best[:] = sol_best
        self.C[:] = autocorr(self.s)
        self._st.alpha = alpha
        self._st.unimproved = unimproved
        self._st.rng_ctr = rng_ctr
        self._st.steps = steps
        F, _, _ = fitness(self.C, alpha)
        for i, w in enumerate(int_to_limbs(F)):
            self._st.F[i] = int(w)
        vl = F if value_local is None else value_local
        for i, w in enumerate(int_to_limbs(vl)):
            self._st.value_local[i] = int(w)
        self._st.psl = psl(self.C)
        self._st.psl_best = psl(autocorr(self.sol_best)) if psl_best is None else psl_best
        self.fbest_seq[:] = s
        for i in range(WL):
            self._st.F_best[i] = self._st.F[i]

    def run(self, nsteps: int, mode: int = MODE_INCREMENTAL) -> np.ndarray:
        tr = np.zeros(nsteps, dtype=TRACE_DTYPE)
        rc = lib().orc_run(ct.byref(self._pc), ct.byref(self._st), nsteps, mode, _ptr(tr) if nsteps else None)
        if rc != 0:
            raise RuntimeError(f"oracle run failed rc={rc}")
        return tr
