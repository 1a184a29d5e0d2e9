"""ctypes binding of include/psl.h.  Argument marshalling only: the search itself runs
in libpsl.so.  Function names mirror the C ABI; ``Context`` bundles them."""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "_build", "libpsl.so")

PSL_OK, PSL_EINVAL, PSL_ENOMEM, PSL_ENOENT, PSL_EBUSY, PSL_ETIMEOUT, PSL_ECUDA, PSL_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
PSL_FORM_BATCHED, PSL_FORM_PLAIN = 0, 1
PSL_QUEUED, PSL_RUNNING, PSL_DONE, PSL_ERROR = 0, 1, 2, 3
WIDE = 12


class PslError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"psl error {code}: {msg}")
        self.code = code


class psl_config(ct.Structure):
    _fields_ = [("n_lmt", ct.c_int32), ("ls_lmt", ct.c_int32), ("flip_lmt", ct.c_int32), ("device", ct.c_int32),
                ("arena_bytes", ct.c_uint64), ("arena", ct.c_void_p), ("stream", ct.c_void_p), ("form", ct.c_int32),
                ("max_walks", ct.c_int32), ("hot_tile_sb", ct.c_int32), ("steps_per_graph", ct.c_int32),
                ("hot_threads", ct.c_int32), ("max_sms", ct.c_int32), ("alpha2_tables", ct.c_int32)]


class psl_walk_params(ct.Structure):
    _fields_ = [("L", ct.c_uint32), ("seed", ct.c_uint64), ("alpha1", ct.c_int32), ("alpha2", ct.c_int32),
                ("budget", ct.c_uint64), ("n_lmt", ct.c_int32), ("ls_lmt", ct.c_int32), ("flip_lmt", ct.c_int32),
                ("topk", ct.c_int32), ("init_seq", ct.c_void_p), ("trace_cap", ct.c_uint32),
                ("shard_rank", ct.c_uint32), ("shard_count", ct.c_uint32)]


class psl_status(ct.Structure):
    _fields_ = [("state", ct.c_int32), ("error", ct.c_int32), ("L", ct.c_uint32), ("alpha", ct.c_uint32),
                ("moves", ct.c_uint64), ("flip_evals", ct.c_uint64), ("switches", ct.c_uint64),
                ("rechecks", ct.c_uint64), ("psl", ct.c_int32), ("psl_best", ct.c_int32),
                ("unimproved", ct.c_uint32), ("pad", ct.c_uint32), ("F", ct.c_double), ("value_local", ct.c_double),
                ("t_submit", ct.c_double), ("t_start", ct.c_double), ("t_done", ct.c_double)]


class psl_walk_state(ct.Structure):
    _fields_ = [("L", ct.c_uint32), ("N", ct.c_uint32), ("alpha", ct.c_uint32), ("unimproved", ct.c_uint32),
                ("psl", ct.c_int32), ("psl_best", ct.c_int32), ("psl_local", ct.c_int32), ("start", ct.c_uint32),
                ("rng_ctr", ct.c_uint64), ("moves", ct.c_uint64), ("F", ct.c_uint32 * WIDE),
                ("value_local", ct.c_uint32 * WIDE), ("state", ct.c_int32), ("pad", ct.c_uint32)]


class psl_kernel_time(ct.Structure):
    _fields_ = [("name", ct.c_char * 24), ("launches", ct.c_uint64), ("total_ms", ct.c_double)]


TRACE_DTYPE = np.dtype([("step", "<u8"), ("start", "<u4"), ("kstar", "<u4"), ("alpha", "<u4"), ("unimproved", "<u4"),
                        ("psl", "<i4"), ("psl_best", "<i4"), ("win_psl", "<i4"), ("win_psl_j", "<u4"),
                        ("flags", "<u4"), ("nflip", "<u4"), ("ncand", "<u4"), ("score_kstar", "<f4"),
                        ("score_min", "<f4"), ("bound", "<f4"), ("scale_e", "<i4"), ("pad", "<u4"), ("value_step", "<f8"),
                        ("value_exact", "<u4", (WIDE,))])

assert TRACE_DTYPE.itemsize == 128  # psl_trace_rec has no implicit padding


class psl_alu_peak_t(ct.Structure):
    _fields_ = [("sm_count", ct.c_int32), ("max_clock_mhz", ct.c_int32), ("blocks_per_sm", ct.c_int32),
                ("threads_per_block", ct.c_int32), ("fadd", ct.c_double), ("alu", ct.c_double), ("mix", ct.c_double),
                ("lookup", ct.c_double), ("popc", ct.c_double), ("ms", ct.c_double * 5)]


EXPORTED = ["psl_config_default", "psl_init", "psl_submit", "psl_submit_ex", "psl_step", "psl_poll", "psl_best",
            "psl_release", "psl_export_state", "psl_trace", "psl_autocorr", "psl_walk_bytes", "psl_shutdown",
            "psl_last_error", "psl_profile", "psl_profile_read", "psl_autotune", "psl_set_hot_config",
            "psl_autocorr_static", "psl_inject_stall", "psl_set_max_sms",
            "psl_best_fitness", "psl_transfer_bytes", "psl_set_steps_per_graph", "psl_alu_peak",
            "psl_shard_layout", "psl_shard_score", "psl_shard_select", "psl_shard_decide", "psl_best_many",
            "psl_hot_variant"]

_lib = None


def lib_path() -> str:
    return _LIB


def lib():
    """Loads libpsl.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise ImportError(f"{_LIB} is missing: build it with paper_2107_09801_gb300.build.build() "
                              "(the search has no CPU fallback)")
        L = ct.CDLL(_LIB)
        P = ct.c_void_p
        sig = {
            "psl_config_default": (None, [ct.POINTER(psl_config)]),
            "psl_init": (ct.c_int, [ct.POINTER(psl_config), ct.POINTER(P)]),
            "psl_submit": (ct.c_int64, [P, ct.c_uint32, ct.c_uint64, ct.c_double, ct.c_double, ct.c_uint64]),
            "psl_submit_ex": (ct.c_int64, [P, ct.POINTER(psl_walk_params)]),
            "psl_step": (ct.c_int, [P, ct.c_uint32]),
            "psl_poll": (ct.c_int, [P, ct.c_int64, ct.POINTER(psl_status)]),
            "psl_best": (ct.c_int, [P, ct.c_int64, ct.POINTER(ct.c_int32), P, ct.c_size_t]),
            "psl_release": (ct.c_int, [P, ct.c_int64]),
            "psl_export_state": (ct.c_int, [P, ct.c_int64, ct.POINTER(psl_walk_state), P, P, P, P, ct.c_size_t]),
            "psl_trace": (ct.c_int, [P, ct.c_int64, P, ct.c_size_t]),
            "psl_autocorr": (ct.c_int, [P, P, ct.c_uint32, ct.c_uint32, P]),
            "psl_walk_bytes": (ct.c_uint64, [ct.c_uint32, ct.c_int32, ct.c_uint32]),
            "psl_shutdown": (None, [P]),
            "psl_last_error": (ct.c_char_p, [P]),
            "psl_profile": (ct.c_int, [P, ct.c_int]),
            "psl_profile_read": (ct.c_int, [P, ct.POINTER(psl_kernel_time), ct.c_size_t]),
            "psl_autotune": (ct.c_int, [P, ct.c_int]),
            "psl_set_hot_config": (ct.c_int, [P, ct.c_int32, ct.c_int32]),
            "psl_hot_variant": (ct.c_int, [P, ct.c_char_p, ct.c_int32]),
            "psl_autocorr_static": (ct.c_int, [P, ct.c_uint32, P, P]),
            "psl_inject_stall": (ct.c_int, [P, ct.c_int64]),
            "psl_set_max_sms": (ct.c_int, [P, ct.c_int32]),
            "psl_best_fitness": (ct.c_int, [P, ct.c_int64, P, P, P, ct.c_size_t]),
            "psl_transfer_bytes": (ct.c_int, [P, ct.POINTER(ct.c_uint64), ct.POINTER(ct.c_uint64)]),
            "psl_set_steps_per_graph": (ct.c_int, [P, ct.c_int32]),
            "psl_alu_peak": (ct.c_int, [ct.c_int32, P, ct.POINTER(psl_alu_peak_t)]),
            "psl_shard_layout": (ct.c_int, [P, ct.c_int64, ct.POINTER(ct.c_uint32), ct.POINTER(ct.c_uint32),
                                            ct.POINTER(ct.c_uint32)]),
            "psl_shard_score": (ct.c_int, [P, ct.c_int64, P, ct.c_size_t]),
            "psl_shard_select": (ct.c_int, [P, ct.c_int64, P, P, ct.c_size_t]),
            "psl_shard_decide": (ct.c_int, [P, ct.c_int64, P, ct.c_size_t]),
            "psl_best_many": (ct.c_int, [P, P, ct.c_size_t, P, P, ct.c_size_t]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def limbs_to_int(limbs) -> int:
    v = 0
    for i, w in enumerate(limbs):
        v |= int(w) << (32 * i)
    if v >> (32 * WIDE - 1):
        v -= 1 << (32 * WIDE)
    return v


# ---- C-ABI mirrors ---------------------------------------------------------------------------
def psl_config_default() -> psl_config:
    c = psl_config()
    lib().psl_config_default(ct.byref(c))
    return c


def psl_last_error(ctx) -> str:
    r = lib().psl_last_error(ctx)
    return r.decode() if r else ""


def _check(ctx, rc: int) -> int:
    if rc < 0:
        raise PslError(rc, psl_last_error(ctx))
    return rc


def psl_init(cfg: psl_config):
    h = ct.c_void_p()
    _check(None, lib().psl_init(ct.byref(cfg), ct.byref(h)))
    return h


def psl_submit(ctx, L, seed, alpha1, alpha2, budget) -> int:
    return _check(ctx, lib().psl_submit(ctx, L, seed, float(alpha1), float(alpha2), budget))


def psl_submit_ex(ctx, p: psl_walk_params) -> int:
    return _check(ctx, lib().psl_submit_ex(ctx, ct.byref(p)))


def psl_step(ctx, max_moves: int) -> int:
    return _check(ctx, lib().psl_step(ctx, max_moves))


def psl_poll(ctx, wid: int) -> dict:
    st = psl_status()
    _check(ctx, lib().psl_poll(ctx, wid, ct.byref(st)))
    return {f: getattr(st, f) for f, _ in psl_status._fields_ if f != "pad"}


def psl_best(ctx, wid: int, L: int):
    seq = np.zeros(L, dtype=np.int8)
    p = ct.c_int32()
    _check(ctx, lib().psl_best(ctx, wid, ct.byref(p), _ptr(seq), L))
    return int(p.value), seq


def psl_release(ctx, wid: int) -> None:
    _check(ctx, lib().psl_release(ctx, wid))


def psl_export_state(ctx, wid: int, L: int) -> dict:
    st = psl_walk_state()
    piv, lb, sb = (np.zeros(L, dtype=np.int8) for _ in range(3))
    C = np.zeros(L, dtype=np.int32)
    _check(ctx, lib().psl_export_state(ctx, wid, ct.byref(st), _ptr(piv), _ptr(lb), _ptr(sb), _ptr(C), L))
    d = {f: getattr(st, f) for f, _ in psl_walk_state._fields_ if f not in ("pad", "F", "value_local")}
    d["F"] = limbs_to_int(st.F)
    d["value_local"] = limbs_to_int(st.value_local)
    d.update(pivot=piv, local_best=lb, sol_best=sb, C=C)
    return d


def psl_trace(ctx, wid: int, cap: int) -> np.ndarray:
    out = np.zeros(cap, dtype=TRACE_DTYPE)
    n = _check(ctx, lib().psl_trace(ctx, wid, _ptr(out) if cap else None, cap))
    return out[:n]


def psl_autocorr(ctx, seqs: np.ndarray) -> np.ndarray:
    seqs = np.ascontiguousarray(np.atleast_2d(seqs), dtype=np.int8)
    n, L = seqs.shape
    C = np.zeros((n, L), dtype=np.int32)
    _check(ctx, lib().psl_autocorr(ctx, _ptr(seqs), n, L, _ptr(C)))
    return C


def psl_autocorr_static(seq_dev_ptr: int, L: int, C_dev_ptr: int, stream: int | None = None) -> None:
    """Autocorrelation of one sequence in device memory with the library's built-in
    scratch, for callers that cannot allocate device memory (see include/psl.h)."""
    rc = lib().psl_autocorr_static(seq_dev_ptr, L, C_dev_ptr, stream)
    if rc < 0:
        raise PslError(rc, "psl_autocorr_static failed")


def psl_alu_peak(device: int = 0, stream: int | None = None) -> dict:
    """Measured issue rates of the CUDA-core pipes (the neighbourhood kernel's roofline)."""
    out = psl_alu_peak_t()
    rc = lib().psl_alu_peak(device, stream, ct.byref(out))
    if rc < 0:
        raise PslError(rc, "psl_alu_peak failed")
    d = {f: getattr(out, f) for f, _ in psl_alu_peak_t._fields_ if f != "ms"}
    d["ms"] = list(out.ms)
    return d


def psl_walk_bytes(L: int, n_lmt: int = 6912, trace_cap: int = 0) -> int:
    return int(lib().psl_walk_bytes(L, n_lmt, trace_cap))


def psl_shutdown(ctx) -> None:
    lib().psl_shutdown(ctx)


def psl_autotune(ctx, reps: int = 3) -> tuple[int, int]:
    r = _check(ctx, lib().psl_autotune(ctx, reps))
    return r & 0xFFFF, r >> 16


def psl_set_hot_config(ctx, threads: int, tile_sb: int) -> None:
    _check(ctx, lib().psl_set_hot_config(ctx, threads, tile_sb))


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown-gpu"


def psl_profile(ctx, enable: bool | int) -> None:
    _check(ctx, lib().psl_profile(ctx, int(enable)))


def psl_profile_read(ctx) -> dict:
    arr = (psl_kernel_time * 16)()
    n = _check(ctx, lib().psl_profile_read(ctx, arr, 16))
    return {arr[k].name.decode(): (int(arr[k].launches), float(arr[k].total_ms)) for k in range(n)}


# ---- convenience wrapper ---------------------------------------------------------------------
class Context:
    """One library context.  Device memory may come from a torch tensor (``arena_tensor``)
    and work may be issued on a torch stream (``stream``); torch is plumbing only."""

    def __init__(self, *, form: str = "batched", arena_bytes: int = 0, arena_tensor=None, stream=None,
                 max_walks: int = 4096, n_lmt: int = 6912, ls_lmt: int = 2000, flip_lmt: int = 10, device: int = 0,
                 hot_tile_sb: int = 0, steps_per_graph: int = 0, hot_threads: int = 0, max_sms: int = 0,
                 alpha2_tables: bool = False):
        cfg = psl_config_default()
        cfg.n_lmt, cfg.ls_lmt, cfg.flip_lmt, cfg.device = n_lmt, ls_lmt, flip_lmt, device
        cfg.form = PSL_FORM_PLAIN if form == "plain" else PSL_FORM_BATCHED
        cfg.max_walks, cfg.hot_tile_sb, cfg.steps_per_graph = max_walks, hot_tile_sb, steps_per_graph
        cfg.hot_threads = hot_threads
        cfg.max_sms = max_sms
        cfg.alpha2_tables = 1 if alpha2_tables else 0
        self._arena_tensor = arena_tensor
        if arena_tensor is not None:
            cfg.arena = arena_tensor.data_ptr()
            cfg.arena_bytes = arena_tensor.numel() * arena_tensor.element_size()
        else:
            cfg.arena_bytes = arena_bytes
        if stream is not None:
            cfg.stream = stream if isinstance(stream, int) else stream.cuda_stream
        self.h = psl_init(cfg)
        self.L_of: dict[int, int] = {}

    def submit(self, L, seed, alpha1, alpha2, budget) -> int:
        wid = psl_submit(self.h, L, seed, alpha1, alpha2, budget)
        self.L_of[wid] = L
        return wid

    def submit_ex(self, L, seed, alpha1=4, alpha2=13, budget=2000, *, n_lmt=0, ls_lmt=-1, flip_lmt=0, topk=1,
                  init_seq=None, trace_cap=0, shard_rank=0, shard_count=0) -> int:
        seq = None if init_seq is None else np.ascontiguousarray(init_seq, dtype=np.int8)
        p = psl_walk_params(L, seed, alpha1, alpha2, budget, n_lmt, ls_lmt, flip_lmt, topk,
                            None if seq is None else seq.ctypes.data, trace_cap, shard_rank, shard_count)
        wid = psl_submit_ex(self.h, p)
        self.L_of[wid] = L
        return wid

    def step(self, max_moves: int) -> int:
        return psl_step(self.h, max_moves)

    def run(self, chunk: int = 1 << 30) -> None:
        while self.step(chunk) > 0:
            pass

    def poll(self, wid: int) -> dict:
        return psl_poll(self.h, wid)

    def best(self, wid: int):
        return psl_best(self.h, wid, self.L_of[wid])

    def best_many(self, wids) -> tuple[np.ndarray, np.ndarray]:
        """(PSL of each walk's best sequence, the sequences as rows of +-1 int8, padded with 0
        to the longest L), copied back together."""
        wids = np.ascontiguousarray(wids, dtype=np.int64)
        cap = max((self.L_of.get(int(w), 0) for w in wids), default=0)
        psl = np.zeros(len(wids), dtype=np.int32)
        seqs = np.zeros((len(wids), cap), dtype=np.int8)
        _check(self.h, lib().psl_best_many(self.h, wids.ctypes.data, len(wids), psl.ctypes.data,
                                           seqs.ctypes.data, cap))
        return psl, seqs

    def release(self, wid: int) -> None:
        psl_release(self.h, wid)
        self.L_of.pop(wid, None)

    def export_state(self, wid: int) -> dict:
        return psl_export_state(self.h, wid, self.L_of[wid])

    def trace(self, wid: int, cap: int) -> np.ndarray:
        return psl_trace(self.h, wid, cap)

    def autocorr(self, seqs) -> np.ndarray:
        return psl_autocorr(self.h, seqs)

    def autotune(self, reps: int = 3, cache: str | None = None) -> tuple[int, int]:
        """Picks the neighbourhood-kernel configuration for the running walks.  With a
        cache file, a previous choice for the same GPU and length bucket is reused."""
        key = None
        if cache:
            import json
            Ls = [L for w, L in self.L_of.items()]
            key = f"{_gpu_name()}|L<=2^{max(Ls).bit_length() if Ls else 0}|walks>={1 << max(len(Ls), 1).bit_length() >> 1}"
            try:
                table = json.load(open(cache))
            except Exception:
                table = {}
            if key in table:
                t, sb = table[key]
                self._set_hot(t, sb)
                return t, sb
        t, sb = psl_autotune(self.h, reps)
        if cache:
            table[key] = [t, sb]
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return t, sb

    def hot_variant(self) -> str:
        """Name of the neighbourhood kernel the next step launches (queued walks admitted)."""
        buf = ct.create_string_buffer(64)
        rc = lib().psl_hot_variant(self.h, buf, 64)
        if rc < 0:
            raise PslError(rc, "psl_hot_variant failed")
        return buf.value.decode()

    def _set_hot(self, threads: int, tile_sb: int) -> None:
        psl_set_hot_config(self.h, threads, tile_sb)

    def best_fitness(self, wid: int):
        """(exact lowest F over the visited pivots, its sequence as +-1 int8) of a walk whose
        phases share one exponent; with alpha = 2, F is the merit-factor energy."""
        L = self.L_of[wid]
        limbs = (ct.c_uint32 * 12)()
        seq = np.zeros(L, dtype=np.int8)
        _check(self.h, lib().psl_best_fitness(self.h, wid, ct.addressof(limbs), None, seq.ctypes.data, L))
        return sum(int(v) << (32 * i) for i, v in enumerate(limbs)), seq

    def set_max_sms(self, max_sms: int) -> int:
        """Sizes the persistent kernels for max_sms SMs from the next step on (0 = all);
        returns the SM count in use."""
        return _check(self.h, lib().psl_set_max_sms(self.h, max_sms))

    # ---- single-walk k-sharding (one step = score, exchange, select, exchange, decide) ----
    def shard_layout(self, wid: int) -> tuple[int, int, int]:
        """(k-chunks, window size N, most re-check words of a step) of a sharded walk."""
        a, b, c = ct.c_uint32(), ct.c_uint32(), ct.c_uint32()
        _check(self.h, lib().psl_shard_layout(self.h, wid, ct.byref(a), ct.byref(b), ct.byref(c)))
        return int(a.value), int(b.value), int(c.value)

    def shard_score(self, wid: int) -> np.ndarray:
        """This rank's partial FP32 scores, float32 [ksplit, N]; other ranks' chunks are zero."""
        ks, n, _ = self.shard_layout(wid)
        parts = np.zeros((ks, n), dtype=np.float32)
        _check(self.h, lib().psl_shard_score(self.h, wid, parts.ctypes.data, parts.size))
        return parts

    def shard_select(self, wid: int, parts: np.ndarray) -> np.ndarray:
        """Selection on the summed scores, then this rank's exact re-check words (uint32)."""
        parts = np.ascontiguousarray(parts, dtype=np.float32)
        _, _, cap = self.shard_layout(wid)
        out = np.zeros(cap, dtype=np.uint32)
        m = _check(self.h, lib().psl_shard_select(self.h, wid, parts.ctypes.data, out.ctypes.data, cap))
        return out[:m]

    def shard_decide(self, wid: int, rc_words: np.ndarray) -> int:
        """The exact decision and update from the summed re-check words; returns the walk state."""
        rc_words = np.ascontiguousarray(rc_words, dtype=np.uint32)
        return _check(self.h, lib().psl_shard_decide(self.h, wid, rc_words.ctypes.data if rc_words.size else None,
                                                      rc_words.size))

    def inject_stall(self, wid: int) -> None:
        """Test hook: the walk's next neighbourhood pass runs out its bounded waits."""
        _check(self.h, lib().psl_inject_stall(self.h, wid))

    def profile(self, enable: bool | int = True) -> None:
        """True / 1: time every kernel; 2: the neighbourhood kernel only; False / 0: off."""
        _check(self.h, lib().psl_profile(self.h, int(enable)))

    def transfer_bytes(self) -> tuple[int, int]:
        """(host->device, device->host) bytes the context has copied since it was created."""
        a, b = ct.c_uint64(), ct.c_uint64()
        _check(self.h, lib().psl_transfer_bytes(self.h, ct.byref(a), ct.byref(b)))
        return int(a.value), int(b.value)

    def set_steps_per_graph(self, steps: int) -> None:
        """Steps per CUDA graph launch (0 = plain launches); captures the graph now when walks run."""
        _check(self.h, lib().psl_set_steps_per_graph(self.h, steps))

    def profile_read(self) -> dict:
        return psl_profile_read(self.h)

    def close(self) -> None:
        if self.h:
            psl_shutdown(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
