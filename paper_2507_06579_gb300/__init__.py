"""Eisenstein discriminants on GB300 (sm_103a): Python binding.

Thin ctypes marshalling over the C-ABI of ``include/eis.h``; every step of
the computation runs in the CUDA kernels of ``libeis_gb300.so`` (built
in-tree by :func:`build`).  There is no CPU fallback: if the library is not
built, or no GPU is present, the calls raise.

The functions mirror the C entry points::

    ctx = Context(device=0)
    ctx.count_range(lo, hi)                  # eis_count_range
    ctx.classify_range(lo, hi)               # eis_classify_range (bit-packed)
    ctx.classify_range_u8(lo, hi)            # eis_classify_range_u8
    ctx.classify_range_log(lo, hi)           # eis_classify_range_log
    ctx.is_eisenstein(d)                     # eis_is_eisenstein
    ctx.count_batch(los, his)                # eis_count_batch
    plan = ctx.plan_create(los, his, mode)   # eis_plan_* (device-resident pipeline)

Device outputs may be torch CUDA tensors (their ``data_ptr()`` is passed);
streams may be ``torch.cuda.Stream`` objects.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

LIB_PATH = _build.LIB

EIS_OK = 0
EIS_EINVAL = -1
EIS_ENOTD = -2
EIS_ERANGE = -3
EIS_ENOMEM = -4
EIS_ETIMEOUT = -5
EIS_EDEVICE = -6
EIS_ESTEPS = -7
EIS_EBUSY = -8
EIS_ENOTFOUND = -9
EIS_ETOOLARGE = -10
EIS_ECANCELED = -11
EIS_REQ_COUNT = 0
EIS_REQ_MEMBER = 1
EIS_NOALLOC_MAX_CANDIDATES = 1 << 20

EIS_D_LIMIT = 1 << 44

EIS_MODE_PLAIN = 0
EIS_MODE_PERSISTENT = 1

EIS_PLAN_CLASSES = 1
EIS_PLAN_PRIMES = 2

EIS_OPT_MODE = 1
EIS_OPT_CTAS_PER_SM = 2
EIS_OPT_THREADS = 3
EIS_OPT_STEP_LIMIT = 4
EIS_OPT_USE_GRAPH = 5
EIS_OPT_GIANT_THRESHOLD = 6
EIS_OPT_GIANT_STRIDE = 7
EIS_OPT_GIANT_COMPOSE = 8
EIS_OPT_MEM_BUDGET = 9
EIS_OPT_MEM_IN_USE = 10
EIS_OPT_GIANT_KERNEL = 11
EIS_OPT_MARK_EVERY = 12
EIS_OPT_BSGS_CHUNK = 13
EIS_OPT_BSGS_WALK_CAP = 14
EIS_OPT_BSGS_WINDOW = 15
EIS_GIANT_LANE = 0
EIS_GIANT_WARP = 1
EIS_COMPOSE_TEXTBOOK = 0
EIS_COMPOSE_NUCOMP = 1

_lock = threading.Lock()
_lib = None


class EisError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().eis_strerror(code).decode()
        if code == EIS_EDEVICE:
            msg += " [%s]" % lib().eis_last_cuda_error_string().decode()
        super().__init__("%s failed: %s (%d)" % (where, msg, code))


class Stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_uint64), ("in_D", ctypes.c_uint64),
                ("in_E", ctypes.c_uint64), ("baby_steps", ctypes.c_uint64),
                ("giant_steps", ctypes.c_uint64), ("deferred", ctypes.c_uint64),
                ("ms_total", ctypes.c_double), ("ms_walk", ctypes.c_double),
                ("ms_sieve", ctypes.c_double), ("ms_giant", ctypes.c_double),
                ("launches", ctypes.c_int), ("sm_count", ctypes.c_int),
                ("search_steps", ctypes.c_uint64)]

    def as_dict(self):
        """The fields as a plain dict."""
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile libeis_gb300.so for sm_103a (nvcc) if it is out of date."""
    return _build.build(force=force)


class TuneRow(ctypes.Structure):
    _fields_ = [("d_hi", ctypes.c_uint64), ("nbaby", ctypes.c_int32), ("mark_every", ctypes.c_int32)]


EIS_TUNE_MAX_ROWS = 8


class TuneResult(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("giant_threshold", ctypes.c_int64),
                ("giant_stride", ctypes.c_int64), ("ms_best", ctypes.c_double),
                ("ms_default", ctypes.c_double), ("trials", ctypes.c_int32),
                ("giant_kernel", ctypes.c_int32), ("mark_every", ctypes.c_int32),
                ("bsgs_chunk", ctypes.c_int64)]

    def as_dict(self):
        """The fields as a plain dict."""
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("slot_candidates", ctypes.c_uint64),
                ("slot_requests", ctypes.c_uint32), ("max_pending", ctypes.c_uint32),
                ("giant_after", ctypes.c_uint32), ("giant_max", ctypes.c_uint32),
                ("fail_launches", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "requests_submitted", "requests_done", "rejected", "batches", "parts",
        "max_batch_parts", "pending_parts", "reserved_bytes", "deferred")]

    def as_dict(self):
        """The fields as a plain dict."""
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


# (name, restype, argtypes) of every exported symbol declared in include/eis.h
_VP, _U64, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
_P = ctypes.POINTER
SIGNATURES = [
    ("eis_create", _I32, [_P(_VP), _I32, _U64]),
    ("eis_destroy", _I32, [_VP]),
    ("eis_strerror", ctypes.c_char_p, [_I32]),
    ("eis_last_cuda_error_string", ctypes.c_char_p, []),
    ("eis_set_option", _I32, [_VP, _I32, _I64]),
    ("eis_get_option", _I32, [_VP, _I32, _P(_I64)]),
    ("eis_get_stats", _I32, [_VP, _P(Stats)]),
    ("eis_count_range", _I32, [_VP, _U64, _U64, _P(_U64)]),
    ("eis_classify_range", _I32, [_VP, _U64, _U64, _VP, _VP, _I32, _P(_U64), _VP]),
    ("eis_classify_range_u8", _I32, [_VP, _U64, _U64, _VP, _I32, _P(_U64), _VP]),
    ("eis_classify_range_log", _I32, [_VP, _U64, _U64, _VP, _I32, _VP]),
    ("eis_is_eisenstein", _I32, [_VP, _U64, _P(_I32)]),
    ("eis_count_batch", _I32, [_VP, _VP, _VP, _SZ, _VP]),
    ("eis_autotune", _I32, [_VP, _U64, _U64, _P(TuneResult)]),
    ("eis_set_tune_table", _I32, [_VP, _VP, _SZ]),
    ("eis_get_tune_table", _I32, [_VP, _VP, _SZ, _P(_SZ)]),
    ("eis_autotune_decades", _I32, [_VP, _U64, _U64, _VP, _SZ, _P(_SZ)]),
    ("eis_classify_range_noalloc", _I32, [_I32, _U64, _U64, _VP, _VP, _P(_U64), _VP]),
    ("eis_plan_create", _I32, [_VP, _VP, _VP, _SZ, _I32, _P(_VP)]),
    ("eis_plan_create_ex", _I32, [_VP, _VP, _VP, _SZ, _I32, ctypes.c_uint32, _P(_VP)]),
    ("eis_plan_class_counts", _I32, [_VP, _VP]),
    ("eis_class_counts", _I32, [_VP, _U64, _U64, _I32, _VP]),
    ("eis_plan_launch", _I32, [_VP, _VP]),
    ("eis_plan_counts", _I32, [_VP, _VP]),
    ("eis_plan_counts_D", _I32, [_VP, _VP]),
    ("eis_plan_bitmaps", _I32, [_VP, _P(_VP), _P(_VP), _VP, _P(_U64)]),
    ("eis_plan_copy_bitmaps", _I32, [_VP, _VP, _VP, _I32]),
    ("eis_plan_stats", _I32, [_VP, _P(Stats)]),
    ("eis_plan_destroy", _I32, [_VP]),
    ("eis_server_create", _I32, [_VP, _P(ServerConfig), _P(_VP)]),
    ("eis_server_submit", _I32, [_VP, _I32, _U64, _U64, _P(_U64)]),
    ("eis_server_poll", _I32, [_VP, _U64, _P(_I32)]),
    ("eis_server_wait", _I32, [_VP, _U64, ctypes.c_double, _P(_U64), _P(ctypes.c_double)]),
    ("eis_server_cancel", _I32, [_VP, _U64]),
    ("eis_server_stats", _I32, [_VP, _P(ServerStats)]),
    ("eis_server_destroy", _I32, [_VP]),
    ("eis_server_replay", _I32, [_VP, _SZ, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                 _P(ctypes.c_double)]),
]


def lib():
    """Load libeis_gb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libeis_gb300.so is not built; run "
                                   "paper_2507_06579_gb300.build() (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != EIS_OK:
        raise EisError(rc, where)


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _u64_array(vals):
    a = np.ascontiguousarray(np.asarray(vals, dtype=np.uint64))
    return a


def num_candidates(lo: int, hi: int):
    """(n, d0): candidates d == 5 (mod 8) in [lo, hi) and the first one."""
    d0 = lo + ((13 - lo % 8) % 8)
    return (max(0, (hi - d0 + 7) // 8) if hi > d0 else 0), d0


class Plan:
    """A device-resident pipeline over fixed intervals (eis_plan_*)."""

    def __init__(self, ctx: "Context", los, his, mode: int, flags: int = 0):
        self.ctx = ctx
        self.los = _u64_array(los)
        self.his = _u64_array(his)
        self.n = len(self.los)
        self.flags = flags
        h = ctypes.c_void_p()
        _check(lib().eis_plan_create_ex(ctx.handle, self.los.ctypes.data, self.his.ctypes.data,
                                        self.n, mode, flags, ctypes.byref(h)), "eis_plan_create_ex")
        self.handle = h

    def class_counts(self):
        """(n, 3) array: per interval the number of d with eps_d == omega^g
        mod 2O_K, g = 0, 1, 2 (needs EIS_PLAN_CLASSES)."""
        out = np.zeros(3 * max(self.n, 1), dtype=np.uint64)
        _check(lib().eis_plan_class_counts(self.handle, out.ctypes.data), "eis_plan_class_counts")
        return out[: 3 * self.n].reshape(self.n, 3)

    def launch(self, stream=None):
        """Enqueue one full pass (the plan's CUDA graph) on `stream`, by default the context's
        stream; asynchronous, as eis_plan_launch."""
        _check(lib().eis_plan_launch(self.handle, _stream_handle(stream)), "eis_plan_launch")

    def counts(self):
        """Per-interval #E (d in E) of the last launch."""
        out = np.zeros(max(self.n, 1), dtype=np.uint64)
        _check(lib().eis_plan_counts(self.handle, out.ctypes.data), "eis_plan_counts")
        return out[: self.n]

    def counts_D(self):
        """Per-interval #D (square-free candidates) of the last launch."""
        out = np.zeros(max(self.n, 1), dtype=np.uint64)
        _check(lib().eis_plan_counts_D(self.handle, out.ctypes.data), "eis_plan_counts_D")
        return out[: self.n]

    def stats(self) -> dict:
        """Counts and device times of the last launch (eis_plan_stats)."""
        st = Stats()
        _check(lib().eis_plan_stats(self.handle, ctypes.byref(st)), "eis_plan_stats")
        return st.as_dict()

    def bitmaps(self):
        """(flags_ptr, sqfree_ptr, word_offsets, total_words) -- device pointers."""
        f, s = ctypes.c_void_p(), ctypes.c_void_p()
        off = np.zeros(max(self.n, 1), dtype=np.uint64)
        tot = ctypes.c_uint64()
        _check(lib().eis_plan_bitmaps(self.handle, ctypes.byref(f), ctypes.byref(s),
                                      off.ctypes.data, ctypes.byref(tot)), "eis_plan_bitmaps")
        return f.value, s.value, off[: self.n], int(tot.value)

    def copy_bitmaps(self):
        """Host copies (flags, sqfree) of the plan's bitmaps (uint32 words)."""
        _, _, _, tot = self.bitmaps()
        f = np.zeros(max(tot, 1), dtype=np.uint32)
        s = np.zeros(max(tot, 1), dtype=np.uint32)
        _check(lib().eis_plan_copy_bitmaps(self.handle, f.ctypes.data, s.ctypes.data, 0),
               "eis_plan_copy_bitmaps")
        return f[:tot], s[:tot]

    def destroy(self):
        """Free the plan's device buffers and graph (idempotent)."""
        if self.handle:
            lib().eis_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (eis_server_*)."""

    def __init__(self, ctx: "Context", slots: int = 0, slot_candidates: int = 0,
                 slot_requests: int = 0, max_pending: int = 0, giant_after: int = 0,
                 giant_max: int = 0, fail_launches: int = 0):
        self.ctx = ctx
        cfg = ServerConfig(slots, slot_candidates, slot_requests, max_pending, giant_after,
                           giant_max, fail_launches)
        h = ctypes.c_void_p()
        _check(lib().eis_server_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)),
               "eis_server_create")
        self.handle = h

    def submit_count(self, lo: int, hi: int) -> int:
        """Queue #E over [lo, hi); returns the request id."""
        rid = ctypes.c_uint64()
        _check(lib().eis_server_submit(self.handle, EIS_REQ_COUNT, lo, hi, ctypes.byref(rid)),
               "eis_server_submit")
        return int(rid.value)

    def submit_member(self, d: int) -> int:
        """Queue the membership query 'is d in E'; returns the request id."""
        rid = ctypes.c_uint64()
        _check(lib().eis_server_submit(self.handle, EIS_REQ_MEMBER, d, d + 1, ctypes.byref(rid)),
               "eis_server_submit")
        return int(rid.value)

    def poll(self, rid: int) -> bool:
        """True once request rid has finished (does not wait)."""
        done = ctypes.c_int()
        _check(lib().eis_server_poll(self.handle, rid, ctypes.byref(done)), "eis_server_poll")
        return bool(done.value)

    def wait(self, rid: int, timeout_ms: float = 60_000.0):
        """(status, result, latency_us); status is an EIS_* code (EIS_ETIMEOUT
        leaves the request queued)."""
        res = ctypes.c_uint64()
        lat = ctypes.c_double()
        rc = lib().eis_server_wait(self.handle, rid, timeout_ms, ctypes.byref(res), ctypes.byref(lat))
        return rc, int(res.value), float(lat.value)

    def cancel(self, rid: int):
        """Drop request rid if it has not finished."""
        _check(lib().eis_server_cancel(self.handle, rid), "eis_server_cancel")

    def stats(self) -> dict:
        """Server counters: requests, batches, parts, reserved memory."""
        st = ServerStats()
        _check(lib().eis_server_stats(self.handle, ctypes.byref(st)), "eis_server_stats")
        return st.as_dict()

    def replay(self, t_arrival_s, kinds, los, his):
        """Native load replay -> dict of numpy arrays (results, status,
        latency_us) and the wall time."""
        n = len(t_arrival_s)
        t = np.ascontiguousarray(np.asarray(t_arrival_s, dtype=np.float64))
        k = np.ascontiguousarray(np.asarray(kinds, dtype=np.int32))
        lo, hi = _u64_array(los), _u64_array(his)
        res = np.zeros(max(n, 1), dtype=np.uint64)
        st = np.zeros(max(n, 1), dtype=np.int32)
        lat = np.zeros(max(n, 1), dtype=np.float64)
        wall = ctypes.c_double()
        rc = lib().eis_server_replay(self.handle, n, t.ctypes.data, k.ctypes.data, lo.ctypes.data,
                                     hi.ctypes.data, res.ctypes.data, st.ctypes.data,
                                     lat.ctypes.data, ctypes.byref(wall))
        return {"rc": rc, "results": res[:n], "status": st[:n], "latency_us": lat[:n],
                "wall_s": float(wall.value)}

    def close(self):
        """Stop the server and free its slots (idempotent)."""
        if getattr(self, "handle", None):
            lib().eis_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One device context (eis_create / eis_destroy)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, mode: int | None = None):
        h = ctypes.c_void_p()
        _check(lib().eis_create(ctypes.byref(h), device, mem_budget_bytes), "eis_create")
        self.handle = h
        self.device = device
        if mode is not None:
            self.set_option(EIS_OPT_MODE, mode)

    def close(self):
        """Release the context and every device resource it owns (idempotent)."""
        if getattr(self, "handle", None):
            lib().eis_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- options / stats
    def set_option(self, key: int, value: int):
        """Set an EIS_OPT_* option (raises EisError on an invalid value)."""
        _check(lib().eis_set_option(self.handle, key, int(value)), "eis_set_option")

    def get_option(self, key: int) -> int:
        """Current value of an EIS_OPT_* option."""
        v = ctypes.c_int64()
        _check(lib().eis_get_option(self.handle, key, ctypes.byref(v)), "eis_get_option")
        return int(v.value)

    def stats(self) -> dict:
        """Counts, steps and times of the context's last call (eis_get_stats)."""
        st = Stats()
        _check(lib().eis_get_stats(self.handle, ctypes.byref(st)), "eis_get_stats")
        return st.as_dict()

    # -- entry points
    def count_range(self, lo: int, hi: int) -> int:
        """#E over the half-open range [lo, hi)."""
        out = ctypes.c_uint64()
        _check(lib().eis_count_range(self.handle, lo, hi, ctypes.byref(out)), "eis_count_range")
        return int(out.value)

    def pi_E(self, x: int) -> int:
        """pi_E(x) = #{d in E : d <= x}."""
        return self.count_range(0, x + 1)

    def classify_range(self, lo: int, hi: int, flags_out=None, sqfree_out=None, stream=None):
        """Bit-packed flags / square-free words.  With no outputs given, returns
        host numpy uint32 arrays (flags, sqfree, count).  Torch CUDA tensors as
        outputs are written on the device."""
        n, _ = num_candidates(lo, hi)
        nw = (n + 31) // 32
        cnt = ctypes.c_uint64()
        if flags_out is None and sqfree_out is None:
            f = np.zeros(max(nw, 1), dtype=np.uint32)
            s = np.zeros(max(nw, 1), dtype=np.uint32)
            _check(lib().eis_classify_range(self.handle, lo, hi, f.ctypes.data, s.ctypes.data, 0,
                                            ctypes.byref(cnt), _stream_handle(stream)),
                   "eis_classify_range")
            return f[:nw], s[:nw], int(cnt.value)
        on_dev = 1 if _is_device(flags_out if flags_out is not None else sqfree_out) else 0
        _check(lib().eis_classify_range(self.handle, lo, hi, _ptr(flags_out), _ptr(sqfree_out),
                                        on_dev, ctypes.byref(cnt), _stream_handle(stream)),
               "eis_classify_range")
        return flags_out, sqfree_out, int(cnt.value)

    def classify_range_u8(self, lo: int, hi: int, codes_out=None, stream=None):
        """One byte per candidate d == 5 (mod 8) of [lo, hi): 0 not in D, 1 in D \\ E, 2 in E.
        Returns (codes, #E); a torch CUDA tensor as codes_out is written on the device."""
        n, _ = num_candidates(lo, hi)
        cnt = ctypes.c_uint64()
        if codes_out is None:
            codes = np.zeros(max(n, 1), dtype=np.uint8)
            _check(lib().eis_classify_range_u8(self.handle, lo, hi, codes.ctypes.data, 0,
                                               ctypes.byref(cnt), _stream_handle(stream)),
                   "eis_classify_range_u8")
            return codes[:n], int(cnt.value)
        _check(lib().eis_classify_range_u8(self.handle, lo, hi, _ptr(codes_out),
                                           1 if _is_device(codes_out) else 0, ctypes.byref(cnt),
                                           _stream_handle(stream)), "eis_classify_range_u8")
        return codes_out, int(cnt.value)

    def classify_range_log(self, lo: int, hi: int, stream=None):
        """One byte per candidate: 0 not in D, else 1 + log_omega(eps_d mod 2O_K)."""
        n, _ = num_candidates(lo, hi)
        out = np.zeros(max(n, 1), dtype=np.uint8)
        _check(lib().eis_classify_range_log(self.handle, lo, hi, out.ctypes.data, 0,
                                            _stream_handle(stream)), "eis_classify_range_log")
        return out[:n]

    def is_eisenstein(self, d: int) -> bool:
        """True if d is in E; raises EisError with code EIS_ENOTD if d is not in D."""
        r = ctypes.c_int()
        _check(lib().eis_is_eisenstein(self.handle, d, ctypes.byref(r)), "eis_is_eisenstein")
        return bool(r.value)

    def count_batch(self, los, his):
        """#E of each range [los[i], his[i]) in one persistent launch."""
        lo = _u64_array(los)
        hi = _u64_array(his)
        assert lo.shape == hi.shape
        out = np.zeros(max(len(lo), 1), dtype=np.uint64)
        _check(lib().eis_count_batch(self.handle, lo.ctypes.data, hi.ctypes.data, len(lo),
                                     out.ctypes.data), "eis_count_batch")
        return out[: len(lo)]

    def set_tune_table(self, rows):
        """Install per-decade lane-search settings: rows of (d_hi, nbaby,
        mark_every), d_hi increasing (eis_set_tune_table); [] removes them."""
        arr = (TuneRow * max(len(rows), 1))(*[TuneRow(int(a), int(b), int(c)) for a, b, c in rows])
        _check(lib().eis_set_tune_table(self.handle, ctypes.addressof(arr), len(rows)),
               "eis_set_tune_table")

    def tune_table(self):
        """The installed per-decade settings as (d_hi, nbaby, mark_every) rows."""
        arr = (TuneRow * EIS_TUNE_MAX_ROWS)()
        n = ctypes.c_size_t()
        _check(lib().eis_get_tune_table(self.handle, ctypes.addressof(arr), EIS_TUNE_MAX_ROWS,
                                        ctypes.byref(n)), "eis_get_tune_table")
        return [(arr[i].d_hi, arr[i].nbaby, arr[i].mark_every) for i in range(n.value)]

    def autotune_decades(self, lo: int, hi: int):
        """Time the walk and the lane search per decade of [lo, hi) and keep
        the fastest settings in the context's table (eis_autotune_decades);
        returns the rows found, (d_hi, nbaby, mark_every), nbaby = 0 = walk."""
        arr = (TuneRow * 16)()
        n = ctypes.c_size_t()
        _check(lib().eis_autotune_decades(self.handle, int(lo), int(hi), ctypes.addressof(arr), 16,
                                          ctypes.byref(n)), "eis_autotune_decades")
        return [(arr[i].d_hi, arr[i].nbaby, arr[i].mark_every) for i in range(min(n.value, 16))]

    def autotune(self, lo: int, hi: int, cache_path: str | None = None) -> dict:
        """Pick the persistent-walk and giant-step settings for the d-range of
        the sample [lo, hi) (eis_autotune) and keep them in this context.
        With cache_path, results are stored per decade of hi in a JSON file
        and reused instead of re-timing."""
        import json
        import math
        key = "decade_%d" % int(math.log10(max(hi, 10)))
        cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        if key in cache:
            r = cache[key]
            self.set_option(EIS_OPT_CTAS_PER_SM, r["ctas_per_sm"])
            self.set_option(EIS_OPT_GIANT_THRESHOLD, r["giant_threshold"])
            self.set_option(EIS_OPT_GIANT_STRIDE, r["giant_stride"])
            if "giant_kernel" in r:
                self.set_option(EIS_OPT_GIANT_KERNEL, r["giant_kernel"])
                self.set_option(EIS_OPT_BSGS_CHUNK, r["bsgs_chunk"])
            return dict(r, cached=True)
        res = TuneResult()
        _check(lib().eis_autotune(self.handle, lo, hi, ctypes.byref(res)), "eis_autotune")
        r = res.as_dict()
        if cache_path:
            cache[key] = r
            tmp = cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, cache_path)
        return dict(r, cached=False)

    def plan_create(self, los, his, mode: int = EIS_MODE_PERSISTENT, flags: int = 0) -> Plan:
        """A reusable plan over the ranges [los[i], his[i]) (see Plan)."""
        return Plan(self, los, his, mode, flags)

    def class_counts(self, lo: int, hi: int, primes_only: bool = False):
        """[#{eps_d == 1}, #{eps_d == omega}, #{eps_d == omega^2}] over [lo, hi)."""
        out = np.zeros(3, dtype=np.uint64)
        _check(lib().eis_class_counts(self.handle, lo, hi, 1 if primes_only else 0,
                                      out.ctypes.data), "eis_class_counts")
        return [int(x) for x in out]


def _is_device(t) -> bool:
    return hasattr(t, "is_cuda") and bool(t.is_cuda)


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t)
