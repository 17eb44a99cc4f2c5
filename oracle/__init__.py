"""CPU oracle for Eisenstein discriminants -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import this package.  The product path
(``paper_2507_06579_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, integers only); this module
builds it with gcc and exposes thin ctypes wrappers:

* ``walk_mod2(d)``      Oracle-B: Appendix A baby steps with theta kept
                        modulo 2O_K, full period -> (theta code, period)
* ``unit_exact(d)``     Oracle-A: the exact fundamental unit (Section 1,
                        eps_d = (x0 + y0 sqrt d)/2) with its norm verified
* ``classify_range``    per-candidate codes 0 (not in D), 1 (D \\ E), 2 (E)
* ``count_range``       (#D, #E, rho steps) over [lo, hi)
* ``pell_smallest``     Lemma 1.1(ii) brute force
* ``narrow_classno``    Lemma 1.1(iv) via cycles of reduced forms
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_ENOTD = -1
ORC_EINVARIANT = -2
ORC_ENORM = -3


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, pthreads)."""
    newer = os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h")))
    if newer and not force:
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-Wall", "-Wextra", "-fPIC", "-shared",
           "-pthread", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Unit(ctypes.Structure):
    _fields_ = [("period", ctypes.c_uint64), ("norm", ctypes.c_int),
                ("flag", ctypes.c_int), ("theta", ctypes.c_int),
                ("x0_lo", ctypes.c_uint64), ("y0_lo", ctypes.c_uint64),
                ("y0_fits", ctypes.c_int), ("x0_fits", ctypes.c_int),
                ("y0_bits", ctypes.c_uint64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB: load a prebuilt variant (the mutation tests plant
            # mistakes in a copy of oracle.c and load it this way)
            path = os.environ.get("ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            u64, i32 = ctypes.c_uint64, ctypes.c_int
            L.orc_isqrt.restype = u64
            L.orc_isqrt.argtypes = [u64]
            L.orc_is_squarefree.restype = i32
            L.orc_is_squarefree.argtypes = [u64]
            L.orc_in_D.restype = i32
            L.orc_in_D.argtypes = [u64]
            L.orc_walk_mod2.restype = i32
            L.orc_walk_mod2.argtypes = [u64, ctypes.POINTER(i32), ctypes.POINTER(u64)]
            L.orc_unit_exact.restype = i32
            L.orc_unit_exact.argtypes = [u64, ctypes.POINTER(_Unit)]
            L.orc_pell_smallest.restype = u64
            L.orc_pell_smallest.argtypes = [u64, u64, ctypes.POINTER(u64), ctypes.POINTER(i32)]
            L.orc_narrow_classno.restype = ctypes.c_int64
            L.orc_narrow_classno.argtypes = [u64]
            L.orc_classify_range.restype = i32
            L.orc_classify_range.argtypes = [u64, u64, i32, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]
            L.orc_count_range.restype = i32
            L.orc_count_range.argtypes = [u64, u64, i32, ctypes.POINTER(u64 * 3)]
            L.orc_sqfree_range.restype = i32
            L.orc_sqfree_range.argtypes = [u64, u64, i32, ctypes.c_void_p, ctypes.POINTER(u64)]
            L.orc_is_prime.restype = i32
            L.orc_is_prime.argtypes = [u64]
            L.orc_classify_range_primes.restype = i32
            L.orc_classify_range_primes.argtypes = [u64, u64, i32, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_count_range_primes.restype = i32
            L.orc_count_range_primes.argtypes = [u64, u64, i32, ctypes.POINTER(u64 * 3)]
            L.orc_num_candidates.restype = u64
            L.orc_num_candidates.argtypes = [u64, u64, ctypes.POINTER(u64)]
            L.orc_default_threads.restype = i32
            L.orc_default_threads.argtypes = []
            _lib = L
    return _lib


def isqrt(n: int) -> int:
    return int(lib().orc_isqrt(n))


def is_squarefree(n: int) -> bool:
    return bool(lib().orc_is_squarefree(n))


def is_prime(n: int) -> bool:
    return bool(lib().orc_is_prime(n))


def classify_range_primes(lo: int, hi: int, nthreads: int = 0, thetas: bool = False):
    """Per-candidate codes over the primes == 5 (mod 8) of [lo, hi): 0 (not
    prime), 1 (prime not in E), 2 (prime in E); optionally theta codes."""
    n, d0 = num_candidates(lo, hi)
    codes = np.zeros(n, dtype=np.uint8)
    th = np.zeros(n, dtype=np.uint8) if thetas else None
    rc = lib().orc_classify_range_primes(lo, hi, nthreads, codes.ctypes.data if n else None,
                                         th.ctypes.data if (th is not None and n) else None)
    if rc != ORC_OK:
        raise RuntimeError("orc_classify_range_primes(%d, %d) failed with %d" % (lo, hi, rc))
    out = {"d0": d0, "codes": codes}
    if th is not None:
        out["thetas"] = th
    return out


def count_range_primes(lo: int, hi: int, nthreads: int = 0):
    """(#primes == 5 mod 8, #(E cap P), rho steps) over [lo, hi)."""
    out = (ctypes.c_uint64 * 3)()
    rc = lib().orc_count_range_primes(lo, hi, nthreads, ctypes.byref(out))
    if rc != ORC_OK:
        raise RuntimeError("orc_count_range_primes(%d, %d) failed with %d" % (lo, hi, rc))
    return int(out[0]), int(out[1]), int(out[2])


def in_D(d: int) -> bool:
    return bool(lib().orc_in_D(d))


def walk_mod2(d: int):
    """(rc, theta, period): theta = x + 2y for eps_d = x + y*omega mod 2O_K."""
    th = ctypes.c_int(0)
    per = ctypes.c_uint64(0)
    rc = lib().orc_walk_mod2(d, ctypes.byref(th), ctypes.byref(per))
    return rc, th.value, per.value


def unit_exact(d: int) -> dict:
    u = _Unit()
    rc = lib().orc_unit_exact(d, ctypes.byref(u))
    if rc != ORC_OK:
        raise ValueError("orc_unit_exact(%d) failed with %d" % (d, rc))
    return {"period": u.period, "norm": u.norm, "flag": bool(u.flag), "theta": u.theta,
            "x0": u.x0_lo if u.x0_fits else None, "y0": u.y0_lo if u.y0_fits else None,
            "y0_parity": u.y0_lo & 1, "y0_bits": u.y0_bits}


def pell_smallest(d: int, ymax: int):
    """Smallest y <= ymax with x^2 - d y^2 = +-4 -> (y, x, sign) or None."""
    x = ctypes.c_uint64(0)
    sg = ctypes.c_int(0)
    y = lib().orc_pell_smallest(d, ymax, ctypes.byref(x), ctypes.byref(sg))
    if y == 0:
        return None
    return int(y), int(x.value), int(sg.value)


def narrow_classno(D: int) -> int:
    h = int(lib().orc_narrow_classno(D))
    if h < 0:
        raise ValueError("orc_narrow_classno(%d) failed" % D)
    return h


def num_candidates(lo: int, hi: int):
    d0 = ctypes.c_uint64(0)
    n = lib().orc_num_candidates(lo, hi, ctypes.byref(d0))
    return int(n), int(d0.value)


def default_threads() -> int:
    return int(lib().orc_default_threads())


def classify_range(lo: int, hi: int, nthreads: int = 0, periods: bool = False,
                   thetas: bool = False):
    """Per-candidate uint8 codes (0 not in D, 1 in D \\ E, 2 in E) for
    d = d0 + 8k in [lo, hi); optionally the periods (uint32) and theta codes."""
    n, d0 = num_candidates(lo, hi)
    codes = np.zeros(n, dtype=np.uint8)
    per = np.zeros(n, dtype=np.uint32) if periods else None
    th = np.zeros(n, dtype=np.uint8) if thetas else None
    rc = lib().orc_classify_range(
        lo, hi, nthreads, codes.ctypes.data if n else None,
        per.ctypes.data if (per is not None and n) else None,
        th.ctypes.data if (th is not None and n) else None)
    if rc != ORC_OK:
        raise RuntimeError("orc_classify_range(%d, %d) failed with %d" % (lo, hi, rc))
    out = {"d0": d0, "codes": codes}
    if per is not None:
        out["periods"] = per
    if th is not None:
        out["thetas"] = th
    return out


def sqfree_range(lo: int, hi: int, nthreads: int = 0, flags: bool = True):
    """(per-candidate uint8 1/0 membership in D or None, #D) over [lo, hi)."""
    n, _ = num_candidates(lo, hi)
    arr = np.zeros(n, dtype=np.uint8) if flags else None
    cnt = ctypes.c_uint64(0)
    rc = lib().orc_sqfree_range(lo, hi, nthreads,
                                arr.ctypes.data if (arr is not None and n) else None,
                                ctypes.byref(cnt))
    if rc != ORC_OK:
        raise RuntimeError("orc_sqfree_range(%d, %d) failed with %d" % (lo, hi, rc))
    return arr, int(cnt.value)


def count_range(lo: int, hi: int, nthreads: int = 0):
    """(#D, #E, total rho steps) over [lo, hi) by Oracle-B."""
    out = (ctypes.c_uint64 * 3)()
    rc = lib().orc_count_range(lo, hi, nthreads, ctypes.byref(out))
    if rc != ORC_OK:
        raise RuntimeError("orc_count_range(%d, %d) failed with %d" % (lo, hi, rc))
    return int(out[0]), int(out[1]), int(out[2])
