"""CPU oracle for UTF-16 toWellFormed / isWellFormed -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never imports it and never falls back to it.

The arithmetic is in ``utf16_oracle.c`` (plain scalar C, the definition of
Section 1 of the paper with the string-end rule of Section 3.1); this module
only compiles it with gcc and marshals numpy arrays.  ``*_threads`` helpers
run the same scalar function over disjoint index ranges on several threads:
the rule reads only in[i-1], in[i] and in[i+1] of the whole string, so the
ranges give exactly the single-thread result.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "utf16_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile utf16_oracle.c into liboracle.so (gcc -O2, no vector flags)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u16p = ctypes.POINTER(ctypes.c_uint16)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64 = ctypes.c_int64
        lib.oracle_unit_is_bad.argtypes = [u16p, i64, i64]
        lib.oracle_unit_is_bad.restype = ctypes.c_int
        lib.oracle_to_well_formed_range.argtypes = [u16p, i64, i64, i64, u16p]
        lib.oracle_to_well_formed.argtypes = [u16p, i64, u16p]
        lib.oracle_first_bad.argtypes = [u16p, i64]
        lib.oracle_first_bad.restype = i64
        lib.oracle_first_bad_range.argtypes = [u16p, i64, i64, i64]
        lib.oracle_first_bad_range.restype = i64
        lib.oracle_to_well_formed_batch.argtypes = [u16p, i64p, i64, u16p]
        lib.oracle_first_bad_batch.argtypes = [u16p, i64p, i64, i64p]
        lib.oracle_illseq.argtypes = [u16p, i64, u8p]
        lib.oracle_code_point.argtypes = [ctypes.c_uint16, ctypes.c_uint16]
        lib.oracle_code_point.restype = ctypes.c_uint32
        _lib = lib
    return _lib


def _u16(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint16)
    return a


def _ptr16(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))


def _ptr64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def to_well_formed(units) -> np.ndarray:
    """Repaired copy of ``units`` (Section 1 rule, string ends as outside)."""
    a = _u16(units)
    out = np.empty_like(a)
    _load().oracle_to_well_formed(_ptr16(a), a.size, _ptr16(out))
    return out


def first_bad(units) -> int:
    """Index of the first unit that repair replaces, or len(units)."""
    a = _u16(units)
    return int(_load().oracle_first_bad(_ptr16(a), a.size))


def is_well_formed(units) -> bool:
    a = _u16(units)
    return first_bad(a) == a.size


def unit_is_bad(units, i: int) -> bool:
    a = _u16(units)
    return bool(_load().oracle_unit_is_bad(_ptr16(a), a.size, i))


def to_well_formed_batch(units, offsets) -> np.ndarray:
    """Per-string repair; units outside [offsets[0], offsets[-1]) are copied."""
    a = _u16(units)
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    out = a.copy()
    _load().oracle_to_well_formed_batch(_ptr16(a), _ptr64(offs), offs.size - 1, _ptr16(out))
    return out


def first_bad_batch(units, offsets) -> np.ndarray:
    a = _u16(units)
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    fb = np.empty(offs.size - 1, dtype=np.int64)
    _load().oracle_first_bad_batch(_ptr16(a), _ptr64(offs), offs.size - 1, _ptr64(fb))
    return fb


def illseq(units) -> np.ndarray:
    """Section 3.1 step-two flags isHigh(in[i-1]) XOR isLow(in[i])."""
    a = _u16(units)
    flags = np.empty(a.size, dtype=np.uint8)
    _load().oracle_illseq(_ptr16(a), a.size, flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return flags


def code_point(h: int, l: int) -> int:
    return int(_load().oracle_code_point(h, l))


def _ranges(n: int, parts: int):
    step = -(-n // parts) if n else 0
    return [(lo, min(n, lo + step)) for lo in range(0, n, step)] if n else []


def to_well_formed_threads(units: np.ndarray, out: np.ndarray | None = None, threads: int | None = None):
    """Same result as ``to_well_formed``; disjoint ranges on ``threads`` threads."""
    a = _u16(units)
    if out is None:
        out = np.empty_like(a)
    threads = threads or os.cpu_count() or 1
    lib = _load()
    pa, po = _ptr16(a), _ptr16(out)

    def run(r):
        lib.oracle_to_well_formed_range(pa, a.size, r[0], r[1], po)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, _ranges(a.size, threads)))
    return out


def first_bad_threads(units: np.ndarray, threads: int | None = None) -> int:
    a = _u16(units)
    threads = threads or os.cpu_count() or 1
    lib = _load()
    pa = _ptr16(a)
    rs = _ranges(a.size, threads)

    def run(r):
        return lib.oracle_first_bad_range(pa, a.size, r[0], r[1])

    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(run, rs))
    for (lo, hi), v in zip(rs, res):
        if v < hi:
            return int(v)
    return a.size
