"""Seeded synthetic UTF-16 workloads shared by the tests and the benchmark.

The arithmetic of repair and validation lives neither here nor in the C file
beside this module: both only draw input strings.  The CUDA path and the CPU
oracle are both fed from what these functions return.

Workload shapes (all seeded, all in native-order uint16 code units):

* ``mixed(n, lone_rate)``: per position 70% ASCII, 20% BMP non-surrogate,
  8% valid pair (scaled by 1 - lone_rate), lone surrogates at ``lone_rate``,
  half high and half low.  The 1 MiB string uses lone_rate 0.02 (the 70/20/8/2
  mix); the 1 GiB string uses 0, 1e-6 and 1e-2.
* ``uniform_surrogates(n)``, ``shifted_alternating(n)``, ``all_high(n)``: the
  three adversarial 512 MiB strings.
* ``ragged_batch(count)``: log-normal lengths (mu = ln 32, sigma = 1.5)
  clipped to [0, 65536], content mixed at 1% lone rate, 10% of non-empty
  strings forced to start with a low or end with a high surrogate.
* ``request_lengths(count)``: serving request lengths, 80% U[16,256],
  19% U[1024,65536], 1% U[1048576,16777216].
* ``paper_mix(n, pair_rate, lone_rate)``: the paper's Section 4 generator
  shape (pairs among characters, lone surrogates among the other units,
  ASCII otherwise).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libworkloads.so")
_lock = threading.Lock()
_lib = None

SEED_BASE = 0x260106349

SMALL_MIXED_UNITS = 524_288          # 1 MiB string
LARGE_MIXED_UNITS = 536_870_912      # 1 GiB string
ADVERSARIAL_UNITS = 268_435_456      # 512 MiB strings
RAGGED_STRINGS = 1_000_000
SHIFT_PERIOD = 4093


def build(force: bool = False) -> str:
    """Compile gen.c into libworkloads.so next to it (gcc, plain C)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u16p = ctypes.POINTER(ctypes.c_uint16)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.wl_fill_mix.argtypes = [u16p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double]
        lib.wl_fill_paper.argtypes = [u16p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_double]
        lib.wl_fill_uniform_surrogates.argtypes = [u16p, ctypes.c_int64, ctypes.c_uint64]
        lib.wl_fill_shifted_alternating.argtypes = [u16p, ctypes.c_int64, ctypes.c_int64]
        lib.wl_lognormal_lengths.argtypes = [i64p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int64]
        lib.wl_lognormal_lengths.restype = ctypes.c_int64
        lib.wl_request_lengths.argtypes = [i64p, ctypes.c_int64, ctypes.c_uint64]
        lib.wl_request_lengths.restype = ctypes.c_int64
        lib.wl_fill_ragged.argtypes = [u16p, i64p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                       ctypes.c_double]
        _lib = lib
    return _lib


def _u16p(a: np.ndarray):
    assert a.dtype == np.uint16 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))


def _i64p(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def empty_units(n: int, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        return np.empty(n, dtype=np.uint16)
    assert out.dtype == np.uint16 and out.size >= n
    return out[:n]


def mixed(n: int, lone_rate: float, seed: int = SEED_BASE, out: np.ndarray | None = None) -> np.ndarray:
    a = empty_units(n, out)
    _load().wl_fill_mix(_u16p(a), n, seed, float(lone_rate))
    return a


def paper_mix(n: int, pair_rate: float, lone_rate: float, seed: int = SEED_BASE,
              out: np.ndarray | None = None) -> np.ndarray:
    a = empty_units(n, out)
    _load().wl_fill_paper(_u16p(a), n, seed, float(pair_rate), float(lone_rate))
    return a


def uniform_surrogates(n: int, seed: int = SEED_BASE + 2, out: np.ndarray | None = None) -> np.ndarray:
    a = empty_units(n, out)
    _load().wl_fill_uniform_surrogates(_u16p(a), n, seed)
    return a


def shifted_alternating(n: int, period: int = SHIFT_PERIOD, out: np.ndarray | None = None) -> np.ndarray:
    a = empty_units(n, out)
    _load().wl_fill_shifted_alternating(_u16p(a), n, period)
    return a


def all_high(n: int, out: np.ndarray | None = None) -> np.ndarray:
    a = empty_units(n, out)
    a.fill(0xDBFF)
    return a


def lognormal_lengths(count: int, seed: int, mu: float = math.log(32.0), sigma: float = 1.5,
                      clip: int = 65536) -> np.ndarray:
    lens = np.empty(count, dtype=np.int64)
    _load().wl_lognormal_lengths(_i64p(lens), count, seed, mu, sigma, clip)
    return lens


def request_lengths(count: int, seed: int = SEED_BASE + 4) -> np.ndarray:
    lens = np.empty(count, dtype=np.int64)
    _load().wl_request_lengths(_i64p(lens), count, seed)
    return lens


def offsets_from_lengths(lens: np.ndarray, start: int = 0) -> np.ndarray:
    offs = np.empty(lens.size + 1, dtype=np.int64)
    offs[0] = start
    np.cumsum(lens, out=offs[1:])
    offs[1:] += start
    return offs


def fill_ragged(units: np.ndarray, offsets: np.ndarray, seed: int, lone_rate: float,
                forced: float) -> np.ndarray:
    count = offsets.size - 1
    assert units.size >= offsets[-1]
    _load().wl_fill_ragged(_u16p(units), _i64p(offsets), count, seed, float(lone_rate), float(forced))
    return units


def ragged_batch(count: int = RAGGED_STRINGS, seed: int = SEED_BASE + 3, lone_rate: float = 0.01,
                 forced: float = 0.10, clip: int = 65536):
    """Returns (units, offsets) for a ragged batch of ``count`` strings."""
    lens = lognormal_lengths(count, seed, clip=clip)
    offs = offsets_from_lengths(lens)
    units = np.zeros(int(offs[-1]), dtype=np.uint16)
    fill_ragged(units, offs, seed ^ 0x5EED, lone_rate, forced)
    return units, offs


# Named workloads, by what they are.
def small_mixed():
    """1 MiB string, 70/20/8/2 mix (out-of-place repair plus first-error index)."""
    return mixed(SMALL_MIXED_UNITS, 0.02, seed=SEED_BASE + 0)


def large_mixed(lone_rate: float, out: np.ndarray | None = None):
    """1 GiB string, mix at the given lone-surrogate rate."""
    return mixed(LARGE_MIXED_UNITS, lone_rate, seed=SEED_BASE + 1, out=out)


def adversarial(kind: str, n: int = ADVERSARIAL_UNITS, out: np.ndarray | None = None):
    """512 MiB adversarial strings: 'uniform', 'shifted' or 'all_high'."""
    if kind == "uniform":
        return uniform_surrogates(n, out=out)
    if kind == "shifted":
        return shifted_alternating(n, out=out)
    if kind == "all_high":
        return all_high(n, out=out)
    raise ValueError(kind)
