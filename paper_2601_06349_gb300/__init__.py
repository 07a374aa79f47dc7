"""utf16wf on GB300: UTF-16 toWellFormed / isWellFormed as CUDA kernels.

Thin Python binding over the C ABI of ``libutf16wf.so`` (declared in
``include/utf16wf.h``).  Every step of repair and validation runs in the CUDA
kernels of that library; this module only marshals tensors (device memory
and streams come from PyTorch) and raises on error status codes.  There is no
CPU fallback: importing the functions without the built library raises.

Code units are 16-bit tensors (``torch.uint16`` or ``torch.int16``, the bit
pattern is what counts), contiguous, on a CUDA device.  Offsets of ragged
batches are ``torch.int64`` CUDA tensors with ``num_strings + 1`` entries.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libutf16wf.so")

OK, EINVAL, EOVERLAP, ECUDA, ETIMEOUT, ENOMEM, ECLOSED, EAGAIN = 0, -1, -2, -3, -4, -5, -6, -7

_lock = threading.Lock()
_lib = None


class Utf16Error(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


class Config(ctypes.Structure):
    """Launch configuration (utf16_config in include/utf16wf.h)."""
    _fields_ = [("single_variant", ctypes.c_int), ("single_units_per_thread", ctypes.c_int),
                ("single_blocks_per_sm", ctypes.c_int), ("batch_units_per_thread", ctypes.c_int),
                ("batch_prefetch", ctypes.c_int), ("batch_blocks_per_sm", ctypes.c_int),
                ("check_variant", ctypes.c_int), ("inplace_unit_stores", ctypes.c_int),
                ("inplace_variant", ctypes.c_int), ("check_blocks_per_sm", ctypes.c_int),
                ("inplace_blocks_per_sm", ctypes.c_int), ("batch_check_prefetch", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("vector_bytes", ctypes.c_int),
                ("repair_variant", ctypes.c_int), ("repair_units_per_thread", ctypes.c_int),
                ("repair_blocks_per_sm", ctypes.c_int), ("repair_block_threads", ctypes.c_int),
                ("check_block_threads", ctypes.c_int), ("inplace_block_threads", ctypes.c_int)]
    # Fields whose "not set" value is -1 (0 is a setting of its own).
    _UNSET = {"repair_variant": -1, "repair_blocks_per_sm": -1}

    def __init__(self, **fields):
        super().__init__(**{**self._UNSET, **fields})

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


VARIANT_LDG, VARIANT_LDG_PREFETCH, VARIANT_TMA = 0, 1, 2
ECANCELED = -9


class ServerOptions(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_batch_strings", ctypes.c_int64),
                ("max_batch_bytes", ctypes.c_int64), ("max_inflight_batches", ctypes.c_int),
                ("staging_bytes", ctypes.c_int64), ("small_request_bytes", ctypes.c_int64),
                ("inject_fail_mod", ctypes.c_int64), ("direct_host_access", ctypes.c_int),
                ("inject_copy_fail_mod", ctypes.c_int64), ("inject_copy_fail_step", ctypes.c_int)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("first_bad", ctypes.c_int64), ("n", ctypes.c_int64),
                ("arrival_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64), ("status", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("units", ctypes.c_int64), ("max_batch_requests", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("inflight_batches", ctypes.c_int64), ("arena_used_bytes", ctypes.c_int64)]


def _declare(lib):
    c_u16p = ctypes.c_void_p
    i64 = ctypes.c_int64
    vp = ctypes.c_void_p
    sig = {
        "utf16_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "utf16_to_well_formed": ([vp, vp, i64, vp], ctypes.c_int),
        "utf16_to_well_formed_inplace": ([vp, i64, vp], ctypes.c_int),
        "utf16_to_well_formed_first_bad": ([vp, vp, i64, vp, vp], ctypes.c_int),
        "utf16_is_well_formed": ([vp, i64, vp, vp], ctypes.c_int),
        "utf16_to_well_formed_batch": ([vp, vp, vp, i64, vp], ctypes.c_int),
        "utf16_to_well_formed_batch_inplace": ([vp, vp, i64, vp], ctypes.c_int),
        "utf16_is_well_formed_batch": ([vp, vp, i64, vp, vp], ctypes.c_int),
        "utf16_to_well_formed_host": ([c_u16p, c_u16p, i64, vp], ctypes.c_int),
        "utf16_init_device": ([], ctypes.c_int),
        "utf16_get_config": ([ctypes.POINTER(Config)], ctypes.c_int),
        "utf16_set_config": ([ctypes.POINTER(Config)], ctypes.c_int),
        "utf16_autotune_single": ([vp, vp, i64, ctypes.c_int, ctypes.POINTER(Config)], ctypes.c_int),
        "utf16_autotune_batch": ([vp, vp, vp, i64, ctypes.c_int, ctypes.POINTER(Config)], ctypes.c_int),
        "utf16_check_device_errors": ([], ctypes.c_int),
        "utf16_autotune": ([ctypes.c_int, vp, ctypes.c_int], ctypes.c_int),
        "utf16_get_tuned": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(Config)], ctypes.c_int),
        "utf16_set_tuned": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(Config)], ctypes.c_int),
        "utf16_error_positions": ([vp, i64, vp, i64, vp, vp], ctypes.c_int),
        "utf16_check_offsets": ([vp, i64, vp, vp], ctypes.c_int),
        "utf16_set_checked": ([ctypes.c_int], ctypes.c_int),
        "utf16_get_checked": ([], ctypes.c_int),
        "utf16_selftest_bounded_wait": ([i64], ctypes.c_int),
        "utf16_to_well_formed_first_bad_noalloc": ([vp, vp, i64, vp, vp], ctypes.c_int),
        "utf16_release_device": ([], ctypes.c_int),
        "utf16_server_default_options": ([ctypes.POINTER(ServerOptions)], ctypes.c_int),
        "utf16_server_create": ([ctypes.POINTER(ServerOptions), ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "utf16_server_clock_ns": ([], ctypes.c_int64),
        "utf16_server_submit": ([vp, vp, vp, i64, i64, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "utf16_server_cancel": ([vp, ctypes.c_uint64], ctypes.c_int),
        "utf16_server_next": ([vp, ctypes.POINTER(Completion), i64], ctypes.c_int),
        "utf16_server_stats_get": ([vp, ctypes.POINTER(ServerStats)], ctypes.c_int),
        "utf16_server_destroy": ([vp], ctypes.c_int),
        "utf16_server_replay": ([vp, vp, vp, vp, i64, ctypes.c_double, ctypes.c_uint64, vp, vp], ctypes.c_int),
        "utf16_plain_replay": ([vp, vp, vp, i64, ctypes.c_double, ctypes.c_uint64, vp, vp], ctypes.c_int),
        "utf16_plain_replay_streams": ([vp, vp, vp, i64, ctypes.c_double, ctypes.c_uint64, ctypes.c_int, vp, vp],
                                       ctypes.c_int),
        "utf16_arena_create": ([i64, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "utf16_arena_alloc": ([vp, i64], ctypes.c_int64),
        "utf16_arena_free_oldest": ([vp], ctypes.c_int),
        "utf16_arena_used": ([vp], ctypes.c_int64),
        "utf16_arena_destroy": ([vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def lib():
    """The loaded C library (ctypes).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise ImportError(f"{LIB_PATH} is missing: build it with "
                                      "`python -m paper_2601_06349_gb300.build` (needs nvcc)")
                _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def strerror(code: int) -> str:
    return lib().utf16_strerror(code).decode()


def _check(rc: int, where: str):
    if rc != OK:
        raise Utf16Error(rc, where)


# ---------------------------------------------------------------- tensors
def _torch():
    import torch
    return torch


def _units(t, name="units"):
    torch = _torch()
    if t.dtype not in (torch.uint16, torch.int16):
        raise TypeError(f"{name} must be torch.uint16 or torch.int16, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _stream(stream, device):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def to_well_formed(inp, out=None, *, stream=None):
    """Repaired copy of ``inp`` (or into ``out``; ``out`` may be ``inp``)."""
    torch = _torch()
    _units(inp, "inp")
    if out is None:
        out = torch.empty_like(inp)
    _units(out, "out")
    if out.numel() != inp.numel():
        raise ValueError("out must have as many units as inp")
    with torch.cuda.device(inp.device):
        _check(lib().utf16_to_well_formed(inp.data_ptr(), out.data_ptr(), inp.numel(),
                                          _stream(stream, inp.device)), "utf16_to_well_formed")
    return out


def to_well_formed_(buf, *, stream=None):
    """Repair ``buf`` in place (stores only 16-byte blocks that change)."""
    torch = _torch()
    _units(buf, "buf")
    with torch.cuda.device(buf.device):
        _check(lib().utf16_to_well_formed_inplace(buf.data_ptr(), buf.numel(), _stream(stream, buf.device)),
               "utf16_to_well_formed_inplace")
    return buf


def to_well_formed_first_bad(inp, out=None, first_bad=None, *, stream=None):
    """Repair and first-error index in one pass.  Returns (out, first_bad),
    ``first_bad`` a one-element int64 CUDA tensor written in stream order."""
    torch = _torch()
    _units(inp, "inp")
    if out is None:
        out = torch.empty_like(inp)
    _units(out, "out")
    if first_bad is None:
        first_bad = torch.empty(1, dtype=torch.int64, device=inp.device)
    with torch.cuda.device(inp.device):
        _check(lib().utf16_to_well_formed_first_bad(inp.data_ptr(), out.data_ptr(), inp.numel(),
                                                    first_bad.data_ptr(), _stream(stream, inp.device)),
               "utf16_to_well_formed_first_bad")
    return out, first_bad


def first_error_index(inp, first_bad=None, *, stream=None):
    """isWellFormed: one-element int64 CUDA tensor (asynchronous) holding the
    index of the first mismatched unit, or len(inp)."""
    torch = _torch()
    _units(inp, "inp")
    if first_bad is None:
        first_bad = torch.empty(1, dtype=torch.int64, device=inp.device)
    with torch.cuda.device(inp.device):
        _check(lib().utf16_is_well_formed(inp.data_ptr(), inp.numel(), first_bad.data_ptr(),
                                          _stream(stream, inp.device)), "utf16_is_well_formed")
    return first_bad


def first_error_index_sync(inp, *, stream=None) -> int:
    """isWellFormed with a host result (the call waits for the stream)."""
    torch = _torch()
    _units(inp, "inp")
    v = ctypes.c_int64(-1)
    with torch.cuda.device(inp.device):
        _check(lib().utf16_is_well_formed(inp.data_ptr(), inp.numel(), ctypes.addressof(v),
                                          _stream(stream, inp.device)), "utf16_is_well_formed")
    return v.value


def error_positions(inp, capacity=None, *, stream=None):
    """Indices of all mismatched units (unordered) as an int64 CUDA tensor of
    length min(count, capacity), and the total count (the call waits)."""
    torch = _torch()
    _units(inp, "inp")
    if capacity is None:
        capacity = inp.numel()
    pos = torch.empty(max(int(capacity), 1), dtype=torch.int64, device=inp.device)
    cnt = ctypes.c_int64(-1)
    with torch.cuda.device(inp.device):
        _check(lib().utf16_error_positions(inp.data_ptr(), inp.numel(), pos.data_ptr(), int(capacity),
                                           ctypes.addressof(cnt), _stream(stream, inp.device)),
               "utf16_error_positions")
    return pos[:min(cnt.value, int(capacity))], cnt.value


def is_well_formed(inp, *, stream=None) -> bool:
    return first_error_index_sync(inp, stream=stream) == inp.numel()


def _offsets(offsets):
    torch = _torch()
    if offsets.dtype != torch.int64 or not offsets.is_cuda or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous int64 CUDA tensor")
    return offsets


def to_well_formed_batch(units, offsets, out=None, *, stream=None):
    """Repair each string units[offsets[s]:offsets[s+1]] on its own."""
    torch = _torch()
    _units(units)
    _offsets(offsets)
    if out is None:
        out = units.clone()
    _units(out, "out")
    with torch.cuda.device(units.device):
        _check(lib().utf16_to_well_formed_batch(units.data_ptr(), out.data_ptr(), offsets.data_ptr(),
                                                offsets.numel() - 1, _stream(stream, units.device)),
               "utf16_to_well_formed_batch")
    return out


def to_well_formed_batch_(units, offsets, *, stream=None):
    torch = _torch()
    _units(units)
    _offsets(offsets)
    with torch.cuda.device(units.device):
        _check(lib().utf16_to_well_formed_batch_inplace(units.data_ptr(), offsets.data_ptr(), offsets.numel() - 1,
                                                        _stream(stream, units.device)),
               "utf16_to_well_formed_batch_inplace")
    return units


def first_error_index_batch(units, offsets, first_bad=None, *, stream=None):
    """Per-string first-error index relative to each string (its length when
    well formed), as an int64 CUDA tensor."""
    torch = _torch()
    _units(units)
    _offsets(offsets)
    count = offsets.numel() - 1
    if first_bad is None:
        first_bad = torch.empty(max(count, 0), dtype=torch.int64, device=units.device)
    with torch.cuda.device(units.device):
        _check(lib().utf16_is_well_formed_batch(units.data_ptr(), offsets.data_ptr(), count, first_bad.data_ptr(),
                                                _stream(stream, units.device)), "utf16_is_well_formed_batch")
    return first_bad


def check_offsets(offsets, *, stream=None) -> int:
    """Smallest index violating "offsets[0] >= 0 and non-decreasing" of a
    device int64 offsets tensor, or -1 when it is valid (waits for the
    stream)."""
    _offsets(offsets)
    out = ctypes.c_int64(0)
    with _torch().cuda.device(offsets.device):
        _check(lib().utf16_check_offsets(offsets.data_ptr(), offsets.numel() - 1, ctypes.byref(out),
                                         _stream(stream, offsets.device)), "utf16_check_offsets")
    return out.value


def set_checked(on: bool) -> None:
    """Checked mode: the batch calls validate their offsets first (one pass
    and a wait for the stream) and raise on invalid offsets."""
    _check(lib().utf16_set_checked(1 if on else 0), "utf16_set_checked")


def get_checked() -> bool:
    return lib().utf16_get_checked() != 0


def to_well_formed_host(host_in, host_out=None):
    """Repair a host (CPU) buffer through the device; returns (out, first_bad).
    ``host_in`` / ``host_out``: CPU tensors of 16-bit units or numpy uint16
    arrays.  Pinned buffers, and pageable ones on a device that reads pageable
    memory coherently (GB300 over NVLink-C2C), take one fused pass over the
    host link; other buffers a staged copy pipeline."""
    import numpy as np
    if host_out is None:
        if isinstance(host_in, np.ndarray):
            host_out = np.empty_like(host_in)
        else:
            host_out = _torch().empty_like(host_in, pin_memory=host_in.is_pinned())
    pin, n = _host_ptr(host_in)
    pout, n_out = _host_ptr(host_out)
    if n_out != n:
        raise ValueError("host_in and host_out lengths differ")
    fb = ctypes.c_int64(-1)
    _check(lib().utf16_to_well_formed_host(ctypes.c_void_p(pin), ctypes.c_void_p(pout), n, ctypes.addressof(fb)),
           "utf16_to_well_formed_host")
    return host_out, fb.value


def init_device():
    _check(lib().utf16_init_device(), "utf16_init_device")


def release_device():
    _check(lib().utf16_release_device(), "utf16_release_device")


def get_config() -> Config:
    c = Config()
    _check(lib().utf16_get_config(ctypes.byref(c)), "utf16_get_config")
    return c


def set_config(cfg: Config | None = None, **fields) -> Config:
    """Set the current device's default launch configuration (clears tuned
    entries).  Fields not given keep their current value."""
    c = get_config() if cfg is None else cfg
    for k, v in fields.items():
        setattr(c, k, int(v))
    _check(lib().utf16_set_config(ctypes.byref(c)), "utf16_set_config")
    return c


def autotune_single(inp, out=None, reps: int = 5) -> Config:
    """Time every configuration on this string (out-of-place repair with the
    first-error index) and keep the fastest for its size bucket."""
    torch = _torch()
    _units(inp, "inp")
    if out is None:
        out = torch.empty_like(inp)
    best = Config()
    with torch.cuda.device(inp.device):
        _check(lib().utf16_autotune_single(inp.data_ptr(), out.data_ptr(), inp.numel(), reps, ctypes.byref(best)),
               "utf16_autotune_single")
    return best


def autotune_batch(units, offsets, out=None, reps: int = 5) -> Config:
    """Time every batch configuration on this batch and keep the fastest for
    its bucket of string count."""
    torch = _torch()
    _units(units)
    _offsets(offsets)
    if out is None:
        out = torch.empty_like(units)
    best = Config()
    with torch.cuda.device(units.device):
        _check(lib().utf16_autotune_batch(units.data_ptr(), out.data_ptr(), offsets.data_ptr(), offsets.numel() - 1,
                                          reps, ctypes.byref(best)), "utf16_autotune_batch")
    return best


def check_device_errors():
    """Raise if a kernel gave up a bounded wait since the last check."""
    _check(lib().utf16_check_device_errors(), "utf16_check_device_errors")


# ------------------------------------------------------------------ serving
def _host_ptr(buf):
    """(address, units) of a host buffer: numpy uint16 array or CPU tensor."""
    import numpy as np
    if isinstance(buf, np.ndarray):
        if buf.dtype != np.uint16 or not buf.flags.c_contiguous:
            raise TypeError("host buffers must be contiguous uint16 arrays")
        return buf.ctypes.data, buf.size
    torch = _torch()
    if buf.is_cuda or buf.dtype not in (torch.uint16, torch.int16):
        raise TypeError("host buffers must be CPU tensors of 16-bit units")
    return buf.data_ptr(), buf.numel()


class Server:
    """Continuous-batching repair engine on the current device (see
    utf16_server_* in include/utf16wf.h).  Host buffers given to submit() are
    kept referenced here until their completion has been returned by next()."""

    def __init__(self, **options):
        o = ServerOptions()
        _check(lib().utf16_server_default_options(ctypes.byref(o)), "utf16_server_default_options")
        for k, v in options.items():
            setattr(o, k, int(v))
        h = ctypes.c_void_p()
        _check(lib().utf16_server_create(ctypes.byref(o), ctypes.byref(h)), "utf16_server_create")
        self._h = h
        self._refs = {}
        self.options = o

    def submit(self, host_in, host_out, arrival_ns: int = 0) -> int:
        pin, n = _host_ptr(host_in)
        pout, n2 = _host_ptr(host_out)
        if n2 != n:
            raise ValueError("host_out must have as many units as host_in")
        t = ctypes.c_uint64()
        _check(lib().utf16_server_submit(self._h, pin, pout, n, arrival_ns, ctypes.byref(t)), "utf16_server_submit")
        self._refs[t.value] = (host_in, host_out)
        return t.value

    def cancel(self, ticket: int) -> bool:
        rc = lib().utf16_server_cancel(self._h, ticket)
        if rc not in (OK, EAGAIN):
            _check(rc, "utf16_server_cancel")
        return rc == OK

    def next(self, timeout_us: int = -1):
        c = Completion()
        rc = lib().utf16_server_next(self._h, ctypes.byref(c), timeout_us)
        if rc in (EAGAIN, ETIMEOUT):
            return None
        _check(rc, "utf16_server_next")
        self._refs.pop(c.ticket, None)
        return {"ticket": c.ticket, "first_bad": c.first_bad, "n": c.n, "status": c.status,
                "latency_s": (c.done_ns - c.arrival_ns) * 1e-9}

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().utf16_server_stats_get(self._h, ctypes.byref(st)), "utf16_server_stats_get")
        return {name: getattr(st, name) for name, _ in st._fields_}

    def replay(self, inputs, outputs, rate_per_s: float, seed: int = 1):
        """Poisson replay of the requests through this server; returns
        (latencies in s, first_bad or negative status) as numpy arrays."""
        return _replay(self._h, inputs, outputs, rate_per_s, seed)

    def close(self):
        if self._h:
            _check(lib().utf16_server_destroy(self._h), "utf16_server_destroy")
            self._h = None
            self._refs.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def clock_ns() -> int:
    return lib().utf16_server_clock_ns()


def _replay(handle, inputs, outputs, rate_per_s, seed, streams=0):
    import numpy as np
    count = len(inputs)
    ins = (ctypes.c_void_p * count)()
    outs = (ctypes.c_void_p * count)()
    lens = np.empty(count, dtype=np.int64)
    for i, (a, b) in enumerate(zip(inputs, outputs)):
        pa, na = _host_ptr(a)
        pb, nb = _host_ptr(b)
        if na != nb:
            raise ValueError("input and output lengths differ")
        ins[i], outs[i], lens[i] = pa, pb, na
    lat = np.zeros(count, dtype=np.float64)
    fb = np.zeros(count, dtype=np.int64)
    if handle is None and streams:
        rc = lib().utf16_plain_replay_streams(ins, outs, lens.ctypes.data, count, float(rate_per_s), seed,
                                              int(streams), lat.ctypes.data, fb.ctypes.data)
    elif handle is None:
        rc = lib().utf16_plain_replay(ins, outs, lens.ctypes.data, count, float(rate_per_s), seed,
                                      lat.ctypes.data, fb.ctypes.data)
    else:
        rc = lib().utf16_server_replay(handle, ins, outs, lens.ctypes.data, count, float(rate_per_s), seed,
                                       lat.ctypes.data, fb.ctypes.data)
    _check(rc, "replay")
    return lat, fb


def plain_replay(inputs, outputs, rate_per_s: float, seed: int = 1, streams: int = 0):
    """The same replay with one plain launch per request (H2D, fused kernel,
    D2H, wait), in arrival order: one request at a time (streams = 0), or
    pipelined over `streams` host threads with a stream each."""
    return _replay(None, inputs, outputs, rate_per_s, seed, streams)


class Arena:
    """The serving engine's FIFO ring allocator (host-side offsets only)."""

    def __init__(self, capacity: int):
        h = ctypes.c_void_p()
        _check(lib().utf16_arena_create(capacity, ctypes.byref(h)), "utf16_arena_create")
        self._h = h

    def alloc(self, size: int) -> int:
        return lib().utf16_arena_alloc(self._h, size)

    def free_oldest(self) -> bool:
        return lib().utf16_arena_free_oldest(self._h) == OK

    def used(self) -> int:
        return lib().utf16_arena_used(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().utf16_arena_destroy(self._h)
            self._h = None


def autotune_histogram(op: str, length_histogram) -> None:
    """Tune from a histogram of lengths (bucket b = lengths in [2^b, 2^(b+1)))
    on synthetic text: op "single" (one string per non-empty bucket) or
    "batch" (one batch with the histogram's mix of string lengths)."""
    import numpy as np
    h = np.ascontiguousarray(np.asarray(length_histogram, dtype=np.int64))
    code = {"single": 0, "batch": 1}[op]
    _check(lib().utf16_autotune(code, h.ctypes.data, h.size), "utf16_autotune")


def save_tuning(path: str) -> dict:
    """Write the current device's tuned entries to a JSON file keyed by GPU
    name; returns what was written."""
    import json
    torch = _torch()
    name = torch.cuda.get_device_name()
    entries = {}
    for op, key in ((0, "single"), (1, "batch")):
        for bucket in range(64):
            c = Config()
            if lib().utf16_get_tuned(op, bucket, ctypes.byref(c)) == OK:
                entries.setdefault(key, {})[str(bucket)] = c.as_dict()
    data = {}
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[name] = entries
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    return entries


def load_tuning(path: str) -> int:
    """Restore tuned entries saved for this GPU name; returns how many."""
    import json
    torch = _torch()
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return 0
    entries = data.get(torch.cuda.get_device_name(), {})
    count = 0
    for op, key in ((0, "single"), (1, "batch")):
        for bucket, fields in entries.get(key, {}).items():
            c = Config(**{k: int(v) for k, v in fields.items() if k in dict(Config._fields_)})
            _check(lib().utf16_set_tuned(op, int(bucket), ctypes.byref(c)), "utf16_set_tuned")
            count += 1
    return count
