"""The oracle's pins are sensitive: each plausible mistake planted in a copy of
the oracle's C source (a dropped term, a wrong neighbour index, a border off by
one, a string end treated as a partner) fails at least one pin.

The mutants are compiled into a temporary directory on the CPU; the committed
oracle is never modified.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from test_oracle import all_strings, greedy_repair
from conftest import read_golden
import workloads

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "utf16_oracle.c")

MUTANTS = {
    "high_range_off_by_one": ("u >= 0xD800 && u <= 0xDBFF", "u >= 0xD800 && u < 0xDBFF"),
    "low_range_starts_late": ("u >= 0xDC00 && u <= 0xDFFF", "u >= 0xDC01 && u <= 0xDFFF"),
    "low_check_dropped": ("    if (is_low(in[i])) {\n", "    if (0 && is_low(in[i])) {\n"),
    "high_looks_left": ("(i + 1 < n) && is_low(in[i + 1])", "(i > 0) && is_low(in[i - 1])"),
    "low_looks_right": ("(i > 0) && is_high(in[i - 1])", "(i + 1 < n) && is_high(in[i + 1])"),
    "string_end_pairs": ("(i + 1 < n) && is_low(in[i + 1])", "(i + 1 >= n) || is_low(in[i + 1])"),
    "string_start_pairs": ("(i > 0) && is_high(in[i - 1])", "(i == 0) || is_high(in[i - 1])"),
    "wrong_replacement": ("? 0xFFFD : in[i]", "? 0xFFFE : in[i]"),
    "first_bad_off_by_one": ("if (oracle_unit_is_bad(in, n, i)) return i;\n    return n;",
                             "if (oracle_unit_is_bad(in, n, i)) return i + 1;\n    return n;"),
    "batch_ignores_boundaries": ("oracle_to_well_formed(in + a, b - a, out + a);",
                                 "oracle_to_well_formed_range(in + offsets[0], offsets[count] - offsets[0], "
                                 "a - offsets[0], b - offsets[0], out + offsets[0]);"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, name
    mutated = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    c.write_text(mutated)
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-o", str(so), str(c)])
    lib = ctypes.CDLL(str(so))
    u16p = ctypes.POINTER(ctypes.c_uint16)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_to_well_formed_batch.argtypes = [u16p, i64p, ctypes.c_int64, u16p]
    lib.oracle_first_bad_batch.argtypes = [u16p, i64p, ctypes.c_int64, i64p]
    lib.oracle_to_well_formed.argtypes = [u16p, ctypes.c_int64, u16p]
    return lib


def _pins_pass(lib):
    strings = list(all_strings(4))
    lens = np.array([len(s) for s in strings], dtype=np.int64)
    offs = workloads.offsets_from_lengths(lens)
    units = np.array([u for s in strings for u in s], dtype=np.uint16)
    out = units.copy()
    fb = np.empty(len(strings), dtype=np.int64)
    p16 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))
    p64 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    lib.oracle_to_well_formed_batch(p16(units), p64(offs), len(strings), p16(out))
    lib.oracle_first_bad_batch(p16(units), p64(offs), len(strings), p64(fb))
    for k, s in enumerate(strings):
        want = greedy_repair(s)
        if out[offs[k]:offs[k + 1]].tolist() != want:
            return False
        ch = [i for i in range(len(s)) if want[i] != s[i]]
        if fb[k] != (ch[0] if ch else len(s)):
            return False
    rows = read_golden("fig3_worked_example.txt")
    inp = np.array([int(r[1], 16) for r in rows[:31]], dtype=np.uint16)
    o = np.empty_like(inp)
    lib.oracle_to_well_formed(p16(inp), 31, p16(o))
    return o.tolist() == [int(r[8], 16) for r in rows[:31]]


def test_unmutated_source_passes(tmp_path):
    lib = _build_mutant(tmp_path, "identity", "0xFFFD", "0xFFFD")
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    assert not _pins_pass(lib), f"pin suite did not catch mutant {name}"
