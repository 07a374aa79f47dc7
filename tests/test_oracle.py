"""Pins for the CPU oracle against facts that do not come from the oracle.

* brute force: every string of length 0..5 over a 10-symbol alphabet that
  straddles every class border, against an independent left-to-right greedy
  matcher (a sequential scan, not the oracle's local rule);
* the worked example of Fig. 3 (output column and the illseq column of the
  Section 3.1 second step), from tests/golden;
* the Section 1 code-point formula on the paper's example pair;
* closed forms of the adversarial strings and of the error-free mix;
* invariants: well-formed output, idempotence, length, untouched
  non-surrogates, FFFD only where a surrogate was, kept pairs decode into the
  supplementary planes, and the neighbour-verdict stability that makes the
  in-place GPU form race-free.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads
from conftest import read_golden

ALPHABET = [0x0041, 0x00E9, 0xD7FF, 0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0xE000, 0xFFFD, 0xFFFF]


def greedy_repair(s):
    """Sequential scan: keep a high+low pair and step over both; replace any
    other surrogate; keep everything else."""
    out = []
    i = 0
    while i < len(s):
        u = s[i]
        if 0xD800 <= u <= 0xDBFF and i + 1 < len(s) and 0xDC00 <= s[i + 1] <= 0xDFFF:
            out.append(u)
            out.append(s[i + 1])
            i += 2
        elif 0xD800 <= u <= 0xDFFF:
            out.append(0xFFFD)
            i += 1
        else:
            out.append(u)
            i += 1
    return out


def all_strings(max_len=5):
    for k in range(max_len + 1):
        for t in itertools.product(ALPHABET, repeat=k):
            yield list(t)


@pytest.fixture(scope="module")
def exhaustive():
    strings = list(all_strings())
    lens = np.array([len(s) for s in strings], dtype=np.int64)
    offs = workloads.offsets_from_lengths(lens)
    units = np.array([u for s in strings for u in s], dtype=np.uint16)
    return strings, units, offs


def test_exhaustive_count(exhaustive):
    strings, units, offs = exhaustive
    assert len(strings) == sum(10 ** k for k in range(6)) == 111_111
    assert units.size == sum(k * 10 ** k for k in range(6))


def test_exhaustive_batch_against_greedy(exhaustive):
    strings, units, offs = exhaustive
    out = oracle.to_well_formed_batch(units, offs)
    fb = oracle.first_bad_batch(units, offs)
    for s_idx, s in enumerate(strings):
        a, b = offs[s_idx], offs[s_idx + 1]
        want = greedy_repair(s)
        got = out[a:b].tolist()
        assert got == want, (s, got, want)
        changed = [i for i in range(len(s)) if want[i] != s[i]]
        assert fb[s_idx] == (changed[0] if changed else len(s)), s


def test_exhaustive_single_string_matches_batch(exhaustive):
    strings, units, offs = exhaustive
    out = oracle.to_well_formed_batch(units, offs)
    fb = oracle.first_bad_batch(units, offs)
    for s_idx in range(0, len(strings), 7):
        a, b = offs[s_idx], offs[s_idx + 1]
        s = units[a:b]
        assert np.array_equal(oracle.to_well_formed(s), out[a:b])
        assert oracle.first_bad(s) == fb[s_idx]


def test_batch_neighbours_are_outside():
    # A high surrogate that ends one string stays unpaired even when the next
    # string starts with a low surrogate.
    units = np.array([0xD800, 0xDC00], dtype=np.uint16)
    assert oracle.to_well_formed(units).tolist() == [0xD800, 0xDC00]
    offs = np.array([0, 1, 2], dtype=np.int64)
    assert oracle.to_well_formed_batch(units, offs).tolist() == [0xFFFD, 0xFFFD]
    assert oracle.first_bad_batch(units, offs).tolist() == [0, 0]
    # empty strings between them change nothing
    offs = np.array([0, 1, 1, 1, 2], dtype=np.int64)
    assert oracle.first_bad_batch(units, offs).tolist() == [0, 0, 0, 0]


def test_fig3_worked_example():
    rows = read_golden("fig3_worked_example.txt")
    assert len(rows) == 32
    inp = np.array([int(r[1], 16) for r in rows], dtype=np.uint16)
    lookback = [int(r[2], 16) for r in rows]
    illseq_col = [int(r[7]) for r in rows]
    out_col = np.array([int(r[8], 16) for r in rows], dtype=np.uint16)
    string = inp[:31]  # row 31 is the U+0000 that follows the string
    assert inp[31] == 0
    assert lookback == [0] + inp[:31].tolist()
    got = oracle.to_well_formed(string)
    assert got.tolist() == out_col[:31].tolist()
    assert np.nonzero(got != string)[0].tolist() == [10, 21]
    assert oracle.first_bad(string) == 10
    assert not oracle.is_well_formed(string)
    # Section 3.1 step two over the string and its trailing U+0000
    assert oracle.illseq(inp).tolist() == illseq_col
    # Section 3.1 step three locates the units: a high surrogate flagged one
    # unit later, a low surrogate flagged at itself.
    fl = illseq_col
    is_h = [0xD800 <= u <= 0xDBFF for u in inp.tolist()]
    is_l = [0xDC00 <= u <= 0xDFFF for u in inp.tolist()]
    located = [i for i in range(31) if (is_h[i] and fl[i + 1]) or (is_l[i] and fl[i])]
    assert located == [10, 21]


def test_code_point_examples():
    for h, l, cp in read_golden("code_point_example.txt"):
        assert oracle.code_point(int(h, 16), int(l, 16)) == int(cp, 16)


def _check_invariants(units):
    out = oracle.to_well_formed(units)
    n = units.size
    assert out.size == n
    assert oracle.first_bad(out) == n
    assert np.array_equal(oracle.to_well_formed(out), out)
    surr = (units >= 0xD800) & (units <= 0xDFFF)
    assert np.array_equal(out[~surr], units[~surr])
    changed = out != units
    assert np.all(out[changed] == 0xFFFD)
    assert np.all(surr[changed])
    # kept surrogates come in (high, low) pairs that decode into the
    # supplementary planes
    kept = np.nonzero(surr & ~changed)[0]
    highs = kept[(units[kept] >= 0xD800) & (units[kept] <= 0xDBFF)]
    lows = kept[(units[kept] >= 0xDC00)]
    assert highs.size == lows.size
    assert np.array_equal(highs + 1, lows)
    for h_idx in highs[:2000]:
        cp = oracle.code_point(int(units[h_idx]), int(units[h_idx + 1]))
        assert 0x10000 <= cp <= 0x10FFFF
    fb = oracle.first_bad(units)
    ch = np.nonzero(changed)[0]
    assert fb == (int(ch[0]) if ch.size else n)
    return out


@pytest.mark.parametrize("lone_rate", [0.0, 1e-3, 0.02, 0.3])
def test_invariants_mixed(lone_rate):
    units = workloads.mixed(200_003, lone_rate, seed=1234)
    out = _check_invariants(units)
    if lone_rate == 0.0:
        assert np.array_equal(out, units)


def test_invariants_adversarial():
    for kind in ("uniform", "shifted", "all_high"):
        _check_invariants(workloads.adversarial(kind, n=100_001))


def test_all_high_closed_form():
    units = workloads.all_high(10_000)
    out = oracle.to_well_formed(units)
    assert np.all(out == 0xFFFD)
    assert oracle.first_bad(units) == 0


@pytest.mark.parametrize("n", [4093 * 64 + 144, 268_435_456])
def test_shifted_alternating_closed_form(n):
    # Units (i + floor(i/4093)) odd are 0xDC00, else 0xD800: each 4093-unit
    # period is H L ... H (odd length) and the next starts with H, so exactly
    # the last unit of every complete period, 4093k + 4092, is replaced.
    units = workloads.shifted_alternating(n)
    out = oracle.to_well_formed(units)
    bad = np.nonzero(out != units)[0]
    k = n // 4093
    assert bad.size == k
    assert np.array_equal(bad, 4093 * np.arange(k, dtype=np.int64) + 4092)
    assert oracle.first_bad(units) == 4092
    if n == 268_435_456:
        assert bad.size == 65_584


def test_uniform_surrogates_half_bad():
    # A uniform surrogate is high or low with probability 1/2 each; a high is
    # bad when its right neighbour is not low (1/2), a low when its left
    # neighbour is not high (1/2): the bad share is 1/2.
    units = workloads.uniform_surrogates(1_000_000, seed=99)
    frac = float(np.mean(oracle.to_well_formed(units) != units))
    assert abs(frac - 0.5) < 0.005


def test_neighbour_verdict_stability(exhaustive):
    """Replacing one bad unit by FFFD leaves every other unit's verdict alone:
    a replaced high had a non-low right neighbour, a replaced low a non-high
    left neighbour, and FFFD is neither."""
    strings, units, offs = exhaustive
    out = oracle.to_well_formed_batch(units, offs)
    mod_units, mod_lens, orig_flags, which = [], [], [], []
    for s_idx, s in enumerate(strings):
        a, b = offs[s_idx], offs[s_idx + 1]
        flags = (out[a:b] != units[a:b])
        for i in np.nonzero(flags)[0]:
            t = list(s)
            t[i] = 0xFFFD
            mod_units.extend(t)
            mod_lens.append(len(t))
            orig_flags.append(flags)
            which.append(i)
    mu = np.array(mod_units, dtype=np.uint16)
    mo = workloads.offsets_from_lengths(np.array(mod_lens, dtype=np.int64))
    mout = oracle.to_well_formed_batch(mu, mo)
    assert len(which) > 100_000
    for j, i in enumerate(which):
        a, b = mo[j], mo[j + 1]
        f = (mout[a:b] != mu[a:b])
        expect = orig_flags[j].copy()
        expect[i] = False  # the replaced unit itself is now FFFD
        assert np.array_equal(f, expect)


def test_threaded_helpers_match():
    units = workloads.mixed(1_000_003, 0.01, seed=7)
    ref = oracle.to_well_formed(units)
    for t in (1, 3, 8):
        assert np.array_equal(oracle.to_well_formed_threads(units, threads=t), ref)
        assert oracle.first_bad_threads(units, threads=t) == oracle.first_bad(units)
    clean = workloads.mixed(500_000, 0.0, seed=8)
    assert oracle.first_bad_threads(clean, threads=4) == clean.size


def test_empty_and_tiny():
    assert oracle.to_well_formed(np.zeros(0, np.uint16)).size == 0
    assert oracle.first_bad(np.zeros(0, np.uint16)) == 0
    assert oracle.to_well_formed([0xDC00]).tolist() == [0xFFFD]
    assert oracle.to_well_formed([0xD800]).tolist() == [0xFFFD]
    assert oracle.to_well_formed([0xD800, 0xDC00]).tolist() == [0xD800, 0xDC00]
    assert oracle.to_well_formed([0xDC00, 0xD800]).tolist() == [0xFFFD, 0xFFFD]
