"""Ragged-batch CUDA path against the per-string oracle, bit-exact, through
the C ABI: every string of length <= 5 over the border alphabet as one batch
(at several base misalignments and a nonzero first offset), the 1,000,000
string log-normal batch, and degenerate batches (all empty, one string, runs
of empty strings, strings longer than a chunk)."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import CANARY, Guarded, first_diff
from test_oracle import all_strings

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_06349_gb300 as p
    p.init_device()
    return p


def _run_all_forms(pkg, units, offs, a_in=0, a_out=0, label=""):
    """units: host array the offsets index; returns nothing, asserts parity."""
    import torch
    want = oracle.to_well_formed_batch(units, offs)
    want_fb = oracle.first_bad_batch(units, offs)
    lo, hi = int(offs[0]), int(offs[-1])
    d_off = torch.from_numpy(offs).cuda()
    gi = Guarded(units.size, a_in, units)
    # out of place: units outside [lo, hi) of `out` must stay untouched
    go = Guarded(units.size, a_out, np.full(units.size, CANARY, np.uint16))
    pkg.to_well_formed_batch(gi.view, d_off, go.view)
    got = go.get()
    assert np.array_equal(got[lo:hi], want[lo:hi]), (label, a_in, a_out, first_diff(got[lo:hi], want[lo:hi]))
    assert np.all(got[:lo] == CANARY) and np.all(got[hi:] == CANARY), label
    assert go.canaries_ok()
    # per-string first-error index
    fb = pkg.first_error_index_batch(gi.view, d_off)
    got_fb = fb.cpu().numpy()
    assert np.array_equal(got_fb, want_fb), (label, first_diff(got_fb, want_fb))
    assert np.array_equal(gi.get(), units)
    # in place
    gp = Guarded(units.size, a_in, units)
    pkg.to_well_formed_batch_(gp.view, d_off)
    got = gp.get()
    assert np.array_equal(got, want), (label, first_diff(got, want))
    assert gp.canaries_ok()


@pytest.fixture(scope="module")
def exhaustive_batch():
    strings = list(all_strings())
    lens = np.array([len(s) for s in strings], dtype=np.int64)
    units = np.array([u for s in strings for u in s], dtype=np.uint16)
    return units, lens


@pytest.mark.parametrize("a_in,a_out", [(0, 0), (3, 3), (1, 6), (7, 2), (5, 4)])
def test_exhaustive_alphabet_batch(pkg, exhaustive_batch, a_in, a_out):
    units, lens = exhaustive_batch
    offs = workloads.offsets_from_lengths(lens)
    _run_all_forms(pkg, units, offs, a_in, a_out, "exhaustive")


def test_exhaustive_batch_nonzero_start(pkg, exhaustive_batch):
    units, lens = exhaustive_batch
    pre = np.full(1001, 0xD800, np.uint16)  # outside the batch range: never read as neighbours
    post = np.full(999, 0xDC00, np.uint16)
    all_units = np.concatenate([pre, units, post])
    offs = workloads.offsets_from_lengths(lens, start=pre.size)
    _run_all_forms(pkg, all_units, offs, 2, 5, "exhaustive+start")


def test_lognormal_batch_million_strings(pkg):
    units, offs = workloads.ragged_batch()
    assert offs.size == 1_000_001
    _run_all_forms(pkg, units, offs, 0, 0, "ragged 1M")


def test_degenerate_batches(pkg):
    rng = np.random.default_rng(5)
    alph = np.array([0x41, 0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0xFFFD], np.uint16)
    cases = []
    # all empty
    cases.append((np.full(10, 0xD800, np.uint16), np.full(50, 4, np.int64)))
    # one string
    u = alph[rng.integers(0, alph.size, 70_001)]
    cases.append((u, np.array([0, u.size], np.int64)))
    # runs of empty strings between short ones, and long strings spanning chunks
    lens = []
    for _ in range(3000):
        r = rng.random()
        lens.append(0 if r < 0.4 else (int(rng.integers(1, 8)) if r < 0.8 else int(rng.integers(900, 5000))))
    lens = np.array(lens, np.int64)
    offs = workloads.offsets_from_lengths(lens, start=3)
    u = alph[rng.integers(0, alph.size, int(offs[-1]) + 5)]
    cases.append((u, offs))
    # every string length 1 (each surrogate is alone)
    u = alph[rng.integers(0, alph.size, 20_000)]
    cases.append((u, np.arange(u.size + 1, dtype=np.int64)))
    for k, (u, offs) in enumerate(cases):
        _run_all_forms(pkg, u, offs, k % 8, (3 * k) % 8, f"degenerate {k}")


def test_string_counts_around_the_lengths_pass(pkg):
    """The per-string results start from each string's length, which a small
    kernel writes four strings per thread, 1,024 per block, in one pass of up
    to four times the batch grid: counts around those sizes, and one just
    past a full pass (its grid-stride loop then runs twice), with tiny strings
    so that most strings share a chunk."""
    import torch
    rng = np.random.default_rng(17)
    alph = np.array([0x41, 0xD800, 0xDBFF, 0xDC00, 0xDFFF], np.uint16)
    # the default check grid is two 512-thread blocks per SM
    full_pass = 4 * 1024 * 2 * torch.cuda.get_device_properties(0).multi_processor_count
    for count in (1, 2, 3, 4, 5, 255, 256, 257, 1023, 1024, 1025, 4095, 4096, 4097, full_pass - 1, full_pass,
                  full_pass + 7):
        lens = rng.integers(0, 4, count).astype(np.int64)
        offs = workloads.offsets_from_lengths(lens, start=int(rng.integers(0, 9)))
        units = alph[rng.integers(0, alph.size, int(offs[-1]) + 3)]
        d_off = torch.from_numpy(offs).cuda()
        gi = Guarded(units.size, int(count % 8), units)
        got = pkg.first_error_index_batch(gi.view, d_off).cpu().numpy()
        want = oracle.first_bad_batch(units, offs)
        assert np.array_equal(got, want), (count, first_diff(got, want))
    pkg.check_device_errors()


def test_batch_boundary_pairs(pkg):
    # H | L across a string boundary stays unpaired; inside a string it pairs.
    u = np.array([0x41, 0xD800, 0xDC00, 0xD800, 0xDC00, 0x42] * 1000, np.uint16)
    lens = np.array([2, 1, 3] * 1000, np.int64)  # splits the first pair, keeps the second
    offs = workloads.offsets_from_lengths(lens)
    _run_all_forms(pkg, u, offs, 0, 0, "boundary pairs")


def test_check_offsets(pkg):
    """utf16_check_offsets reports the smallest index that breaks
    "offsets[0] >= 0, non-decreasing", or -1, for host and device results."""
    import ctypes
    import torch
    lens = workloads.lognormal_lengths(200_000, seed=71)
    good = workloads.offsets_from_lengths(lens.astype(np.int64), start=5)
    d = torch.from_numpy(good).cuda()
    assert pkg.check_offsets(d) == -1
    assert pkg.check_offsets(d[:1]) == -1  # no strings
    cases = {0: None, 1: None, 777: None, 123_456: None, good.size - 1: None}
    for i in cases:
        bad = good.copy()
        if i == 0:
            bad[0] = -1
        else:
            bad[i] = bad[i - 1] - 1
        assert pkg.check_offsets(torch.from_numpy(bad).cuda()) == i, i
    two = good.copy()
    two[500] = two[499] - 3
    two[90_000] = -7
    assert pkg.check_offsets(torch.from_numpy(two).cuda()) == 500
    res = torch.full((1,), 99, dtype=torch.int64, device="cuda")  # device result, stream ordered
    s = torch.cuda.current_stream()
    assert pkg.lib().utf16_check_offsets(torch.from_numpy(two).cuda().data_ptr(), two.size - 1, res.data_ptr(),
                                         ctypes.c_void_p(s.cuda_stream)) == 0
    assert int(res.item()) == 500
    # every entry point of the batch path keeps working after a check on the same stream
    units = workloads.mixed(int(good[-1]), 1e-2, seed=72)
    out = pkg.to_well_formed_batch(torch.from_numpy(units.view(np.int16)).cuda(), d)
    lo, hi = int(good[0]), int(good[-1])
    assert np.array_equal(out.cpu().numpy().view(np.uint16)[lo:hi], oracle.to_well_formed_batch(units, good)[lo:hi])


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")  # the refused call captures nothing
def test_checked_mode(pkg):
    """In checked mode every batch entry point rejects invalid offsets with
    UTF16_EINVAL before launching (buffers untouched), accepts valid ones,
    and refuses to run inside a stream capture."""
    import torch
    lens = workloads.lognormal_lengths(50_000, seed=73)
    good = workloads.offsets_from_lengths(lens.astype(np.int64), start=2)
    units = workloads.mixed(int(good[-1]) + 8, 1e-2, seed=74)
    want = oracle.to_well_formed_batch(units, good)
    want_fb = oracle.first_bad_batch(units, good)
    bad = good.copy()
    bad[1234] = bad[1233] - 1
    d_u = torch.from_numpy(units.view(np.int16)).cuda()
    d_good = torch.from_numpy(good).cuda()
    d_bad = torch.from_numpy(bad).cuda()
    was = pkg.get_checked()
    pkg.set_checked(True)
    try:
        out = torch.full_like(d_u, 0x1234)
        fb = torch.full((good.size - 1,), -5, dtype=torch.int64, device="cuda")
        buf = d_u.clone()
        for call in (lambda: pkg.to_well_formed_batch(d_u, d_bad, out),
                     lambda: pkg.to_well_formed_batch_(buf, d_bad),
                     lambda: pkg.first_error_index_batch(d_u, d_bad, fb)):
            with pytest.raises(pkg.Utf16Error) as e:
                call()
            assert e.value.code == pkg.EINVAL
        torch.cuda.synchronize()
        assert bool((out == 0x1234).all()) and bool((fb == -5).all()) and torch.equal(buf, d_u)
        lo, hi = int(good[0]), int(good[-1])
        pkg.to_well_formed_batch(d_u, d_good, out)
        assert np.array_equal(out.cpu().numpy().view(np.uint16)[lo:hi], want[lo:hi])
        pkg.first_error_index_batch(d_u, d_good, fb)
        assert np.array_equal(fb.cpu().numpy(), want_fb)
        pkg.to_well_formed_batch_(buf, d_good)
        assert np.array_equal(buf.cpu().numpy().view(np.uint16)[lo:hi], want[lo:hi])
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.graph(g, stream=s):
                rc = pkg.lib().utf16_to_well_formed_batch(d_u.data_ptr(), out.data_ptr(), d_good.data_ptr(),
                                                          good.size - 1, ctypes.c_void_p(s.cuda_stream))
        assert rc == pkg.EINVAL
    finally:
        pkg.set_checked(was)
    pkg.check_device_errors()
