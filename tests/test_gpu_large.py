"""Sizes beyond 2^31 units: 64-bit unit indices through the kernels, the
first-error reductions, the error list and the ragged-batch offsets search."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu

BIG = (1 << 31) + 4099  # 4 GiB and a ragged tail


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_06349_gb300 as p
    p.init_device()
    return p


def test_string_beyond_2_31_units(pkg):
    import torch
    u = workloads.mixed(BIG, 0.0, seed=4242)  # well formed (pairs, no lone surrogates)
    planted = [(1 << 31) + 5, (1 << 31) + 2001, BIG - 1]
    for p in planted:
        u[p - 1:p + 2] = 0x41
        u[p] = 0xDC00  # a low surrogate after ASCII
        if 0xD800 <= u[p - 2] <= 0xDBFF:  # its low was overwritten
            u[p - 2] = 0x42
        if p + 2 < u.size and 0xDC00 <= u[p + 2] <= 0xDFFF:
            u[p + 2] = 0x42
    want_fb = oracle.first_bad_threads(u)
    assert want_fb == planted[0]
    want = oracle.to_well_formed_threads(u)
    d_in = to_dev(u)
    d_out = torch.empty_like(d_in)
    _, fb = pkg.to_well_formed_first_bad(d_in, d_out)
    got = to_host(d_out)
    assert np.array_equal(got, want), first_diff(got, want)
    del got
    assert int(fb.item()) == want_fb
    assert pkg.first_error_index_sync(d_in) == want_fb
    pos, count = pkg.error_positions(d_in, capacity=16)
    assert count == len(planted)
    assert sorted(pos[:count].cpu().numpy().tolist()) == planted
    del d_out
    pkg.to_well_formed_(d_in)
    got = to_host(d_in)
    assert np.array_equal(got, want), first_diff(got, want)
    del d_in, got
    torch.cuda.empty_cache()


def test_batch_beyond_2_31_units(pkg):
    import torch
    rng = np.random.default_rng(31)
    lens = rng.integers(35_000_000, 40_000_000, 64).astype(np.int64)
    lens[[3, 17, 40]] = 0  # empty strings, one of them among the long ones
    lens = np.concatenate([lens, rng.integers(0, 300, 5000).astype(np.int64)])  # short strings after 2^31
    offs = workloads.offsets_from_lengths(lens, start=3)
    assert offs[-1] > (1 << 31)
    units = workloads.mixed(int(offs[-1]), 1e-6, seed=4343)
    # strings that start or end with a lone surrogate on both sides of 2^31
    for s in range(lens.size):
        if lens[s] > 2 and s % 7 == 0:
            units[offs[s]] = 0xDC00
        if lens[s] > 2 and s % 11 == 0:
            units[offs[s + 1] - 1] = 0xD800
    want = oracle.to_well_formed_batch(units, offs)
    want_fb = oracle.first_bad_batch(units, offs)
    d_u = to_dev(units)
    d_o = torch.from_numpy(offs).cuda()
    got = to_host(pkg.to_well_formed_batch(d_u, d_o))
    lo, hi = int(offs[0]), int(offs[-1])
    assert np.array_equal(got[lo:hi], want[lo:hi]), first_diff(got[lo:hi], want[lo:hi])
    del got
    fb = pkg.first_error_index_batch(d_u, d_o).cpu().numpy()
    assert np.array_equal(fb, want_fb), first_diff(fb, want_fb)
    assert pkg.check_offsets(d_o) == -1
    pkg.to_well_formed_batch_(d_u, d_o)
    got = to_host(d_u)
    assert np.array_equal(got[lo:hi], want[lo:hi])
    del d_u, got
    torch.cuda.empty_cache()
