"""The seeded workload generators: deterministic, exact lengths, and the
distribution shapes the measured workloads are defined by."""
import math

import numpy as np

import workloads


def _classes(u):
    hi = (u >= 0xD800) & (u <= 0xDBFF)
    lo = (u >= 0xDC00) & (u <= 0xDFFF)
    ascii_ = (u >= 0x20) & (u <= 0x7E)
    return hi, lo, ascii_


def test_mixed_is_deterministic():
    a = workloads.mixed(100_000, 0.02, seed=5)
    b = workloads.mixed(100_000, 0.02, seed=5)
    c = workloads.mixed(100_000, 0.02, seed=6)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_mixed_shape():
    u = workloads.mixed(2_000_000, 0.02, seed=11)
    hi, lo, ascii_ = _classes(u)
    # per drawn character: 70% ascii, 20% bmp, 8% pair (2 units), 2% lone
    chars = 2_000_000 / 1.08
    assert abs(ascii_.sum() / chars - 0.70) < 0.01
    assert abs(hi.sum() / chars - (0.08 + 0.01)) < 0.005
    assert abs(lo.sum() / chars - (0.08 + 0.01)) < 0.005
    assert np.all((u >= 0x20))


def test_error_free_mix_has_only_pairs():
    u = workloads.mixed(1_000_000, 0.0, seed=3)
    hi, lo, _ = _classes(u)
    idx = np.nonzero(hi)[0]
    assert np.all(lo[idx + 1])
    assert hi.sum() == lo.sum()


def test_adversarial_shapes():
    u = workloads.adversarial("uniform", n=100_000)
    assert np.all((u >= 0xD800) & (u <= 0xDFFF))
    s = workloads.adversarial("shifted", n=10_000)
    assert s[0] == 0xD800 and s[1] == 0xDC00 and s[4092] == 0xD800 and s[4093] == 0xD800
    assert np.all(workloads.adversarial("all_high", n=100) == 0xDBFF)


def test_ragged_lengths_shape():
    lens = workloads.lognormal_lengths(1_000_000, seed=workloads.SEED_BASE + 3)
    assert lens.min() >= 0 and lens.max() <= 65536
    assert abs(float(np.median(lens)) - 32) <= 1
    assert 0.005 < np.mean(lens == 0) < 0.02
    mean_expected = math.exp(math.log(32) + 1.5 ** 2 / 2)
    assert abs(lens.mean() / mean_expected - 1) < 0.05


def test_ragged_batch_forced_boundaries():
    units, offs = workloads.ragged_batch(count=20_000, seed=77)
    assert offs[0] == 0 and offs[-1] == units.size and np.all(np.diff(offs) >= 0)
    starts_low = 0
    ends_high = 0
    nonempty = 0
    for s in range(20_000):
        a, b = offs[s], offs[s + 1]
        if b > a:
            nonempty += 1
            starts_low += 0xDC00 <= units[a] <= 0xDFFF
            ends_high += 0xD800 <= units[b - 1] <= 0xDBFF
    # 5% forced each way, plus the mix's own chance (~1-5%)
    assert 0.05 < starts_low / nonempty < 0.09
    assert 0.05 < ends_high / nonempty < 0.11


def test_request_lengths_shape():
    lens = workloads.request_lengths(200_000)
    small = (lens >= 16) & (lens <= 256)
    mid = (lens >= 1024) & (lens <= 65536)
    big = (lens >= 1 << 20) & (lens <= 1 << 24)
    assert np.all(small | mid | big)
    assert abs(small.mean() - 0.80) < 0.01
    assert abs(mid.mean() - 0.19) < 0.01
    assert abs(big.mean() - 0.01) < 0.002
