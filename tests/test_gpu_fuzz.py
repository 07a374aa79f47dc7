"""Seeded fuzzing of every entry point against the oracle: random lengths
(0 .. 200,000 units), random input and output misalignment (0..7 units),
content from several distributions (border alphabet, mixed text at random
lone rates, surrogate-only runs, long runs of one value), and random ragged
batches with empty strings and strings that cross many chunks."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import Guarded, first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu

BORDER = np.array([0x0000, 0x0041, 0x00E9, 0xD7FF, 0xD800, 0xD83D, 0xDBFF, 0xDC00, 0xDE0A, 0xDFFF, 0xE000,
                   0xFFFD, 0xFFFF], np.uint16)


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_06349_gb300 as p
    p.init_device()
    return p


def _random_string(rng, n):
    kind = rng.integers(0, 5)
    if kind == 0:
        return BORDER[rng.integers(0, BORDER.size, n)]
    if kind == 1:
        return workloads.mixed(n, float(rng.choice([0.0, 1e-4, 1e-2, 0.2])), seed=int(rng.integers(1 << 40)))
    if kind == 2:
        return (0xD800 + rng.integers(0, 2048, n)).astype(np.uint16)
    if kind == 3:  # long runs of one value with sparse surrogates
        u = np.full(n, rng.choice([0x41, 0xD800, 0xDC00]), np.uint16)
        k = rng.integers(0, max(1, n // 100) + 1)
        u[rng.integers(0, max(n, 1), k)] = BORDER[rng.integers(0, BORDER.size, k)]
        return u
    u = workloads.mixed(n, 0.01, seed=int(rng.integers(1 << 40)))  # pairs straddling every position
    return u


def _length(rng):
    r = rng.random()
    if r < 0.3:
        return int(rng.integers(0, 64))
    if r < 0.7:
        return int(rng.integers(64, 20_000))
    return int(rng.integers(20_000, 200_000))


@pytest.mark.parametrize("seed", range(4))
def test_fuzz_single_string(pkg, seed):
    rng = np.random.default_rng(1000 + seed)
    for it in range(60):
        n = _length(rng)
        u = _random_string(rng, n)
        want = oracle.to_well_formed(u)
        want_fb = oracle.first_bad(u)
        a_in, a_out = int(rng.integers(0, 8)), int(rng.integers(0, 8))
        gi = Guarded(max(n, 1), a_in, u if n else np.zeros(1, np.uint16))
        go = Guarded(max(n, 1), a_out)
        vi, vo = gi.view[:n], go.view[:n]
        op = it % 5
        if op == 0:
            _, fb = pkg.to_well_formed_first_bad(vi, vo)
            assert np.array_equal(to_host(vo), want), (seed, it, n, a_in, a_out, first_diff(to_host(vo), want))
            assert int(fb.item()) == want_fb
        elif op == 1:
            pkg.to_well_formed(vi, vo)
            assert np.array_equal(to_host(vo), want), (seed, it, n)
        elif op == 2:
            pkg.to_well_formed_(vi)
            assert np.array_equal(to_host(vi), want), (seed, it, n)
        elif op == 3:
            assert pkg.first_error_index_sync(vi) == want_fb, (seed, it, n)
            assert int(pkg.first_error_index(vi).item()) == want_fb
        else:
            pos, count = pkg.error_positions(vi, capacity=max(n, 1))
            wpos = np.nonzero(want != u)[0]
            assert count == wpos.size and np.array_equal(np.sort(pos.cpu().numpy()), wpos), (seed, it, n)
        assert gi.canaries_ok() and go.canaries_ok(), (seed, it)


@pytest.mark.parametrize("seed", range(4))
def test_fuzz_ragged_batches(pkg, seed):
    import torch
    rng = np.random.default_rng(2000 + seed)
    for it in range(12):
        count = int(rng.integers(1, 3000))
        lens = np.where(rng.random(count) < 0.2, 0,
                        np.where(rng.random(count) < 0.9, rng.integers(1, 300, count), rng.integers(300, 20_000, count)))
        start = int(rng.integers(0, 50))
        offs = workloads.offsets_from_lengths(lens.astype(np.int64), start=start)
        total = int(offs[-1]) + int(rng.integers(0, 50))
        units = _random_string(rng, total)
        want = oracle.to_well_formed_batch(units, offs)
        want_fb = oracle.first_bad_batch(units, offs)
        a = int(rng.integers(0, 8))
        gi = Guarded(units.size, a, units)
        d_off = torch.from_numpy(offs).cuda()
        out = pkg.to_well_formed_batch(gi.view, d_off)
        got = to_host(out)
        lo, hi = int(offs[0]), int(offs[-1])
        assert np.array_equal(got[lo:hi], want[lo:hi]), (seed, it, first_diff(got[lo:hi], want[lo:hi]))
        fb = pkg.first_error_index_batch(gi.view, d_off).cpu().numpy()
        assert np.array_equal(fb, want_fb), (seed, it, first_diff(fb, want_fb))
        pkg.to_well_formed_batch_(gi.view, d_off)
        assert np.array_equal(gi.get(), want), (seed, it)
        assert gi.canaries_ok()


@pytest.mark.parametrize("seed", range(3))
def test_fuzz_ragged_launch_shapes(pkg, seed):
    """Random ragged batches under a random launch shape each: chunk width,
    block size, lane load width, next chunk in flight and blocks per SM, with
    the input and a separate output misaligned at random (every store class).
    Units of the output outside [offsets[0], offsets[count]) keep their
    canary value, as the entry points promise."""
    import torch
    from gpu_util import CANARY
    rng = np.random.default_rng(3000 + seed)
    saved = pkg.get_config()
    try:
        for it in range(40):
            cfg = dict(batch_units_per_thread=int(rng.choice([2, 4])), block_threads=int(rng.choice([128, 256, 512])),
                       vector_bytes=int(rng.choice([8, 16, 32])), batch_prefetch=int(rng.integers(0, 2)),
                       batch_check_prefetch=int(rng.integers(0, 2)), batch_blocks_per_sm=int(rng.integers(0, 3)))
            pkg.set_config(**cfg)
            count = int(rng.integers(1, 4000))
            r = rng.random(count)
            lens = np.where(r < 0.25, 0, np.where(r < 0.85, rng.integers(1, 120, count),
                                                  rng.integers(120, 9000, count)))
            start = int(rng.integers(0, 40))
            offs = workloads.offsets_from_lengths(lens.astype(np.int64), start=start)
            total = int(offs[-1]) + int(rng.integers(0, 40))
            units = _random_string(rng, total)
            want = oracle.to_well_formed_batch(units, offs)
            want_fb = oracle.first_bad_batch(units, offs)
            lo, hi = int(offs[0]), int(offs[-1])
            a_in, a_out = int(rng.integers(0, 16)), int(rng.integers(0, 16))
            gi = Guarded(max(total, 1), a_in, units if total else np.zeros(1, np.uint16))
            go = Guarded(max(total, 1), a_out)
            vi, vo = gi.view[:total], go.view[:total]
            d_off = torch.from_numpy(offs).cuda()
            pkg.to_well_formed_batch(vi, d_off, vo)
            got = to_host(vo)
            tag = (seed, it, cfg, a_in, a_out, count, total)
            assert np.array_equal(got[lo:hi], want[lo:hi]), (tag, first_diff(got[lo:hi], want[lo:hi]))
            assert np.all(got[:lo] == CANARY) and np.all(got[hi:] == CANARY), tag
            fb = pkg.first_error_index_batch(vi, d_off).cpu().numpy()
            assert np.array_equal(fb, want_fb), (tag, first_diff(fb, want_fb))
            pkg.to_well_formed_batch_(vi, d_off)
            assert np.array_equal(to_host(vi), want), tag
            assert gi.canaries_ok() and go.canaries_ok(), tag
    finally:
        pkg.set_config(saved)
    pkg.check_device_errors()


@pytest.mark.parametrize("seed", range(3))
def test_fuzz_single_launch_shapes(pkg, seed):
    """Random single strings under a random launch shape each: data path of
    the fused repair, the plain repair, the check and in-place repair (128-bit
    loads, next chunk in flight, TMA), units per thread, unit stores in place,
    block size and blocks per SM, at random input and output misalignment."""
    rng = np.random.default_rng(4000 + seed)
    saved = pkg.get_config()
    try:
        for it in range(80):
            cfg = dict(single_variant=int(rng.integers(0, 3)), check_variant=int(rng.integers(0, 3)),
                       inplace_variant=int(rng.integers(0, 3)), single_units_per_thread=int(rng.choice([0, 2, 4])),
                       inplace_unit_stores=int(rng.integers(0, 2)), block_threads=int(rng.choice([0, 128, 256, 512])),
                       single_blocks_per_sm=int(rng.integers(0, 4)), check_blocks_per_sm=int(rng.integers(0, 4)),
                       inplace_blocks_per_sm=int(rng.integers(0, 4)), repair_variant=int(rng.integers(-1, 3)),
                       repair_units_per_thread=int(rng.choice([0, 2, 4])), repair_blocks_per_sm=int(rng.integers(-1, 3)),
                       repair_block_threads=int(rng.choice([0, 128, 256, 512])),
                       check_block_threads=int(rng.choice([0, 128, 256, 512])),
                       inplace_block_threads=int(rng.choice([0, 128, 256, 512])))
            pkg.set_config(**cfg)
            n = _length(rng)
            u = _random_string(rng, n)
            want = oracle.to_well_formed(u)
            want_fb = oracle.first_bad(u)
            a_in, a_out = int(rng.integers(0, 8)), int(rng.integers(0, 8))
            gi = Guarded(max(n, 1), a_in, u if n else np.zeros(1, np.uint16))
            go = Guarded(max(n, 1), a_out)
            vi, vo = gi.view[:n], go.view[:n]
            tag = (seed, it, cfg, n, a_in, a_out)
            pkg.to_well_formed(vi, vo)
            assert np.array_equal(to_host(vo), want), (tag, "plain", first_diff(to_host(vo), want))
            _, fb = pkg.to_well_formed_first_bad(vi, vo)
            assert np.array_equal(to_host(vo), want), (tag, first_diff(to_host(vo), want))
            assert int(fb.item()) == want_fb, tag
            assert int(pkg.first_error_index(vi).item()) == want_fb, tag
            pkg.to_well_formed_(vi)
            assert np.array_equal(to_host(vi), want), tag
            assert gi.canaries_ok() and go.canaries_ok(), tag
    finally:
        pkg.set_config(saved)
    pkg.check_device_errors()
