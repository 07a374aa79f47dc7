"""Every launch configuration gives the oracle's result, bit-exact: the
single-string kernel with 128-bit loads (with and without next-chunk
prefetch, 2 or 4 vectors per thread), the TMA-staged kernel, reduced grids,
and the batch kernel with 2 or 4 vectors per thread, with and without
prefetch.  Also the autotuner's choice, and that no kernel gave up a bounded
wait."""
import itertools

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import Guarded, first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu

# (data path, chunk width, blocks per SM, threads per block)
SINGLE = [(0, 4, 0, 0), (0, 2, 0, 0), (1, 4, 0, 0), (1, 2, 0, 0), (2, 4, 0, 0), (2, 4, 1, 0), (0, 4, 1, 0),
          (1, 2, 2, 0), (0, 4, 0, 128), (1, 4, 0, 512), (0, 2, 0, 512), (1, 2, 3, 128), (2, 4, 0, 512)]
BATCH = [(0, 0, 0), (4, 0, 0), (2, 0, 0), (4, 1, 0), (2, 1, 0), (4, 0, 1)]


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_06349_gb300 as p
    p.init_device()
    saved = p.get_config()
    yield p
    p.set_config(saved)


@pytest.fixture(scope="module")
def strings():
    big = workloads.mixed(40_000_123, 1e-2, seed=31)
    shifted = workloads.shifted_alternating(20_000_003)
    clean = workloads.mixed(30_000_001, 0.0, seed=32)
    return {"mixed": (big, oracle.to_well_formed_threads(big), oracle.first_bad(big)),
            "shifted": (shifted, oracle.to_well_formed_threads(shifted), oracle.first_bad(shifted)),
            "clean": (clean, clean, clean.size)}


@pytest.mark.parametrize("variant,u,bps,bt", SINGLE)
def test_single_configurations(pkg, strings, variant, u, bps, bt):
    import torch
    # the plain repair (no first-error index) on its own settings: this shape,
    # with the fused form on another data path
    pkg.set_config(single_variant=(variant + 1) % 3, single_units_per_thread=u, single_blocks_per_sm=bps,
                   check_variant=variant, inplace_variant=variant, block_threads=bt, repair_variant=variant,
                   repair_units_per_thread=u, repair_blocks_per_sm=bps)
    for name, (src, want, want_fb) in strings.items():
        for a_in, a_out in ((0, 0), (3, 3), (5, 1)):
            gi = Guarded(src.size, a_in, src)
            go = Guarded(src.size, a_out)
            pkg.to_well_formed(gi.view, go.view)
            got = go.get()
            assert np.array_equal(got, want), (name, variant, u, a_in, a_out, "plain", first_diff(got, want))
            assert go.canaries_ok()
    pkg.set_config(single_variant=variant, single_units_per_thread=u, single_blocks_per_sm=bps,
                   check_variant=variant, inplace_variant=variant, block_threads=bt, repair_variant=-1,
                   repair_units_per_thread=0, repair_blocks_per_sm=-1)
    for name, (src, want, want_fb) in strings.items():
        for a_in, a_out in ((0, 0), (3, 3), (5, 1)):
            gi = Guarded(src.size, a_in, src)
            go = Guarded(src.size, a_out)
            _, fb = pkg.to_well_formed_first_bad(gi.view, go.view)
            got = go.get()
            assert np.array_equal(got, want), (name, variant, u, a_in, a_out, first_diff(got, want))
            assert int(fb.item()) == want_fb, (name, variant, u)
            assert go.canaries_ok()
            assert pkg.first_error_index_sync(gi.view) == want_fb, (name, variant, u)
            pkg.to_well_formed_(gi.view)
            assert np.array_equal(gi.get(), want), (name, variant, u, "in place")
            assert gi.canaries_ok()
    # small strings around the tile edges of the TMA kernel (8192 units)
    rng = np.random.default_rng(variant * 10 + u)
    alph = np.array([0x41, 0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0xFFFD], np.uint16)
    for n in (1, 7, 8, 9, 8191, 8192, 8193, 16383, 16384, 16385, 16400, 24583, 40961):
        uu = alph[rng.integers(0, alph.size, n)]
        want = oracle.to_well_formed(uu)
        for a in (0, 1, 7):
            gi = Guarded(n, a, uu)
            go = Guarded(n, a)
            _, fb = pkg.to_well_formed_first_bad(gi.view, go.view)
            assert np.array_equal(go.get(), want), (n, a, variant, u)
            assert int(fb.item()) == oracle.first_bad(uu)
            assert pkg.first_error_index_sync(gi.view) == oracle.first_bad(uu)
    torch.cuda.synchronize()
    pkg.check_device_errors()


@pytest.mark.parametrize("u,pf,bps", BATCH)
def test_batch_configurations(pkg, u, pf, bps):
    pkg.set_config(batch_units_per_thread=u, batch_prefetch=pf, batch_blocks_per_sm=bps, batch_check_prefetch=pf)
    from test_gpu_batch import _run_all_forms
    units, offs = workloads.ragged_batch(count=200_000, seed=77)
    _run_all_forms(pkg, units, offs, 0, 0, f"batch u={u} pf={pf}")
    _run_all_forms(pkg, units, offs, 3, 6, f"batch u={u} pf={pf} misaligned")
    pkg.check_device_errors()


@pytest.mark.parametrize("bt", [128, 256, 512])
@pytest.mark.parametrize("vb", [8, 16, 32])
def test_batch_block_and_vector_widths(pkg, bt, vb):
    """Every batch form at both chunk widths with 128-, 256- or 512-thread
    blocks and 8-, 16- or 32-byte lane loads, aligned and misaligned (store
    classes 2 to 32), on a log-normal batch and one of tiny strings."""
    from test_gpu_batch import _run_all_forms
    units, offs = workloads.ragged_batch(count=60_000, seed=78)
    rng = np.random.default_rng(vb * 1000 + bt)
    tiny = np.where(rng.random(40_000) < 0.3, 0, rng.integers(1, 6, 40_000)).astype(np.int64)
    t_offs = workloads.offsets_from_lengths(tiny, start=3)
    t_units = np.array([0x41, 0xD800, 0xDBFF, 0xDC00, 0xDFFF], np.uint16)[rng.integers(0, 5, int(t_offs[-1]) + 8)]
    for u in (2, 4):
        pkg.set_config(batch_units_per_thread=u, batch_prefetch=0, batch_blocks_per_sm=0, batch_check_prefetch=0,
                       block_threads=bt, vector_bytes=vb)
        for a_in, a_out in ((0, 0), (3, 6), (5, 13), (8, 0)):
            _run_all_forms(pkg, units, offs, a_in, a_out, f"bt={bt} vb={vb} u={u}")
        _run_all_forms(pkg, t_units, t_offs, 1, 1, f"tiny bt={bt} vb={vb} u={u}")
    pkg.set_config(block_threads=0, vector_bytes=0)
    pkg.check_device_errors()


@pytest.mark.parametrize("u,pf,bps", BATCH)
def test_batch_split_pairs_at_every_start_position(pkg, u, pf, bps):
    """Pairs cut by string starts at every position of a chunk, its slices
    and vectors: a text of high-low pairs (a few units replaced by ASCII or
    lone surrogates) split into strings of 0-4 units, then into a mix with
    strings longer than a chunk.  A start at an odd position splits a pair."""
    pkg.set_config(batch_units_per_thread=u, batch_prefetch=pf, batch_blocks_per_sm=bps, batch_check_prefetch=pf)
    from test_gpu_batch import _run_all_forms
    rng = np.random.default_rng(1000 + 10 * u + pf)
    n = 300_000
    units = np.tile(np.array([0xD800, 0xDC00], np.uint16), n // 2)
    noise = rng.random(n) < 0.02
    units[noise] = rng.choice(np.array([0x41, 0xD800, 0xDBFF, 0xDC00, 0xDFFF], np.uint16), int(noise.sum()))
    short = rng.integers(0, 5, n)
    mixed = np.where(rng.random(n) < 0.3, rng.integers(200, 1500, n), rng.integers(0, 5, n))
    for label, lens in (("short", short), ("mixed", mixed)):
        total = np.cumsum(lens)
        lens = lens[: int(np.searchsorted(total, n - 8))]
        offs = workloads.offsets_from_lengths(lens.astype(np.int64), start=1)
        for a_in, a_out in ((0, 0), (3, 5), (7, 1)):
            _run_all_forms(pkg, units, offs, a_in, a_out, f"split pairs {label} u={u} pf={pf}")
    pkg.check_device_errors()


@pytest.mark.parametrize("u,pf,bps", BATCH)
def test_batch_window_straddles_chunk_end(pkg, u, pf, bps):
    """The per-string check reads windows of 32 offsets.  With strings of
    q = chunk/32 units and one of 2q per chunk, a chunk holds more than 31
    starts, its first window ends just before the chunk's end and the next
    window starts just after it: the string holding the next chunk's first
    unit is the last of the earlier window.  A lone low surrogate 6 units into
    every chunk lies in that string."""
    pkg.set_config(batch_units_per_thread=u, batch_prefetch=pf, batch_blocks_per_sm=bps, batch_check_prefetch=pf)
    from test_gpu_batch import _run_all_forms
    cu = 256 * u
    q = cu // 32
    chunks = 40_000  # several chunks per warp of the persistent grid, so prefetched windows are used
    lens = np.array([q] * 31 + [2 * q] + ([q] * 30 + [2 * q]) * (chunks - 1), np.int64)
    offs = workloads.offsets_from_lengths(lens)
    units = np.full(int(offs[-1]) + 8, 0x41, np.uint16)
    units[np.arange(1, chunks) * cu + 6] = 0xDC00
    units[np.arange(1, chunks, 7) * cu - 1] = 0xD800  # and some high surrogates cut by the chunk end
    _run_all_forms(pkg, units, offs, 0, 0, f"straddle u={u} pf={pf}")
    pkg.check_device_errors()


def test_config_fields_by_form_are_validated(pkg):
    """The settings of the plain repair and the per-form block sizes accept
    their documented values and reject others (nothing is changed then)."""
    saved = pkg.get_config()
    try:
        pkg.set_config(repair_variant=2, repair_units_per_thread=4, repair_blocks_per_sm=0, repair_block_threads=512,
                       check_block_threads=128, inplace_block_threads=256)
        for field, bad in (("repair_variant", 3), ("repair_variant", -2), ("repair_units_per_thread", 3),
                           ("repair_blocks_per_sm", -2), ("repair_block_threads", 64), ("check_block_threads", 1024),
                           ("inplace_block_threads", 300)):
            before = pkg.get_config().as_dict()
            with pytest.raises(pkg.Utf16Error):
                pkg.set_config(**{field: bad})
            assert pkg.get_config().as_dict() == before, field
    finally:
        pkg.set_config(saved)


def test_autotuner_choice_is_correct(pkg):
    import torch
    u = workloads.mixed(64 << 20, 1e-2, seed=51)
    d = to_dev(u)
    out = torch.empty_like(d)
    cfg = pkg.autotune_single(d, out, reps=3)
    assert cfg.single_variant in (0, 1, 2)
    assert cfg.repair_variant in (-1, 0, 1, 2) and cfg.repair_units_per_thread in (0, 2, 4)
    assert {cfg.repair_block_threads, cfg.check_block_threads, cfg.inplace_block_threads} <= {0, 128, 256, 512}
    want = oracle.to_well_formed_threads(u)
    out.zero_()
    _, fb = pkg.to_well_formed_first_bad(d, out)
    assert np.array_equal(to_host(out), want)
    assert int(fb.item()) == oracle.first_bad(u)
    out.zero_()
    pkg.to_well_formed(d, out)
    assert np.array_equal(to_host(out), want)
    assert pkg.first_error_index_sync(d) == oracle.first_bad(u)
    out.copy_(d)
    pkg.to_well_formed_(out)
    assert np.array_equal(to_host(out), want)
    units, offs = workloads.ragged_batch(count=300_000, seed=52)
    du = to_dev(units)
    do = torch.from_numpy(offs).cuda()
    bcfg = pkg.autotune_batch(du, do, reps=3)
    assert bcfg.batch_units_per_thread in (0, 2, 4)
    got = to_host(pkg.to_well_formed_batch(du, do))
    assert np.array_equal(got, oracle.to_well_formed_batch(units, offs))
    pkg.check_device_errors()


def test_bounded_wait_gives_up_and_reports(pkg):
    """A wait on a barrier that nothing completes gives up after its limit
    (here 50 ms) and raises the device-error flag that the host reads; the
    context stays usable."""
    import time
    lib = pkg.lib()
    pkg.check_device_errors()  # start clean
    t0 = time.perf_counter()
    assert lib.utf16_selftest_bounded_wait(50_000_000) == pkg.ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert lib.utf16_check_device_errors() == pkg.ETIMEOUT
    assert lib.utf16_check_device_errors() == 0  # read and cleared
    # the device still works
    u = workloads.mixed(100_000, 1e-2, seed=5)
    d = to_dev(u)
    assert pkg.first_error_index_sync(d) == oracle.first_bad(u)


def test_tuning_cache_round_trip(pkg, tmp_path):
    import torch
    u = workloads.mixed(4 << 20, 1e-2, seed=53)
    d = to_dev(u)
    cfg = pkg.autotune_single(d, torch.empty_like(d), reps=2)
    path = str(tmp_path / "tuning.json")
    saved = pkg.save_tuning(path)
    assert "single" in saved and str((u.size).bit_length() - 1) in saved["single"]
    pkg.set_config(pkg.get_config())  # clears tuned entries
    assert pkg.lib().utf16_get_tuned(0, u.size.bit_length() - 1, pkg.Config()) == pkg.EAGAIN
    assert pkg.load_tuning(path) >= 1
    c = pkg.Config()
    assert pkg.lib().utf16_get_tuned(0, u.size.bit_length() - 1, c) == 0
    assert c.as_dict() == cfg.as_dict()


def test_autotune_from_length_histogram(pkg):
    """utf16_autotune tunes size buckets (single strings) and a string-count
    bucket (batches) on synthetic text; the tuned configurations then give
    the oracle's results."""
    import torch
    saved = pkg.get_config()
    try:
        pkg.set_config(saved)  # clear tuned entries
        hist = np.zeros(32, np.int64)
        hist[12] = 5
        hist[22] = 1
        pkg.autotune_histogram("single", hist)
        for b in (12, 22):
            c = pkg.Config()
            assert pkg.lib().utf16_get_tuned(0, b, c) == 0, b
        assert pkg.lib().utf16_get_tuned(0, 13, pkg.Config()) == pkg.EAGAIN
        bh = np.zeros(20, np.int64)
        bh[0] = 50
        bh[5] = 20_000
        bh[11] = 300
        pkg.autotune_histogram("batch", bh)
        total = int(bh.sum())
        assert pkg.lib().utf16_get_tuned(1, total.bit_length() - 1, pkg.Config()) == 0
        # results under the tuned entries
        u = workloads.mixed((1 << 22) + 5, 1e-2, seed=77)
        d = to_dev(u)
        out, fb = pkg.to_well_formed_first_bad(d)
        assert np.array_equal(to_host(out), oracle.to_well_formed_threads(u))
        assert int(fb.item()) == oracle.first_bad(u)
        lens = workloads.lognormal_lengths(total, seed=78)
        offs = workloads.offsets_from_lengths(lens)
        units = workloads.mixed(int(offs[-1]), 1e-2, seed=79)
        d_u = to_dev(units)
        d_o = torch.from_numpy(offs).cuda()
        got = to_host(pkg.to_well_formed_batch(d_u, d_o))
        assert np.array_equal(got, oracle.to_well_formed_batch(units, offs))
        fbb = pkg.first_error_index_batch(d_u, d_o).cpu().numpy()
        assert np.array_equal(fbb, oracle.first_bad_batch(units, offs))
    finally:
        pkg.set_config(saved)


def test_chunk_width_by_size(pkg):
    """The default chunk width (0) is chosen by size: both sides of the switch
    (40,960 units per SM) give the oracle's results in every mode."""
    import torch
    saved = pkg.get_config()
    try:
        pkg.set_config(saved, single_units_per_thread=0)
        assert pkg.get_config().single_units_per_thread == 0
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        for n in (sms * 40960 - 1, sms * 40960 + 3):
            u = workloads.mixed(n, 1e-3, seed=n % 1000)
            want, want_fb = oracle.to_well_formed_threads(u), oracle.first_bad_threads(u)
            d = to_dev(u)
            out = torch.empty_like(d)
            _, fb = pkg.to_well_formed_first_bad(d, out)
            assert np.array_equal(to_host(out), want) and int(fb.item()) == want_fb, n
            assert pkg.first_error_index_sync(d) == want_fb, n
            pkg.to_well_formed_(d)
            assert np.array_equal(to_host(d), want), n
    finally:
        pkg.set_config(saved)
    pkg.check_device_errors()
