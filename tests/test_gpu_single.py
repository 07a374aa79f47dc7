"""Single-string CUDA path against the oracle, bit-exact (integer work: the
tolerance is zero), through the C ABI.

* a sweep of small lengths (0..70 and sizes around every tile edge) at every
  misalignment of the input (0..7 units) and of the output relative to it,
  with guard bands, for out-of-place, fused first-error, in-place and
  read-only entry points, device and host first-error pointers;
* the full-size strings in the launch configuration the benchmark times:
  1 MiB mixed, 1 GiB mixed at lone rates 0 / 1e-6 / 1e-2, the three 512 MiB
  adversarial strings;
* isWellFormed's early exit, stream independence of the scratch slots, and
  the pipelined host-buffer entry point (chunk edges inside surrogate pairs).
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import Guarded, first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu

ALPHABET = np.array([0x0041, 0x00E9, 0xD7FF, 0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0xE000, 0xFFFD, 0xFFFF], np.uint16)


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_06349_gb300 as p
    p.init_device()
    return p


def _sweep_sizes():
    sizes = list(range(0, 71))
    for edge in (256, 512, 1024, 2048, 4096, 8192, 65536):
        sizes += [edge - 9, edge - 1, edge, edge + 1, edge + 9]
    sizes += [100_003, 262_147]
    return sorted(set(s for s in sizes if s >= 0))


def _content(n, rng):
    if n < 4096:
        return ALPHABET[rng.integers(0, ALPHABET.size, n)]
    u = workloads.mixed(n, 0.02, seed=int(rng.integers(1 << 30)))
    # sprinkle surrogates so that every chunk takes the slow path somewhere
    idx = rng.integers(0, n, n // 50)
    u[idx] = ALPHABET[rng.integers(0, ALPHABET.size, idx.size)]
    return u


def test_small_sweep_all_alignments(pkg):
    import torch
    rng = np.random.default_rng(2026)
    for n in _sweep_sizes():
        offs = range(8) if n < 5000 else (0, 3)
        for a_in in offs:
            u = _content(n, rng)
            want = oracle.to_well_formed(u)
            want_fb = oracle.first_bad(u)
            gi = Guarded(n, a_in, u)
            for a_out in (range(8) if n < 300 else (a_in, (a_in + 1) % 8, (a_in + 4) % 8)):
                go = Guarded(n, a_out)
                pkg.to_well_formed(gi.view, go.view)
                got = go.get()
                assert np.array_equal(got, want), (n, a_in, a_out, first_diff(got, want))
                assert go.canaries_ok(), (n, a_in, a_out)
                go2 = Guarded(n, a_out)
                _, fb = pkg.to_well_formed_first_bad(gi.view, go2.view)
                assert np.array_equal(go2.get(), want), (n, a_in, a_out)
                assert int(fb.item()) == want_fb, (n, a_in, a_out)
                assert go2.canaries_ok()
            # read-only check: device and host result pointers
            assert int(pkg.first_error_index(gi.view).item()) == want_fb, (n, a_in)
            assert pkg.first_error_index_sync(gi.view) == want_fb, (n, a_in)
            assert np.array_equal(gi.get(), u)
            assert gi.canaries_ok()
            # in place
            gp = Guarded(n, a_in, u)
            pkg.to_well_formed_(gp.view)
            assert np.array_equal(gp.get(), want), (n, a_in, first_diff(gp.get(), want))
            assert gp.canaries_ok()
    torch.cuda.synchronize()


def test_in_place_same_pointer_via_out_of_place_entry(pkg):
    u = workloads.mixed(300_001, 0.05, seed=5)
    g = Guarded(u.size, 3, u)
    pkg.to_well_formed(g.view, g.view)
    assert np.array_equal(g.get(), oracle.to_well_formed(u))
    assert g.canaries_ok()


def _full_check(pkg, u, label):
    import torch
    want = oracle.to_well_formed_threads(u)
    want_fb = oracle.first_bad_threads(u)
    d_in = to_dev(u)
    d_out = torch.empty_like(d_in)
    # fused out-of-place + first-error (the benchmarked launch)
    _, fb = pkg.to_well_formed_first_bad(d_in, d_out)
    got = to_host(d_out)
    assert np.array_equal(got, want), (label, first_diff(got, want))
    assert int(fb.item()) == want_fb, label
    # read-only
    assert pkg.first_error_index_sync(d_in) == want_fb, label
    # out-of-place without first-error
    d_out.fill_(0)
    pkg.to_well_formed(d_in, d_out)
    assert np.array_equal(to_host(d_out), want), label
    # in place (input no longer needed)
    pkg.to_well_formed_(d_in)
    got = to_host(d_in)
    assert np.array_equal(got, want), (label, first_diff(got, want))
    del d_in, d_out
    torch.cuda.empty_cache()
    return want_fb, int(np.count_nonzero(want != u))


def test_small_mixed_string(pkg):
    u = workloads.small_mixed()
    fb, nbad = _full_check(pkg, u, "1 MiB mixed")
    assert nbad > 0 and fb < 100


@pytest.mark.parametrize("lone_rate", [0.0, 1e-6, 1e-2])
def test_large_mixed_string(pkg, lone_rate):
    u = workloads.large_mixed(lone_rate)
    fb, nbad = _full_check(pkg, u, f"1 GiB mixed p={lone_rate}")
    if lone_rate == 0.0:
        assert nbad == 0 and fb == u.size


@pytest.mark.parametrize("kind", ["uniform", "shifted", "all_high"])
def test_adversarial_string(pkg, kind):
    u = workloads.adversarial(kind)
    fb, nbad = _full_check(pkg, u, kind)
    if kind == "shifted":
        assert nbad == 65_584 and fb == 4092
    if kind == "all_high":
        assert nbad == u.size and fb == 0


def test_is_well_formed_early_exit_positions(pkg):
    n = 50_000_000
    base = workloads.mixed(n, 0.0, seed=17)
    for pos in (0, 1, 255, 256, 1023, 1024, 12_345_678, n - 2, n - 1):
        u = base.copy()
        u[pos] = 0xDC00 if pos == 0 else 0xD800
        if pos > 0 and 0xD800 <= u[pos - 1] <= 0xDBFF:
            u[pos - 1] = 0x41  # keep the planted error the first one
        want = oracle.first_bad(u)
        d = to_dev(u)
        assert pkg.first_error_index_sync(d) == want, pos
        assert int(pkg.first_error_index(d).item()) == want, pos
    d = to_dev(base)
    assert pkg.first_error_index_sync(d) == n
    assert pkg.is_well_formed(d)


def test_streams_use_independent_slots(pkg):
    import torch
    strings = [workloads.mixed(3_000_000 + 7 * i, 1e-4 * (i + 1), seed=100 + i) for i in range(6)]
    wants = [oracle.first_bad(s) for s in strings]
    devs = [to_dev(s) for s in strings]
    streams = [torch.cuda.Stream() for _ in range(3)]
    results = []
    for rep in range(3):
        for i, d in enumerate(devs):
            s = streams[i % 3]
            with torch.cuda.stream(s):
                results.append((i, pkg.first_error_index(d, stream=s)))
    torch.cuda.synchronize()
    for i, t in results:
        assert int(t.item()) == wants[i]


@pytest.mark.parametrize("units_per_thread", [0, 4])
@pytest.mark.parametrize("pageable_direct", ["0", "1"])
@pytest.mark.parametrize("chunk", [4096, 1 << 20])
def test_host_pipeline_chunk_edges(pkg, chunk, pageable_direct, units_per_thread):
    """Pageable host buffers: the staged three-stream pipeline (direct passes
    off), and the direct pass where the device reads pageable memory
    coherently (else the pipeline again).  The pipeline repairs each chunk in
    place with the units just outside it as neighbours; with 4-vector chunks
    that is the bit-word kernel, which must not replace those neighbours
    (surrogate-dense text puts unpaired surrogates on both sides of every
    chunk edge)."""
    os.environ["UTF16WF_HOST_CHUNK_UNITS"] = str(chunk)
    os.environ["UTF16WF_HOST_PAGEABLE_DIRECT"] = pageable_direct
    saved = pkg.get_config()
    pkg.set_config(single_units_per_thread=units_per_thread)
    try:
        for kind, u in (("shifted", workloads.shifted_alternating(3 * chunk + 77)),
                        ("mixed", workloads.mixed(5 * chunk + 3, 0.01, seed=3)),
                        ("uniform", workloads.uniform_surrogates(2 * chunk + 1, seed=4))):
            want = oracle.to_well_formed(u)
            out, fb = pkg.to_well_formed_host(u)
            assert np.array_equal(out, want), (kind, first_diff(out, want))
            assert fb == oracle.first_bad(u), kind
            v = u.copy()
            out2, fb2 = pkg.to_well_formed_host(v, v)  # in place on the host buffer
            assert np.array_equal(v, want) and fb2 == fb, kind
    finally:
        os.environ.pop("UTF16WF_HOST_CHUNK_UNITS", None)
        os.environ.pop("UTF16WF_HOST_PAGEABLE_DIRECT", None)
        pkg.set_config(saved)


def test_host_pipeline_pinned_large(pkg):
    import torch
    u = workloads.large_mixed(1e-2)
    want = oracle.to_well_formed_threads(u)
    h_in = torch.from_numpy(u.view(np.int16)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    out, fb = pkg.to_well_formed_host(h_in, h_out)
    got = out.numpy().view(np.uint16)
    assert np.array_equal(got, want), first_diff(got, want)
    assert fb == oracle.first_bad_threads(u)


def test_raw_c_abi_host_first_bad_pointer(pkg):
    """Direct ctypes call: host first-error pointer makes the call blocking."""
    import torch
    u = workloads.mixed(777_777, 1e-3, seed=9)
    d = to_dev(u)
    v = ctypes.c_int64(-7)
    rc = pkg.lib().utf16_is_well_formed(d.data_ptr(), u.size, ctypes.addressof(v),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0 and v.value == oracle.first_bad(u)
    out = torch.empty_like(d)
    w = ctypes.c_int64(-7)
    rc = pkg.lib().utf16_to_well_formed_first_bad(d.data_ptr(), out.data_ptr(), u.size, ctypes.addressof(w), None)
    assert rc == 0 and w.value == v.value
    assert np.array_equal(to_host(out), oracle.to_well_formed(u))


def _plant(base, edge, kind):
    """One mismatch next to unit `edge` of a string of non-surrogates and
    pairs (with a neighbour or two rewritten so that it stays the only one
    nearby)."""
    u = base.copy()
    u[edge - 3:edge + 3] = 0x41
    if 0xD800 <= u[edge - 4] <= 0xDBFF:  # its low was overwritten
        u[edge - 4] = 0x42
    if 0xDC00 <= u[edge + 3] <= 0xDFFF:  # its high was overwritten
        u[edge + 3] = 0x42
    if kind == "lone_high_last":       # last unit of the chunk before `edge`: a high with no low after it
        u[edge - 1] = 0xD800
    elif kind == "lone_low_first":     # first unit of the chunk: a low with no high before it
        u[edge] = 0xDC00
    elif kind == "pair_across":        # a valid pair across the chunk edge (no mismatch at all)
        u[edge - 1], u[edge] = 0xD83D, 0xDE0A
    elif kind == "lone_high_first":
        u[edge] = 0xDBFF
    elif kind == "lone_low_last":
        u[edge - 1] = 0xDFFF
    return u


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("units_per_thread", [2, 4])
def test_check_mismatch_at_chunk_edges(pkg, variant, units_per_thread):
    """The read-only check clears whole chunks with the step-two test; a
    mismatch in a chunk's first or last unit (the last one is only visible
    through the unit after the chunk) must still be found, and a pair across
    two chunks must not be reported."""
    chunk_units = 256 * units_per_thread
    base = workloads.mixed(300_000, 0.0, seed=61)
    saved = pkg.get_config()
    pkg.set_config(check_variant=variant, single_units_per_thread=units_per_thread)
    try:
        for a in (0, 5):
            for k in (3, 101):
                edge = k * chunk_units - a  # first unit of warp chunk k for a string misaligned by a units
                for kind in ("lone_high_last", "lone_low_first", "pair_across", "lone_high_first", "lone_low_last"):
                    u = _plant(base, edge, kind)
                    want = oracle.first_bad(u)
                    if kind == "pair_across":
                        assert want == u.size
                    else:
                        assert edge - 1 <= want <= edge, (kind, want, edge)
                    g = Guarded(u.size, a, u)
                    assert pkg.first_error_index_sync(g.view) == want, (variant, units_per_thread, a, k, kind)
                    assert int(pkg.first_error_index(g.view).item()) == want, (variant, units_per_thread, a, k, kind)
    finally:
        pkg.set_config(saved)


def test_bench_launch_configuration_full_size(pkg):
    """The benchmarked step in the launch configuration the bench uses: the
    autotuner's choice for the 1 GiB string at 1e-2 lone surrogates, then the
    fused repair, the check, the repair alone and in-place repair, each
    against the oracle."""
    import torch
    u = workloads.large_mixed(1e-2)
    want = oracle.to_well_formed_threads(u)
    want_fb = oracle.first_bad_threads(u)
    saved = pkg.get_config()
    try:
        d_in = to_dev(u)
        d_out = torch.empty_like(d_in)
        cfg = pkg.autotune_single(d_in, d_out, reps=2)
        _, fb = pkg.to_well_formed_first_bad(d_in, d_out)
        got = to_host(d_out)
        assert np.array_equal(got, want), (cfg.as_dict(), first_diff(got, want))
        assert int(fb.item()) == want_fb
        assert pkg.first_error_index_sync(d_in) == want_fb
        d_out.zero_()
        pkg.to_well_formed(d_in, d_out)  # the repair alone, on its own tuned settings
        got = to_host(d_out)
        assert np.array_equal(got, want), (cfg.as_dict(), "plain", first_diff(got, want))
        pkg.to_well_formed_(d_in)
        assert np.array_equal(to_host(d_in), want), cfg.as_dict()
        del d_in, d_out
        torch.cuda.empty_cache()
    finally:
        pkg.set_config(saved)


def test_host_api_pinned_direct_and_mixed(pkg):
    """Host-buffer API: both buffers pinned (one pass over the host link),
    in place on a pinned buffer, misaligned pinned views, and a pinned input
    with a pageable output (staged chunks) all give the oracle's result."""
    import torch
    rng = np.random.default_rng(83)
    for n in (1, 7, 8, 3 * 4096 + 5, 1_000_003):
        u = workloads.mixed(n, 1e-2, seed=int(rng.integers(1 << 30)))
        want, want_fb = oracle.to_well_formed(u), oracle.first_bad(u)
        for a in (0, 3):
            base_in = torch.zeros(n + 8, dtype=torch.int16).pin_memory()
            base_in[a:a + n] = torch.from_numpy(u.view(np.int16))
            h_in = base_in[a:a + n]
            h_out = torch.zeros(n + 8, dtype=torch.int16).pin_memory()[5 - a:5 - a + n]
            out, fb = pkg.to_well_formed_host(h_in, h_out)
            assert np.array_equal(out.numpy().view(np.uint16), want) and fb == want_fb, (n, a, "pinned")
            assert np.all(base_in[:a].numpy() == 0) and np.all(base_in[a + n:].numpy() == 0)
            out2, fb2 = pkg.to_well_formed_host(h_in, h_in)  # in place, pinned
            assert np.array_equal(h_in.numpy().view(np.uint16), want) and fb2 == want_fb, (n, a, "in place")
            h_in[:] = torch.from_numpy(u.view(np.int16))
            pageable = np.zeros(n, np.uint16)
            out3, fb3 = pkg.to_well_formed_host(h_in, pageable)
            assert np.array_equal(pageable, want) and fb3 == want_fb, (n, a, "pinned in, pageable out")


def test_readme_example(pkg):
    """The usage example of the README, as written there."""
    import torch
    wf = pkg
    s = torch.tensor([0x48, 0xD800, 0x69, 0xD83D, 0xDE0A], dtype=torch.uint16, device="cuda")
    out, first_bad = wf.to_well_formed_first_bad(s)
    assert out.cpu().tolist() == [0x48, 0xFFFD, 0x69, 0xD83D, 0xDE0A]
    assert first_bad.cpu().tolist() == [1]
    offsets = torch.tensor([0, 2, 5], dtype=torch.int64, device="cuda")
    assert wf.first_error_index_batch(s, offsets).cpu().tolist() == [1, 3]
