"""Launches captured into CUDA graphs: after utf16_init_device() the entry
points with device outputs neither allocate nor synchronise, so a graph
captured once replays the fused single-string call, the ragged batch (repair
and per-string check) and a long mix of back-to-back reductions on new
contents of the same buffers, with the oracle's results every time."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_06349_gb300 as p
    p.init_device()
    return p


def test_single_string_graph_replay(pkg):
    import torch
    n = workloads.SMALL_MIXED_UNITS
    d_in = to_dev(workloads.small_mixed())
    d_out = torch.empty_like(d_in)
    fb = torch.empty(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pkg.to_well_formed_first_bad(d_in, d_out, fb)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pkg.to_well_formed_first_bad(d_in, d_out, fb)
    for seed in range(5):
        u = workloads.mixed(n, 0.02 if seed % 2 else 0.0, seed=700 + seed)
        d_in.copy_(to_dev(u))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(to_host(d_out), oracle.to_well_formed(u)), seed
        assert int(fb.item()) == oracle.first_bad(u), seed


def test_ragged_batch_graph_replay(pkg):
    import torch
    units, offs = workloads.ragged_batch(count=100_000, seed=71)
    d_u = to_dev(units)
    d_o = torch.from_numpy(offs).cuda()
    d_out = torch.empty_like(d_u)
    fbb = torch.empty(offs.size - 1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pkg.to_well_formed_batch(d_u, d_o, d_out)
        pkg.first_error_index_batch(d_u, d_o, fbb)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pkg.to_well_formed_batch(d_u, d_o, d_out)
        pkg.first_error_index_batch(d_u, d_o, fbb)
    for seed in range(3):
        u2 = units.copy()
        workloads.fill_ragged(u2, offs, seed=900 + seed, lone_rate=0.02, forced=0.2)
        d_u.copy_(to_dev(u2))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(to_host(d_out), oracle.to_well_formed_batch(u2, offs)), seed
        assert np.array_equal(fbb.cpu().numpy(), oracle.first_bad_batch(u2, offs)), seed


def test_back_to_back_reductions_in_one_graph(pkg):
    """Many reductions back to back on one stream, captured in one graph so
    that consecutive grids overlap as far as the library lets them: one-block
    and many-block grids, strings with and without errors, the fused repair,
    the read-only check (with its early exit), the error list and the offsets
    check, each with its own device result.  Every result must be the
    oracle's on every replay (the completion counter and the minimum are reset
    by each launch for the next)."""
    import torch
    rng = np.random.default_rng(77)
    sizes = [1, 9, 1000, 8192, 8193, 65_536, 300_001, 1_000_000]
    strings, outs = [], []
    for k, n in enumerate(sizes):
        strings.append(to_dev(workloads.mixed(n, 0.0, seed=800 + k)))
        outs.append(torch.empty_like(strings[-1]))
    calls = 48
    picks = rng.integers(0, len(sizes), calls)
    kinds = rng.integers(0, 3, calls)  # 0 repair + first error, 1 check, 2 error list
    res = torch.full((calls,), -7, dtype=torch.int64, device="cuda")
    pos = torch.empty((calls, 64), dtype=torch.int64, device="cuda")
    offs = workloads.offsets_from_lengths(rng.integers(0, 50, 20_000).astype(np.int64))
    bad = offs.copy()
    bad[12_345] = bad[12_344] - 1
    d_offs = [torch.from_numpy(offs).cuda(), torch.from_numpy(bad).cuda()]
    ores = torch.full((2,), -7, dtype=torch.int64, device="cuda")
    lib = pkg.lib()
    import ctypes

    def run(stream):
        h = ctypes.c_void_p(stream.cuda_stream)
        for i in range(calls):
            d, o, n = strings[picks[i]], outs[picks[i]], sizes[picks[i]]
            r = res[i:i + 1].data_ptr()
            if kinds[i] == 0:
                rc = lib.utf16_to_well_formed_first_bad(d.data_ptr(), o.data_ptr(), n, r, h)
            elif kinds[i] == 1:
                rc = lib.utf16_is_well_formed(d.data_ptr(), n, r, h)
            else:
                rc = lib.utf16_error_positions(d.data_ptr(), n, pos[i].data_ptr(), 64, r, h)
            assert rc == 0, (i, rc)
            if i % 16 == 0:
                for j in range(2):
                    assert lib.utf16_check_offsets(d_offs[j].data_ptr(), offs.size - 1, ores[j:j + 1].data_ptr(),
                                                   h) == 0

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run(s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run(torch.cuda.current_stream())
    for rep in range(4):
        # new contents: errors in some strings, none in others
        hosts = []
        for k, n in enumerate(sizes):
            u = workloads.mixed(n, float(rng.choice([0.0, 1e-5, 1e-2])), seed=int(rng.integers(1 << 40)))
            strings[k].copy_(to_dev(u))
            hosts.append(u)
        res.fill_(-7)
        ores.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        got = res.cpu().numpy()
        for i in range(calls):
            u = hosts[picks[i]]
            if kinds[i] == 2:
                assert got[i] == int(np.count_nonzero(oracle.to_well_formed(u) != u)), (rep, i)
            else:
                assert got[i] == oracle.first_bad(u), (rep, i, kinds[i], sizes[picks[i]])
        assert ores.cpu().numpy().tolist() == [-1, 12_345]
    pkg.check_device_errors()
