"""Launches captured into CUDA graphs: after utf16_init_device() the entry
points with device outputs neither allocate nor synchronise, so a graph
captured once replays the fused single-string call and the ragged batch
(repair and per-string check) on new contents of the same buffers, with the
oracle's results every time."""
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
