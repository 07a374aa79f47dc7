"""Full error report (every replaced index and the count) and in-place
repair with unit-granularity stores, against the oracle; and the paper's own
workload shapes (Section 4: 1,000,000 units with 0.1 % pairs and 0 % / 0.1 %
lone surrogates; the 1024-unit 5 % low / 5 % high / 90 % ASCII string)."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import Guarded, first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_06349_gb300 as p
    p.init_device()
    saved = p.get_config()
    yield p
    p.set_config(saved)


def _cases():
    yield "mixed", workloads.mixed(3_000_001, 1e-2, seed=61)
    yield "clean", workloads.mixed(1_000_003, 0.0, seed=62)
    yield "shifted", workloads.shifted_alternating(2_000_000)
    yield "uniform", workloads.uniform_surrogates(500_001, seed=63)
    yield "all_high", workloads.all_high(70_000)
    yield "paper_0", workloads.paper_mix(1_000_000, 0.001, 0.0, seed=64)
    yield "paper_0.1", workloads.paper_mix(1_000_000, 0.001, 0.001, seed=65)
    yield "browser_1024", workloads.paper_mix(1024, 0.0, 0.10, seed=66)


@pytest.mark.parametrize("name,u", list(_cases()))
def test_error_positions_match_oracle(pkg, name, u):
    want = np.nonzero(oracle.to_well_formed(u) != u)[0]
    for a in (0, 3):
        g = Guarded(u.size, a, u)
        pos, count = pkg.error_positions(g.view)
        assert count == want.size, (name, a)
        got = np.sort(pos.cpu().numpy())
        assert np.array_equal(got, want), (name, a, first_diff(got, want))
    if want.size > 10:
        pos, count = pkg.error_positions(to_dev(u), capacity=want.size // 3)
        got = pos.cpu().numpy()
        assert count == want.size and got.size == want.size // 3
        assert np.unique(got).size == got.size and np.all(np.isin(got, want))


def test_error_positions_small_sweep(pkg):
    rng = np.random.default_rng(67)
    alph = np.array([0x41, 0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0xFFFD], np.uint16)
    for n in list(range(0, 40)) + [255, 256, 257, 1023, 1024, 1025, 4097]:
        u = alph[rng.integers(0, alph.size, n)]
        want = np.nonzero(oracle.to_well_formed(u) != u)[0]
        g = Guarded(max(n, 1), 5, u if n else np.zeros(1, np.uint16))
        view = g.view[:n]
        pos, count = pkg.error_positions(view, capacity=max(n, 1))
        assert count == want.size, n
        assert np.array_equal(np.sort(pos.cpu().numpy()), want), n


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("name,u", list(_cases()))
def test_in_place_unit_stores(pkg, name, u, variant):
    pkg.set_config(inplace_unit_stores=1, inplace_variant=variant)
    want = oracle.to_well_formed(u)
    for a in (0, 7):
        g = Guarded(u.size, a, u)
        pkg.to_well_formed_(g.view)
        assert np.array_equal(g.get(), want), (name, a, first_diff(g.get(), want))
        assert g.canaries_ok()
    pkg.set_config(inplace_unit_stores=0)


@pytest.mark.parametrize("name,u", [c for c in _cases() if c[0].startswith(("paper", "browser"))])
def test_paper_workloads(pkg, name, u):
    d = to_dev(u)
    out, fb = pkg.to_well_formed_first_bad(d)
    assert np.array_equal(to_host(out), oracle.to_well_formed(u)), name
    assert int(fb.item()) == oracle.first_bad(u), name
