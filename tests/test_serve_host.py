"""Host-side logic of the serving engine, without a GPU: the FIFO ring used
for admission against the HBM budget never hands out overlapping or
out-of-range blocks, frees strictly oldest-first, reports what it holds, and
never refuses a block that fits an empty ring."""
import random

import pytest


@pytest.fixture(scope="module")
def pkg():
    from paper_2601_06349_gb300 import build
    build.build()
    import paper_2601_06349_gb300 as p
    return p


@pytest.mark.parametrize("seed", range(6))
def test_ring_properties(pkg, seed):
    rng = random.Random(seed)
    cap = rng.choice([1000, 4096, 1 << 20])
    a = pkg.Arena(cap)
    live = []  # (off, size) oldest first
    refused_when_empty = 0
    for _ in range(4000):
        if live and rng.random() < 0.45:
            assert a.free_oldest()
            live.pop(0)
        else:
            size = rng.randint(1, cap // rng.choice([1, 2, 3, 8, 50]))
            off = a.alloc(size)
            if off < 0:
                if not live:
                    refused_when_empty += 1
                continue
            assert 0 <= off and off + size <= cap
            for o, s in live:
                assert off + size <= o or o + s <= off, "overlap with a live block"
            live.append((off, size))
        assert a.used() == sum(s for _, s in live)
    assert refused_when_empty == 0
    while live:
        assert a.free_oldest()
        live.pop(0)
    assert a.used() == 0
    assert not a.free_oldest()
    assert a.alloc(cap) == 0


def test_ring_rejects_oversize(pkg):
    a = pkg.Arena(100)
    assert a.alloc(101) == -1
    assert a.alloc(0) == -1
    assert a.alloc(100) == 0
    assert a.alloc(1) == -1
