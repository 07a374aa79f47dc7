"""Serving engine (continuous batching) against the oracle, through the C ABI:
every request's result and first-error index equal the oracle's, the same
alone and in a mix under load; small budgets force admission to wait for
completions; host-injected admission failures and cancellations leave every
other request exact; the plain per-request replay agrees too."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import first_diff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_06349_gb300 as p
    p.init_device()
    return p


def _requests(count, seed, big=True):
    rng = np.random.default_rng(seed)
    lens = workloads.request_lengths(count, seed=seed)
    if not big:
        lens = np.minimum(lens, 70_000)
    lens[::97] = 0  # a few empty requests
    reqs = []
    for i, n in enumerate(lens):
        u = workloads.mixed(int(n), 1e-3, seed=seed * 100_003 + i)
        if n > 2 and rng.random() < 0.3:
            u[0] = 0xDC00  # starts with a low surrogate
        if n > 2 and rng.random() < 0.3:
            u[-1] = 0xD800  # ends with a high surrogate
        reqs.append(u)
    return reqs


def _expect(reqs):
    return [(oracle.to_well_formed(u), oracle.first_bad(u)) for u in reqs]


def test_submit_next_matches_oracle(pkg):
    reqs = _requests(300, 11)
    want = _expect(reqs)
    outs = [np.zeros_like(u) for u in reqs]
    with pkg.Server(hbm_budget_bytes=96 << 20, max_inflight_batches=3, small_request_bytes=64 << 10,
                    staging_bytes=16 << 20, max_batch_bytes=64 << 20) as srv:
        tickets = {srv.submit(u, o): i for i, (u, o) in enumerate(zip(reqs, outs))}
        got = {}
        while len(got) < len(reqs):
            c = srv.next(timeout_us=30_000_000)
            assert c is not None, "timed out waiting for completions"
            got[tickets[c["ticket"]]] = c
        st = srv.stats()
    for i, (w, fb) in enumerate(want):
        assert got[i]["status"] == 0
        assert got[i]["first_bad"] == fb, i
        assert np.array_equal(outs[i], w), i
    assert st["batches"] >= 2


def test_same_alone_and_in_the_mix(pkg):
    reqs = _requests(400, 12)
    want = _expect(reqs)
    alone = [np.zeros_like(u) for u in reqs]
    alone_fb = []
    with pkg.Server(hbm_budget_bytes=512 << 20) as srv:
        for u, o in zip(reqs, alone):  # one at a time: each request is a batch of its own
            srv.submit(u, o)
            c = srv.next(timeout_us=30_000_000)
            assert c is not None and c["status"] == 0
            alone_fb.append(c["first_bad"])
        mix = [np.zeros_like(u) for u in reqs]
        lat, fb = srv.replay(reqs, mix, rate_per_s=50_000, seed=3)  # arrivals overlap: batched together
        st = srv.stats()
    assert st["max_batch_requests"] > 1, "the mix never formed a multi-request batch"
    for i, (w, f) in enumerate(want):
        assert np.array_equal(alone[i], w) and alone_fb[i] == f, i
        assert np.array_equal(mix[i], alone[i]) and fb[i] == alone_fb[i], i
    assert np.all(lat > 0)


@pytest.mark.parametrize("direct", [1, 0])
def test_pinned_host_buffers(pkg, direct):
    """Pinned buffers: small requests gathered / scattered by the GPU itself
    (direct) or staged through pinned staging; large ones by copy engines."""
    import torch
    reqs = _requests(300, 13)
    want = _expect(reqs)
    ins = [torch.from_numpy(u.view(np.int16)).pin_memory() for u in reqs]
    outs = [torch.full_like(t, 0x5A5A).pin_memory() for t in ins]
    with pkg.Server(small_request_bytes=32 << 10, direct_host_access=direct) as srv:
        lat, fb = srv.replay(ins, outs, rate_per_s=0, seed=4)
        lat2, fb2 = srv.replay(ins, outs, rate_per_s=20_000, seed=5)
    for i, (w, f) in enumerate(want):
        assert np.array_equal(outs[i].numpy().view(np.uint16), w) and fb[i] == f and fb2[i] == f, i


def test_pinned_and_pageable_in_one_batch(pkg):
    import torch
    reqs = _requests(300, 17, big=False)
    want = _expect(reqs)
    ins, outs = [], []
    for i, u in enumerate(reqs):
        if i % 3 == 0:  # pageable numpy buffers: staged
            ins.append(u.copy())
            outs.append(np.zeros_like(u))
        else:           # pinned: gathered / scattered by the GPU; odd offsets exercise unaligned copies
            t = torch.from_numpy(np.concatenate([np.zeros(i % 8, np.uint16), u]).view(np.int16)).pin_memory()
            ins.append(t[i % 8:])
            outs.append(torch.zeros(u.size + 8, dtype=torch.int16).pin_memory()[(i * 5) % 8:][:u.size])
    with pkg.Server(max_inflight_batches=2, direct_host_access=1) as srv:
        lat, fb = srv.replay(ins, outs, rate_per_s=0, seed=6)
        st = srv.stats()
    assert st["max_batch_requests"] > 10
    for i, (w, f) in enumerate(want):
        got = outs[i] if isinstance(outs[i], np.ndarray) else outs[i].numpy().view(np.uint16)
        assert np.array_equal(got, w), (i, first_diff(got, w))
        assert fb[i] == f, (i, fb[i], f)


@pytest.mark.parametrize("host_pass_sms", ["", "0"])
def test_large_requests_in_pinned_buffers(pkg, host_pass_sms):
    """Large requests whose buffers kernels can reach are repaired where they
    are by one fused pass each (out of place, or in place when input and
    output are the same buffer), at any unit offset, in batches with staged
    small requests; pageable ones too where the device reads pageable memory
    coherently.  A partially overlapping pair, and every large request with
    host passes off, goes through the copy engines."""
    import os
    import torch
    os.environ["UTF16WF_SERVE_HOST_PASS_SMS"] = host_pass_sms
    rng = np.random.default_rng(41)
    reqs, ins, outs, same = [], [], [], []
    for i in range(48):
        kind = i % 4
        n = int(rng.integers(300_000, 1_200_000)) if kind != 3 else int(rng.integers(1, 3000))
        u = workloads.mixed(n, float(rng.choice([0.0, 1e-4, 1e-2])), seed=4100 + i)
        if i % 11 == 0:
            u[0], u[-1] = 0xDC00, 0xD800  # errors at both ends
        reqs.append(u)
        off = int(rng.integers(0, 8))
        if kind == 0:    # pinned, distinct buffers, odd offsets
            ins.append(torch.from_numpy(np.concatenate([np.zeros(off, np.uint16), u]).view(np.int16)).pin_memory()[off:])
            outs.append(torch.zeros(n + 8, dtype=torch.int16).pin_memory()[(off * 3) % 8:][:n])
        elif kind == 1:  # pinned, one buffer in place
            t = torch.from_numpy(np.concatenate([np.zeros(off, np.uint16), u]).view(np.int16)).pin_memory()[off:]
            ins.append(t)
            outs.append(t)
        elif kind == 2:  # pageable: host passes where the device reads pageable memory, else copy engines
            if i % 8 == 2:
                v = u.copy()  # one buffer, in place
                ins.append(v)
                outs.append(v)
            else:
                ins.append(u.copy())
                outs.append(np.zeros_like(u))
        else:            # small, staged
            ins.append(torch.from_numpy(u.view(np.int16)).pin_memory())
            outs.append(torch.zeros(n, dtype=torch.int16).pin_memory())
    # a partially overlapping pinned pair: output = input shifted by 3 units
    n = 400_000
    u = workloads.mixed(n, 1e-2, seed=4199)
    buf = torch.zeros(n + 3, dtype=torch.int16).pin_memory()
    buf[:n] = torch.from_numpy(u.view(np.int16))
    reqs.append(u)
    ins.append(buf[:n])
    outs.append(buf[3:])
    want = _expect(reqs)
    try:
        with pkg.Server(max_inflight_batches=3) as srv:
            lat, fb = srv.replay(ins, outs, rate_per_s=0, seed=8)
    finally:
        os.environ.pop("UTF16WF_SERVE_HOST_PASS_SMS", None)
    for i, (w, f) in enumerate(want):
        got = outs[i] if isinstance(outs[i], np.ndarray) else outs[i].numpy().view(np.uint16)
        assert np.array_equal(got, w), (i, first_diff(got, w))
        assert fb[i] == f, (i, fb[i], f)


def test_injected_admission_failures_leave_others_exact(pkg):
    reqs = _requests(200, 14, big=False)
    want = _expect(reqs)
    outs = [np.full_like(u, 0x5A5A) for u in reqs]
    with pkg.Server(inject_fail_mod=7) as srv:
        tickets = [srv.submit(u, o) for u, o in zip(reqs, outs)]
        res = {}
        while len(res) < len(reqs):
            c = srv.next(timeout_us=30_000_000)
            assert c is not None
            res[c["ticket"]] = c
    failed = 0
    for i, t in enumerate(tickets):
        c = res[t]
        if reqs[i].size and t % 7 == 6:
            assert c["status"] == pkg.ENOMEM
            assert np.all(outs[i] == 0x5A5A)  # untouched
            failed += 1
        else:
            assert c["status"] == 0 and c["first_bad"] == want[i][1], i
            assert np.array_equal(outs[i], want[i][0]), i
    assert failed > 10


@pytest.mark.parametrize("step", [0, 1])
def test_injected_copy_failures_leave_others_exact(pkg, step):
    """A copy step that fails (injected on the host in every third launched
    batch: its host-to-device copies for step 0, its device-to-host copies
    for step 1) completes that batch's requests with UTF16_ECUDA and leaves
    their outputs untouched (these small requests are staged, and the engine
    copies staged results back only on success).  Every other request is
    exact, and the engine goes on serving the batches after a failed one."""
    reqs = _requests(300, 16 + step, big=False)
    want = _expect(reqs)
    outs = [np.full_like(u, 0x5A5A) for u in reqs]
    with pkg.Server(inject_copy_fail_mod=3, inject_copy_fail_step=step, max_batch_strings=16,
                    max_inflight_batches=2) as srv:
        tickets = [srv.submit(u, o) for u, o in zip(reqs, outs)]
        res = {}
        while len(res) < len(reqs):
            c = srv.next(timeout_us=30_000_000)
            assert c is not None
            res[c["ticket"]] = c
        st = srv.stats()
    failed = ok = 0
    for i, t in enumerate(tickets):
        c = res[t]
        if c["status"] == pkg.ECUDA:
            assert np.all(outs[i] == 0x5A5A), i  # untouched
            failed += 1
        else:
            assert c["status"] == 0 and c["first_bad"] == want[i][1], i
            assert np.array_equal(outs[i], want[i][0]), i
            ok += 1
    assert st["batches"] >= 19  # at most 8 requests (16 strings) per batch
    assert failed > 0 and ok > failed
    pkg.check_device_errors()


def test_cancel_before_admission(pkg):
    reqs = _requests(400, 15, big=False)
    want = _expect(reqs)
    outs = [np.zeros_like(u) for u in reqs]
    with pkg.Server(max_inflight_batches=1, max_batch_strings=8) as srv:
        tickets = [srv.submit(u, o) for u, o in zip(reqs, outs)]
        cancelled = {t for t in tickets[200:] if srv.cancel(t)}
        res = {}
        while len(res) < len(reqs):
            c = srv.next(timeout_us=30_000_000)
            assert c is not None
            res[c["ticket"]] = c
    assert cancelled, "nothing was still pending to cancel"
    for i, t in enumerate(tickets):
        if t in cancelled:
            assert res[t]["status"] == pkg.ECANCELED
        else:
            assert res[t]["status"] == 0 and res[t]["first_bad"] == want[i][1]
            assert np.array_equal(outs[i], want[i][0]), i


def test_plain_replay_matches(pkg):
    reqs = _requests(150, 16)
    want = _expect(reqs)
    outs = [np.zeros_like(u) for u in reqs]
    lat, fb = pkg.plain_replay(reqs, outs, rate_per_s=0, seed=5)
    for i, (w, f) in enumerate(want):
        assert np.array_equal(outs[i], w) and fb[i] == f, i
    # pipelined over several streams: the same results, every request completed
    for streams in (1, 4, 8):
        outs = [np.zeros_like(u) for u in reqs]
        lat, fb = pkg.plain_replay(reqs, outs, rate_per_s=0, seed=5, streams=streams)
        for i, (w, f) in enumerate(want):
            assert np.array_equal(outs[i], w) and fb[i] == f, (streams, i)
        assert np.all(lat >= 0)


def test_oversize_request_rejected(pkg):
    with pkg.Server(hbm_budget_bytes=1 << 20, max_batch_bytes=1 << 19) as srv:
        big = np.zeros(1 << 20, np.uint16)
        with pytest.raises(pkg.Utf16Error):
            srv.submit(big, big)


def test_request_longer_than_batch_target(pkg):
    """max_batch_bytes bounds packing only: a request longer than it is served
    as a batch of its own, between packed batches of small requests."""
    rng = np.random.default_rng(31)
    reqs = []
    for i in range(60):
        n = int(rng.integers(100_000, 300_000)) if i % 10 == 3 else int(rng.integers(1, 2000))
        reqs.append(workloads.mixed(n, 1e-2, seed=3100 + i))
    want = _expect(reqs)
    outs = [np.zeros_like(u) for u in reqs]
    with pkg.Server(hbm_budget_bytes=64 << 20, max_batch_bytes=64 << 10) as srv:
        lat, fb = srv.replay(reqs, outs, 0, seed=3)
        st = srv.stats()
    for i, (w, f) in enumerate(want):
        assert np.array_equal(outs[i], w) and fb[i] == f, i
    assert st["rejected"] == 0 and st["batches"] >= 6


def test_aligned_padding_fits_reservation(pkg):
    """Admission reserves arena space for the launch layout, where staged
    requests are packed first and every directly copied request starts at a
    16-byte boundary.  Alternating direct requests of 8k+1 units with staged
    ones of 8k+7 units makes that layout much longer than the arrival-order
    one; every request must still come back exact."""
    import torch
    rng = np.random.default_rng(29)
    reqs = []
    for i in range(400):
        n = int(8 * rng.integers(0, 40) + (1 if i % 2 == 0 else 7))
        u = workloads.mixed(n, 1e-2, seed=2900 + i)
        reqs.append(u)
    want = _expect(reqs)
    for rep in range(3):
        ins, outs = [], []
        for i, u in enumerate(reqs):
            if i % 2 == 1:
                ins.append(u.copy())
                outs.append(np.zeros_like(u))
            else:
                ins.append(torch.from_numpy(u.view(np.int16).copy()).pin_memory())
                outs.append(torch.zeros(u.size, dtype=torch.int16).pin_memory())
        with pkg.Server(max_inflight_batches=2, direct_host_access=1, hbm_budget_bytes=64 << 20) as srv:
            _, fb = srv.replay(ins, outs, rate_per_s=0, seed=rep)
        for i, (w, f) in enumerate(want):
            got = outs[i] if isinstance(outs[i], np.ndarray) else outs[i].numpy().view(np.uint16)
            assert fb[i] == f, (rep, i, fb[i], f)
            assert np.array_equal(got, w), (rep, i, first_diff(got, w))
