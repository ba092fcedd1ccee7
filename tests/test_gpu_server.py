"""GPU tests of the sort server (continuous batching, admission by a
device-memory budget): every request's result equals the oracle's, and is
bit-identical whether the request ran alone or in a mix of other requests.
Tolerance is zero: sorted integers either match or they do not."""
import time

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")

from paper_1511_03404_gb300 import rs  # noqa: E402

pytestmark = pytest.mark.gpu


def make_trace(count, seed, max_log2=18):
    """Mixed requests: u32 pairs or u64 keys (by the parity of a draw),
    log-uniform sizes in [2^10, 2^max_log2], uniform keys."""
    raw = inputs.mt19937(seed, 3 * count)
    reqs = []
    for i in range(count):
        u = raw[2 * i] / 2**32
        n = int(2 ** (10 + (max_log2 - 10) * u))
        if raw[2 * count + i] % 2 == 0:
            k = inputs.keys(np.uint32, "uniform", n, seed=seed * 100000 + i)
            v = inputs.values(np.uint32, n)
        else:
            k = inputs.keys(np.uint64, "uniform", n, seed=seed * 100000 + i)
            v = None
        reqs.append((k, v))
    return reqs


class Req:
    def __init__(self, k, v):
        self.k, self.v = k, v
        self.ok = np.empty_like(k)
        self.ov = np.empty_like(v) if v is not None else None
        self.c = rs.rs_request(k.dtype.itemsize, 0 if v is None else v.dtype.itemsize, k.size, 0,
                               8 * k.dtype.itemsize, k.ctypes.data,
                               None if v is None else v.ctypes.data, self.ok.ctypes.data,
                               None if v is None else self.ov.ctypes.data)


def wait_all(server, handles, timeout_s=120):
    pending = dict(handles)
    status = {}
    t0 = time.time()
    while pending:
        for h in list(pending):
            st, done = rs.rs_poll(server, h)
            if done:
                status[pending.pop(h)] = st
        if time.time() - t0 > timeout_s:
            raise TimeoutError(f"{len(pending)} requests not done")
        time.sleep(0.0005)
    return status


def run(server, reqs, sequential=False):
    out = [Req(k, v) for k, v in reqs]
    if sequential:
        for i, r in enumerate(out):
            st, h = rs.rs_submit(server, r.c)
            rs.check(st, "rs_submit")
            assert wait_all(server, {h: i}) == {i: rs.RS_OK}
    else:
        handles = {}
        for i, r in enumerate(out):
            st, h = rs.rs_submit(server, r.c)
            rs.check(st, "rs_submit")
            handles[h] = i
        status = wait_all(server, handles)
        assert all(s == rs.RS_OK for s in status.values()), status
    return out


@pytest.fixture
def server():
    st, srv = rs.rs_server_create(1 << 30, 8)
    rs.check(st, "rs_server_create")
    yield srv
    rs.check(rs.rs_server_destroy(srv))


def test_mixed_trace_matches_oracle(server):
    reqs = make_trace(120, seed=3)
    out = run(server, reqs)
    for r in out:
        ek, ev = oracle.lsd_sort(r.k, r.v)
        assert np.array_equal(r.ok, ek)
        if r.v is not None:
            assert np.array_equal(r.ov, ev)
    st, stats = rs.rs_server_stats(server)
    rs.check(st)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["service_p99_ms"] >= stats["service_p50_ms"] > 0
    assert stats["wait_p99_ms"] >= stats["wait_p50_ms"] >= 0
    # the per-request trace: one record per request, times in order
    st, trace = rs.rs_server_trace(server)
    rs.check(st, "rs_server_trace")
    assert len(trace) == len(reqs)
    assert sorted(t["n"] for t in trace) == sorted(int(k.size) for k, _ in reqs)
    for t in trace:
        assert 0 <= t["submit_s"] <= t["admit_s"] <= t["done_s"]
        assert 0 <= t["stream"] < 8 and t["batched"] in (0, 1)


def test_short_requests_queued_together_share_one_launch():
    """Short u32 pair requests that wait together (every stream busy with a
    longer sort) are admitted as one batched segmented sort; a short request
    that is alone in the queue runs as its own sort instead of a batch of one."""
    st, server = rs.rs_server_create(4 << 30, 8)
    rs.check(st, "rs_server_create")
    try:
        _short_requests_batch(server)
    finally:
        rs.check(rs.rs_server_destroy(server))


def _short_requests_batch(server):
    st, cfg = rs.rs_server_get_config(server)
    rs.check(st)
    # long sorts (a few ms each, copies included) on all eight streams, none
    # counted as "large" (which would keep them to three at a time), so the
    # short requests submitted right after them have to queue
    rs.check(rs.rs_server_set_config(server, dict(cfg, large_n=1 << 30)))
    busy = [(inputs.keys(np.uint64, "uniform", 1 << 23, seed=40 + i), None) for i in range(8)]
    short = [(inputs.keys(np.uint32, "gaussian", 3000 + 17 * i, seed=60 + i),
              inputs.values(np.uint32, 3000 + 17 * i)) for i in range(24)]
    # short 64-bit key requests batch as well (one batch per type)
    short += [(inputs.keys(np.uint64, "bucket", 5000 + 31 * i, seed=90 + i), None)
              for i in range(12)]
    out = run(server, busy + short)
    for r in out:
        ek, ev = oracle.lsd_sort(r.k, r.v)
        assert np.array_equal(r.ok, ek)
        if r.v is not None:
            assert np.array_equal(r.ov, ev)
    st, stats = rs.rs_server_stats(server)
    rs.check(st)
    assert stats["batches"] >= 2 and stats["batched_requests"] >= 2 * stats["batches"]
    st, trace = rs.rs_server_trace(server)
    rs.check(st)
    assert sum(t["batched"] for t in trace) == stats["batched_requests"]
    assert any(t["batched"] and t["key_bytes"] == 8 for t in trace)
    assert any(t["batched"] and t["key_bytes"] == 4 for t in trace)
    # alone: one short request on an idle server is not a batch
    rs.check(rs.rs_server_reset_stats(server))
    out = run(server, short[:1])
    assert np.array_equal(out[0].ok, oracle.lsd_sort(out[0].k, out[0].v)[0])
    st, stats = rs.rs_server_stats(server)
    rs.check(st)
    assert stats["batches"] == 0 and stats["completed"] == 1


def test_same_result_alone_and_in_the_mix():
    reqs = make_trace(60, seed=11, max_log2=17)
    st, alone_srv = rs.rs_server_create(1 << 30, 1)
    rs.check(st)
    try:
        alone = run(alone_srv, reqs, sequential=True)
    finally:
        rs.rs_server_destroy(alone_srv)
    # a tight budget and several streams: requests queue, batch and overlap
    st, mix_srv = rs.rs_server_create(48 << 20, 6)
    rs.check(st)
    try:
        mixed = run(mix_srv, reqs)
        st, stats = rs.rs_server_stats(mix_srv)
        assert stats["pool_peak_bytes"] <= 48 << 20
        assert stats["max_queued"] > 1
    finally:
        rs.rs_server_destroy(mix_srv)
    for a, m in zip(alone, mixed):
        assert np.array_equal(a.ok, m.ok)
        if a.v is not None:
            assert np.array_equal(a.ov, m.ov)


def test_rejections_and_cancel():
    st, srv = rs.rs_server_create(8 << 20, 1)
    rs.check(st)
    try:
        big = np.zeros(1 << 22, dtype=np.uint32)  # footprint > the whole 8 MiB budget
        r = Req(big, np.arange(big.size, dtype=np.uint32))
        assert rs.rs_submit(srv, r.c)[0] == rs.RS_ERR_INVALID
        bad = rs.rs_request(4, 8, 100, 0, 32, None, None, None, None)
        assert rs.rs_submit(srv, bad)[0] == rs.RS_ERR_INVALID
        # one stream, several requests: the later ones queue; cancel one
        reqs = [Req(inputs.keys(np.uint64, "uniform", 1 << 17, seed=s), None) for s in range(6)]
        handles = {}
        for i, q in enumerate(reqs):
            st, h = rs.rs_submit(srv, q.c)
            rs.check(st)
            handles[h] = i
        last = max(handles)
        c = rs.rs_cancel(srv, last)
        assert c in (rs.RS_OK, rs.RS_ERR_BUSY)
        status = wait_all(srv, handles)
        if c == rs.RS_OK:
            assert status[handles[last]] == rs.RS_ERR_CANCELLED
        assert rs.rs_poll(srv, last)[0] == rs.RS_ERR_NOT_FOUND
        for h, i in handles.items():
            if status[i] == rs.RS_OK:
                assert np.array_equal(reqs[i].ok, np.sort(reqs[i].k))
    finally:
        rs.rs_server_destroy(srv)


def test_config_policies_same_results():
    """Every scheduling policy gives the oracle's results: no batching, every
    request large with one at a time, large requests on default-priority
    streams, and copies through the shared copy queues."""
    reqs = make_trace(40, seed=21, max_log2=17)
    st, srv = rs.rs_server_create(1 << 30, 4)
    rs.check(st)
    try:
        st, cfg = rs.rs_server_get_config(srv)
        rs.check(st)
        assert cfg == {"batch_max_n": 1 << 14, "max_batch_keys": 1 << 22, "large_n": 1 << 21,
                       "max_large": 3, "large_low_priority": 1, "shared_copy_queues": 0}
        for bad in ({"batch_max_n": 1 << 23}, {"max_batch_keys": (1 << 30) + 1},
                    {"large_n": 0}, {"max_large": 0}, {"max_large": 65},
                    {"large_low_priority": 2}, {"shared_copy_queues": 2}):
            assert rs.rs_server_set_config(srv, dict(cfg, **bad)) == rs.RS_ERR_INVALID
        assert rs.rs_server_get_config(srv)[1] == cfg  # a rejected setting changes nothing
        for policy in ({"batch_max_n": 0},
                       {"large_n": 1, "max_large": 1},
                       {"large_n": 1 << 12, "large_low_priority": 0},
                       {"large_n": 1 << 12, "shared_copy_queues": 1}):
            rs.check(rs.rs_server_set_config(srv, dict(cfg, **policy)), "rs_server_set_config")
            rs.check(rs.rs_server_reset_stats(srv))
            out = run(srv, reqs)
            for r in out:
                ek, ev = oracle.lsd_sort(r.k, r.v)
                assert np.array_equal(r.ok, ek)
                if r.v is not None:
                    assert np.array_equal(r.ov, ev)
            st, stats = rs.rs_server_stats(srv)
            assert stats["completed"] == len(reqs)
            if policy.get("batch_max_n") == 0:
                assert stats["batches"] == 0
    finally:
        rs.rs_server_destroy(srv)


def test_completion_queue(server):
    """rs_server_completed hands out every finished request once, and
    rs_poll then reports its status."""
    reqs = make_trace(30, seed=5, max_log2=16)
    out = [Req(k, v) for k, v in reqs]
    handles = {}
    for i, r in enumerate(out):
        st, h = rs.rs_submit(server, r.c)
        rs.check(st, "rs_submit")
        handles[h] = i
    seen = []
    t0 = time.time()
    while len(seen) < len(handles):
        st, fin = rs.rs_server_completed(server, 7)
        rs.check(st, "rs_server_completed")
        assert len(fin) <= 7
        seen += fin
        if time.time() - t0 > 120:
            raise TimeoutError("requests not done")
        time.sleep(0.0005)
    assert sorted(seen) == sorted(handles)  # each exactly once
    for h in seen:
        assert rs.rs_poll(server, h) == (rs.RS_OK, True)
    assert rs.rs_server_completed(server, 8) == (rs.RS_OK, [])
    for r in out:
        assert np.array_equal(r.ok, oracle.lsd_sort(r.k, r.v)[0])
