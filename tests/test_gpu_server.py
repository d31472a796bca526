"""The request loop (continuous batching): requests submitted while others are
on the GPU are admitted as memory frees up, batched and labelled; every result
must equal the oracle's and the result of the same request labelled alone."""
import ctypes
import threading
import time

import numpy as np
import pytest

import lattices as L
import oracle
import paper_1603_08357_gb300 as ccl

pytestmark = pytest.mark.gpu


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        t = int(rng.integers(0, 3))
        if t == 0:
            lat = L.honeycomb(int(rng.integers(2, 90)), L.PC_HONEYCOMB, 100 + r)
        elif t == 1:
            lat = L.triangle(int(rng.integers(2, 120)), L.PC_TRIANGLE, 100 + r)
        else:
            lat = L.cayley(3, int(rng.integers(1, 12)), 0.5, 100 + r, perm_seed=r)
        out.append(lat)
    return out


def _submit(srv, lat):
    st, ticket = ccl.ccl_server_submit(srv, lat.n, lat.nnz, lat.row_ptr, lat.col_idx, lat.open_bits)
    assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
    return ticket


def _wait(srv, ticket, n):
    out = np.full(n, -1, np.int32)
    st = ccl.ccl_server_wait(srv, ticket, out, 60_000)
    assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
    return out


def test_mixed_stream_matches_alone_and_oracle():
    reqs = _requests(300, 7)
    srv = ccl.ccl_server_create(0, n_streams=3, max_batch=64)
    try:
        # alone: one request in flight at a time
        alone = [_wait(srv, _submit(srv, lat), lat.n) for lat in reqs[:40]]
        # in the mix: everything submitted from two threads, then collected
        tickets = [None] * len(reqs)

        def feed(idx):
            for k in idx:
                tickets[k] = _submit(srv, reqs[k])
                time.sleep(0.0002)
        th = [threading.Thread(target=feed, args=(range(s, len(reqs), 2),)) for s in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        mixed = [_wait(srv, tickets[k], reqs[k].n) for k in range(len(reqs))]
        stats = ccl.ccl_server_stats_get(srv)
    finally:
        srv.close()
    for k, lat in enumerate(reqs):
        want = oracle.uf_label(lat)
        assert np.array_equal(mixed[k], want), k
        if k < len(alone):
            assert np.array_equal(alone[k], mixed[k])
    assert stats.completed == 340 and stats.rejected == 0
    assert stats.batches < stats.completed          # requests were batched together
    assert 0 < stats.p50_ms <= stats.p99_ms <= stats.max_ms


def test_rejection_and_unknown_ticket():
    srv = ccl.ccl_server_create(0, n_streams=1, hbm_budget=1 << 20)
    try:
        big = L.triangle(400, 0.3, 1)                      # needs more than 1 MiB on the device
        st, _ = ccl.ccl_server_submit(srv, big.n, big.nnz, big.row_ptr, big.col_idx, big.open_bits)
        assert st == ccl.CCL_ERR_REJECTED
        small = L.triangle(8, 0.5, 2)
        t = _submit(srv, small)
        assert np.array_equal(_wait(srv, t, small.n), oracle.uf_label(small))
        assert ccl.ccl_server_wait(srv, 987654, None, 10) == ccl.CCL_ERR_NOT_FOUND
        assert ccl.ccl_server_stats_get(srv).rejected == 1
    finally:
        srv.close()


def test_admission_waits_for_memory():
    """A budget that holds only a few requests at a time: later requests wait
    for earlier ones to finish, and all complete correctly."""
    reqs = [L.triangle(150, L.PC_TRIANGLE, s) for s in range(24)]
    one = 4 * (reqs[0].n + 1) + 4 * reqs[0].nnz + 8 * reqs[0].nnz + 4 * reqs[0].n
    srv = ccl.ccl_server_create(0, n_streams=2, hbm_budget=3 * one)
    try:
        tickets = [_submit(srv, lat) for lat in reqs]
        outs = [_wait(srv, t, lat.n) for t, lat in zip(tickets, reqs)]
    finally:
        srv.close()
    for lat, got in zip(reqs, outs):
        assert np.array_equal(got, oracle.uf_label(lat))


def test_wait_timeout_keeps_the_ticket():
    """A wait that times out leaves the ticket pending; a later wait returns
    the labels."""
    lat = L.triangle(1500, L.PC_TRIANGLE, 9)
    srv = ccl.ccl_server_create(0, n_streams=1)
    try:
        t = _submit(srv, lat)
        out = np.full(lat.n, -1, np.int32)
        st = ccl.ccl_server_wait(srv, t, out, 0)
        assert st in (ccl.CCL_OK, ccl.CCL_ERR_TIMEOUT)
        if st == ccl.CCL_ERR_TIMEOUT:
            assert np.array_equal(_wait(srv, t, lat.n), oracle.uf_label(lat))
        else:
            assert np.array_equal(out, oracle.uf_label(lat))
            assert ccl.ccl_server_wait(srv, t, out, 0) == ccl.CCL_ERR_NOT_FOUND
    finally:
        ccl.ccl_server_destroy(srv)


def test_nocopy_requests_match_oracle():
    """Requests submitted without a copy (arrays kept alive by the caller),
    mixed with copied ones, give the oracle's labels."""
    reqs = _requests(120, 13)
    srv = ccl.ccl_server_create(0, n_streams=2, max_batch=32)
    try:
        tickets = []
        for k, lat in enumerate(reqs):
            if k % 2:
                st, t = ccl.ccl_server_submit_nocopy(srv, lat.n, lat.nnz, lat.row_ptr, lat.col_idx, lat.open_bits)
                assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
            else:
                t = _submit(srv, lat)
            tickets.append(t)
        for t, lat in zip(tickets, reqs):
            assert np.array_equal(_wait(srv, t, lat.n), oracle.uf_label(lat))
    finally:
        ccl.ccl_server_destroy(srv)


def test_destroy_with_waiters_blocked():
    """ccl_server_destroy while other threads wait on their tickets: every
    wait returns, either with the oracle's labels (labelled before the stop)
    or CCL_ERR_REJECTED with its output untouched (dropped), and destroy
    returns only after the waiters have left."""
    lat = L.triangle(2000, L.PC_TRIANGLE, 21)
    want = oracle.uf_label(lat)
    srv = ccl.ccl_server_create(0, n_streams=1, max_batch=1)
    tickets = []
    for _ in range(128):
        st, t = ccl.ccl_server_submit_nocopy(srv, lat.n, lat.nnz, lat.row_ptr, lat.col_idx, lat.open_bits)
        assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
        tickets.append(t)
    watched = tickets[:4] + tickets[-28:]      # the last ones are labelled last
    outs = [np.full(lat.n, -1, np.int32) for _ in watched]
    status = [None] * len(watched)
    class Handle:       # the raw handle: srv.close() clears srv's own
        _as_parameter_ = ctypes.c_void_p(srv.handle)

    def waiter(k):
        status[k] = ccl.ccl_server_wait(Handle, watched[k], outs[k], 60_000)

    threads = [threading.Thread(target=waiter, args=(k,)) for k in range(len(watched))]
    for th in threads:
        th.start()
    # destroy may only overlap waits already in progress: wait until every
    # thread is inside ccl_server_wait (or already returned)
    deadline = time.monotonic() + 10
    while ccl.ccl_server_stats_get(srv).waiting + sum(s is not None for s in status) < len(watched):
        assert time.monotonic() < deadline
        time.sleep(0.0005)
    srv.close()
    for th in threads:
        th.join(timeout=10)
        assert not th.is_alive()
    dropped = 0
    for st, out in zip(status, outs):
        if st == ccl.CCL_OK:
            assert np.array_equal(out, want)
        else:
            assert st == ccl.CCL_ERR_REJECTED, ccl.ccl_status_string(st)
            assert (out == -1).all()
            dropped += 1
    assert dropped >= 1


def test_empty_and_edgeless_requests():
    """Requests with no sites and with sites but no entries, mixed with
    ordinary ones, copied and not copied."""
    empty = L.Lattice("e", 0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(1, np.uint32), 0, 0)
    isolated = L.Lattice("i", 77, 0, np.zeros(78, np.int32), np.zeros(0, np.int32), np.zeros(1, np.uint32), 0, 0)
    reqs = [empty, L.triangle(50, L.PC_TRIANGLE, 1), isolated, empty, L.honeycomb(40, L.PC_HONEYCOMB, 2), isolated]
    srv = ccl.ccl_server_create(0, n_streams=2, max_batch=4)
    try:
        tickets = []
        for k, lat in enumerate(reqs):
            submit = ccl.ccl_server_submit if k % 2 else ccl.ccl_server_submit_nocopy
            st, t = submit(srv, lat.n, lat.nnz, lat.row_ptr, lat.col_idx if lat.nnz else lat.row_ptr,
                           lat.open_bits)
            assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
            tickets.append(t)
        for t, lat in zip(tickets, reqs):
            out = np.full(max(lat.n, 1), -1, np.int32)
            st = ccl.ccl_server_wait(srv, t, out, 60_000)
            assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
            assert np.array_equal(out[:lat.n], oracle.uf_label(lat))
    finally:
        srv.close()


def test_failed_batch_launch_is_reported(monkeypatch):
    """A batch whose launch fails (here its first launch, made to fail by the
    server's test hook as a failed workspace allocation would) ends its
    request with that error, not with CCL_OK and unwritten labels; the server
    then labels the next request correctly."""
    monkeypatch.setenv("CCL_SERVER_FAIL_BATCH", "1")
    srv = ccl.ccl_server_create(0, n_streams=1, max_batch=8)
    monkeypatch.delenv("CCL_SERVER_FAIL_BATCH")
    try:
        lat = L.triangle(64, L.PC_TRIANGLE, 5)
        out = np.full(lat.n, -1, np.int32)
        st = ccl.ccl_server_wait(srv, _submit(srv, lat), out, 60_000)
        assert st == ccl.CCL_ERR_OUT_OF_MEMORY, ccl.ccl_status_string(st)
        assert np.array_equal(_wait(srv, _submit(srv, lat), lat.n), oracle.uf_label(lat))
    finally:
        ccl.ccl_server_destroy(srv)


def test_kept_workspace_is_counted_and_freed():
    """The workspace a context keeps after a large batch counts against the
    budget; when it alone blocks the next request, the idle context frees it
    and the request is labelled (a budget that fits one large request's
    buffer and workspace share, but not that plus the workspace kept from the
    previous batch)."""
    big = L.triangle(1024, L.PC_TRIANGLE, 6)
    nnz = big.nnz
    per_req = 4 * (big.n + 1) + 4 * nnz + 4 * ((nnz + 31) // 32) + 4 * big.n + 4 * 256 + 12 * nnz
    srv = ccl.ccl_server_create(0, n_streams=2, max_batch=1, hbm_budget=int(per_req * 1.2))
    try:
        want = oracle.uf_label(big)
        for _ in range(4):      # each request after the first needs the kept workspace freed
            assert np.array_equal(_wait(srv, _submit(srv, big), big.n), want)
    finally:
        ccl.ccl_server_destroy(srv)
