"""ccl_label_noalloc, the allocation-free entry point, against ccl_label.

Some callers cannot allocate device memory while they run (a latency-bound
loop that cannot absorb cudaMalloc's device-wide synchronisation, or a
process whose device memory belongs to another allocator). The entry point
serves them from one fixed device array inside the library. This file is
named so that pytest collects it last; it passes alone in a fresh process and
after the other tests.
"""
import numpy as np
import pytest
import torch

import lattices as L
import oracle
import paper_1603_08357_gb300 as ccl
from ccl_testutil import DEV, gpu_label, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(lat):
    rp, ci, bits = to_dev(lat)
    out = torch.full((lat.n,), -5, dtype=torch.int32, device=DEV)
    st = ccl.ccl_label_noalloc(lat.n, lat.nnz, rp, ci, bits, out)
    assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
    return out.cpu().numpy()


def test_noalloc_matches_ccl_label_twice(ctx):
    lats = [L.triangle(500, L.PC_TRIANGLE, 3), L.cayley(3, 15, 0.5, 4, perm_seed=5),
            L.honeycomb(256, L.PC_HONEYCOMB, 1)]
    for lat in lats:
        want = gpu_label(ctx, lat)
        # two calls in a row: the shared scratch keeps the previous call's contents
        first = _noalloc(lat)
        second = _noalloc(lat)
        assert np.array_equal(first, want)
        assert np.array_equal(second, want)
        assert np.array_equal(first, oracle.uf_label(lat))


def test_noalloc_allocates_nothing_after_the_first_call():
    """After the first call on the device (which loads the library's device
    code and with it the fixed array), further calls leave the device's free
    memory unchanged: every buffer here exists before the calls."""
    lat = L.triangle(560, L.PC_TRIANGLE, 8)     # 1,881,600 entries, within the limit
    rp, ci, bits = to_dev(lat)
    out = torch.full((lat.n,), -5, dtype=torch.int32, device=DEV)
    assert ccl.ccl_label_noalloc(lat.n, lat.nnz, rp, ci, bits, out) == ccl.CCL_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        out.fill_(-5)
        assert ccl.ccl_label_noalloc(lat.n, lat.nnz, rp, ci, bits, out) == ccl.CCL_OK
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(out.cpu().numpy(), oracle.uf_label(lat))


def test_noalloc_at_its_limit():
    """Exactly 2^21 CSR entries (the largest input its scratch holds): the
    oracle's labels."""
    rng = np.random.default_rng(21)
    n, m = 400000, 1 << 20
    u = rng.integers(0, n, m); v = rng.integers(0, n, m)
    op = rng.random(m) < 0.5
    rows = np.concatenate([u, v]); cols = np.concatenate([v, u]); bitv = np.concatenate([op, op])
    order = np.argsort(rows, kind="stable")
    rp = np.zeros(n + 1, np.int64); np.add.at(rp, rows[order] + 1, 1)
    lat = L.Lattice("random", n, len(cols), np.cumsum(rp).astype(np.int32), cols[order].astype(np.int32),
                    L.pack_bits(bitv[order]), 0.5, 21)
    assert lat.nnz == 1 << 21
    assert np.array_equal(_noalloc(lat), oracle.uf_label(lat))


def test_noalloc_rejects_beyond_its_scratch():
    big_nnz = (1 << 21) + 1
    st = ccl.ccl_label_noalloc(10, big_nnz, 0, 0, 0, 0)
    assert st == ccl.CCL_ERR_INVALID_ARGUMENT
