"""GPU parity of the dense strided neighbour-list input (Section 3: slot k
of site i is nn[i + k*N]) against the oracle, on every lattice family, with
empty slots between used ones, widths past the register path, device-drawn
bonds, malformed slots and the degenerate sizes."""
import dataclasses

import numpy as np
import pytest
import torch

import lattices as L
import oracle
import paper_1603_08357_gb300 as ccl
from ccl_testutil import DEV

pytestmark = pytest.mark.gpu


def dense_dev(nn, bits):
    return (torch.from_numpy(np.ascontiguousarray(nn, np.int32)).to(DEV),
            torch.from_numpy(np.ascontiguousarray(bits, np.uint32).view(np.int32)).to(DEV))


def gpu_dense(ctx, n, W, nn, bits, expect=ccl.CCL_OK):
    d_nn, d_bits = dense_dev(nn if W else np.zeros(1, np.int32), bits)
    out = torch.full((max(n, 1),), -7, dtype=torch.int32, device=DEV)
    st = ccl.ccl_label_dense(ctx, n, W, d_nn if W else None, d_bits if W else None, out)
    assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
    st = ccl.ccl_sync(ctx)
    assert st == expect, ccl.ccl_status_string(st)
    return out[:n].cpu().numpy()


CASES = [
    ("triangle", dict(L=301, p=L.PC_TRIANGLE, seed=1)),
    ("honeycomb", dict(L=150, p=L.PC_HONEYCOMB, seed=2, periodic_y=False)),
    ("cayley", dict(z=3, shells=15, p=0.5, seed=3, perm_seed=3)),
    ("cayley", dict(z=5, shells=7, p=0.25, seed=4)),
    ("square", dict(L=333, p=0.5, seed=5)),
    ("cubic", dict(L=47, p=L.PC_CUBIC, seed=6, periodic_y=False)),
]


@pytest.mark.parametrize("kind,kw", CASES)
@pytest.mark.parametrize("slot_seed,extra", [(None, 0), (11, 0), (12, 6)])
def test_dense_matches_oracle(ctx, kind, kw, slot_seed, extra):
    lat = L.make_instance(dict(kind=kind, **kw))
    W, nn, bits = L.to_dense(lat, int(np.diff(lat.row_ptr).max()) + extra, slot_seed)
    want = oracle.dense_uf_label(lat.n, W, nn, bits)
    assert np.array_equal(want, oracle.uf_label(lat))
    assert np.array_equal(gpu_dense(ctx, lat.n, W, nn, bits), want)


@pytest.mark.parametrize("p", [0.0, 0.3, 0.7, 1.0])
def test_dense_multigraph(ctx, p):
    lat = L.random_graph(20000, 45000, 9, self_loops=True, asymmetric=0.0)
    lat = dataclasses.replace(lat, open_bits=oracle.keyed_bits(lat, 5, p))
    for slot_seed in (None, 1):
        W, nn, bits = L.to_dense(lat, None, slot_seed)
        assert np.array_equal(gpu_dense(ctx, lat.n, W, nn, bits), oracle.dense_uf_label(lat.n, W, nn, bits))


@pytest.mark.parametrize("kind,kw", CASES[:2] + CASES[4:])
def test_dense_random_matches_oracle_and_csr(ctx, kind, kw):
    lat = L.make_instance(dict(kind=kind, **kw))
    W, nn, _ = L.to_dense(lat, None, 21)
    d_nn, _ = dense_dev(nn, np.zeros(1, np.uint32))
    rp = torch.from_numpy(lat.row_ptr).to(DEV)
    ci = torch.from_numpy(lat.col_idx).to(DEV)
    for seed, p in ((3, kw["p"]), (2**64 - 5, 0.9 * kw["p"])):
        want = oracle.dense_uf_label(lat.n, W, nn, oracle.dense_keyed_bits(lat.n, W, nn, seed, p))
        out = torch.empty(lat.n, dtype=torch.int32, device=DEV)
        assert ccl.ccl_label_dense_random(ctx, lat.n, W, d_nn, seed, p, out) == ccl.CCL_OK
        assert ccl.ccl_sync(ctx) == ccl.CCL_OK
        assert np.array_equal(out.cpu().numpy(), want)
        out2 = torch.empty(lat.n, dtype=torch.int32, device=DEV)
        assert ccl.ccl_label_random(ctx, lat.n, lat.nnz, rp, ci, seed, p, out2) == ccl.CCL_OK
        assert ccl.ccl_sync(ctx) == ccl.CCL_OK
        assert np.array_equal(out2.cpu().numpy(), want)      # same realisation from CSR input


def test_dense_degenerate(ctx):
    # width 0: every site alone
    assert np.array_equal(gpu_dense(ctx, 1000, 0, None, np.zeros(1, np.uint32)), np.arange(1000))
    # one site; all slots empty; ragged n (not a multiple of 32 or of a tile)
    assert gpu_dense(ctx, 1, 3, np.full(3, -1, np.int32), np.full(1, 0xFFFFFFFF, np.uint32)).tolist() == [0]
    lat = L.triangle(37, 0.6, 3)                      # 1369 sites
    W, nn, bits = L.to_dense(lat)
    assert np.array_equal(gpu_dense(ctx, lat.n, W, nn, bits), oracle.uf_label(lat))
    # n == 0 does nothing
    assert ccl.ccl_label_dense(ctx, 0, 4, None, None, None) == ccl.CCL_OK
    # argument errors are reported before any launch
    t = torch.zeros(8, dtype=torch.int32, device=DEV)
    assert ccl.ccl_label_dense(ctx, 4, -1, t, t, t) == ccl.CCL_ERR_INVALID_ARGUMENT
    assert ccl.ccl_label_dense(ctx, 4, ccl.CCL_DENSE_MAX_WIDTH + 1, t, t, t) == ccl.CCL_ERR_INVALID_ARGUMENT
    assert ccl.ccl_label_dense(ctx, 4, 2, None, t, t) == ccl.CCL_ERR_INVALID_ARGUMENT
    assert ccl.ccl_label_dense_random(ctx, 4, 2, t, 1, -0.5, t) == ccl.CCL_ERR_INVALID_ARGUMENT


@pytest.mark.parametrize("bad", [-2, 1000, 2**31 - 1])
def test_dense_bad_slot_is_reported(ctx, bad):
    lat = L.square(30, 0.5, 1)
    W, nn, bits = L.to_dense(lat)
    nn = nn.copy()
    nn[17 + 2 * lat.n] = bad
    gpu_dense(ctx, lat.n, W, nn, bits, expect=ccl.CCL_ERR_INDEX_OUT_OF_RANGE)
    # the context stays usable
    W, nn, bits = L.to_dense(lat)
    assert np.array_equal(gpu_dense(ctx, lat.n, W, nn, bits), oracle.uf_label(lat))


def test_dense_graph_replay_and_wide_rows(ctx):
    """Repeated identical calls replay a graph; a width past the register
    path (12 slots, 6 used) takes the general scan."""
    lat = L.cubic(40, 0.3, 8)
    W, nn, bits = L.to_dense(lat, 12, 4)
    want = oracle.dense_uf_label(lat.n, W, nn, bits)
    d_nn, d_bits = dense_dev(nn, bits)
    out = torch.empty(lat.n, dtype=torch.int32, device=DEV)
    for _ in range(3):
        out.fill_(-1)
        assert ccl.ccl_label_dense(ctx, lat.n, W, d_nn, d_bits, out) == ccl.CCL_OK
        assert ccl.ccl_sync(ctx) == ccl.CCL_OK
        assert np.array_equal(out.cpu().numpy(), want)
    assert ccl.ccl_get_stats(ctx).used_graph == 1


def test_dense_full_size_triangle(ctx):
    """The 4096^2 triangle lattice at p_c as a dense list, site by site."""
    lat = L.triangle(4096, 0.3473, 2)
    W, nn, bits = L.to_dense(lat)
    assert np.array_equal(gpu_dense(ctx, lat.n, W, nn, bits), oracle.uf_label(lat))


def _chorded_ring(n, chords, p, seed):
    """Ring i -- i+1 plus chords i -- i+c (periodic), bonds open with
    probability p; degree at most 2 + 2 * len(chords)."""
    rng = np.random.default_rng(seed)
    i = np.arange(n)
    us = [i] + [i for _ in chords]
    vs = [(i + 1) % n] + [(i + c) % n for c in chords]
    u = np.concatenate(us); v = np.concatenate(vs)
    keep = u != v
    u, v = u[keep], v[keep]
    op = rng.random(len(u)) < p
    rows = np.concatenate([u, v]); cols = np.concatenate([v, u]); bitv = np.concatenate([op, op])
    order = np.argsort(rows, kind="stable")
    rows, cols, bitv = rows[order], cols[order], bitv[order]
    rp = np.zeros(n + 1, np.int64); np.add.at(rp, rows + 1, 1)
    return L.Lattice("ring", n, len(cols), np.cumsum(rp).astype(np.int32), cols.astype(np.int32),
                     L.pack_bits(bitv), p, seed)


@pytest.mark.parametrize("W", [1, 2, 7, 8, 9])
@pytest.mark.parametrize("n", [1, 31, 1025, 70001])
def test_dense_width_boundaries(ctx, W, n):
    """Widths at the edges of the dense kernels (8 is the widest the staged
    kernel takes, 9 the narrowest of the general one), used slots scattered
    over the row, ragged site counts."""
    if W == 1:                                              # a matching: degree 1
        i = np.arange(0, n - 1, 2)
        u, v = i, i + 1
        op = np.random.default_rng(W + n).random(len(u)) < 0.6
        rows = np.concatenate([u, v]); cols = np.concatenate([v, u]); bitv = np.concatenate([op, op])
        order = np.argsort(rows, kind="stable")
        rp = np.zeros(n + 1, np.int64); np.add.at(rp, rows[order] + 1, 1)
        lat = L.Lattice("matching", n, len(cols), np.cumsum(rp).astype(np.int32),
                        cols[order].astype(np.int32), L.pack_bits(bitv[order]), 0.6, 0)
    else:
        lat = _chorded_ring(n, [7, 13][: (W - 2) // 2] if W >= 4 else [], 0.45, W * 1000 + n)
    deg = int(np.diff(lat.row_ptr).max()) if lat.n else 0
    assert deg <= W
    for slot_seed in (None, 3):
        Wd, nn, bits = L.to_dense(lat, W, slot_seed)
        assert Wd == W
        want = oracle.dense_uf_label(lat.n, W, nn, bits)
        assert np.array_equal(want, oracle.uf_label(lat))
        assert np.array_equal(gpu_dense(ctx, lat.n, W, nn, bits), want)
