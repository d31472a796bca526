"""Full-size parity: the single-instance workloads at their stated sizes, in
the launch configuration the benchmark times (default options, graph replay),
compared site by site with the oracle's union-find labels.

  honeycomb 256x256 cells (131,072 sites), p = 0.6527
  triangle 4096x4096 (16,777,216 sites), p = 0.3473
  Bethe z=3, 24 shells, random position (50,331,646 sites), p = 0.5
  triangle 16384x16384 (268,435,456 sites), p = 0.3473  (the largest served instance)

plus the largest input the int32 CSR allows: a triangle lattice whose
2,147,344,344 entries sit just under 2^31 - 1 (every entry, slot and bit
index near the top of its range).
"""
import numpy as np
import pytest
import torch

import lattices as L
import oracle
import paper_1603_08357_gb300 as ccl
from ccl_testutil import DEV, to_dev

pytestmark = pytest.mark.gpu

CASES = {
    "hc256": dict(kind="honeycomb", L=256, p=0.6527, seed=1),
    "tri4096": dict(kind="triangle", L=4096, p=0.3473, seed=2),
    "bethe24": dict(kind="cayley", z=3, shells=24, p=0.5, seed=3, perm_seed=3),
    "tri16384": dict(kind="triangle", L=16384, p=0.3473, seed=5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_full_size_matches_oracle(ctx, name):
    lat = L.make_instance(CASES[name])
    rp, ci, bits = to_dev(lat)
    out = torch.empty(lat.n, dtype=torch.int32, device=DEV)
    for _ in range(2):                       # first call captures, second replays the graph
        out.fill_(-1)
        assert ccl.ccl_label(ctx, lat.n, lat.nnz, rp, ci, bits, out) == ccl.CCL_OK
        assert ccl.ccl_sync(ctx) == ccl.CCL_OK
    got = out.cpu().numpy()
    del rp, ci, bits, out
    torch.cuda.empty_cache()
    want = oracle.uf_label(lat)
    assert np.array_equal(got, want), int(np.count_nonzero(got != want))
    if lat.kind == "cayley":
        # forest identity at full size: clusters = sites - open bonds
        assert np.count_nonzero(got == np.arange(lat.n)) == lat.n - lat.n_open_bonds


def test_maximum_csr_size(ctx):
    """Triangle 18918 x 18918: 357,890,724 sites and 6 L^2 = 2,147,344,344 CSR
    entries, the largest triangle lattice whose entry count fits int32."""
    Ls = 18918
    assert 6 * Ls * Ls < 2**31 - 1 < 6 * (Ls + 1) ** 2
    lat = L.triangle(Ls, 0.3473, 7)
    rp, ci, bits = to_dev(lat)
    out = torch.full((lat.n,), -1, dtype=torch.int32, device=DEV)
    assert ccl.ccl_label(ctx, lat.n, lat.nnz, rp, ci, bits, out) == ccl.CCL_OK
    assert ccl.ccl_sync(ctx) == ccl.CCL_OK
    got = out.cpu().numpy()
    assert ccl.ccl_get_stats(ctx).nnz == lat.nnz
    del rp, ci, bits, out
    torch.cuda.empty_cache()
    want = oracle.uf_label(lat)
    assert np.array_equal(got, want), int(np.count_nonzero(got != want))


def test_batched_mix_full_size_matches_oracle():
    """The whole batched workload: 4096 mixed honeycomb / triangle / Cayley
    instances (about 2.1e9 sites, 7.3e9 CSR entries) in one ccl_label_batched
    call with the autotuned settings (graph replay on the second call), every
    label against the union-find oracle run over all host cores; then the
    same batch through ccl_label_batched_host."""
    b = L.make_batch(L.batched_mix_specs(4096, seed=4))
    want, _ = oracle.uf_label_batched_threads(b)
    c = ccl.ccl_context_create(0)
    try:
        rp = torch.from_numpy(b.row_ptr).to(DEV)
        ci = torch.from_numpy(b.col_idx).to(DEV)
        bits = torch.from_numpy(b.open_bits.view(np.int32)).to(DEV)
        out = torch.empty(b.n_total, dtype=torch.int32, device=DEV)
        st, _ = ccl.ccl_autotune_batched(c, b.k, b.site_off, b.ent_off, rp, ci, bits, out)
        assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
        for _ in range(2):
            out.fill_(-1)
            assert ccl.ccl_label_batched(c, b.k, b.site_off, b.ent_off, rp, ci, bits, out) == ccl.CCL_OK
            assert ccl.ccl_sync(c) == ccl.CCL_OK
            got = out.cpu().numpy()
            bad = np.flatnonzero(got != want)
            assert bad.size == 0, f"{bad.size} labels differ, first at site {bad[0]}"
        del rp, ci, bits, out
        torch.cuda.empty_cache()
        h = np.full(b.n_total, -1, np.int32)
        st = ccl.ccl_label_batched_host(c, b.k, b.site_off, b.ent_off, b.row_ptr, b.col_idx, b.open_bits, h)
        assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
        assert np.array_equal(h, want)
    finally:
        ccl.ccl_context_destroy(c)
