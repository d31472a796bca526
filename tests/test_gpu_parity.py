"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Labels are integers and canonical (smallest site of the cluster, Section 3),
so the bar is bit-exact equality on every site. Inputs are the seeded
generator's lattices and random multigraphs; sizes span many 32-site chunks
with ragged tails, the staged and the direct row paths, empty and degenerate
inputs. The residual-pair count of step (i) is compared with the oracle's
sequential run of Section 3.
"""
import numpy as np
import pytest
import torch

import lattices as L
import oracle
import paper_1603_08357_gb300 as ccl
from ccl_testutil import DEV, gpu_label, gpu_label_batched, to_dev
from conftest import load_golden

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["worked_example.txt", "row_max_rule.txt", "duplicate_min.txt"])
def test_golden(ctx, name):
    g = load_golden(name)
    rp = np.array(g["row_ptr"], np.int32)
    lat = L.Lattice("golden", g["n"][0], int(rp[-1]), rp, np.array(g["col_idx"], np.int32),
                    L.pack_bits(np.array(g["open"], bool)), 0.0, 0)
    assert gpu_label(ctx, lat).tolist() == g["label"]
    st = ccl.ccl_get_stats(ctx)
    assert st.residual_pairs == sum(len(v) for v in g.get("residual", {}).values())


@pytest.mark.parametrize("seed", range(40))
def test_random_multigraphs(ctx, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.choice([1, 2, 31, 32, 33, 64, 65, 200, 1000, 4097]))
    m = int(rng.integers(0, 3 * n + 2))
    lat = L.random_graph(n, m, 500 + seed, asymmetric=0.3 if seed % 3 == 0 else 0.0,
                         p=float(rng.uniform(0.2, 0.9)))
    want = oracle.uf_label(lat)
    assert np.array_equal(gpu_label(ctx, lat), want)
    assert ccl.ccl_get_stats(ctx).residual_pairs == oracle.steps_label(lat)["n_residual"]


def test_heavy_rows_direct_path(ctx):
    """A hub of degree 5000 and chunks with more than 256 entries take the
    unstaged path of step (i)."""
    n = 6000
    hub_edges = [(5999, j) for j in range(0, 5000)]
    rng = np.random.default_rng(3)
    extra = [(int(a), int(b)) for a, b in rng.integers(0, n, (3000, 2))]
    edges = hub_edges + extra
    u = np.array([a for a, b in edges]); v = np.array([b for a, b in edges])
    op = rng.random(len(edges)) < 0.5
    rows = np.concatenate([u, v]); cols = np.concatenate([v, u]); bitv = np.concatenate([op, op])
    order = np.argsort(rows, kind="stable")
    rows, cols, bitv = rows[order], cols[order], bitv[order]
    rp = np.zeros(n + 1, np.int64); np.add.at(rp, rows + 1, 1); rp = np.cumsum(rp).astype(np.int32)
    lat = L.Lattice("hub", n, len(cols), rp, cols.astype(np.int32), L.pack_bits(bitv), 0.5, 0)
    assert np.array_equal(gpu_label(ctx, lat), oracle.uf_label(lat))


def _csr_from_edges(n, u, v, op):
    rows = np.concatenate([u, v]); cols = np.concatenate([v, u]); bitv = np.concatenate([op, op])
    order = np.argsort(rows, kind="stable")
    rows, cols, bitv = rows[order], cols[order], bitv[order]
    rp = np.zeros(n + 1, np.int64); np.add.at(rp, rows + 1, 1); rp = np.cumsum(rp).astype(np.int32)
    return L.Lattice("edges", n, len(cols), rp, cols.astype(np.int32), L.pack_bits(bitv), 0.5, 0)


@pytest.mark.parametrize("hub_degrees", [(20000,), (9000, 9000, 40)])
def test_tile_entries_beyond_one_stage(ctx, hub_degrees):
    """Tiles whose CSR entries exceed what one shared-memory stage holds
    (7168 columns): the stage holds part of the range, the rest is read from
    global memory, and every row of the tile takes the bounds-checked path."""
    n = 50000
    rng = np.random.default_rng(sum(hub_degrees))
    us, vs = [], []
    for h, deg in enumerate(hub_degrees):
        hub = 1500 + 3 * h                          # hubs share one 1024-site tile
        nb = rng.choice(np.delete(np.arange(n), hub), deg, replace=False)
        us.append(np.full(deg, hub)); vs.append(nb)
    ring = np.arange(n - 1)
    us.append(ring); vs.append(ring + 1)
    u = np.concatenate(us); v = np.concatenate(vs)
    op = rng.random(len(u)) < 0.35
    lat = _csr_from_edges(n, u, v, op)
    tile = lat.row_ptr[2048] - lat.row_ptr[1024]
    assert tile > 7168
    assert np.array_equal(gpu_label(ctx, lat), oracle.uf_label(lat))
    assert ccl.ccl_get_stats(ctx).residual_pairs == oracle.steps_label(lat)["n_residual"]


def test_tile_entries_beyond_one_stage_batched(ctx):
    """The same overflowing tile inside a batch, after an instance whose entry
    count leaves the hub instance's bits starting mid-word (bit offset not a
    multiple of 32)."""
    from ccl_testutil import gpu_label_batched
    rng = np.random.default_rng(11)
    n = 30000
    nb = rng.choice(np.delete(np.arange(n), 1500), 15000, replace=False)
    ring = np.arange(n - 1)
    u = np.concatenate([np.full(15000, 1500), ring]); v = np.concatenate([nb, ring + 1])
    hub = _csr_from_edges(n, u, v, rng.random(len(u)) < 0.4)
    lats = [L.random_graph(37, 29, 5, p=0.6), hub, L.triangle(33, L.PC_TRIANGLE, 6)]
    assert lats[0].nnz % 32 != 0
    K = len(lats)
    site_off = np.zeros(K + 1, np.int64); site_off[1:] = np.cumsum([x.n for x in lats])
    ent_off = np.zeros(K + 1, np.int64); ent_off[1:] = np.cumsum([x.nnz for x in lats])
    row_ptr = np.concatenate([x.row_ptr for x in lats]).astype(np.int32)
    col_idx = np.concatenate([x.col_idx for x in lats]).astype(np.int32)
    bitv = np.concatenate([L.unpack_bits(x.open_bits, x.nnz) for x in lats])
    b = L.Batch(site_off, ent_off, row_ptr, col_idx, L.pack_bits(bitv), [{"kind": "edges"}] * K)
    got = gpu_label_batched(ctx, b)
    for k, x in enumerate(lats):
        assert np.array_equal(got[int(site_off[k]):int(site_off[k + 1])], oracle.uf_label(x)), k
    assert ccl.ccl_get_stats(ctx).residual_pairs == sum(oracle.steps_label(x)["n_residual"] for x in lats)


def _lattice_cases():
    out = []
    for p in [0.0, 0.25, None, 0.75, 1.0]:
        out.append(("honeycomb", dict(L=37), p))
        out.append(("triangle", dict(L=45), p))
        out.append(("cayley", dict(z=3, shells=11, perm_seed=None), p))
        out.append(("cayley", dict(z=4, shells=7, perm_seed=5), p))
    out.append(("triangle", dict(L=200, periodic_y=False), None))
    out.append(("honeycomb", dict(L=150, periodic_y=False), None))
    return out


@pytest.mark.parametrize("kind,kw,p", _lattice_cases())
def test_lattices(ctx, kind, kw, p):
    if p is None:
        p = {"honeycomb": L.PC_HONEYCOMB, "triangle": L.PC_TRIANGLE}.get(kind) or 1.0 / (kw["z"] - 1)
    spec = dict(kind=kind, p=p, seed=77, **kw)
    lat = L.make_instance(spec)
    want = oracle.uf_label(lat)
    got = gpu_label(ctx, lat)
    assert np.array_equal(got, want)
    assert ccl.ccl_get_stats(ctx).residual_pairs == oracle.steps_label(lat)["n_residual"]


@pytest.mark.parametrize("z,S", [(3, 14), (5, 7)])
def test_standard_bethe_has_no_residual_pairs(ctx, z, S):
    for p in (0.3, 1.0 / (z - 1), 0.9):
        lat = L.cayley(z, S, p, 9)
        assert np.array_equal(gpu_label(ctx, lat), oracle.uf_label(lat))
        assert ccl.ccl_get_stats(ctx).residual_pairs == 0


@pytest.mark.parametrize("threads", [64, 128, 256, 512])
@pytest.mark.parametrize("pre", [0, 1])
@pytest.mark.parametrize("link", [0, 1])
@pytest.mark.parametrize("refill", [0, 1])
@pytest.mark.parametrize("order", [0, 1])
def test_launch_options_same_labels(threads, pre, link, refill, order):
    c = ccl.ccl_context_create(0)
    try:
        for opt, val in ((ccl.CCL_OPT_BLOCK_THREADS, threads), (ccl.CCL_OPT_PRE_ANALYSIS, pre),
                         (ccl.CCL_OPT_LINK_MODE, link), (ccl.CCL_OPT_REFILL, refill),
                         (ccl.CCL_OPT_ANALYSIS_ORDER, order),
                         (ccl.CCL_OPT_CTAS_PER_SM, 1 if threads == 64 else 0)):
            assert ccl.ccl_set_option(c, opt, val) == ccl.CCL_OK
        lat = L.triangle(300, 0.52, 11)
        want = oracle.uf_label(lat)
        for graphs in (0, 1):
            ccl.ccl_set_option(c, ccl.CCL_OPT_USE_GRAPHS, graphs)
            for _ in range(2):
                assert np.array_equal(gpu_label(c, lat), want)
    finally:
        ccl.ccl_context_destroy(c)


def test_profile_step_times(ctx):
    lat = L.triangle(512, L.PC_TRIANGLE, 5)
    ccl.ccl_set_option(ctx, ccl.CCL_OPT_PROFILE, 1)
    try:
        assert np.array_equal(gpu_label(ctx, lat), oracle.uf_label(lat))
        t = ccl.ccl_get_step_times(ctx)
        assert len(t) == 5 and all(v >= 0 for v in t) and t[0] > 0 and t[4] == 1
    finally:
        ccl.ccl_set_option(ctx, ccl.CCL_OPT_PROFILE, 0)


def test_edge_cases(ctx):
    empty = L.Lattice("e", 0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(1, np.uint32), 0, 0)
    assert gpu_label(ctx, empty).size == 0
    iso = L.Lattice("iso", 70, 0, np.zeros(71, np.int32), np.zeros(0, np.int32), np.zeros(1, np.uint32), 0, 0)
    assert np.array_equal(gpu_label(ctx, iso), np.arange(70))
    one = L.Lattice("one", 1, 2, np.array([0, 2], np.int32), np.array([0, 0], np.int32),
                    np.array([3], np.uint32), 0, 0)
    assert gpu_label(ctx, one).tolist() == [0]
    assert ccl.ccl_label(ctx, -1, 0, 0, 0, 0, 0) == ccl.CCL_ERR_INVALID_ARGUMENT
    assert ccl.ccl_label(ctx, 5, 0, None, None, None, None) == ccl.CCL_ERR_INVALID_ARGUMENT


def test_kernel_checks_report_bad_input(ctx):
    """Out-of-range indices and inconsistent row pointers are caught by the
    kernels' own bounds checks and reported by ccl_sync; the bad entries are
    skipped, never dereferenced."""
    lat = L.triangle(40, 0.5, 1)
    ci = lat.col_idx.copy(); ci[100] = lat.n + 5; ci[2000] = -3
    bad = L.Lattice("bad", lat.n, lat.nnz, lat.row_ptr, ci, lat.open_bits, 0.5, 0)
    gpu_label(ctx, bad, expect_status=ccl.CCL_ERR_INDEX_OUT_OF_RANGE)
    rp = lat.row_ptr.copy(); rp[500] = rp[502]      # rows no longer monotone
    bad = L.Lattice("bad", lat.n, lat.nnz, rp, lat.col_idx, lat.open_bits, 0.5, 0)
    gpu_label(ctx, bad, expect_status=ccl.CCL_ERR_INDEX_OUT_OF_RANGE)
    bad = L.Lattice("bad", lat.n, lat.nnz - 6, lat.row_ptr, lat.col_idx, lat.open_bits, 0.5, 0)
    got = gpu_label(ctx, bad, expect_status=ccl.CCL_ERR_INDEX_OUT_OF_RANGE)
    assert got.shape == (lat.n,)
    # the context is usable afterwards
    assert np.array_equal(gpu_label(ctx, lat), oracle.uf_label(lat))


def test_validate(ctx):
    lat = L.triangle(64, 0.4, 2)
    rp, ci, bits = to_dev(lat)
    assert ccl.ccl_validate(ctx, lat.n, lat.nnz, rp, ci, bits) == ccl.CCL_OK
    asym = L.random_graph(500, 900, 4, asymmetric=0.5)
    rp, ci, bits = to_dev(asym)
    assert ccl.ccl_validate(ctx, asym.n, asym.nnz, rp, ci, bits) == ccl.CCL_ERR_ASYMMETRIC
    ci2 = lat.col_idx.copy(); ci2[7] = lat.n
    rp, ci, bits = to_dev(L.Lattice("b", lat.n, lat.nnz, lat.row_ptr, ci2, lat.open_bits, 0, 0))
    assert ccl.ccl_validate(ctx, lat.n, lat.nnz, rp, ci, bits) == ccl.CCL_ERR_INDEX_OUT_OF_RANGE


def test_host_path(ctx):
    lat = L.cayley(3, 12, 0.5, 4, perm_seed=8)
    out = np.full(lat.n, -1, np.int32)
    st = ccl.ccl_label_host(ctx, lat.n, lat.nnz, lat.row_ptr, lat.col_idx, lat.open_bits, out)
    assert st == ccl.CCL_OK
    assert np.array_equal(out, oracle.uf_label(lat))


def test_autotune(ctx):
    c = ccl.ccl_context_create(0)
    try:
        lat = L.triangle(256, L.PC_TRIANGLE, 3)
        rp, ci, bits = to_dev(lat)
        out = torch.empty(lat.n, dtype=torch.int32, device=DEV)
        st, best = ccl.ccl_autotune(c, lat.n, lat.nnz, rp, ci, bits, out)
        assert st == ccl.CCL_OK and best > 0
        assert np.array_equal(out.cpu().numpy(), oracle.uf_label(lat))
        assert np.array_equal(gpu_label(c, lat), oracle.uf_label(lat))
    finally:
        ccl.ccl_context_destroy(c)


def _mixed_specs(K, seed):
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(K):
        t = int(rng.integers(0, 4))
        if t == 0:
            specs.append(dict(kind="honeycomb", L=int(rng.integers(2, 60)), p=float(rng.uniform(0.5, 0.8)), seed=k))
        elif t == 1:
            specs.append(dict(kind="triangle", L=int(rng.integers(2, 70)), p=float(rng.uniform(0.2, 0.5)), seed=k))
        elif t == 2:
            specs.append(dict(kind="cayley", z=int(rng.integers(3, 7)), shells=int(rng.integers(0, 6)),
                              p=float(rng.uniform(0.1, 0.9)), seed=k, perm_seed=k if k % 2 else None))
        else:
            specs.append(dict(kind="triangle", L=int(rng.integers(1, 4)), p=0.5, seed=k))
    return specs


@pytest.mark.parametrize("graphs", [0, 1])
def test_batched_matches_oracle_and_single(ctx, graphs):
    b = L.make_batch(_mixed_specs(150, 21))
    ccl.ccl_set_option(ctx, ccl.CCL_OPT_USE_GRAPHS, graphs)
    try:
        got = gpu_label_batched(ctx, b)
        again = gpu_label_batched(ctx, b)
    finally:
        ccl.ccl_set_option(ctx, ccl.CCL_OPT_USE_GRAPHS, 1)
    assert np.array_equal(got, again)
    want = oracle.uf_label_batched(b)
    assert np.array_equal(got, want)
    pairs = ccl.ccl_get_stats(ctx).residual_pairs
    tot = 0
    for k in range(b.k):
        inst = b.instance(k)
        s0, s1 = b.site_off[k], b.site_off[k + 1]
        assert np.array_equal(gpu_label(ctx, inst), got[s0:s1])
        tot += oracle.steps_label(inst)["n_residual"]
    assert pairs == tot


@pytest.mark.parametrize("K", [1, 3, 150])
def test_batched_host_path(ctx, K):
    """ccl_label_batched_host: host arrays in, labels out, the instances
    labelled in groups, each through all four steps, with the label downloads
    of earlier groups overlapping the uploads of later ones (K = 1: one group;
    K = 3: empty groups, one-instance groups and an empty instance); equal to
    the oracle and to the device-array call, twice in a row (buffers reused),
    and the statistics count the residual pairs of every group."""
    specs = _mixed_specs(K, 40 + K)
    if K == 3:
        specs[1] = dict(kind="triangle", L=0, p=0.5, seed=1)     # an empty instance in the middle
    b = L.make_batch(specs)
    want = oracle.uf_label_batched(b)
    for _ in range(2):
        out = np.full(b.n_total, -3, np.int32)
        st = ccl.ccl_label_batched_host(ctx, b.k, b.site_off, b.ent_off, b.row_ptr, b.col_idx,
                                        b.open_bits, out)
        assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
        assert np.array_equal(out, want)
    stats = ccl.ccl_get_stats(ctx)
    assert stats.n_inst == b.k and stats.n_sites == b.n_total
    assert stats.residual_pairs == sum(oracle.steps_label(L.make_instance(sp))["n_residual"] for sp in specs)
    assert np.array_equal(gpu_label_batched(ctx, b), want)
    assert ccl.ccl_get_stats(ctx).n_inst == b.k


def test_batched_host_path_large_groups(ctx):
    """Instances big enough that every upload group holds several step-(i)
    bands, in a batch whose bits start mid-word for most instances."""
    specs = [dict(kind="triangle", L=700, p=L.PC_TRIANGLE, seed=1), dict(kind="honeycomb", L=33, p=0.6, seed=2),
             dict(kind="cayley", z=3, shells=14, p=0.5, seed=3, perm_seed=3),
             dict(kind="triangle", L=513, p=0.36, seed=4), dict(kind="honeycomb", L=600, p=0.65, seed=5)]
    b = L.make_batch(specs)
    out = np.full(b.n_total, -3, np.int32)
    st = ccl.ccl_label_batched_host(ctx, b.k, b.site_off, b.ent_off, b.row_ptr, b.col_idx, b.open_bits, out)
    assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
    assert np.array_equal(out, oracle.uf_label_batched(b))


@pytest.mark.parametrize("window,group,park", [(64, 0, 0), (512, 16, 1), (2048, 1, 1), (65536, 3, 0),
                                               (1024, 0, 1)])
def test_window_and_super_chunk_settings_same_labels(window, group, park):
    """Every step-(iii) window length, step-(ii)/(iv) super-chunk run length
    and parking setting gives the oracle's labels, single and batched (the
    run length splits instances across super-chunks), with step (ii) on;
    the statistics report the settings used."""
    lat = L.triangle(700, L.PC_TRIANGLE, 12)
    b = L.make_batch(_mixed_specs(60, 13) + [dict(kind="honeycomb", L=400, p=L.PC_HONEYCOMB, seed=3),
                                             dict(kind="cayley", z=3, shells=15, p=0.5, seed=4, perm_seed=4)])
    c = ccl.ccl_context_create(0)
    try:
        for opt, v in ((ccl.CCL_OPT_REDUCE_WINDOW, window), (ccl.CCL_OPT_ANALYSIS_GROUP, group),
                       (ccl.CCL_OPT_ANALYSIS_PARK, park), (ccl.CCL_OPT_PRE_ANALYSIS, 1)):
            assert ccl.ccl_set_option(c, opt, v) == ccl.CCL_OK
            assert ccl.ccl_get_option(c, opt) == v
        assert np.array_equal(gpu_label(c, lat), oracle.uf_label(lat))
        st = ccl.ccl_get_stats(c)
        assert (st.reduce_window, st.analysis_group, st.analysis_park, st.pre_analysis) == (window, group, park, 1)
        assert np.array_equal(gpu_label_batched(c, b), oracle.uf_label_batched(b))
        assert ccl.ccl_set_option(c, ccl.CCL_OPT_ANALYSIS_PARK, 2) == ccl.CCL_ERR_INVALID_ARGUMENT
        assert ccl.ccl_set_option(c, ccl.CCL_OPT_REDUCE_WINDOW, 63) == ccl.CCL_ERR_INVALID_ARGUMENT
        assert ccl.ccl_set_option(c, ccl.CCL_OPT_ANALYSIS_GROUP, -2) == ccl.CCL_ERR_INVALID_ARGUMENT
    finally:
        ccl.ccl_context_destroy(c)


@pytest.mark.parametrize("pre", [0, 1])
def test_iteration_cap_reports_nonconvergence(pre):
    """The failure path of the iteration caps (Algorithm 1's merge loop and
    the root chases of steps (ii)/(iv)): with CCL_OPT_ITER_CAP = 1 a triangle
    lattice at p_c (long label chains) cannot finish, ccl_sync returns
    CCL_ERR_NONCONVERGED, single and batched; with the cap cleared the same
    context labels correctly again."""
    lat = L.triangle(512, L.PC_TRIANGLE, 3)
    b = L.make_batch(_mixed_specs(20, 5) + [dict(kind="triangle", L=300, p=L.PC_TRIANGLE, seed=9)])
    c = ccl.ccl_context_create(0)
    try:
        ccl.ccl_set_option(c, ccl.CCL_OPT_PRE_ANALYSIS, pre)
        assert ccl.ccl_set_option(c, ccl.CCL_OPT_ITER_CAP, 1) == ccl.CCL_OK
        assert ccl.ccl_get_option(c, ccl.CCL_OPT_ITER_CAP) == 1
        for _ in range(2):
            gpu_label(c, lat, expect_status=ccl.CCL_ERR_NONCONVERGED)
        out = torch.empty(b.n_total, dtype=torch.int32, device=DEV)
        from ccl_testutil import batch_to_dev
        brp, bci, bbits = batch_to_dev(b)
        assert ccl.ccl_label_batched(c, b.k, b.site_off, b.ent_off, brp, bci, bbits, out) == ccl.CCL_OK
        assert ccl.ccl_sync(c) == ccl.CCL_ERR_NONCONVERGED
        assert ccl.ccl_set_option(c, ccl.CCL_OPT_ITER_CAP, 0) == ccl.CCL_OK
        assert np.array_equal(gpu_label(c, lat), oracle.uf_label(lat))
        assert np.array_equal(gpu_label_batched(c, b), oracle.uf_label_batched(b))
        assert ccl.ccl_set_option(c, ccl.CCL_OPT_ITER_CAP, -1) == ccl.CCL_ERR_INVALID_ARGUMENT
    finally:
        ccl.ccl_context_destroy(c)


def test_two_streams_two_contexts():
    c1, c2 = ccl.ccl_context_create(0), ccl.ccl_context_create(0)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = L.triangle(700, L.PC_TRIANGLE, 1)
    b = L.cayley(3, 16, 0.5, 2, perm_seed=3)
    da, db = to_dev(a), to_dev(b)
    torch.cuda.synchronize()
    oa = torch.empty(a.n, dtype=torch.int32, device=DEV)
    ob = torch.empty(b.n, dtype=torch.int32, device=DEV)
    for _ in range(3):
        assert ccl.ccl_label(c1, a.n, a.nnz, *da, oa, s1) == ccl.CCL_OK
        assert ccl.ccl_label(c2, b.n, b.nnz, *db, ob, s2) == ccl.CCL_OK
    assert ccl.ccl_sync(c1, s1) == ccl.CCL_OK and ccl.ccl_sync(c2, s2) == ccl.CCL_OK
    assert np.array_equal(oa.cpu().numpy(), oracle.uf_label(a))
    assert np.array_equal(ob.cpu().numpy(), oracle.uf_label(b))
    ccl.ccl_context_destroy(c1)
    ccl.ccl_context_destroy(c2)


def test_graph_replay_keyed_on_sizes(ctx):
    """Same device buffers and chunk count, different n / nnz: the cached graph
    of the first call must not be replayed for the second."""
    a = L.random_graph(40, 60, 1)
    b = L.random_graph(50, 90, 2)
    rp = torch.zeros(64, dtype=torch.int32, device=DEV)
    ci = torch.zeros(256, dtype=torch.int32, device=DEV)
    bits = torch.zeros(8, dtype=torch.int32, device=DEV)
    out = torch.zeros(64, dtype=torch.int32, device=DEV)
    for lat in (a, b, a, b):
        rp[:lat.n + 1] = torch.from_numpy(lat.row_ptr).to(DEV)
        ci[:lat.nnz] = torch.from_numpy(lat.col_idx).to(DEV)
        bits[:lat.open_bits.size] = torch.from_numpy(lat.open_bits.view(np.int32)).to(DEV)
        assert ccl.ccl_label(ctx, lat.n, lat.nnz, rp, ci, bits, out) == ccl.CCL_OK
        assert ccl.ccl_sync(ctx) == ccl.CCL_OK
        assert np.array_equal(out[:lat.n].cpu().numpy(), oracle.uf_label(lat))


def test_graph_replay_reads_new_contents():
    """Same buffers and sizes, new bond bits written in place between calls:
    the replayed graph labels what the buffers hold now (single and batched)."""
    c = ccl.ccl_context_create(0)
    try:
        _replay_new_contents(c)
    finally:
        ccl.ccl_context_destroy(c)


def _replay_new_contents(ctx):
    from ccl_testutil import batch_to_dev
    lats = [L.triangle(130, p, seed) for p, seed in ((0.30, 1), (0.45, 2), (0.30, 3), (0.60, 4))]
    rp, ci, bits = to_dev(lats[0])
    out = torch.empty(lats[0].n, dtype=torch.int32, device=DEV)
    for k, lat in enumerate(lats):
        assert np.array_equal(lat.row_ptr, lats[0].row_ptr) and np.array_equal(lat.col_idx, lats[0].col_idx)
        bits.copy_(torch.from_numpy(lat.open_bits.view(np.int32)).to(DEV))
        out.fill_(-1)
        assert ccl.ccl_label(ctx, lat.n, lat.nnz, rp, ci, bits, out) == ccl.CCL_OK
        assert ccl.ccl_sync(ctx) == ccl.CCL_OK
        assert np.array_equal(out.cpu().numpy(), oracle.uf_label(lat))
        if k:
            assert ccl.ccl_get_stats(ctx).used_graph == 1
    specs = [dict(kind="honeycomb", L=40, p=0.65, seed=1), dict(kind="cayley", z=3, shells=9, p=0.5, seed=2, perm_seed=2)]
    b0 = L.make_batch(specs)
    brp, bci, bbits = batch_to_dev(b0)
    bout = torch.empty(b0.n_total, dtype=torch.int32, device=DEV)
    for k, seed in enumerate((5, 6, 7)):
        b = L.make_batch([dict(sp, seed=seed + i) for i, sp in enumerate(specs)])
        assert np.array_equal(b.col_idx, b0.col_idx)
        bbits.copy_(torch.from_numpy(b.open_bits.view(np.int32)).to(DEV))
        bout.fill_(-1)
        assert ccl.ccl_label_batched(ctx, b.k, b.site_off, b.ent_off, brp, bci, bbits, bout) == ccl.CCL_OK
        assert ccl.ccl_sync(ctx) == ccl.CCL_OK
        got = bout.cpu().numpy()
        for i in range(b.k):
            assert np.array_equal(got[int(b.site_off[i]):int(b.site_off[i + 1])], oracle.uf_label(b.instance(i)))
        if k:
            assert ccl.ccl_get_stats(ctx).used_graph == 1


@pytest.mark.parametrize("refill", [0, 1])
@pytest.mark.parametrize("order", [0, 1])
def test_refill_modes_on_uneven_work(refill, order):
    """Both ways of handing residual pairs to threads, on inputs whose chains
    differ widely in length: a randomly numbered tree, a multigraph, and a
    batch of mixed instances."""
    from ccl_testutil import gpu_label_batched
    c = ccl.ccl_context_create(0)
    try:
        assert ccl.ccl_set_option(c, ccl.CCL_OPT_REFILL, refill) == ccl.CCL_OK
        assert ccl.ccl_set_option(c, ccl.CCL_OPT_PRE_ANALYSIS, 1) == ccl.CCL_OK
        assert ccl.ccl_set_option(c, ccl.CCL_OPT_ANALYSIS_ORDER, order) == ccl.CCL_OK
        for lat in (L.cayley(3, 17, 0.5, 3, perm_seed=5), L.random_graph(50000, 90000, 4),
                    L.triangle(1000, 0.6, 3)):
            assert np.array_equal(gpu_label(c, lat), oracle.uf_label(lat))
        b = L.make_batch(L.batched_mix_specs(48, seed=21))
        got = gpu_label_batched(c, b)
        for k in range(b.k):
            s0, s1 = int(b.site_off[k]), int(b.site_off[k + 1])
            assert np.array_equal(got[s0:s1], oracle.uf_label(b.instance(k)))
        v = ccl.ccl_get_option(c, ccl.CCL_OPT_REFILL)
        assert v == refill
    finally:
        ccl.ccl_context_destroy(c)


def test_autotune_batched_keeps_labels_and_tunes_its_class():
    from ccl_testutil import batch_to_dev
    c = ccl.ccl_context_create(0)
    try:
        b = L.make_batch(L.batched_mix_specs(24, seed=31))
        rp, ci, bits = batch_to_dev(b)
        out = torch.full((b.n_total,), -1, dtype=torch.int32, device=DEV)
        st, best = ccl.ccl_autotune_batched(c, b.k, b.site_off, b.ent_off, rp, ci, bits, out)
        assert st == ccl.CCL_OK and best > 0
        assert ccl.ccl_sync(c) == ccl.CCL_OK
        got = out.cpu().numpy()
        for k in range(b.k):
            s0, s1 = int(b.site_off[k]), int(b.site_off[k + 1])
            assert np.array_equal(got[s0:s1], oracle.uf_label(b.instance(k)))
        out.fill_(-1)
        assert ccl.ccl_label_batched(c, b.k, b.site_off, b.ent_off, rp, ci, bits, out) == ccl.CCL_OK
        assert ccl.ccl_sync(c) == ccl.CCL_OK
        assert np.array_equal(out.cpu().numpy(), got)
        assert ccl.ccl_autotune_batched(c, 0, [0], [0], rp, ci, bits, out)[0] == ccl.CCL_OK
    finally:
        ccl.ccl_context_destroy(c)


def test_tune_cache_file_roundtrip(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("CCL_TUNE_CACHE", str(path))
    lat = L.triangle(512, 0.35, 3)
    want = oracle.uf_label(lat)
    rp, ci, bits = to_dev(lat)
    out = torch.empty(lat.n, dtype=torch.int32, device=DEV)
    c = ccl.ccl_context_create(0)
    try:
        st, best = ccl.ccl_autotune(c, lat.n, lat.nnz, rp, ci, bits, out)
        assert st == ccl.CCL_OK and best > 0
        assert np.array_equal(out.cpu().numpy(), want)
    finally:
        ccl.ccl_context_destroy(c)
    rows = [list(map(int, l.split())) for l in path.read_text().splitlines() if l.strip()]
    assert len(rows) >= 1 and all(len(r) == 10 for r in rows)
    assert all(r[1] in (128, 256, 512) and r[3] in (0, 1) and r[4] in (0, 1) for r in rows)
    assert all(r[7] in (0, 256, 512, 1024, 2048) and r[8] in (-1, 0, 8, 16, 32) and r[9] in (-1, 0, 1)
               for r in rows)
    # a new context reads the table back (and the older 7-field lines);
    # malformed lines are skipped
    old_form = " ".join(map(str, rows[0][:7]))
    path.write_text("not a line\n" + path.read_text() + "1 2 3\n" + old_form + "\n")
    c = ccl.ccl_context_create(0)
    try:
        out.fill_(-1)
        assert ccl.ccl_label(c, lat.n, lat.nnz, rp, ci, bits, out) == ccl.CCL_OK
        assert ccl.ccl_sync(c) == ccl.CCL_OK
        assert np.array_equal(out.cpu().numpy(), want)
    finally:
        ccl.ccl_context_destroy(c)


@pytest.mark.parametrize("L_", [255, 256, 257, 700])
def test_host_path_parts(ctx, L_):
    """The host-buffer entry point uploads large inputs in parts and starts
    step (i) on each part as it arrives; sizes around the 64-tile threshold,
    ragged tails, and a multigraph with rows of every length."""
    for lat in (L.triangle(L_, L.PC_TRIANGLE, 4), L.random_graph(L_ * L_, 2 * L_ * L_, 5)):
        out = np.full(lat.n, -1, np.int32)
        st = ccl.ccl_label_host(ctx, lat.n, lat.nnz, lat.row_ptr, lat.col_idx, lat.open_bits, out)
        assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
        assert np.array_equal(out, oracle.uf_label(lat))


def test_host_path_bad_row_ptr(ctx):
    lat = L.triangle(400, 0.4, 6)
    rp = lat.row_ptr.copy()
    rp[lat.n // 2] = lat.nnz + 5                     # past the entries: rejected before any launch
    out = np.empty(lat.n, np.int32)
    st = ccl.ccl_label_host(ctx, lat.n, lat.nnz, rp, lat.col_idx, lat.open_bits, out)
    assert st in (ccl.CCL_ERR_INVALID_ARGUMENT, ccl.CCL_ERR_INDEX_OUT_OF_RANGE)
    assert ccl.ccl_label_host(ctx, lat.n, lat.nnz, lat.row_ptr, lat.col_idx, lat.open_bits, out) == ccl.CCL_OK
    assert np.array_equal(out, oracle.uf_label(lat))


def test_thousands_of_small_random_graphs():
    """2000 random multigraphs of 1..300 sites (self-loops, repeated edges,
    isolated sites) labelled in one batched call, each against the oracle."""
    from ccl_testutil import batch_to_dev
    rng = np.random.default_rng(77)
    lats = []
    for k in range(2000):
        n = int(rng.integers(1, 301))
        m = int(rng.integers(0, 2 * n + 1))
        lats.append(L.random_graph(n, m, 1000 + k, p=float(rng.uniform(0.2, 0.9))))
    K = len(lats)
    site_off = np.zeros(K + 1, np.int64)
    ent_off = np.zeros(K + 1, np.int64)
    site_off[1:] = np.cumsum([x.n for x in lats])
    ent_off[1:] = np.cumsum([x.nnz for x in lats])
    row_ptr = np.concatenate([x.row_ptr for x in lats]).astype(np.int32)        # n_k + 1 each
    col_idx = np.concatenate([x.col_idx for x in lats]).astype(np.int32)
    bitv = np.concatenate([L.unpack_bits(x.open_bits, x.nnz) for x in lats])
    b = L.Batch(site_off, ent_off, row_ptr, col_idx, L.pack_bits(bitv), [{"kind": "random"}] * K)
    assert b.k == K and b.n_total == int(site_off[-1])
    c = ccl.ccl_context_create(0)
    try:
        got = gpu_label_batched(c, b)
    finally:
        ccl.ccl_context_destroy(c)
    for k, x in enumerate(lats):
        assert np.array_equal(got[int(site_off[k]):int(site_off[k + 1])], oracle.uf_label(x)), k


def test_allocation_failure_is_reported_and_recoverable():
    """A workspace the device cannot hold (16 TB of pair slots) is refused with
    CCL_ERR_OUT_OF_MEMORY; the context keeps labelling afterwards."""
    c = ccl.ccl_context_create(0)
    try:
        assert ccl.ccl_reserve(c, 0, 1 << 41, 0) == ccl.CCL_ERR_OUT_OF_MEMORY
        lat = L.triangle(300, 0.4, 8)
        assert np.array_equal(gpu_label(c, lat), oracle.uf_label(lat))
    finally:
        ccl.ccl_context_destroy(c)
