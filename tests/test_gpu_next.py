"""GPU parity of the steps around the labelling: bonds drawn on the device
(ccl_label_random), sequential relabelling with cluster sizes (ccl_relabel)
and the spanning test of Section 4 (ccl_spanning), each against the oracle."""
import dataclasses

import numpy as np
import pytest
import torch

import lattices as L
import oracle
from oracle import stats
import paper_1603_08357_gb300 as ccl
from ccl_testutil import DEV, gpu_label, to_dev

pytestmark = pytest.mark.gpu


def _random_labels(ctx, lat, seed, p):
    rp, ci, _ = to_dev(lat)
    out = torch.full((max(lat.n, 1),), -3, dtype=torch.int32, device=DEV)
    st = ccl.ccl_label_random(ctx, lat.n, lat.nnz, rp, ci if lat.nnz else None, seed, p, out)
    assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
    assert ccl.ccl_sync(ctx) == ccl.CCL_OK
    return out[:lat.n].cpu().numpy()


@pytest.mark.parametrize("kind,kw", [("triangle", dict(L=300)), ("honeycomb", dict(L=211)),
                                     ("cayley", dict(z=3, shells=14, perm_seed=4)),
                                     ("triangle", dict(L=257, periodic_y=False))])
@pytest.mark.parametrize("p", [0.0, 0.35, 0.5, 0.65, 1.0])
def test_label_random_matches_oracle(ctx, kind, kw, p):
    lat = L.make_instance(dict(kind=kind, p=0.5, seed=1, **kw))
    for seed in (7, 2**63 + 11):
        want = oracle.uf_label(dataclasses.replace(lat, open_bits=oracle.keyed_bits(lat, seed, p)))
        assert np.array_equal(_random_labels(ctx, lat, seed, p), want)


def test_label_random_multigraph(ctx):
    lat = L.random_graph(5000, 9000, 3, asymmetric=0.0)
    for seed in range(5):
        want = oracle.uf_label(dataclasses.replace(lat, open_bits=oracle.keyed_bits(lat, seed, 0.55)))
        assert np.array_equal(_random_labels(ctx, lat, seed, 0.55), want)
    rp, ci, _ = to_dev(lat)
    out = torch.empty(lat.n, dtype=torch.int32, device=DEV)
    assert ccl.ccl_label_random(ctx, lat.n, lat.nnz, rp, ci, 1, 1.5, out) == ccl.CCL_ERR_INVALID_ARGUMENT


@pytest.mark.parametrize("kind,kw,p", [("triangle", dict(L=513), L.PC_TRIANGLE),
                                       ("honeycomb", dict(L=300), 0.8),
                                       ("cayley", dict(z=4, shells=9, perm_seed=2), 1 / 3),
                                       ("triangle", dict(L=40), 0.0), ("triangle", dict(L=40), 1.0)])
def test_relabel_and_sizes(ctx, kind, kw, p):
    lat = L.make_instance(dict(kind=kind, p=p, seed=5, **kw))
    lab = gpu_label(ctx, lat)
    d_lab = torch.from_numpy(lab).to(DEV)
    seq = torch.full((lat.n,), -1, dtype=torch.int32, device=DEV)
    sizes = torch.full((lat.n,), -1, dtype=torch.int32, device=DEV)
    nc = torch.zeros(1, dtype=torch.int32, device=DEV)
    assert ccl.ccl_relabel(ctx, lat.n, d_lab, seq, nc, sizes) == ccl.CCL_OK
    assert ccl.ccl_sync(ctx) == ccl.CCL_OK
    want_seq, want_sizes = stats.sequential(lab)
    C = int(nc.item())
    assert C == want_sizes.size == stats.n_clusters(lab)
    assert np.array_equal(seq.cpu().numpy(), want_seq)
    assert np.array_equal(sizes[:C].cpu().numpy(), want_sizes)
    assert ccl.ccl_relabel(ctx, lat.n, d_lab, d_lab, nc) == ccl.CCL_ERR_INVALID_ARGUMENT


def _relabel(ctx, lab, with_sizes=True):
    n = lab.size
    d_lab = torch.from_numpy(lab).to(DEV) if n else torch.zeros(1, dtype=torch.int32, device=DEV)
    seq = torch.full((max(n, 1),), -1, dtype=torch.int32, device=DEV)
    sizes = torch.full((max(n, 1),), -1, dtype=torch.int32, device=DEV) if with_sizes else None
    nc = torch.full((1,), -9, dtype=torch.int32, device=DEV)
    assert ccl.ccl_relabel(ctx, n, d_lab, seq, nc, sizes) == ccl.CCL_OK
    assert ccl.ccl_sync(ctx) == ccl.CCL_OK
    C = int(nc.item())
    return C, seq[:n].cpu().numpy(), (sizes[:C].cpu().numpy() if with_sizes else None)


@pytest.mark.parametrize("n", [0, 1, 31, 8192, 8193])
def test_relabel_block_edges(ctx, n):
    """Site counts at the edges of the relabelling blocks (8192 sites), with
    and without the sizes output."""
    lat = L.random_graph(n, max(0, n // 2), 8, p=0.7) if n else None
    lab = gpu_label(ctx, lat) if n else np.zeros(0, np.int32)
    want_seq, want_sizes = stats.sequential(lab)
    for with_sizes in (True, False):
        C, seq, sizes = _relabel(ctx, lab, with_sizes)
        assert C == want_sizes.size
        assert np.array_equal(seq, want_seq)
        if with_sizes:
            assert np.array_equal(sizes, want_sizes)


def test_relabel_more_blocks_than_scan_threads(ctx):
    """9.4M sites: 1152 relabelling blocks, more than the one-CTA scan has
    threads, so each scan thread sums a run of blocks."""
    lat = L.triangle(3072, L.PC_TRIANGLE, 12)
    lab = gpu_label(ctx, lat)
    assert np.array_equal(lab, oracle.uf_label(lat))
    C, seq, sizes = _relabel(ctx, lab)
    want_seq, want_sizes = stats.sequential(lab)
    assert (lat.n + 8191) // 8192 > 1024
    assert C == want_sizes.size and np.array_equal(seq, want_seq) and np.array_equal(sizes, want_sizes)


def test_spanning_empty_sets_and_bad_sites(ctx):
    """No top (or bottom) sites: -1. Site numbers outside [0, n) are skipped
    and reported by ccl_sync; the result is that of the valid sites."""
    lat = L.triangle(96, 0.7, 3, periodic_y=False)
    lab = gpu_label(ctx, lat)
    top, bot = L.row_sites(lat, 0), L.row_sites(lat, 95)
    want = stats.spanning_label(oracle.uf_label(lat), top, bot)
    assert want >= 0
    d_lab = torch.from_numpy(lab).to(DEV)
    res = torch.zeros(1, dtype=torch.int32, device=DEV)
    dev = lambda a: torch.from_numpy(np.asarray(a, np.int32)).to(DEV)
    assert ccl.ccl_spanning(ctx, lat.n, d_lab, None, 0, dev(bot), bot.size, res) == ccl.CCL_OK
    assert ccl.ccl_sync(ctx) == ccl.CCL_OK and int(res.item()) == -1
    assert ccl.ccl_spanning(ctx, lat.n, d_lab, dev(top), top.size, None, 0, res) == ccl.CCL_OK
    assert ccl.ccl_sync(ctx) == ccl.CCL_OK and int(res.item()) == -1
    bad_top = np.concatenate([[-1, lat.n], top, [lat.n + 5]])
    bad_bot = np.concatenate([bot, [2 ** 31 - 1]])
    assert ccl.ccl_spanning(ctx, lat.n, d_lab, dev(bad_top), bad_top.size, dev(bad_bot), bad_bot.size,
                            res) == ccl.CCL_OK
    assert ccl.ccl_sync(ctx) == ccl.CCL_ERR_INDEX_OUT_OF_RANGE
    assert int(res.item()) == want
    assert np.array_equal(gpu_label(ctx, lat), lab)          # the context is still usable


@pytest.mark.parametrize("kind", ["triangle", "honeycomb"])
def test_spanning(ctx, kind):
    pc = L.PC_TRIANGLE if kind == "triangle" else L.PC_HONEYCOMB
    for Ls, seed in ((64, 1), (200, 2), (513, 3)):
        for p in (pc - 0.05, pc, pc + 0.05):
            lat = L.make_instance(dict(kind=kind, L=Ls, p=p, seed=seed, periodic_y=False))
            lab = gpu_label(ctx, lat)
            top, bot = L.row_sites(lat, 0), L.row_sites(lat, Ls - 1)
            res = torch.zeros(1, dtype=torch.int32, device=DEV)
            d_lab = torch.from_numpy(lab).to(DEV)
            d_top = torch.from_numpy(top.astype(np.int32)).to(DEV)
            d_bot = torch.from_numpy(bot.astype(np.int32)).to(DEV)
            assert ccl.ccl_spanning(ctx, lat.n, d_lab, d_top, top.size, d_bot, bot.size, res) == ccl.CCL_OK
            assert ccl.ccl_sync(ctx) == ccl.CCL_OK
            assert int(res.item()) == stats.spanning_label(oracle.uf_label(lat), top, bot)


def test_random_full_size_triangle(ctx):
    """tri4096 at p_c with device-drawn bonds, compared site by site."""
    lat = L.triangle(4096, 0.5, 2)
    want = oracle.uf_label(dataclasses.replace(lat, open_bits=oracle.keyed_bits(lat, 99, 0.3473)))
    assert np.array_equal(_random_labels(ctx, lat, 99, 0.3473), want)


def test_spanning_curve_matches_oracle(ctx):
    """R_span(p) from the device sampler equals, realisation by realisation,
    the oracle's labels of the same keyed bonds."""
    from paper_1603_08357_gb300 import percolation as P
    for kind, Ls in (("triangle", 24), ("honeycomb", 17)):
        lat = L.make_instance(dict(kind=kind, L=Ls, p=0.0, seed=0, periodic_y=False))
        top, bot = P.boundary_rows(kind, Ls)
        assert np.array_equal(np.sort(top), np.sort(L.row_sites(lat, 0)))
        assert np.array_equal(np.sort(bot), np.sort(L.row_sites(lat, Ls - 1)))
        ps = [P.PC_EXACT[kind] - 0.1, P.PC_EXACT[kind], P.PC_EXACT[kind] + 0.1]
        R = P.Sampler(ctx, lat, top, bot).spanning_curve(ps, 120, seed0=500)
        want = []
        for p in ps:
            hits = 0
            for r in range(120):
                lab = oracle.uf_label(dataclasses.replace(lat, open_bits=oracle.keyed_bits(lat, 500 + r, p)))
                hits += stats.spanning_label(lab, top, bot) >= 0
            want.append(hits / 120)
        assert np.allclose(R, want, rtol=0, atol=1e-12), (kind, R, want)


def test_spanning_crossing_near_exact_threshold(ctx):
    """Curves of two sizes cross near 2 sin(pi/18) (triangle), as in Fig. 6."""
    from paper_1603_08357_gb300 import percolation as P
    pc = P.PC_EXACT["triangle"]
    ps = np.linspace(pc - 0.03, pc + 0.03, 7)
    curves = []
    for Ls in (64, 128):
        lat = L.make_instance(dict(kind="triangle", L=Ls, p=0.0, seed=0, periodic_y=False))
        curves.append(P.Sampler(ctx, lat, *P.boundary_rows("triangle", Ls)).spanning_curve(ps, 1500, 77))
    for R in curves:
        assert np.all(np.diff(R) >= 0) and R[0] < 0.3 and R[-1] > 0.7
    x, err = P.crossing(ps, curves[0], curves[1], 1500)
    assert err is not None and 0 < err < 0.005
    assert x is not None and abs(x - pc) < 0.01, x


def test_stats_after_host_path_grows(ctx):
    """ccl_relabel and ccl_spanning keep working after the host-buffer entry
    point has grown its device buffers on the same context."""
    small = L.make_instance(dict(kind="triangle", L=64, p=0.5, seed=1, periodic_y=False))
    lab = gpu_label(ctx, small)
    d_lab = torch.from_numpy(lab).to(DEV)
    seq = torch.empty(small.n, dtype=torch.int32, device=DEV)
    nc = torch.zeros(1, dtype=torch.int32, device=DEV)
    assert ccl.ccl_relabel(ctx, small.n, d_lab, seq, nc) == ccl.CCL_OK      # scratch allocated
    big = L.make_instance(dict(kind="triangle", L=700, p=0.4, seed=2))
    out = np.empty(big.n, np.int32)
    assert ccl.ccl_label_host(ctx, big.n, big.nnz, big.row_ptr, big.col_idx, big.open_bits, out) == ccl.CCL_OK
    assert np.array_equal(out, oracle.uf_label(big))
    assert ccl.ccl_relabel(ctx, small.n, d_lab, seq, nc) == ccl.CCL_OK
    assert ccl.ccl_sync(ctx) == ccl.CCL_OK
    assert np.array_equal(seq.cpu().numpy(), stats.sequential(lab)[0])


def _largest(ctx, lab):
    res = torch.full((2,), -9, dtype=torch.int32, device=DEV)
    d = torch.from_numpy(np.ascontiguousarray(lab, np.int32)).to(DEV) if lab.size else \
        torch.zeros(1, dtype=torch.int32, device=DEV)
    assert ccl.ccl_largest_cluster(ctx, lab.size, d, res) == ccl.CCL_OK
    return tuple(int(v) for v in res.cpu().numpy())


def test_largest_cluster_matches_oracle(ctx):
    """ccl_largest_cluster against the oracle's statistic: ties go to the
    smaller label (the worked example's two 5-site clusters), lattices from
    p = 0 (all singletons) to p = 1, a randomly numbered tree, sizes across
    warp and grid edges, and no sites."""
    from conftest import load_golden
    g = load_golden("worked_example.txt")
    assert _largest(ctx, np.array(g["label"], np.int32)) == tuple(g["largest"])
    assert _largest(ctx, np.zeros(0, np.int32)) == (0, -1)
    assert _largest(ctx, np.zeros(1, np.int32)) == (1, 0)
    for lat in (L.triangle(300, 0.0, 1), L.triangle(300, 1.0, 1), L.triangle(257, L.PC_TRIANGLE, 2),
                L.honeycomb(129, L.PC_HONEYCOMB, 3), L.cayley(3, 14, 0.5, 4, perm_seed=4),
                L.random_graph(33, 40, 5)):
        lab = gpu_label(ctx, lat)
        assert _largest(ctx, lab) == stats.largest_cluster(oracle.uf_label(lat))
    assert ccl.ccl_sync(ctx) == ccl.CCL_OK


def test_largest_cluster_bad_label_is_reported(ctx):
    lab = np.array([0, 0, 7, 1], np.int32)             # 7 is out of range for n = 4
    assert _largest(ctx, lab) == (2, 0)
    assert ccl.ccl_sync(ctx) == ccl.CCL_ERR_INDEX_OUT_OF_RANGE


def test_sweep_largest_matches_oracle(ctx):
    """The device sweep (device-drawn bonds, spanning and largest cluster per
    realisation) equals, realisation by realisation, the oracle's statistics
    of the same keyed bonds."""
    from paper_1603_08357_gb300 import percolation as P
    for kind, Ls in (("triangle", 40), ("honeycomb", 23)):
        lat = L.make_instance(dict(kind=kind, L=Ls, p=0.0, seed=0, periodic_y=False))
        top, bot = P.boundary_rows(kind, Ls)
        ps = [P.PC_EXACT[kind] - 0.05, P.PC_EXACT[kind], P.PC_EXACT[kind] + 0.05]
        span, big = P.Sampler(ctx, lat, top, bot).sweep(ps, 60, seed0=900)
        for a, p in enumerate(ps):
            for r in range(60):
                lab = oracle.uf_label(dataclasses.replace(lat, open_bits=oracle.keyed_bits(lat, 900 + r, p)))
                assert tuple(big[a, r]) == stats.largest_cluster(lab), (kind, p, r)
                assert bool(span[a, r]) == (stats.spanning_label(lab, top, bot) >= 0)


def test_largest_cluster_crossing_near_exact_threshold(ctx):
    """The finite-size-scaled mean largest cluster S(L, p) L^(-91/48) of two
    sizes crosses near 2 sin(pi/18) (triangle)."""
    from paper_1603_08357_gb300 import percolation as P
    pc = P.PC_EXACT["triangle"]
    ps = np.linspace(pc - 0.03, pc + 0.03, 7)
    curves = []
    for Ls in (64, 128):
        lat = L.make_instance(dict(kind="triangle", L=Ls, p=0.0, seed=0, periodic_y=False))
        _, big = P.Sampler(ctx, lat, *P.boundary_rows("triangle", Ls)).sweep(ps, 1500, 31)
        curves.append(P.scaled_largest(big[..., 0], Ls))
    for m, _ in curves:
        assert np.all(np.diff(m) > 0)
    x, err = P.crossing(ps, curves[0][0], curves[1][0], se=(curves[0][1], curves[1][1]))
    assert x is not None and err is not None and err < 0.01
    assert abs(x - pc) < 0.012, (x, err)


@pytest.mark.parametrize("kind,Ls,reps", [("triangle", 512, 12), ("honeycomb", 362, 12), ("triangle", 4096, 2)])
def test_sweep_at_the_papers_sizes_matches_oracle(ctx, kind, Ls, reps):
    """The device sweep at the sizes of Section 4 (N = 262,144 and 16,777,216
    sites; honeycomb 362 x 362 cells = 262,088 sites): spanning flag and
    largest cluster (size, label) of every realisation equal the oracle's on
    the same keyed bonds."""
    from paper_1603_08357_gb300 import percolation as P
    lat = L.make_instance(dict(kind=kind, L=Ls, p=0.0, seed=0, periodic_y=False))
    top, bot = P.boundary_rows(kind, Ls)
    pc = P.PC_EXACT[kind]
    ps = [pc - 0.003, pc, pc + 0.003]
    span, big = P.Sampler(ctx, lat, top, bot).sweep(ps, reps, seed0=2024)
    for a, p in enumerate(ps):
        for r in range(reps):
            lab = oracle.uf_label(dataclasses.replace(lat, open_bits=oracle.keyed_bits(lat, 2024 + r, p)))
            assert tuple(big[a, r]) == stats.largest_cluster(lab), (kind, Ls, p, r)
            assert bool(span[a, r]) == (stats.spanning_label(lab, top, bot) >= 0), (kind, Ls, p, r)
