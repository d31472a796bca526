"""Pins for the CPU oracle (oracle/) against what the paper and mathematics fix.

* brute force: every bond mask of small multigraphs (<= 12 bonds, self-loops
  and duplicate entries included) against scipy's connected components;
* hand-worked examples of the four steps of Section 3 (tests/golden);
* the forest identity: on a tree, clusters = sites - open bonds, exactly;
* the empty residual lists of a centre-numbered Bethe lattice (Section 4);
* the renaming invariance of a Bethe lattice stored in random position;
* the mean size of the centre cluster of a branching process;
* crossings of the spanning probability near p_c = 1 - 2 sin(pi/18)
  (honeycomb) and 2 sin(pi/18) (triangle), Section 4, Figs. 5-6.
"""
import dataclasses
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import lattices as L
import oracle
from oracle import stats
from conftest import load_golden


def _canonical_from_components(comp: np.ndarray) -> np.ndarray:
    """Smallest member of each component, by first occurrence in site order."""
    _, first = np.unique(comp, return_index=True)
    rep = np.empty(comp.max() + 1 if comp.size else 0, np.int64)
    rep[comp[first]] = first
    return rep[comp].astype(np.int32)


def _scipy_labels(n, edges_open):
    if n == 0:
        return np.zeros(0, np.int32)
    u = np.array([a for a, b in edges_open] or [0], np.int64)
    v = np.array([b for a, b in edges_open] or [0], np.int64)
    w = np.ones(len(edges_open) or 1)
    if not edges_open:
        w[:] = 0
    A = sp.coo_matrix((w, (u, v)), shape=(n, n)).tocsr()
    A.eliminate_zeros()
    _, comp = connected_components(A, directed=False)
    return _canonical_from_components(comp)


def _lattice_from_entries(n, rows_entries):
    """rows_entries[i] = list of (j, bit); returns a lattices.Lattice."""
    row_ptr = np.zeros(n + 1, np.int32)
    cols, bitv = [], []
    for i in range(n):
        for j, b in rows_entries[i]:
            cols.append(j); bitv.append(b)
        row_ptr[i + 1] = len(cols)
    ci = np.array(cols, np.int32)
    return L.Lattice("test", n, len(cols), row_ptr, ci, L.pack_bits(np.array(bitv, bool)), 0.0, 0)


@pytest.mark.parametrize("seed", range(12))
def test_bruteforce_all_masks(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 9))
    m = int(rng.integers(0, 13))
    u = rng.integers(0, n, m)
    v = rng.integers(0, n, m)
    if seed % 3 == 0 and m >= 2:          # force a duplicate edge
        u[1], v[1] = v[0], u[0]
    # CSR listing each edge in both rows; bit of edge t in both copies
    entries = [[] for _ in range(n)]
    for t in range(m):
        a, b = int(u[t]), int(v[t])
        entries[a].append([b, 0, t]); entries[b].append([a, 0, t])
    for mask in range(1 << m):
        rows = [[(j, (mask >> t) & 1) for j, _, t in entries[i]] for i in range(n)]
        lat = _lattice_from_entries(n, rows)
        expect = _scipy_labels(n, [(int(u[t]), int(v[t])) for t in range(m) if (mask >> t) & 1])
        o1 = oracle.uf_label(lat)
        o2 = oracle.bfs_label(lat)
        o3 = oracle.steps_label(lat)["label"]
        assert np.array_equal(o1, expect), (mask, o1, expect)
        assert np.array_equal(o2, expect)
        assert np.array_equal(o3, expect)


@pytest.mark.parametrize("name", ["worked_example.txt", "row_max_rule.txt", "duplicate_min.txt"])
def test_golden_steps(name):
    g = load_golden(name)
    n = g["n"][0]
    rp = np.array(g["row_ptr"], np.int32)
    lat = L.Lattice("golden", n, int(rp[-1]), rp, np.array(g["col_idx"], np.int32),
                    L.pack_bits(np.array(g["open"], bool)), 0.0, 0)
    st = oracle.steps_label(lat)
    assert st["after_init"].tolist() == g["after_init"]
    assert st["after_ii"].tolist() == g["after_ii"]
    assert st["after_iii"].tolist() == g["after_iii"]
    assert st["label"].tolist() == g["label"]
    res = g.get("residual", {})
    for i in range(n):
        assert st["residual"][i].tolist() == res.get(i, []), i
    assert st["n_residual"] == sum(len(v) for v in res.values())
    assert oracle.uf_label(lat).tolist() == g["label"]
    assert oracle.bfs_label(lat).tolist() == g["label"]
    if "largest" in g:
        assert list(stats.largest_cluster(st["label"])) == g["largest"]


@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_agree_and_invariants(seed):
    lat = L.random_graph(3000, 4000, seed, asymmetric=0.3 if seed % 2 else 0.0, p=0.55)
    o1, o2, o3 = oracle.uf_label(lat), oracle.bfs_label(lat), oracle.steps_label(lat)["label"]
    assert np.array_equal(o1, o2) and np.array_equal(o1, o3)
    # the bond set read from row max(i, j): the generator's per-edge state
    u, v = lat.meta["edges"]
    op = lat.meta["open"]
    keep = op & (u != v)
    expect = _scipy_labels(lat.n, list(zip(u[keep].tolist(), v[keep].tolist())))
    assert np.array_equal(o1, expect)
    idx = np.arange(lat.n)
    assert np.all(o1 <= idx) and np.array_equal(o1[o1], o1)
    # every open bond's ends share a label, and a label is the least site carrying it
    assert np.array_equal(o1[u[keep]], o1[v[keep]])
    least = np.full(lat.n, lat.n, np.int64)
    np.minimum.at(least, o1, idx)
    assert np.array_equal(least[o1], o1)


@pytest.mark.parametrize("z,S,p,perm", [(3, 8, 0.5, None), (3, 8, 0.5, 9), (4, 6, 0.4, 5),
                                        (6, 4, 0.9, 2), (3, 10, 1.0, 1), (5, 5, 0.0, None)])
def test_tree_identity(z, S, p, perm):
    """On a forest every open bond joins two clusters: clusters = N - open bonds."""
    for seed in range(3):
        lat = L.cayley(z, S, p, 100 + seed, perm_seed=perm)
        lab = oracle.uf_label(lat)
        assert stats.n_clusters(lab) == lat.n - lat.n_open_bonds
        assert np.array_equal(lab, oracle.bfs_label(lat))


@pytest.mark.parametrize("z,S", [(3, 9), (4, 6), (6, 4)])
@pytest.mark.parametrize("p", [0.25, 0.5, 1.0])
def test_standard_position_has_empty_residual_lists(z, S, p):
    """Section 4: numbered from the centre, every site has at most one lower
    neighbour (its parent), so no residual list survives step (i)."""
    lat = L.cayley(z, S, p, 7)
    st = oracle.steps_label(lat)
    assert st["n_residual"] == 0
    rnd = L.cayley(z, S, 1.0, 7, perm_seed=3)
    assert oracle.steps_label(rnd)["n_residual"] > 0


def test_random_position_is_a_renaming():
    std = L.cayley(3, 9, 0.55, 21)
    rnd = L.cayley(3, 9, 0.55, 21, perm_seed=77)
    P = rnd.meta["perm"]
    a, b = oracle.uf_label(std), oracle.uf_label(rnd)
    # same partition after renaming: sites s, t together in std iff P[s], P[t] together in rnd
    ren = b[P]                                  # label (in rnd numbering) of standard site s
    # each std cluster maps to exactly one rnd cluster and vice versa
    m1 = {}
    for s in range(std.n):
        m1.setdefault(int(a[s]), set()).add(int(ren[s]))
    assert all(len(v) == 1 for v in m1.values())
    assert len({next(iter(v)) for v in m1.values()}) == len(m1)


def _bethe_center_closed_form(z, S, p):
    # Each of the z (z-1)^(k-1) sites of shell k joins the centre's cluster iff
    # the k bonds of its path to the centre are open (a branching process).
    return 1.0 + z * sum(p ** k * (z - 1) ** (k - 1) for k in range(1, S + 1))


@pytest.mark.parametrize("z,S,p", [(3, 10, 0.5), (4, 7, 0.25), (3, 8, 0.7), (5, 5, 0.25)])
def test_bethe_center_cluster_mean(z, S, p):
    """p_c = 1/(z-1) for the Bethe lattice (Section 4): at p_c the mean centre
    cluster grows linearly with the shell count; the Monte Carlo mean of the
    oracle's cluster sizes must match the branching-process expectation."""
    sizes = []
    for seed in range(1500):
        perm = seed if seed % 2 else None
        lat = L.cayley(z, S, p, 5000 + seed, perm_seed=perm)
        lab = oracle.uf_label(lat)
        c = L.cayley_center(lat)
        sizes.append(int(np.count_nonzero(lab == lab[c])))
    sizes = np.array(sizes, float)
    mean, sd = sizes.mean(), sizes.std(ddof=1)
    expect = _bethe_center_closed_form(z, S, p)
    assert abs(mean - expect) < 5 * sd / math.sqrt(sizes.size), (mean, expect)
    if abs(p - 1 / (z - 1)) < 1e-12:
        assert abs(expect - (1 + z * S / (z - 1))) < 1e-9


def _span_prob(make, Ls, p, samples, seed0):
    hits = 0
    for s in range(samples):
        lat = make(Ls, p, seed0 + s)
        lab = oracle.uf_label(lat)
        if stats.spans(lab, L.row_sites(lat, 0), L.row_sites(lat, Ls - 1)):
            hits += 1
    return hits / samples


@pytest.mark.parametrize("kind", ["triangle", "honeycomb"])
def test_spanning_crossing_brackets_pc(kind):
    """R_span(p) curves of different sizes cross at p_c (Section 4): below p_c the
    larger system spans less often, above it more often."""
    pc = L.PC_TRIANGLE if kind == "triangle" else L.PC_HONEYCOMB
    make = (lambda Ls, p, s: L.triangle(Ls, p, s, periodic_y=False)) if kind == "triangle" else \
           (lambda Ls, p, s: L.honeycomb(Ls, p, s, periodic_y=False))
    n = 500
    d = 0.04
    lo_s, lo_b = _span_prob(make, 12, pc - d, n, 1), _span_prob(make, 64, pc - d, n, 2)
    hi_s, hi_b = _span_prob(make, 12, pc + d, n, 3), _span_prob(make, 64, pc + d, n, 4)
    def tol(a, b):   # 4 standard errors of a difference of two binomial proportions
        return 4 * math.sqrt((a * (1 - a) + b * (1 - b)) / n + 1.0 / n ** 2)
    assert lo_s - lo_b > tol(lo_s, lo_b), (lo_s, lo_b)
    assert hi_b - hi_s > tol(hi_s, hi_b), (hi_s, hi_b)


def _mean_largest(kind, Ls, p, reps, seed0):
    """Mean size of the largest cluster over `reps` periodic realisations, and
    its standard error."""
    from concurrent.futures import ThreadPoolExecutor

    def one(r):
        lat = L.make_instance(dict(kind=kind, L=Ls, p=p, seed=seed0 + r), nthreads=1)
        return stats.largest_cluster(oracle.uf_label(lat))[0]
    with ThreadPoolExecutor(8) as ex:
        v = np.array(list(ex.map(one, range(reps))), float)
    return v.mean(), v.std(ddof=1) / math.sqrt(reps)


@pytest.mark.parametrize("kind", ["triangle", "honeycomb"])
def test_largest_cluster_scales_with_the_fractal_dimension(kind):
    """At p_c the largest cluster of an L x L system grows as L^D with the
    exact two-dimensional percolation fractal dimension D = 91/48, so the mean
    largest cluster at 2L over that at L is 2^(91/48) = 3.7214 up to
    corrections that are small at L = 64..128 and within CLT error; slightly
    off p_c the ratio moves far from it (towards 1 below, 4 above). This pins
    the largest-cluster statistic and, through it, the thresholds
    1 - 2 sin(pi/18) and 2 sin(pi/18) (Section 4)."""
    pc = L.PC_TRIANGLE if kind == "triangle" else L.PC_HONEYCOMB
    target = 2 ** (91 / 48)
    a, ea = _mean_largest(kind, 64, pc, 2000, 10_000)
    b, eb = _mean_largest(kind, 128, pc, 2000, 20_000)
    ratio = b / a
    err = ratio * math.hypot(ea / a, eb / b)
    assert abs(ratio - target) < 4 * err + 0.01, (ratio, err)
    lo = _mean_largest(kind, 128, pc - 0.03, 300, 30_000)[0] / _mean_largest(kind, 64, pc - 0.03, 300, 40_000)[0]
    hi = _mean_largest(kind, 128, pc + 0.03, 300, 50_000)[0] / _mean_largest(kind, 64, pc + 0.03, 300, 60_000)[0]
    assert lo < target - 0.8 and hi > target + 0.15, (lo, hi)


def test_largest_cluster_extremes():
    tri = L.triangle(16, 0.0, 1)
    assert stats.largest_cluster(oracle.uf_label(tri)) == (1, 0)      # singletons: the tie goes to site 0
    tri = L.triangle(16, 1.0, 1)
    assert stats.largest_cluster(oracle.uf_label(tri)) == (256, 0)
    assert stats.largest_cluster(np.zeros(0, np.int32)) == (0, -1)
    # two clusters {0, 2} and {1, 3, 4}: the larger wins although its label is larger
    assert stats.largest_cluster(np.array([0, 1, 0, 1, 1], np.int32)) == (3, 1)


def test_extremes():
    tri = L.triangle(16, 0.0, 1)
    assert np.array_equal(oracle.uf_label(tri), np.arange(tri.n))
    tri = L.triangle(16, 1.0, 1)
    assert not oracle.uf_label(tri).any()
    empty = L.Lattice("empty", 0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32),
                      np.zeros(1, np.uint32), 0.0, 0)
    assert oracle.uf_label(empty).size == 0
    bad = L.Lattice("bad", 2, 1, np.array([0, 1, 1], np.int32), np.array([5], np.int32),
                    np.zeros(1, np.uint32), 0.0, 0)
    with pytest.raises(ValueError):
        oracle.uf_label(bad)


def test_batched_oracle_matches_single():
    specs = [dict(kind="honeycomb", L=9, p=0.65, seed=1), dict(kind="cayley", z=4, shells=5, p=0.33,
             seed=2, perm_seed=3), dict(kind="triangle", L=11, p=0.35, seed=4)]
    b = L.make_batch(specs)
    lab = oracle.uf_label_batched(b)
    for k in range(b.k):
        s0, s1 = b.site_off[k], b.site_off[k + 1]
        assert np.array_equal(lab[s0:s1], oracle.bfs_label(b.instance(k)))


def test_oracle_splitmix64_published_vectors():
    # first outputs of SplitMix64 from state 0, as printed by the reference implementation
    assert oracle.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64(0, 2) == 0x06C45D188009454F


def test_keyed_bits_symmetric_and_rate():
    import dataclasses
    tri = L.triangle(128, 0.5, 1)
    for p in (0.0, 0.3, 0.65, 1.0):
        bits = oracle.keyed_bits(tri, 12345, p)
        lat = dataclasses.replace(tri, open_bits=bits)
        b = L.unpack_bits(bits, lat.nnz)
        rows = np.repeat(np.arange(lat.n), np.diff(lat.row_ptr))
        state = {}
        for r, c, v in zip(rows.tolist(), lat.col_idx.tolist(), b.tolist()):
            key = (min(r, c), max(r, c))
            assert state.setdefault(key, v) == v          # both copies agree
        frac = np.mean(list(state.values()))
        assert abs(frac - p) <= 4 * np.sqrt(max(p * (1 - p), 1e-9) / len(state)) + 1e-12


def test_sequential_and_spanning_by_hand():
    g = load_golden("worked_example.txt")
    seq, sizes = stats.sequential(np.array(g["label"], np.int32))
    assert seq.tolist() == [0, 0, 1, 1, 0, 0, 1, 1, 0, 1]          # worked by hand
    assert sizes.tolist() == [5, 5]
    lab = np.array([0, 0, 2, 2, 4, 0], np.int32)                    # clusters {0,1,5}, {2,3}, {4}
    assert stats.spanning_label(lab, np.array([1, 2]), np.array([5, 4])) == 0
    assert stats.spanning_label(lab, np.array([2]), np.array([3, 4])) == 2
    assert stats.spanning_label(lab, np.array([4]), np.array([0, 2])) == -1


# ---- dense strided neighbour lists (Section 3) and the square / cubic lattices

def _dense_cases():
    yield L.triangle(33, L.PC_TRIANGLE, 3)
    yield L.honeycomb(20, 0.7, 4, periodic_y=False)
    yield L.cayley(3, 9, 0.6, 5, perm_seed=2)
    yield L.square(30, 0.5, 6)
    yield L.cubic(9, 0.3, 7, periodic_y=False)
    yield L.random_graph(700, 1500, 8)


@pytest.mark.parametrize("slot_seed,extra", [(None, 0), (3, 0), (4, 5)])
def test_dense_oracle_equals_csr_oracle(slot_seed, extra):
    for lat in _dense_cases():
        W0 = int(np.diff(lat.row_ptr).max())
        W, nn, bits = L.to_dense(lat, W0 + extra, slot_seed)
        assert np.array_equal(oracle.dense_uf_label(lat.n, W, nn, bits), oracle.uf_label(lat))
        assert np.array_equal(oracle.dense_uf_label(lat.n, W, nn, bits), oracle.bfs_label(lat))


def test_dense_by_hand():
    # 4 sites, width 2: 0-1 open, 1-2 closed, 2-3 open, 3-0 open (ring with one gap)
    #   slot 0 of each site: its clockwise neighbour, slot 1: anticlockwise
    n, W = 4, 2
    nn = np.array([1, 2, 3, 0,  3, 0, 1, 2], np.int32)
    state = {(0, 1): 1, (1, 2): 0, (2, 3): 1, (0, 3): 1}
    bits = np.zeros(1, np.uint32)
    for e in range(8):
        i, j = e % n, int(nn[e])
        if state[(min(i, j), max(i, j))]:
            bits[0] |= np.uint32(1 << e)
    assert oracle.dense_uf_label(n, W, nn, bits).tolist() == [0, 0, 0, 0]
    bits2 = bits & ~np.uint32((1 << 3) | (1 << 4))       # close 3-0 in both slots
    assert oracle.dense_uf_label(n, W, nn, bits2).tolist() == [0, 0, 2, 2]
    with pytest.raises(ValueError):
        oracle.dense_to_csr(n, W, np.array([1, 2, 3, 4, -1, -1, -1, -1]))


def test_dense_keyed_bits_match_csr():
    lat = L.triangle(17, 0.3, 1)
    W, nn, _ = L.to_dense(lat, 8, 5)
    want = oracle.uf_label(dataclasses.replace(lat, open_bits=oracle.keyed_bits(lat, 123, 0.4)))
    assert np.array_equal(oracle.dense_uf_label(lat.n, W, nn, oracle.dense_keyed_bits(lat.n, W, nn, 123, 0.4)),
                          want)


def test_square_and_cubic_structure():
    for lat, z in ((L.square(12, 1.0, 1), 4), (L.cubic(6, 1.0, 1), 6)):
        deg = np.diff(lat.row_ptr)
        assert np.all(deg == z)
        A = sp.csr_matrix((np.ones(lat.nnz), lat.col_idx, lat.row_ptr), shape=(lat.n, lat.n))
        assert (A != A.T).nnz == 0
        assert np.all(oracle.uf_label(lat) == 0)
    assert L.cubic(6, 1.0, 1).nnz == 6 * 6 ** 3
    assert L.square(10, 1.0, 1, periodic_y=False).nnz == 4 * 100 - 2 * 10    # no wrap in y
    assert L.cubic(5, 1.0, 1, periodic_y=False).nnz == 6 * 125 - 2 * 25       # no wrap in z
    # every open bond beyond a spanning forest closes a cycle: C >= N - open bonds
    for lat in (L.square(40, 0.3, 2), L.cubic(10, 0.2, 3)):
        lab = oracle.uf_label(lat)
        assert stats.n_clusters(lab) >= lat.n - lat.n_open_bonds


def test_square_crossing_near_half():
    """Spanning curves of two sizes cross near the exact square-lattice
    bond threshold 1/2."""
    ps = [0.44, 0.47, 0.5, 0.53, 0.56]
    R = {}
    for Ls in (16, 48):
        R[Ls] = []
        for p in ps:
            hits = 0
            for s in range(300):
                lat = L.square(Ls, p, 1000 * Ls + s, periodic_y=False)
                hits += stats.spanning_label(oracle.uf_label(lat), L.row_sites(lat, 0),
                                             L.row_sites(lat, Ls - 1)) >= 0
            R[Ls].append(hits / 300)
    d = np.array(R[16]) - np.array(R[48])
    assert d[0] > 0 and d[-1] < 0
    k = int(np.flatnonzero(np.diff(np.sign(d)) != 0)[0])
    x = ps[k] + (ps[k + 1] - ps[k]) * d[k] / (d[k] - d[k + 1])
    assert abs(x - 0.5) < 0.03, (x, R)
