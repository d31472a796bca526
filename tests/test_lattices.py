"""Pins for the seeded input generator (lattices/): published SplitMix64
outputs, lattice geometry (degree, bond count, bipartiteness, faces), Cayley
tree size formula and numbering, CSR/bit symmetry and permutation bijectivity."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import lattices as L


def test_splitmix64_published_vectors():
    # First outputs of SplitMix64 from state 0 (Steele, Lea & Flood 2014; the
    # reference C implementation by Vigna prints these values).
    assert L.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert L.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert L.splitmix64(0, 2) == 0x06C45D188009454F


def _adj(lat, open_only=False):
    rows = np.repeat(np.arange(lat.n), np.diff(lat.row_ptr))
    data = np.ones(lat.nnz)
    if open_only:
        data = L.unpack_bits(lat.open_bits, lat.nnz).astype(float)
    return sp.csr_matrix((data, (rows, lat.col_idx)), shape=(lat.n, lat.n))


def _check_symmetric(lat):
    A = _adj(lat)
    assert (A != A.T).nnz == 0
    Ao = _adj(lat, open_only=True)
    assert (Ao != Ao.T).nnz == 0, "the two copies of a bond disagree"


@pytest.mark.parametrize("Lc", [4, 5, 16])
def test_honeycomb_geometry(Lc):
    lat = L.honeycomb(Lc, 0.5, 7)
    assert lat.n == 2 * Lc * Lc and lat.nnz == 6 * Lc * Lc          # 3 L^2 bonds
    assert np.all(np.diff(lat.row_ptr) == 3)                          # coordination 3
    _check_symmetric(lat)
    rows = np.repeat(np.arange(lat.n), 3)
    assert np.all((rows % 2) != (lat.col_idx % 2))                    # bipartite A-B
    A = _adj(lat)
    A2 = (A @ A).toarray()
    np.fill_diagonal(A2, 0)
    assert A2.max() <= 1                                              # no 4-cycles
    # Euler's formula on the torus, V - E + F = 0, gives F = E - V = L^2 faces;
    # with girth 6 and 3 bonds per site those faces are the L^2 hexagons.
    assert (lat.nnz // 2) - lat.n == Lc * Lc


@pytest.mark.parametrize("Lt", [4, 7, 16])
def test_triangle_geometry(Lt):
    lat = L.triangle(Lt, 0.5, 9)
    assert lat.n == Lt * Lt and lat.nnz == 6 * Lt * Lt
    assert np.all(np.diff(lat.row_ptr) == 6)
    _check_symmetric(lat)
    A = _adj(lat)
    tri = (A @ A @ A).diagonal().sum() / 6
    assert tri == 2 * Lt * Lt                                         # 2 triangles per site


def test_open_boundary_rows():
    lat = L.triangle(8, 1.0, 1, periodic_y=False)
    deg = np.diff(lat.row_ptr)
    assert np.all(deg[:8] == 4) and np.all(deg[-8:] == 4) and np.all(deg[8:-8] == 6)
    _check_symmetric(lat)
    h = L.honeycomb(8, 1.0, 1, periodic_y=False)
    dh = np.diff(h.row_ptr)
    assert np.all(dh[L.row_sites(h, 0)[:8]] == 2)      # A sites of row 0 lose their down bond
    assert np.all(dh[L.row_sites(h, 7)[8:]] == 2)      # B sites of the top row lose their up bond
    _check_symmetric(h)


@pytest.mark.parametrize("z,S", [(3, 1), (3, 6), (4, 4), (5, 3), (6, 3), (2, 5)])
def test_cayley_tree(z, S):
    lat = L.cayley(z, S, 0.5, 3)
    expect = 1 + 2 * S if z == 2 else 1 + z * ((z - 1) ** S - 1) // (z - 2)
    assert lat.n == expect
    assert lat.nnz == 2 * (lat.n - 1)
    _check_symmetric(lat)
    deg = np.diff(lat.row_ptr)
    leaves = z * (z - 1) ** (S - 1)
    assert deg[0] == z
    assert np.all(deg[lat.n - leaves:] == 1)
    assert np.all(deg[1:lat.n - leaves] == z)
    # centre-first numbering: the first entry of each row > 0 is its parent, which is lower
    rows = np.arange(1, lat.n)
    assert np.all(lat.col_idx[lat.row_ptr[rows]] < rows)
    ncomp, _ = sp.csgraph.connected_components(_adj(lat), directed=False)
    assert ncomp == 1


def test_permutation_bijective_and_relabels():
    perm, inv = L.permutation(1000, 11)
    assert np.array_equal(np.sort(perm), np.arange(1000))
    assert np.array_equal(perm[inv], np.arange(1000))
    std = L.cayley(3, 7, 0.6, 5)
    rnd = L.cayley(3, 7, 0.6, 5, perm_seed=11)
    P = rnd.meta["perm"]
    # same bonds, same states, sites renamed by perm
    def bond_set(lat, ren=None):
        rows = np.repeat(np.arange(lat.n), np.diff(lat.row_ptr))
        bits = L.unpack_bits(lat.open_bits, lat.nnz)
        a, b = rows, lat.col_idx
        if ren is not None:
            a, b = ren[a], ren[b]
        return set(zip(a.tolist(), b.tolist(), bits.tolist()))
    assert bond_set(rnd) == bond_set(std, P)


def test_bond_probability():
    lat = L.triangle(256, 0.3, 17)
    frac = lat.n_open_bonds / (lat.nnz // 2)
    assert abs(frac - 0.3) < 4 * math.sqrt(0.3 * 0.7 / (lat.nnz // 2))
    assert L.bond_open(1, 5, 1.0) and not L.bond_open(1, 5, 0.0)


def test_batch_roundtrip():
    specs = [dict(kind="honeycomb", L=5, p=0.6, seed=1), dict(kind="cayley", z=3, shells=4, p=0.5,
             seed=2, perm_seed=3), dict(kind="triangle", L=3, p=0.4, seed=4)]
    b = L.make_batch(specs)
    for k, s in enumerate(specs):
        one = L.make_instance(s)
        got = b.instance(k)
        assert np.array_equal(got.row_ptr, one.row_ptr)
        assert np.array_equal(got.col_idx, one.col_idx)
        assert np.array_equal(L.unpack_bits(got.open_bits, got.nnz),
                              L.unpack_bits(one.open_bits, one.nnz))


def test_workload_sizes():
    assert L.honeycomb(256, L.PC_HONEYCOMB, 1).n_bonds == 196_608
    tri = L.triangle(64, L.PC_TRIANGLE, 2)
    assert tri.nnz == 6 * 64 * 64
    assert L.instance_size(dict(kind="cayley", z=3, shells=24)) == 50_331_646
    assert L.instance_size(dict(kind="triangle", L=16384)) == 268_435_456
    specs = L.batched_mix_specs(64, seed=4)
    assert all(L.instance_size(s) <= 2 * 1024 * 1024 for s in specs)
    assert abs(L.PC_HONEYCOMB + L.PC_TRIANGLE - 1.0) < 1e-15     # duality of the two thresholds


def test_crossing_interpolation():
    from paper_1603_08357_gb300 import percolation as P
    ps = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    ra = np.array([0.0, 0.2, 0.4, 0.6, 1.0])
    rb = np.array([0.0, 0.1, 0.4, 0.8, 1.0])     # cross exactly at 0.3, tie at both ends
    assert P.crossing(ps, ra, rb)[0] == pytest.approx(0.3)
    rb2 = np.array([0.0, 0.1, 0.3, 0.9, 1.0])     # d = 0, .1, .1, -.3, 0 -> crossing at 0.325
    assert P.crossing(ps, ra, rb2)[0] == pytest.approx(0.325)
    assert P.crossing(ps, ra, ra) == (None, None)
