"""Seeded synthetic bond-percolation inputs (Section 4 workloads).

The honeycomb, triangle and Bethe (Cayley tree) lattices of Section 4 as CSR
neighbour lists plus one open/closed bit per CSR entry, and the batched and
served mixes built from them. This module holds none of the labelling
method's arithmetic: it only produces inputs, which the CPU oracle and the
CUDA library both consume. Geometry, numbering and the random stream are
documented in ``gen.c``.

Thresholds used to pick ``p`` (Section 4): p_c = 1 - 2 sin(pi/18) for the
honeycomb lattice, 2 sin(pi/18) for the triangle lattice, 1/(z-1) for the
Bethe lattice of coordination z.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liblattices.so")
_lock = threading.Lock()
_lib = None

PC_HONEYCOMB = 1.0 - 2.0 * math.sin(math.pi / 18.0)
PC_TRIANGLE = 2.0 * math.sin(math.pi / 18.0)
PC_SQUARE = 0.5                 # bond percolation, exact (Sykes & Essam 1964)
PC_CUBIC = 0.2488126            # simple cubic bond percolation (Lorenz & Ziff 1998)


def pc_bethe(z: int) -> float:
    return 1.0 / (z - 1)


def build(force: bool = False) -> str:
    """Compile gen.c into _build/liblattices.so (plain gcc, no arch flags)."""
    src = os.path.join(_HERE, "gen.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


class _Desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("L", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("z", ctypes.c_int32), ("shells", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("perm", ctypes.c_void_p), ("perm_inv", ctypes.c_void_p), ("n", ctypes.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.lat_splitmix64.restype = ctypes.c_uint64
            lib.lat_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.lat_bond_open.restype = ctypes.c_int
            lib.lat_bond_open.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double]
            lib.lat_cayley_nsites.restype = ctypes.c_int64
            lib.lat_cayley_nsites.argtypes = [ctypes.c_int32, ctypes.c_int32]
            lib.lat_count_entries.restype = ctypes.c_int64
            lib.lat_count_entries.argtypes = [ctypes.POINTER(_Desc)]
            lib.lat_fill.restype = ctypes.c_int64
            lib.lat_fill.argtypes = [ctypes.POINTER(_Desc), ctypes.c_uint64, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int64)]
            lib.lat_copy_bits.restype = None
            lib.lat_copy_bits.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_int64]
            lib.lat_permutation.restype = None
            lib.lat_permutation.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p,
                                            ctypes.c_void_p]
            _lib = lib
    return _lib


def splitmix64(seed: int, k: int) -> int:
    """Output number k (0-based) of SplitMix64 started from state ``seed``."""
    return int(_load().lat_splitmix64(seed & (2**64 - 1), k))


def bond_open(seed: int, bond: int, p: float) -> bool:
    return bool(_load().lat_bond_open(seed & (2**64 - 1), bond, p))


def _threads() -> int:
    return max(1, min(os.cpu_count() or 1, 64))


@dataclass
class Lattice:
    """One instance: CSR rows over sites 0..n-1 plus per-entry open bits.

    ``open_bits`` has ceil(nnz/32) uint32 words (at least one); bit e (word
    e >> 5, bit e & 31) is the state of CSR entry e.
    """
    kind: str
    n: int
    nnz: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    open_bits: np.ndarray
    p: float
    seed: int
    n_open_bonds: int = -1
    meta: dict = field(default_factory=dict)

    @property
    def n_bonds(self) -> int:
        return self.nnz // 2


def _desc(kind: str, n: int, L=0, periodic_y=True, z=0, shells=0, perm=None, perm_inv=None):
    d = _Desc()
    d.kind = {"honeycomb": 0, "triangle": 1, "cayley": 2, "square": 3, "cubic": 4}[kind]
    d.L, d.periodic_y, d.z, d.shells, d.n = L, int(bool(periodic_y)), z, shells, n
    d.perm = perm.ctypes.data if perm is not None else None
    d.perm_inv = perm_inv.ctypes.data if perm_inv is not None else None
    return d


def _nsites(kind, L=0, z=0, shells=0) -> int:
    if kind == "honeycomb":
        return 2 * L * L
    if kind in ("triangle", "square"):
        return L * L
    if kind == "cubic":
        return L * L * L
    return int(_load().lat_cayley_nsites(z, shells))


def _fill_into(d: _Desc, seed, p, row_ptr, col_idx, bits, bit_off, nthreads):
    """Fill preallocated views; returns (nnz, open_bonds)."""
    ob = ctypes.c_int64(0)
    nnz = _load().lat_fill(ctypes.byref(d), seed & (2**64 - 1), float(p), row_ptr.ctypes.data,
                           col_idx.ctypes.data, col_idx.size, bits.ctypes.data, bit_off,
                           nthreads, ctypes.byref(ob))
    if nnz < 0:
        raise ValueError("lattice too large for int32 CSR")
    return int(nnz), int(ob.value)


def permutation(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    perm = np.empty(n, np.int32)
    inv = np.empty(n, np.int32)
    _load().lat_permutation(n, seed & (2**64 - 1), perm.ctypes.data, inv.ctypes.data)
    return perm, inv


def _make(kind, seed, p, nthreads=None, **kw) -> Lattice:
    lib = _load()
    n = _nsites(kind, kw.get("L", 0), kw.get("z", 0), kw.get("shells", 0))
    perm = perm_inv = None
    if kind == "cayley" and kw.get("perm_seed") is not None:
        perm, perm_inv = permutation(n, kw["perm_seed"])
    d = _desc(kind, n, L=kw.get("L", 0), periodic_y=kw.get("periodic_y", True), z=kw.get("z", 0),
              shells=kw.get("shells", 0), perm=perm, perm_inv=perm_inv)
    nnz = int(lib.lat_count_entries(ctypes.byref(d)))
    row_ptr = np.empty(n + 1, np.int32)
    col_idx = np.empty(nnz, np.int32)
    bits = np.zeros(max(1, (nnz + 31) // 32), np.uint32)
    nnz2, ob = _fill_into(d, seed, p, row_ptr, col_idx, bits, 0, nthreads or _threads())
    assert nnz2 == nnz
    meta = {k: v for k, v in kw.items()}
    if perm is not None:
        meta["perm"] = perm
    return Lattice(kind, n, nnz, row_ptr, col_idx, bits, p, seed, ob, meta)


def honeycomb(L: int, p: float, seed: int, periodic_y: bool = True, nthreads=None) -> Lattice:
    """Honeycomb bond percolation on L x L unit cells (N = 2 L^2)."""
    lat = _make("honeycomb", seed, p, nthreads, L=L, periodic_y=periodic_y)
    return lat


def triangle(L: int, p: float, seed: int, periodic_y: bool = True, nthreads=None) -> Lattice:
    """Triangle-lattice bond percolation on L x L sites (coordination 6)."""
    return _make("triangle", seed, p, nthreads, L=L, periodic_y=periodic_y)


def square(L: int, p: float, seed: int, periodic_y: bool = True, nthreads=None) -> Lattice:
    """Square-lattice bond percolation on L x L sites (coordination 4)."""
    return _make("square", seed, p, nthreads, L=L, periodic_y=periodic_y)


def cubic(L: int, p: float, seed: int, periodic_y: bool = True, nthreads=None) -> Lattice:
    """Simple-cubic bond percolation on L^3 sites (coordination 6); with
    periodic_y=False the z direction is open."""
    return _make("cubic", seed, p, nthreads, L=L, periodic_y=periodic_y)


def cayley(z: int, shells: int, p: float, seed: int, perm_seed: int | None = None,
           nthreads=None) -> Lattice:
    """Bethe-lattice (Cayley tree) bond percolation, coordination z, `shells` shells.

    perm_seed=None keeps the standard (centre-first) numbering; otherwise the
    sites are stored under a seeded uniform permutation ("random position").
    """
    return _make("cayley", seed, p, nthreads, z=z, shells=shells, perm_seed=perm_seed)


def row_sites(lat: Lattice, y: int) -> np.ndarray:
    """Sites whose cell row is y (honeycomb: both A and B of the cell; cubic:
    the plane z = y)."""
    L = lat.meta["L"]
    if lat.kind in ("triangle", "square"):
        return np.arange(y * L, (y + 1) * L, dtype=np.int64)
    if lat.kind == "cubic":
        return np.arange(y * L * L, (y + 1) * L * L, dtype=np.int64)
    c = np.arange(y * L, (y + 1) * L, dtype=np.int64)
    return np.concatenate([2 * c, 2 * c + 1])


def cayley_center(lat: Lattice) -> int:
    perm = lat.meta.get("perm")
    return int(perm[0]) if perm is not None else 0


def random_graph(n: int, m: int, seed: int, self_loops: bool = True,
                 asymmetric: float = 0.0, p: float = 0.5) -> Lattice:
    """Random multigraph with m edges as a CSR listing each edge in both rows.

    Edge t = {u_t, v_t} has one bond id t. With ``asymmetric`` > 0 that
    fraction of edges draws an independent bit for the copy stored in the
    lower-numbered row, so the two directions can disagree.
    """
    rng = np.random.default_rng(seed)
    u = rng.integers(0, max(n, 1), m) if n > 0 else np.zeros(0, np.int64)
    v = rng.integers(0, max(n, 1), m) if n > 0 else np.zeros(0, np.int64)
    if not self_loops and n > 1:
        same = u == v
        v[same] = (u[same] + 1) % n
    is_open = rng.random(m) < p
    skew = rng.random(m) < asymmetric
    alt = rng.random(m) < p
    # entries: (row, col, bit)
    rows = np.concatenate([u, v]).astype(np.int64)
    cols = np.concatenate([v, u]).astype(np.int64)
    bit_u = np.where((u < v) & skew, alt, is_open)    # copy stored in row u
    bit_v = np.where((v < u) & skew, alt, is_open)    # copy stored in row v
    bitv = np.concatenate([bit_u, bit_v])
    order = np.argsort(rows, kind="stable")
    rows, cols, bitv = rows[order], cols[order], bitv[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    nnz = 2 * m
    bits = pack_bits(bitv)
    return Lattice("random", n, nnz, row_ptr, cols.astype(np.int32), bits, p, seed, -1,
                   {"edges": (u, v), "open": is_open})


def pack_bits(bitv: np.ndarray) -> np.ndarray:
    """Pack a boolean per-entry array into little-endian uint32 words."""
    nnz = bitv.size
    nw = max(1, (nnz + 31) // 32)
    padded = np.zeros(nw * 32, np.uint8)
    padded[:nnz] = bitv.astype(np.uint8)
    b = np.packbits(padded, bitorder="little")
    return b.view("<u4").astype(np.uint32)


def unpack_bits(bits: np.ndarray, nnz: int, bit_off: int = 0) -> np.ndarray:
    b = np.unpackbits(bits.astype("<u4").view(np.uint8), bitorder="little")
    return b[bit_off:bit_off + nnz].astype(bool)


# ---------------------------------------------------------------------------
# Batched instances: concatenated CSR with int64 per-instance offsets.
# ---------------------------------------------------------------------------

@dataclass
class Batch:
    """K instances in concatenated form.

    Instance k owns sites [site_off[k], site_off[k+1]) and entries
    [ent_off[k], ent_off[k+1]); its n_k + 1 local row pointers start at
    row_ptr[site_off[k] + k]; its col_idx values are local site indices; the
    bit of its local entry e is global bit ent_off[k] + e of ``open_bits``.
    """
    site_off: np.ndarray
    ent_off: np.ndarray
    row_ptr: np.ndarray
    col_idx: np.ndarray
    open_bits: np.ndarray
    specs: list

    @property
    def k(self) -> int:
        return len(self.specs)

    @property
    def n_total(self) -> int:
        return int(self.site_off[-1])

    @property
    def nnz_total(self) -> int:
        return int(self.ent_off[-1])

    def aligned_bits(self, nthreads=None):
        """The bits again, each instance starting on a word boundary: returns
        (bits, word_off) with instance k's entry e at bit 32*word_off[k] + e."""
        nnz = np.diff(self.ent_off)
        words = (nnz + 31) // 32
        word_off = np.zeros(self.k + 1, np.int64)
        word_off[1:] = np.cumsum(words)
        out = np.zeros(max(1, int(word_off[-1])), np.uint32)
        lib = _load()

        def one(k):
            lib.lat_copy_bits(self.open_bits.ctypes.data, int(self.ent_off[k]), int(nnz[k]),
                              out.ctypes.data, 32 * int(word_off[k]))
        with ThreadPoolExecutor(max_workers=nthreads or _threads()) as ex:
            list(ex.map(one, range(self.k)))
        return out, word_off

    def instance(self, k: int) -> Lattice:
        s0, s1 = int(self.site_off[k]), int(self.site_off[k + 1])
        e0, e1 = int(self.ent_off[k]), int(self.ent_off[k + 1])
        n, nnz = s1 - s0, e1 - e0
        rp = self.row_ptr[s0 + k: s1 + k + 1]
        ci = self.col_idx[e0:e1]
        bits = pack_bits(unpack_bits(self.open_bits, nnz, e0))
        sp = self.specs[k]
        return Lattice(sp["kind"], n, nnz, rp, ci, bits, sp["p"], sp["seed"], -1, dict(sp))


def _spec_desc(sp):
    n = _nsites(sp["kind"], sp.get("L", 0), sp.get("z", 0), sp.get("shells", 0))
    perm = perm_inv = None
    if sp.get("perm_seed") is not None:
        perm, perm_inv = permutation(n, sp["perm_seed"])
    d = _desc(sp["kind"], n, L=sp.get("L", 0), periodic_y=sp.get("periodic_y", True),
              z=sp.get("z", 0), shells=sp.get("shells", 0), perm=perm, perm_inv=perm_inv)
    return n, d, (perm, perm_inv)


def make_batch(specs: list, nthreads=None) -> Batch:
    """Generate instances described by dicts (kind, L | z, shells, p, seed[, perm_seed])."""
    lib = _load()
    K = len(specs)
    descs, ns, nnzs, keep = [], [], [], []
    for sp in specs:
        n, d, hold = _spec_desc(sp)
        descs.append(d); keep.append(hold); ns.append(n)
        nnzs.append(int(lib.lat_count_entries(ctypes.byref(d))))
    site_off = np.zeros(K + 1, np.int64)
    ent_off = np.zeros(K + 1, np.int64)
    site_off[1:] = np.cumsum(ns)
    ent_off[1:] = np.cumsum(nnzs)
    row_ptr = np.empty(int(site_off[-1]) + K, np.int32)
    col_idx = np.empty(int(ent_off[-1]), np.int32)
    bits = np.zeros(max(1, (int(ent_off[-1]) + 31) // 32), np.uint32)

    def one(k):
        s0, e0 = int(site_off[k]), int(ent_off[k])
        rp = row_ptr[s0 + k: s0 + k + ns[k] + 1]
        ci = col_idx[e0:e0 + nnzs[k]]
        nnz, _ = _fill_into(descs[k], specs[k]["seed"], specs[k]["p"], rp, ci, bits, e0, 1)
        assert nnz == nnzs[k]

    with ThreadPoolExecutor(max_workers=nthreads or _threads()) as ex:
        list(ex.map(one, range(K)))
    return Batch(site_off, ent_off, row_ptr, col_idx, bits, list(specs))


def batched_mix_specs(K: int = 4096, seed: int = 4, max_cayley_sites: int = 2 * 1024 * 1024):
    """The batched workload: K instances, each uniformly honeycomb, triangle or
    Cayley tree. Honeycomb/triangle: L uniform integer in 64..1024. Cayley: z
    uniform in {3,4,5,6}, shells uniform in 8..S_max(z), S_max the largest
    shell count <= 16 with at most ``max_cayley_sites`` sites. p uniform in
    p_c +- 0.05 for the instance's lattice."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(K):
        t = int(rng.integers(0, 3))
        s = {"seed": int(seed * 1_000_003 + k)}
        if t < 2:
            L = int(rng.integers(64, 1025))
            kind = "honeycomb" if t == 0 else "triangle"
            pc = PC_HONEYCOMB if t == 0 else PC_TRIANGLE
            s.update(kind=kind, L=L)
        else:
            z = int(rng.integers(3, 7))
            smax = 16
            while _nsites("cayley", z=z, shells=smax) > max_cayley_sites:
                smax -= 1
            sh = int(rng.integers(8, smax + 1))
            pc = pc_bethe(z)
            s.update(kind="cayley", z=z, shells=sh, perm_seed=int(seed * 7_000_001 + k))
        s["p"] = float(pc + rng.uniform(-0.05, 0.05))
        specs.append(s)
    return specs


def served_specs(n_req: int = 20000, seed: int = 5, lo: float = 1e3, hi: float = 1e7):
    """Requests with sizes log-uniform in [lo, hi] sites over the three lattice
    types at their p_c. Size is matched by the lattice parameter nearest to the
    drawn site count (L for honeycomb/triangle, shells for a z=3 tree)."""
    rng = np.random.default_rng(seed)
    specs = []
    for r in range(n_req):
        target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        t = int(rng.integers(0, 3))
        s = {"seed": int(seed * 1_000_003 + r)}
        if t == 0:
            L = max(2, int(round(math.sqrt(target / 2))))
            s.update(kind="honeycomb", L=L, p=PC_HONEYCOMB)
        elif t == 1:
            L = max(2, int(round(math.sqrt(target))))
            s.update(kind="triangle", L=L, p=PC_TRIANGLE)
        else:
            sh = max(1, int(round(math.log2(max(target - 1, 3) / 3 + 1))))
            s.update(kind="cayley", z=3, shells=sh, p=pc_bethe(3),
                     perm_seed=int(seed * 7_000_001 + r))
        specs.append(s)
    return specs


def make_instance(spec: dict, nthreads=None) -> Lattice:
    kind = spec["kind"]
    if kind == "honeycomb":
        return honeycomb(spec["L"], spec["p"], spec["seed"], spec.get("periodic_y", True), nthreads)
    if kind == "triangle":
        return triangle(spec["L"], spec["p"], spec["seed"], spec.get("periodic_y", True), nthreads)
    if kind == "square":
        return square(spec["L"], spec["p"], spec["seed"], spec.get("periodic_y", True), nthreads)
    if kind == "cubic":
        return cubic(spec["L"], spec["p"], spec["seed"], spec.get("periodic_y", True), nthreads)
    return cayley(spec["z"], spec["shells"], spec["p"], spec["seed"], spec.get("perm_seed"), nthreads)


def instance_size(spec: dict) -> int:
    return _nsites(spec["kind"], spec.get("L", 0), spec.get("z", 0), spec.get("shells", 0))


def to_dense(lat: Lattice, width: int | None = None, slot_seed: int | None = None):
    """The dense strided neighbour list of the same graph and bond states:
    returns (width, nn, bits) with nn int32[width * n] (slot k of site i at
    nn[i + k*n], -1 where empty) and bits uint32[ceil(width*n/32)] (slot e's
    state at bit e). width defaults to the largest degree; with slot_seed
    each row's entries go to seeded random distinct slots (empty slots then
    sit between used ones), else to slots 0..deg-1 in CSR order."""
    n = lat.n
    rp = np.asarray(lat.row_ptr, np.int64)
    deg = np.diff(rp)
    W = int(deg.max()) if n and lat.nnz else 0
    width = W if width is None else int(width)
    if width < W:
        raise ValueError("width below the largest degree")
    nn = np.full(width * n, -1, np.int32)
    bits = np.zeros(max(1, (width * n + 31) // 32), np.uint32)
    if lat.nnz == 0:
        return width, nn, bits
    row = np.repeat(np.arange(n, dtype=np.int64), deg)
    k = np.arange(lat.nnz, dtype=np.int64) - rp[row]
    if slot_seed is not None:
        rng = np.random.default_rng(slot_seed)
        keys = rng.random((n, width)).argsort(axis=1)      # a random slot order per row
        k = keys[row, k]
    slot = row + k * n
    nn[slot] = np.asarray(lat.col_idx, np.int32)
    on = unpack_bits(lat.open_bits, lat.nnz).astype(bool)
    s_on = slot[on]
    np.bitwise_or.at(bits, s_on >> 5, (np.uint32(1) << (s_on & 31).astype(np.uint32)))
    return width, nn, bits
