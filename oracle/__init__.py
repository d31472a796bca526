"""CPU oracle for bond-percolation cluster labelling -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never calls it, and it
shares no code with the library: the only thing both sides use is the input
generator in ``lattices``.

What it computes (Section 3): the canonical cluster label, the smallest site
number of each site's cluster of open bonds, where the bond {i, j} is read
from row max(i, j). Three independent C routines (``ccl_oracle.c``): weighted
union-find, breadth-first search, and the four steps of Section 3 run on one
core. ``stats`` holds the Section 4 measurements made on labels (spanning,
cluster counts, the centre cluster of a Bethe lattice). ``dense_to_csr``
reads the dense strided neighbour list of Section 3 back into CSR rows.

Parity pins (tests/test_oracle_*.py): brute force over every bond mask of
graphs with at most 12 bonds against scipy's connected components; a worked
example computed by hand (tests/golden); the forest identity clusters =
sites - open bonds; the empty residual lists of a centre-numbered Bethe
lattice; the mean centre-cluster size of a branching process; spanning-curve
crossings near 1 - 2 sin(pi/18) and 2 sin(pi/18).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ccl_oracle.c with plain gcc into oracle/_build/liboracle.so."""
    src = os.path.join(_HERE, "ccl_oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            sig = [ctypes.c_int32, ctypes.c_int64, P, P, P, ctypes.c_int64, P]
            for name in ("oracle_uf_label", "oracle_bfs_label"):
                f = getattr(lib, name)
                f.restype = ctypes.c_int
                f.argtypes = sig
            lib.oracle_steps_label.restype = ctypes.c_int
            lib.oracle_steps_label.argtypes = sig + [P, P, P, P, P, P]
            lib.oracle_splitmix64.restype = ctypes.c_uint64
            lib.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_keyed_bits.restype = ctypes.c_int
            lib.oracle_keyed_bits.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, ctypes.c_uint64,
                                              ctypes.c_double, P]
            lib.oracle_uf_label_batched.restype = ctypes.c_int
            lib.oracle_uf_label_batched.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data if a is not None else None


def _args(lat):
    rp = np.ascontiguousarray(lat.row_ptr, np.int32)
    ci = np.ascontiguousarray(lat.col_idx, np.int32)
    bits = np.ascontiguousarray(lat.open_bits, np.uint32)
    if ci.size == 0:
        ci = np.zeros(1, np.int32)
    return rp, ci, bits


def _check(rc):
    if rc == -1:
        raise ValueError("oracle: row pointer or column index out of range")
    if rc == -2:
        raise MemoryError("oracle: allocation failed")


def uf_label(lat) -> np.ndarray:
    """O1: canonical labels by weighted union-find."""
    rp, ci, bits = _args(lat)
    out = np.empty(lat.n, np.int32)
    _check(_load().oracle_uf_label(lat.n, lat.nnz, _ptr(rp), _ptr(ci), _ptr(bits), 0, _ptr(out)))
    return out


def bfs_label(lat) -> np.ndarray:
    """O2: canonical labels by breadth-first search in ascending seed order."""
    rp, ci, bits = _args(lat)
    out = np.empty(lat.n, np.int32)
    _check(_load().oracle_bfs_label(lat.n, lat.nnz, _ptr(rp), _ptr(ci), _ptr(bits), 0, _ptr(out)))
    return out


def steps_label(lat) -> dict:
    """The four steps of Section 3 on one core, with intermediate states.

    Returns dict(label, after_init, after_ii, after_iii, residual) where
    residual[i] is the residual list of site i after step (i).
    """
    rp, ci, bits = _args(lat)
    n = lat.n
    out = np.empty(n, np.int32)
    a0, a1, a2 = (np.empty(n, np.int32) for _ in range(3))
    rptr = np.empty(n + 1, np.int64)
    rj = np.empty(max(1, lat.nnz), np.int32)
    nres = ctypes.c_int64(0)
    _check(_load().oracle_steps_label(n, lat.nnz, _ptr(rp), _ptr(ci), _ptr(bits), 0, _ptr(out),
                                      _ptr(a0), _ptr(a1), _ptr(a2), _ptr(rptr), _ptr(rj),
                                      ctypes.addressof(nres)))
    residual = [rj[rptr[i]:rptr[i + 1]].copy() for i in range(n)] if n <= 100_000 else None
    return dict(label=out, after_init=a0, after_ii=a1, after_iii=a2, residual=residual,
                n_residual=int(nres.value))


def splitmix64(seed: int, k: int) -> int:
    return int(_load().oracle_splitmix64(seed & (2**64 - 1), k))


def keyed_bits(lat, seed: int, p: float) -> np.ndarray:
    """Open bits of the realisation (seed, p) whose bond {lo, hi} is drawn from
    SplitMix64 output number lo * 2^32 + hi (the library's ccl_label_random)."""
    rp, ci, _ = _args(lat)
    bits = np.zeros(max(1, (lat.nnz + 31) // 32), np.uint32)
    _check(_load().oracle_keyed_bits(lat.n, lat.nnz, _ptr(rp), _ptr(ci), seed & (2**64 - 1), float(p),
                                     _ptr(bits)))
    return bits


class _Csr:
    def __init__(self, n, row_ptr, col_idx, open_bits):
        self.n, self.nnz = n, int(col_idx.size)
        self.row_ptr, self.col_idx, self.open_bits = row_ptr, col_idx, open_bits


def dense_to_csr(n: int, width: int, nn: np.ndarray, bits: np.ndarray | None = None):
    """The graph of a dense strided neighbour list (Section 3: slot k of site
    i is nn[i + k*n], -1 = empty) as CSR rows: row i lists the non-empty slots
    of site i in slot order, each with the open bit of its slot (bit i + k*n).
    Raises ValueError for a slot outside [-1, n)."""
    nn = np.asarray(nn, np.int64).reshape(width, n) if width else np.zeros((0, n), np.int64)
    if nn.size and (nn.min() < -1 or nn.max() >= n):
        raise ValueError("dense neighbour list: slot out of range")
    used = (nn >= 0).T                                   # [n, width]: row i, slot k
    rows, ks = np.nonzero(used)                          # row-major: rows ascending, k ascending
    row_ptr = np.zeros(n + 1, np.int32)
    np.cumsum(used.sum(axis=1), out=row_ptr[1:])
    col_idx = nn[ks, rows].astype(np.int32)
    slot = rows + ks * n
    if bits is None:
        open_bits = np.zeros(max(1, (col_idx.size + 31) // 32), np.uint32)
    else:
        b = np.asarray(bits, np.uint32)
        on = ((b[slot >> 5] >> (slot & 31).astype(np.uint32)) & 1).astype(np.uint8)
        open_bits = np.zeros(max(1, (col_idx.size + 31) // 32) * 4, np.uint8)
        packed = np.packbits(on, bitorder="little")
        open_bits[:packed.size] = packed
        open_bits = open_bits.view("<u4").astype(np.uint32)
    return _Csr(n, row_ptr, col_idx, open_bits)


def dense_uf_label(n: int, width: int, nn: np.ndarray, bits: np.ndarray) -> np.ndarray:
    """Canonical labels of a dense strided neighbour list (union-find on the
    same graph as CSR rows)."""
    return uf_label(dense_to_csr(n, width, nn, bits))


def dense_keyed_bits(n: int, width: int, nn: np.ndarray, seed: int, p: float) -> np.ndarray:
    """Slot bits of realisation (seed, p): each non-empty slot gets the state
    ``keyed_bits`` gives its bond {min(i, j), max(i, j)}."""
    g = dense_to_csr(n, width, nn)
    kb = keyed_bits(g, seed, p)
    nnv = np.asarray(nn, np.int64).reshape(width, n) if width else np.zeros((0, n), np.int64)
    rows, ks = np.nonzero((nnv >= 0).T)
    slot = rows + ks * n
    on = ((kb[np.arange(g.nnz) >> 5] >> (np.arange(g.nnz) & 31).astype(np.uint32)) & 1).astype(bool)
    out = np.zeros(max(1, (width * n + 31) // 32), np.uint32)
    s_on = slot[on]
    np.bitwise_or.at(out, s_on >> 5, np.uint32(1) << (s_on & 31).astype(np.uint32))
    return out


def uf_label_batched(batch, k0: int = 0, k1: int | None = None) -> np.ndarray:
    """Union-find labels of instances [k0, k1) of a ``lattices.Batch``;
    returns the concatenated label array of those instances."""
    k1 = batch.k if k1 is None else k1
    out = np.empty(batch.n_total, np.int32)
    ci = batch.col_idx if batch.col_idx.size else np.zeros(1, np.int32)
    _check(_load().oracle_uf_label_batched(k0, k1, _ptr(batch.site_off), _ptr(batch.ent_off),
                                           _ptr(batch.row_ptr), _ptr(ci), _ptr(batch.open_bits),
                                           _ptr(out)))
    return out[int(batch.site_off[k0]):int(batch.site_off[k1])]


def uf_label_batched_threads(batch, threads: int | None = None) -> tuple[np.ndarray, int]:
    """O1 over every instance of a ``lattices.Batch``, whole instances handed
    to host threads (largest first; the C routine runs without the GIL).
    Returns (concatenated labels, threads used)."""
    from concurrent.futures import ThreadPoolExecutor
    threads = threads or os.cpu_count() or 1
    out = np.empty(max(batch.n_total, 1), np.int32)
    ci = batch.col_idx if batch.col_idx.size else np.zeros(1, np.int32)
    lib = _load()
    sizes = np.diff(batch.site_off)
    order = np.argsort(-sizes, kind="stable")

    def one(k):
        k = int(k)
        return lib.oracle_uf_label_batched(k, k + 1, _ptr(batch.site_off), _ptr(batch.ent_off),
                                           _ptr(batch.row_ptr), _ptr(ci), _ptr(batch.open_bits), _ptr(out))

    with ThreadPoolExecutor(max_workers=threads) as ex:
        for rc in ex.map(one, order):
            _check(rc)
    return out[:batch.n_total], threads


from . import stats  # noqa: E402,F401
