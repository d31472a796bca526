"""Section 4 measurements on the GPU: spanning probability R_span(p), its
crossing point between lattice sizes (the threshold estimate of Figs. 5 and 6),
the largest cluster and the crossing of its finite-size-scaled mean
S(L, p) L^(-91/48) between sizes (a second threshold estimate), and the
average time of one realisation at p = 0.5, 1, 1.5 p_c (Fig. 7).

Every realisation runs on the device: ``ccl_label_random`` draws the bonds
inside step (i) and labels them, ``ccl_spanning`` tests whether one cluster
touches both the first and the last row of an open-y lattice, and
``ccl_largest_cluster`` finds the largest cluster. Only three ints per
realisation come back to the host.

Realisation r at every p uses the same seed (seed0 + r). Since a bond is open
iff its uniform draw is below p, the realisations are coupled: raising p only
opens bonds, so each realisation's spanning flag is monotone in p and so is
the estimated curve.

    python -m paper_1603_08357_gb300.percolation --lattice triangle \
        --sizes 512,1024,2048,4096 --realisations 4000
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import binding as B

PC_EXACT = {"triangle": 2 * math.sin(math.pi / 18), "honeycomb": 1 - 2 * math.sin(math.pi / 18)}


def boundary_rows(kind: str, L: int):
    """Sites of the first and last rows of an L x L open-y lattice in the
    numbering of the lattice generator (honeycomb: both sites of each cell)."""
    if kind == "triangle":
        top = np.arange(L, dtype=np.int32)
        bot = np.arange((L - 1) * L, L * L, dtype=np.int32)
    else:
        c0 = np.arange(L, dtype=np.int32)
        c1 = np.arange((L - 1) * L, L * L, dtype=np.int32)
        top = np.concatenate([2 * c0, 2 * c0 + 1])
        bot = np.concatenate([2 * c1, 2 * c1 + 1])
    return top, bot


class Sampler:
    """One open-y lattice resident on the device, sampled at any p and seed."""

    def __init__(self, ctx, lat, top: np.ndarray, bottom: np.ndarray, stream=None):
        import torch
        self.ctx, self.n, self.nnz = ctx, lat.n, lat.nnz
        dev = torch.device("cuda", torch.cuda.current_device())
        self.rp = torch.from_numpy(np.ascontiguousarray(lat.row_ptr, np.int32)).to(dev)
        self.ci = torch.from_numpy(np.ascontiguousarray(lat.col_idx, np.int32)).to(dev)
        self.top = torch.from_numpy(np.ascontiguousarray(top, np.int32)).to(dev)
        self.bot = torch.from_numpy(np.ascontiguousarray(bottom, np.int32)).to(dev)
        self.labels = torch.empty(max(lat.n, 1), dtype=torch.int32, device=dev)
        self.stream = stream
        self.dev = dev

    def realise(self, seed: int, p: float, result_addr: int, largest_addr: int | None = None) -> None:
        """Labels realisation (seed, p) and writes its spanning label (-1 if
        none) to the device int at result_addr and, if largest_addr is given,
        the size and label of its largest cluster to the two device ints
        there; asynchronous."""
        B.check(B.ccl_label_random(self.ctx, self.n, self.nnz, self.rp, self.ci, seed, p, self.labels,
                                   self.stream), "ccl_label_random")
        B.check(B.ccl_spanning(self.ctx, self.n, self.labels, self.top, self.top.numel(), self.bot,
                               self.bot.numel(), result_addr, self.stream), "ccl_spanning")
        if largest_addr is not None:
            B.check(B.ccl_largest_cluster(self.ctx, self.n, self.labels, largest_addr, self.stream),
                    "ccl_largest_cluster")

    def sweep(self, ps, n_real: int, seed0: int = 0):
        """Spanning flags and largest clusters of n_real coupled realisations
        at each p: returns (span [len(ps), n_real] bool, largest
        [len(ps), n_real, 2] int32 of (size, label)), one copy back at the end."""
        import torch
        res = torch.empty((len(ps), n_real), dtype=torch.int32, device=self.dev)
        big = torch.empty((len(ps), n_real, 2), dtype=torch.int32, device=self.dev)
        base, bbase = res.data_ptr(), big.data_ptr()
        for a, p in enumerate(ps):
            for r in range(n_real):
                k = a * n_real + r
                self.realise(seed0 + r, float(p), base + 4 * k, bbase + 8 * k)
        B.check(B.ccl_sync(self.ctx, self.stream), "ccl_sync")
        return (res >= 0).cpu().numpy(), big.cpu().numpy()

    def spanning_curve(self, ps, n_real: int, seed0: int = 0) -> np.ndarray:
        """R_span at each p from n_real coupled realisations."""
        import torch
        res = torch.empty((len(ps), n_real), dtype=torch.int32, device=self.dev)
        base = res.data_ptr()
        for a, p in enumerate(ps):
            for r in range(n_real):
                self.realise(seed0 + r, float(p), base + 4 * (a * n_real + r))
        B.check(B.ccl_sync(self.ctx, self.stream), "ccl_sync")
        return (res >= 0).sum(dim=1).cpu().numpy().astype(np.float64) / n_real

    def time_per_realisation(self, p: float, reps: int, seed0: int = 1 << 40,
                             labelling_only: bool = True) -> float:
        """Average device time (ms) of one realisation at p, by CUDA events
        on the launching stream around reps back-to-back realisations."""
        import torch
        s = self.stream if self.stream is not None else torch.cuda.current_stream()
        res = torch.empty(reps, dtype=torch.int32, device=self.dev)
        for r in range(3):
            self._one(seed0 + r, p, res.data_ptr(), labelling_only)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for r in range(reps):
            self._one(seed0 + 3 + r, p, res.data_ptr() + 4 * r, labelling_only)
        e1.record(s)
        B.check(B.ccl_sync(self.ctx, self.stream), "ccl_sync")
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def _one(self, seed, p, addr, labelling_only):
        if labelling_only:
            B.check(B.ccl_label_random(self.ctx, self.n, self.nnz, self.rp, self.ci, seed, p, self.labels,
                                       self.stream), "ccl_label_random")
        else:
            self.realise(seed, p, addr)


def crossing(ps, ra, rb, n_real: int | None = None, se=None):
    """p where the curves ra and rb cross: linear interpolation of ra - rb
    between neighbouring grid points where it changes sign, skipping points
    where both curves sit at the same value (0 or 1 far from p_c). Returns
    (p_x, err) with err the standard error of the two estimates at p_x
    divided by the difference of the slopes -- binomial errors of spanning
    fractions from n_real realisations, or the given standard errors
    se = (se_a, se_b) per grid point (err is None with neither) -- or
    (None, None) if the curves do not cross."""
    ps = np.asarray(ps, np.float64)
    ra, rb = np.asarray(ra, np.float64), np.asarray(rb, np.float64)
    d = ra - rb
    live = np.flatnonzero(d != 0.0)
    for a, b in zip(live[:-1], live[1:]):
        if d[a] * d[b] < 0:
            if b > a + 1:       # equal estimates on a run of grid points between
                a, b = a + 1, b - 1
                t = 0.5 if b > a else 0.0
            else:
                t = d[a] / (d[a] - d[b])
            x = float(ps[a] + (ps[b] - ps[a]) * t)
            if n_real is None and se is None:
                return x, None
            if se is not None:
                sa, sb = np.asarray(se[0], np.float64), np.asarray(se[1], np.float64)
                var = (sa[a] + t * (sa[b] - sa[a])) ** 2 + (sb[a] + t * (sb[b] - sb[a])) ** 2
            else:
                r1, r2 = ra[a] + t * (ra[b] - ra[a]), rb[a] + t * (rb[b] - rb[a])
                var = (r1 * (1 - r1) + r2 * (1 - r2)) / n_real
            lo, hi = max(a - 1, 0), min(b + 1, len(ps) - 1)
            dslope = abs((d[hi] - d[lo]) / (ps[hi] - ps[lo]))
            return x, float(np.sqrt(var) / dslope)
    return None, None


D_FRACTAL = 91 / 48      # exact fractal dimension of 2-D percolation clusters


def scaled_largest(largest_sizes: np.ndarray, L: int):
    """Mean largest-cluster size over realisations (last axis) scaled by
    L^-D, with its standard error: at p_c it tends to a constant, so the
    scaled curves of different L cross there (finite-size scaling)."""
    v = largest_sizes.astype(np.float64)
    m = v.mean(axis=-1) / L ** D_FRACTAL
    e = v.std(axis=-1, ddof=1) / np.sqrt(v.shape[-1]) / L ** D_FRACTAL
    return m, e


def main(argv=None):
    import torch
    import lattices as Lt
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--lattice", choices=["triangle", "honeycomb"], default="triangle")
    ap.add_argument("--sizes", default="")
    ap.add_argument("--realisations", type=int, default=2000)
    ap.add_argument("--width", type=float, default=0.006, help="half-width of the p grid around p_c")
    ap.add_argument("--points", type=int, default=13)
    ap.add_argument("--timing-reps", type=int, default=50)
    ap.add_argument("--seed", type=int, default=11)
    a = ap.parse_args(argv)
    kind = a.lattice
    sizes = [int(s) for s in a.sizes.split(",")] if a.sizes else (
        [512, 1024, 2048, 4096] if kind == "triangle" else [362, 724, 1448, 2896])
    pc = PC_EXACT[kind]
    ps = np.linspace(pc - a.width, pc + a.width, a.points)
    ctx = B.ccl_context_create(torch.cuda.current_device())
    curves = {}
    for L in sizes:
        lat = (Lt.triangle if kind == "triangle" else Lt.honeycomb)(L, 0.0, 0, periodic_y=False)
        top, bot = boundary_rows(kind, L)
        smp = Sampler(ctx, lat, top, bot)
        t0 = time.perf_counter()
        span, big = smp.sweep(ps, a.realisations, a.seed * 1_000_003 + L)
        wall = time.perf_counter() - t0
        R = span.mean(axis=1)
        S, S_err = scaled_largest(big[..., 0], L)
        times = {f"{m}pc": smp.time_per_realisation(m * pc, a.timing_reps) for m in (0.5, 1.0, 1.5)}
        curves[L] = (R, S, S_err)
        print(json.dumps({"lattice": kind, "L": L, "N": lat.n, "realisations": a.realisations,
                          "p": [round(float(p), 6) for p in ps], "R_span": [round(float(r), 5) for r in R],
                          "largest_scaled": [round(float(x), 6) for x in S],
                          "ms_per_realisation": {k: round(v, 4) for k, v in times.items()},
                          "sweep_wall_s": round(wall, 2)}), flush=True)
        del smp
        torch.cuda.empty_cache()
    pairs = [(sizes[i], sizes[i + 1]) for i in range(len(sizes) - 1)]
    xs = {f"{u}x{v}": crossing(ps, curves[u][0], curves[v][0], a.realisations) for u, v in pairs}
    xl = {f"{u}x{v}": crossing(ps, curves[u][1], curves[v][1], se=(curves[u][2], curves[v][2]))
          for u, v in pairs}
    print(json.dumps({"lattice": kind, "p_c_exact": round(pc, 6), "crossings": xs,
                      "largest_cluster_crossings": xl}), flush=True)
    B.ccl_context_destroy(ctx)


if __name__ == "__main__":
    main()
