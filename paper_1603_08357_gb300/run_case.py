"""Runs one labelling workload through the C ABI a fixed number of times, for
profilers (ncu) and quick checks: no timing, no oracle.

    python -m paper_1603_08357_gb300.run_case --workload tri4096 --steps 3
    python -m paper_1603_08357_gb300.run_case --workload batched --instances 128 --steps 2

The calls after the warm-up run inside an NVTX range named "steps", so a
profiler can be limited to them (ncu --nvtx --nvtx-include "steps/").
Workloads: the single instances of the benchmark (hc256, tri4096, bethe24,
tri16384) and the first --instances instances of the batched mix (seed 4).
Launch settings: the library's defaults, or its autotuner with --autotune.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SINGLE = {
    "hc256": dict(kind="honeycomb", L=256, p=0.6527, seed=1),
    "tri4096": dict(kind="triangle", L=4096, p=0.3473, seed=2),
    "bethe24": dict(kind="cayley", z=3, shells=24, p=0.5, seed=3, perm_seed=3),
    "tri16384": dict(kind="triangle", L=16384, p=0.3473, seed=5),
}


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", choices=sorted(SINGLE) + ["batched"], default="tri4096")
    ap.add_argument("--instances", type=int, default=4096, help="batched: the first this many instances")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--autotune", action="store_true")
    a = ap.parse_args(argv)
    import torch
    import lattices as L
    from . import binding as B
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = B.ccl_context_create(dev.index)
    stream = torch.cuda.current_stream()
    if a.workload == "batched":
        b = L.make_batch(L.batched_mix_specs(4096, seed=4)[:a.instances])
        rp, ci = torch.from_numpy(b.row_ptr).to(dev), torch.from_numpy(b.col_idx).to(dev)
        bits = torch.from_numpy(b.open_bits.view(np.int32)).to(dev)
        out = torch.empty(b.n_total, dtype=torch.int32, device=dev)
        if a.autotune:
            B.check(B.ccl_autotune_batched(ctx, b.k, b.site_off, b.ent_off, rp, ci, bits, out, stream)[0], "autotune")
        call = lambda: B.ccl_label_batched(ctx, b.k, b.site_off, b.ent_off, rp, ci, bits, out, stream)  # noqa: E731
    else:
        lat = L.make_instance(SINGLE[a.workload])
        rp, ci = torch.from_numpy(lat.row_ptr).to(dev), torch.from_numpy(lat.col_idx).to(dev)
        bits = torch.from_numpy(lat.open_bits.view(np.int32)).to(dev)
        out = torch.empty(lat.n, dtype=torch.int32, device=dev)
        if a.autotune:
            B.check(B.ccl_autotune(ctx, lat.n, lat.nnz, rp, ci, bits, out, stream)[0], "autotune")
        call = lambda: B.ccl_label(ctx, lat.n, lat.nnz, rp, ci, bits, out, stream)  # noqa: E731
    for _ in range(a.warmup):
        B.check(call(), "label")
    B.check(B.ccl_sync(ctx, stream), "warm-up")
    torch.cuda.nvtx.range_push("steps")
    for _ in range(a.steps):
        B.check(call(), "label")
    torch.cuda.nvtx.range_pop()
    B.check(B.ccl_sync(ctx, stream), "steps")
    st = B.ccl_get_stats(ctx)
    print(f"{a.workload}: {st.n_inst} instance(s), {st.n_sites} sites, {st.nnz} entries, "
          f"{st.residual_pairs} residual pairs, {a.steps} step(s)")
    B.ccl_context_destroy(ctx)


if __name__ == "__main__":
    main()
