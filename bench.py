#!/usr/bin/env python3
"""Benchmark of the GB300 cluster-labelling path (Komura's generalized GPU CCL).

One step = one pass of the four labelling steps (init, analysis, label
reduction, analysis) over one instance of the workload, inputs resident in
HBM. Default workload: triangle-lattice bond percolation, 4096 x 4096 sites
(16,777,216 sites, 100,663,296 CSR entries), periodic, p = 0.3473, seed 2.

Prints one JSON line (rank 0): sites labelled per second over all ranks,
the roofline of the dominant kernel, the CPU oracle baseline, the end-to-end
figure through the host-buffer entry point, and the clocks seen meanwhile.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME] [--impl ours|reference]

Multi-GPU (torchrun): replicas only -- every rank labels its own seeded
instance, with no collective on the data path; ranks meet at barriers around
the timed region and the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lattices as L  # noqa: E402

CONFIGS = {
    "tri4096": dict(kind="triangle", L=4096, p=0.3473, seed=2,
                    desc="triangle bond percolation 4096x4096 periodic p=0.3473"),
    "hc256": dict(kind="honeycomb", L=256, p=0.6527, seed=1,
                  desc="honeycomb bond percolation 256x256 cells periodic p=0.6527"),
    "bethe24": dict(kind="cayley", z=3, shells=24, p=0.5, seed=3, perm_seed=3,
                    desc="Bethe lattice z=3, 24 shells, random position, p=0.5"),
    "tri16384": dict(kind="triangle", L=16384, p=0.3473, seed=5,
                     desc="triangle bond percolation 16384x16384 periodic p=0.3473"),
}
L2_BYTES = 129 * 1024 * 1024
METRIC = "sites labeled/s per GB300 (batched vs one-at-a-time); achieved HBM GB/s"


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# clocks during the timed region: NVML through ctypes (read-only queries)

class ClockSampler:
    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x100: "display_clock_setting"}

    def __init__(self, index: int, uuid: str | None = None):
        self.samples, self.reasons, self.max_mhz = [], 0, None
        self._stop = threading.Event()
        self._th = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = ctypes.c_void_p()
            found = False
            if uuid:
                u = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
                found = nv.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) == 0
            if not found and nv.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(h)) != 0:
                raise OSError("no handle")
            self.nv, self.h = nv, h
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:   # NVML_CLOCK_SM = 1
                self.max_mhz = int(mx.value)
        except OSError:
            self.nv = None

    def _run(self):
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        fn = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0:
                self.samples.append(int(clk.value))
            if fn(self.h, ctypes.byref(rs)) == 0:
                self.reasons |= int(rs.value)
            time.sleep(0.001)

    def start(self):
        if self.nv is not None:
            self._th = threading.Thread(target=self._run, daemon=True)
            self._th.start()

    def stop(self):
        if self._th is not None:
            self._stop.set()
            self._th.join()
        names = [v for k, v in self.REASONS.items() if self.reasons & k and k != 0x1]
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None,
                "sm_max_mhz": self.max_mhz, "reasons": names, "samples": len(self.samples),
                "source": "nvml" if self.nv is not None else "unavailable"}


# ----------------------------------------------------------------------------
# The CPU-baseline leg and the reference arm: the only places that run the
# oracle. The leg also compares the GPU's labels with the oracle's labels of the
# same input, which it computes anyway.

def oracle_time(lat, budget_s: float, min_reps: int = 1, check=None):
    """Times the oracle's union-find labelling of the full instance on one core,
    repeating until `budget_s` seconds have elapsed; returns (sites/s, reps,
    secs, same) with same = whether `check` equals the oracle's labels (None
    without `check`)."""
    import oracle
    reps, t0 = 0, time.perf_counter()
    labels = None
    while True:
        labels = oracle.uf_label(lat)
        reps += 1
        el = time.perf_counter() - t0
        if reps >= min_reps and el >= budget_s:
            break
    same = None if check is None else bool(np.array_equal(check, labels))
    return lat.n * reps / el, reps, el, same


def oracle_input(lat, seed=None):
    """The instance the oracle labels: lat itself, or (bonds drawn on the
    device) lat with the open bits of realisation (seed, lat.p)."""
    if seed is None:
        return lat
    import dataclasses
    import oracle
    return dataclasses.replace(lat, open_bits=oracle.keyed_bits(lat, seed, lat.p))


def replica_spec(name: str, rank: int) -> dict:
    """The instance rank `rank` labels: the workload with its seeds offset per
    rank (replicas: every rank labels an independent instance of the same
    shape; nothing is exchanged)."""
    c = dict(CONFIGS[name])
    c.pop("desc")
    c["seed"] = c["seed"] + 1000 * rank
    if "perm_seed" in c:
        c["perm_seed"] = c["perm_seed"] + 1000 * rank
    return c


P_OVERRIDE = None      # --p: the bond probability of a single-instance config


def make_workload(name: str, rank: int):
    spec = replica_spec(name, rank)
    desc = CONFIGS[name]["desc"]
    if P_OVERRIDE is not None:
        spec["p"] = P_OVERRIDE
        desc = desc.replace(f"p={CONFIGS[name]['p']}", f"p={P_OVERRIDE}")
    return L.make_instance(spec), desc


def max_over_ranks(value: float, dist, device=None) -> float:
    """The job's step time: the slowest rank's (barrier-bracketed) time."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algorithmic_bytes(n: int, nnz: int, q: int, input_kind: str = "csr", width: int = 0,
                      rows: int | None = None) -> dict:
    """Minimum bytes each step must move (each array read or written once).

    init (csr):          row_ptr 4 rows (n+1, or n+K for K batched instances)
                         + col_idx 4 nnz + bit words 4 ceil(nnz/32)
                         + labels 4n + residual pairs 8q
    init (random):       as csr without the bit words (bonds drawn on the device)
    init (dense):        neighbour slots 4 width n + bit words 4 ceil(width n/32)
                         + labels 4n + pairs 8q
    init (dense-random): neighbour slots 4 width n + labels 4n + pairs 8q
    analysis: labels read 4n + write 4n (each of steps ii and iv)
    reduce:   pairs 8q + two label reads 8q
    """
    if input_kind in ("dense", "dense-random"):
        slots = width * n
        b_in = 4 * slots + (4 * ((slots + 31) // 32) if input_kind == "dense" else 0)
    else:
        b_in = 4 * (n + 1 if rows is None else rows) + 4 * nnz + \
            (4 * ((nnz + 31) // 32) if input_kind == "csr" else 0)
    b_init = b_in + 4 * n + 8 * q
    b_ana = 8 * n
    b_red = 16 * q
    return {"init": b_init, "analysis_ii": b_ana, "reduce": b_red, "analysis_iv": b_ana,
            "path": b_init + 2 * b_ana + b_red}


# The sources of the kernels bench.py times and of the host code that sizes
# and launches them; the request loop and the allocation-free entry do not
# change what those launches run.
KERNEL_SOURCES = ("ccl_api.cu", "ccl_dense.cuh", "ccl_device.cuh", "ccl_stats.cuh", "ccl_types.cuh")


def _source_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(KERNEL_SOURCES):
        with open(os.path.join(ROOT, "paper_1603_08357_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (same hash) or on sources that differ from them
    only outside the kernels and their launches (an entry's
    equivalent_source_hashes, each with the change named in its note); else
    None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        ent = rec.get(f"{kernel}:{workload}")
        h = _source_hash()
        if ent and (ent.get("source_hash") == h or h in ent.get("equivalent_source_hashes", [])):
            return float(ent["dram_bytes_per_launch"]), ent.get("scaled_from")
    except Exception:
        pass
    return None, None


# ----------------------------------------------------------------------------

def _reference_sample(args):
    """What one reference step labels, as (run_step, sites, entries, desc,
    cores): the whole instance (one core) for the single-instance configs;
    for the batched mix its first --reference-instances instances with whole
    instances spread over the host's cores (as the CPU-baseline leg does);
    for the served stream its first 24 requests (one core)."""
    import oracle
    if args.config == "batched":
        specs = L.batched_mix_specs(args.instances, seed=4)[:args.reference_instances]
        sb = L.make_batch(specs)
        cores = os.cpu_count() or 1
        return (lambda: oracle.uf_label_batched_threads(sb, cores), sb.n_total, sb.nnz_total,
                f"batched mix, first {sb.k} instances, whole instances over {cores} threads", cores)
    if args.config == "served":
        lats = [L.make_instance(sp) for sp in L.served_specs(args.requests, seed=5)[:24]]
        desc = "served stream, first 24 requests"
    else:
        lats, desc = [make_workload(args.config, 0)[0]], make_workload(args.config, 0)[1]

    def run_step():
        for x in lats:
            oracle.uf_label(x)
    return run_step, sum(x.n for x in lats), sum(x.nnz for x in lats), desc, 1


def run_reference(args, rank, world):
    if rank != 0:
        return
    one_step, n_step, nnz_step, desc, cores = _reference_sample(args)
    for _ in range(args.warmup):
        one_step()
    t_all = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    wall = time.perf_counter() - t_all
    ms = 1e3 * wall / args.steps
    value = n_step / (ms / 1e3)
    line = {
        "impl": "reference", "value": value, "unit": "sites/s",
        "metric": METRIC if args.config == "batched" else (
            "sites labeled/s (served)" if args.config == "served" else "sites labeled/s"),
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": args.config, "desc": desc, "n_sites": n_step, "nnz": nnz_step,
                   "l2": "inputs larger than L2 (no flush)" if nnz_step * 4 > L2_BYTES else "L2-resident"},
        "cpu_baseline": {"value": value, "unit": "sites/s", "cores": cores, "kind": "oracle",
                         "sample": f"union-find oracle over {desc} ({n_step} sites), one pass per step"},
        "e2e": {"value": value, "unit": "sites/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1603_08357_gb300 as ccl

    lat, desc = make_workload(args.config, rank)
    kind = args.input
    rp = torch.from_numpy(lat.row_ptr).to(dev)
    ci = torch.from_numpy(lat.col_idx).to(dev)
    bits = torch.from_numpy(lat.open_bits.view(np.int32)).to(dev)
    labels = torch.empty(lat.n, dtype=torch.int32, device=dev)
    width, h_nn, h_dbits = 0, None, None
    if kind in ("dense", "dense-random"):
        # the same graph and bond states as a dense strided neighbour list
        width, h_nn, h_dbits = L.to_dense(lat)
        d_nn = torch.from_numpy(h_nn).to(dev)
        d_dbits = torch.from_numpy(h_dbits.view(np.int32)).to(dev)
    seed_of = lambda k: (lat.seed * 1_000_003 + k) & (2**64 - 1)  # noqa: E731
    step_no = [0]
    ctx = ccl.ccl_context_create(local)
    stream = torch.cuda.current_stream(dev)
    tuned = None
    if not args.no_autotune:
        st_t, best_ms = ccl.ccl_autotune(ctx, lat.n, lat.nnz, rp, ci, bits, labels, stream)
        ccl.check(st_t, "ccl_autotune")
        tuned = {"best_ms": best_ms}
    opts = {name: ccl.ccl_get_option(ctx, o) for name, o in (
        ("threads", ccl.CCL_OPT_BLOCK_THREADS), ("ctas_per_sm", ccl.CCL_OPT_CTAS_PER_SM),
        ("pre_analysis", ccl.CCL_OPT_PRE_ANALYSIS), ("link_mode", ccl.CCL_OPT_LINK_MODE),
        ("refill", ccl.CCL_OPT_REFILL), ("analysis_order", ccl.CCL_OPT_ANALYSIS_ORDER))}

    def step():
        if kind == "csr":
            st = ccl.ccl_label(ctx, lat.n, lat.nnz, rp, ci, bits, labels, stream)
        elif kind == "dense":
            st = ccl.ccl_label_dense(ctx, lat.n, width, d_nn, d_dbits, labels, stream)
        elif kind == "random":       # a new realisation every step
            st = ccl.ccl_label_random(ctx, lat.n, lat.nnz, rp, ci, seed_of(step_no[0]), lat.p, labels, stream)
        else:
            st = ccl.ccl_label_dense_random(ctx, lat.n, width, d_nn, seed_of(step_no[0]), lat.p, labels, stream)
        step_no[0] += 1
        if st != ccl.CCL_OK:
            raise ccl.CclError(st, kind)

    for _ in range(max(args.warmup, 3)):
        step()
    ccl.check(ccl.ccl_sync(ctx, stream), "warm-up")

    # correctness guard: the CPU-baseline leg compares every label of the last
    # timed step with the oracle's labels of the same instance (rank 0, N=1)
    stats = ccl.ccl_get_stats(ctx)
    q = int(stats.residual_pairs)
    opts.update(_settings(stats))

    # timed region: K steps, per-step CUDA events on the launching stream; the
    # library records events between its kernels (profiling ring) so that the
    # dominant kernel's mean duration comes from the same steps
    ccl.ccl_set_option(ctx, ccl.CCL_OPT_PROFILE, 1)
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(local, uuid)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    for k in range(args.steps):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    st = ccl.ccl_sync(ctx, stream)
    ccl.check(st, "timed steps")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_local = sum(step_ms) / args.steps
    kern = ccl.ccl_get_step_times(ctx)
    ccl.ccl_set_option(ctx, ccl.CCL_OPT_PROFILE, 0)
    ms = max_over_ranks(ms_local, dist, dev)

    # graph-replay steps (the production path) for comparison
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        step()
    g1.record(stream)
    torch.cuda.synchronize()
    ms_graph = g0.elapsed_time(g1) / args.steps

    # end-to-end from pinned host memory: csr through the host-buffer entry
    # point; the other inputs copy their arrays in, label, and copy labels out
    last_seed = seed_of(step_no[0] - 1)
    last_labels = labels.cpu().numpy()
    h_lab = torch.empty(lat.n, dtype=torch.int32).pin_memory()
    e_steps = max(1, min(args.steps, 10))
    if kind == "csr":
        h_rp = torch.from_numpy(lat.row_ptr).pin_memory()
        h_ci = torch.from_numpy(lat.col_idx).pin_memory()
        h_bits = torch.from_numpy(lat.open_bits.view(np.int32)).pin_memory()
        h2d = 4 * (lat.n + 1) + 4 * lat.nnz + 4 * lat.open_bits.size
        entry = "ccl_label_host (pinned host buffers)"

        def e2e_step():
            s = ccl.ccl_label_host(ctx, lat.n, lat.nnz, h_rp.data_ptr(), h_ci.data_ptr(),
                                   h_bits.data_ptr(), h_lab.data_ptr(), stream)
            if s != ccl.CCL_OK:
                raise ccl.CclError(s, "ccl_label_host")
    else:
        host_in = ([torch.from_numpy(lat.row_ptr), torch.from_numpy(lat.col_idx)] if kind == "random" else
                   [torch.from_numpy(h_nn)] + ([torch.from_numpy(h_dbits.view(np.int32))] if kind == "dense" else []))
        host_in = [t.pin_memory() for t in host_in]
        dev_in = [rp, ci] if kind == "random" else ([d_nn] + ([d_dbits] if kind == "dense" else []))
        h2d = sum(t.numel() * 4 for t in host_in)
        entry = {"dense": "ccl_label_dense", "random": "ccl_label_random",
                 "dense-random": "ccl_label_dense_random"}[kind] + " with pinned H2D/D2H copies"

        def e2e_step():
            for h, d in zip(host_in, dev_in):
                d.copy_(h, non_blocking=True)
            step()
            h_lab.copy_(labels, non_blocking=True)
            ccl.check(ccl.ccl_sync(ctx, stream), "e2e")

    for _ in range(2):
        e2e_step()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e_steps):
        e2e_step()
    e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / e_steps, dist, dev)

    ok_sample = None
    if rank == 0:
        peak, peak_src = _peaks()
        ab = algorithmic_bytes(lat.n, lat.nnz, q, kind, width)
        names = ["init", "analysis_ii", "reduce", "analysis_iv"]
        dom = max(range(4), key=lambda i: kern[i] if kern[i] > 0.005 else -1)
        dom_name = names[dom]
        achieved = ab[dom_name] / (kern[dom] / 1e3) / 1e9
        workload = args.config if kind == "csr" else f"{args.config}/{kind}"
        traffic, scaled = _ncu_traffic(dom_name, workload)
        cpu = None
        if not args.no_cpu_baseline and world == 1:      # the CPU baseline is an N=1 figure
            # the leg's oracle labels also check the labels of the last timed step
            ref = oracle_input(lat, last_seed if kind in ("random", "dense-random") else None)
            v, reps, secs, ok_sample = oracle_time(ref, args.cpu_seconds, check=last_labels)
            cpu = {"value": v, "unit": "sites/s", "cores": 1, "kind": "oracle",
                   "sample": f"union-find oracle over the full instance ({lat.n} sites), "
                             f"{reps} pass(es) in {secs:.1f} s, 1 thread"}
        kernels = {names[i]: ({"ms": kern[i], "alg_bytes": ab[names[i]],
                               "alg_gbs": ab[names[i]] / (kern[i] / 1e3) / 1e9}
                              if kern[i] > 0.005 else {"ms": kern[i], "skipped": True})
                   for i in range(4)}
        value = world * lat.n / (ms / 1e3)
        line = {
            "metric": "sites labeled/s", "value": value, "unit": "sites/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": workload, "desc": desc, "p": lat.p, "input": kind, "width": width or None,
                       "n_sites": lat.n, "nnz": lat.nnz,
                       "residual_pairs": q, "options": opts, "autotune": tuned,
                       "l2": "inputs larger than L2 (no flush)" if lat.nnz * 4 > L2_BYTES
                       else "inputs L2-resident (no flush)",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "edges_per_s": world * (lat.nnz // 2) / (ms / 1e3),
            "path_alg_gbs": ab["path"] / (ms / 1e3) / 1e9,
            "ms_per_step_graph_replay": ms_graph,
            "kernels": kernels,
            "roofline": {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_src} hbm_gbs (copy, burst)",
                         "traffic_note": scaled},
            "cpu_baseline": cpu,
            "e2e": {"value": world * lat.n / (e_ms / 1e3), "unit": "sites/s",
                    "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 4 * lat.n, "ms_per_step": e_ms,
                    "entry": entry},
            "gpu_launches": args.steps * (4 if opts["pre_analysis"] else 3),
            "clocks": clk,
            "parity_last_step": ok_sample,      # from the CPU-baseline leg (None without it)
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _phases(st) -> dict:
    """The request loop's latency by phase (p50 / p99 in ms)."""
    names = ("admit", "upload", "wait_launch", "gpu_and_return")
    return {n: [round(st.phase_p50_ms[k], 3), round(st.phase_p99_ms[k], 3)] for k, n in enumerate(names)}


def _settings(stats) -> dict:
    """The settings the library reports for its last call (tuned, set or
    chosen by size)."""
    return {k: int(getattr(stats, k)) for k in ("pre_analysis", "link_mode", "refill", "analysis_order",
                                                 "reduce_window", "analysis_group", "analysis_park")}


def _pinned(a: np.ndarray) -> np.ndarray:
    """A copy of a host array in a pinned host allocation (cudaHostAlloc
    through torch), as a numpy array sharing that memory."""
    import torch
    return torch.from_numpy(a.view(np.int32)).pin_memory().numpy().view(a.dtype)


def run_batched(args, rank, world, local):
    """The batched workload (the metric's headline): K mixed instances labelled
    by one pass of the four steps (ccl_label_batched), against the same
    instances labelled one ccl_label call at a time, both in this run.

    value: batched sites/s from per-step CUDA events, inputs resident in HBM.
    roofline: the dominant kernel of the batched step (per-kernel events of
    the same timed steps) against the measured copy bandwidth.
    e2e: ccl_label_batched_host from pinned host allocations (inputs up,
    labels down, inside the timed region).
    cpu_baseline: the union-find oracle over every instance of the batch,
    whole instances spread over the host's cores; it also checks every label
    of the last timed step."""
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1603_08357_gb300 as ccl
    t_gen = time.perf_counter()
    specs = L.batched_mix_specs(args.instances, seed=4 + 1000 * rank)
    b = L.make_batch(specs)
    abits, word_off = b.aligned_bits()
    t_gen = time.perf_counter() - t_gen
    # the concatenated arrays move into pinned host allocations (the host side
    # of the e2e leg, and what every other leg reads too)
    t_pin = time.perf_counter()
    import dataclasses
    b = dataclasses.replace(b, row_ptr=_pinned(b.row_ptr), col_idx=_pinned(b.col_idx),
                            open_bits=_pinned(b.open_bits))
    t_pin = time.perf_counter() - t_pin
    rp = torch.from_numpy(b.row_ptr).to(dev)
    ci = torch.from_numpy(b.col_idx).to(dev)
    bits = torch.from_numpy(b.open_bits.view(np.int32)).to(dev)
    labels = torch.empty(b.n_total, dtype=torch.int32, device=dev)
    ctx = ccl.ccl_context_create(local)
    stream = torch.cuda.current_stream(dev)
    tuned = None
    if not args.no_autotune:
        st_t, best_ms = ccl.ccl_autotune_batched(ctx, b.k, b.site_off, b.ent_off, rp, ci, bits, labels, stream)
        ccl.check(st_t, "ccl_autotune_batched")
        tuned = {"best_ms": best_ms}

    def step():
        st = ccl.ccl_label_batched(ctx, b.k, b.site_off, b.ent_off, rp, ci, bits, labels, stream)
        if st != ccl.CCL_OK:
            raise ccl.CclError(st, "ccl_label_batched")

    for _ in range(max(args.warmup, 3)):
        step()
    ccl.check(ccl.ccl_sync(ctx, stream), "warm-up")
    stats = ccl.ccl_get_stats(ctx)
    q = int(stats.residual_pairs)
    opts = _settings(stats)

    # timed region: per-step CUDA events on the launching stream; the library
    # records events between its kernels for every timed step (profiling ring)
    ccl.ccl_set_option(ctx, ccl.CCL_OPT_PROFILE, 1)
    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    for k in range(args.steps):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ccl.check(ccl.ccl_sync(ctx, stream), "timed steps")
    ms = max_over_ranks(sum(a.elapsed_time(c) for a, c in ev) / args.steps, dist, dev)
    kern = ccl.ccl_get_step_times(ctx)
    ccl.ccl_set_option(ctx, ccl.CCL_OPT_PROFILE, 0)
    got = labels.cpu().numpy()

    # graph replay of the same call (the production path), for comparison
    step()
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(max(1, min(args.steps, 5))):
        step()
    g1.record(stream)
    torch.cuda.synchronize()
    ms_graph = g0.elapsed_time(g1) / max(1, min(args.steps, 5))

    # one instance per call (graphs off: every instance is a new shape)
    one = ccl.ccl_context_create(local)
    ccl.ccl_set_option(one, ccl.CCL_OPT_USE_GRAPHS, 0)
    out1 = torch.empty_like(labels)
    rp0, ci0, ab0, lab0 = rp.data_ptr(), ci.data_ptr(), torch.from_numpy(abits.view(np.int32)).to(dev), out1.data_ptr()
    ab0p = ab0.data_ptr()
    so, eo = b.site_off, b.ent_off

    def one_step():
        for k in range(b.k):
            n_k, nnz_k = int(so[k + 1] - so[k]), int(eo[k + 1] - eo[k])
            st = ccl.ccl_label(one, n_k, nnz_k, rp0 + 4 * (int(so[k]) + k), ci0 + 4 * int(eo[k]),
                               ab0p + 4 * int(word_off[k]), lab0 + 4 * int(so[k]), stream)
            if st != ccl.CCL_OK:
                raise ccl.CclError(st, "ccl_label")

    one_step()
    ccl.check(ccl.ccl_sync(one, stream), "one-at-a-time warm-up")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, min(args.steps, 3))
    if dist:
        dist.barrier()
    e0.record(stream)
    for _ in range(reps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_one = max_over_ranks(e0.elapsed_time(e1) / reps, dist, dev)
    same = bool(torch.equal(out1, labels))
    del out1, ab0
    ccl.ccl_context_destroy(one)

    # end to end from pinned host allocations through ccl_label_batched_host;
    # the device copies of the inputs are dropped first (the context keeps
    # buffers of its own for the host path)
    del rp, ci, bits
    torch.cuda.empty_cache()
    h_lab = _pinned(np.empty(b.n_total, np.int32))
    h2d = b.row_ptr.nbytes + b.col_idx.nbytes + b.open_bits.nbytes
    d2h = h_lab.nbytes

    def e2e_step():
        st = ccl.ccl_label_batched_host(ctx, b.k, b.site_off, b.ent_off, b.row_ptr, b.col_idx, b.open_bits,
                                        h_lab, stream)
        if st != ccl.CCL_OK:
            raise ccl.CclError(st, "ccl_label_batched_host")

    e2e_step()
    e_steps = max(1, min(args.steps, 3))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    e_step_ms = []
    for _ in range(e_steps):
        t1 = time.perf_counter()
        e2e_step()
        e_step_ms.append(1e3 * (time.perf_counter() - t1))
    e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / e_steps, dist, dev)
    e2e_same = bool(np.array_equal(h_lab, got))

    if rank == 0:
        peak, peak_src = _peaks()
        ab = algorithmic_bytes(b.n_total, b.nnz_total, q, "csr", rows=b.n_total + b.k)
        names = ["init", "analysis_ii", "reduce", "analysis_iv"]
        dom = max(range(4), key=lambda i: kern[i] if kern[i] > 0.005 else -1)
        dom_name = names[dom]
        achieved = ab[dom_name] / (kern[dom] / 1e3) / 1e9
        traffic, scaled = _ncu_traffic(dom_name, "batched")
        kernels = {names[i]: ({"ms": kern[i], "alg_bytes": ab[names[i]],
                               "alg_gbs": ab[names[i]] / (kern[i] / 1e3) / 1e9}
                              if kern[i] > 0.005 else {"ms": kern[i], "skipped": True})
                   for i in range(4)}
        cpu, ok = None, None
        if not args.no_cpu_baseline and world == 1:      # the CPU baseline is an N=1 figure
            import oracle
            t2 = time.perf_counter()
            want, threads = oracle.uf_label_batched_threads(b)
            el = time.perf_counter() - t2
            ok = bool(np.array_equal(got, want))
            cpu = {"value": b.n_total / el, "unit": "sites/s", "cores": threads, "kind": "oracle",
                   "sample": f"union-find oracle over all {b.k} instances of the batch ({b.n_total} sites) "
                             f"in {el:.1f} s, whole instances spread over {threads} threads"}
        line = {
            "metric": METRIC, "value": world * b.n_total / (ms / 1e3), "unit": "sites/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "batched", "instances": b.k, "n_sites": b.n_total, "nnz": b.nnz_total,
                       "desc": "4096 mixed honeycomb / triangle / Cayley-tree instances at p_c +- 0.05, "
                               "concatenated CSR with int64 offsets",
                       "residual_pairs": q, "generation_s": t_gen, "pinning_s": t_pin, "options": opts,
                       "autotune": tuned,
                       "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "one_at_a_time": {"value": world * b.n_total / (ms_one / 1e3), "unit": "sites/s",
                              "ms_per_step": ms_one, "calls_per_step": b.k, "entry": "ccl_label",
                              "speedup_batched": ms_one / ms, "labels_identical": same},
            "edges_per_s": world * (b.nnz_total // 2) / (ms / 1e3),
            "path_alg_gbs": ab["path"] / (ms / 1e3) / 1e9,
            "ms_per_step_graph_replay": ms_graph,
            "kernels": kernels,
            "roofline": {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "alg_bytes_per_launch": ab[dom_name],
                         "peak_source": f"{peak_src} hbm_gbs (copy, burst)", "traffic_note": scaled},
            "cpu_baseline": cpu,
            "e2e": {"value": world * b.n_total / (e_ms / 1e3), "unit": "sites/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e_ms,
                    "step_ms": [round(x, 2) for x in e_step_ms],
                    "entry": "ccl_label_batched_host (pinned host allocations)",
                    "labels_identical": e2e_same},
            "gpu_launches": args.steps * (4 if opts["pre_analysis"] else 3),
            "clocks": clk,
            "parity_all_instances": ok,       # every label of the last timed step vs the oracle
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_served(args, rank, world, local):
    """The served workload: a stream of requests (log-uniform 1e3..1e7 sites,
    the three lattice types at p_c) through the request loop (ccl_server_*),
    host arrays in, labels back in host memory, against the same stream
    labelled one ccl_label_host call at a time from the same host memory.
    First the capacity with a bounded number of requests in flight (closed
    loop, both submission modes), then Poisson arrivals at fractions of that
    capacity (open loop) for the latency percentiles. The stream repeats a
    pool of distinct pre-generated requests (the whole stream would not fit in
    host memory); the pool's arrays and the result buffers live in pinned
    host allocations, as a serving process keeps its request buffers."""
    import dataclasses
    import torch
    torch.cuda.set_device(local)
    import paper_1603_08357_gb300 as ccl
    t_gen = time.perf_counter()
    specs = L.served_specs(args.requests, seed=5 + 1000 * rank)
    pool = [L.make_instance(sp) for sp in specs[:args.pool]]
    t_gen = time.perf_counter() - t_gen
    pool = [dataclasses.replace(lat, row_ptr=_pinned(lat.row_ptr), col_idx=_pinned(lat.col_idx),
                                open_bits=_pinned(lat.open_bits)) for lat in pool]
    req = [pool[r % len(pool)] for r in range(args.requests)]
    total_sites = sum(lat.n for lat in req)
    mean_sites = total_sites / len(req)
    out_bufs = {id(lat): _pinned(np.empty(lat.n, np.int32)) for lat in pool}
    keep_idx = set(range(0, len(req), max(1, len(req) // args.parity_sample)))

    def submit_with(fn, name):
        def sub(srv, lat):
            while True:
                st, t = fn(srv, lat.n, lat.nnz, lat.row_ptr, lat.col_idx, lat.open_bits)
                if st == ccl.CCL_OK:
                    return t
                if st != ccl.CCL_ERR_REJECTED:
                    raise ccl.CclError(st, name)
                time.sleep(0.0005)
        return sub
    submit_nocopy = submit_with(ccl.ccl_server_submit_nocopy, "ccl_server_submit_nocopy")
    submit = submit_with(ccl.ccl_server_submit, "ccl_server_submit")

    def new_server():
        srv = ccl.ccl_server_create(local, n_streams=args.streams, max_batch=1024, host_staging_bytes=8 << 30)
        for lat in pool[:16]:                                   # warm-up
            ccl.check(ccl.ccl_server_wait(srv, submit_nocopy(srv, lat), out_bufs[id(lat)], 600_000), "warm-up")
        return srv

    def collect(srv, tickets, keep=None, sem=None):
        """Waits for every ticket with args.waiters client threads (thread t
        takes requests t, t + waiters, ... in order), as a serving front end
        with several connections would; labels of the kept requests go to
        buffers of their own."""
        errors = []

        def waiter(t):
            try:
                for k in range(t, len(req), args.waiters):
                    while tickets[k] is None:
                        time.sleep(0.00005)
                    lat = req[k]
                    buf = np.empty(lat.n, np.int32) if keep is not None and k in keep_idx else out_bufs[id(lat)]
                    ccl.check(ccl.ccl_server_wait(srv, tickets[k], buf, 600_000), "ccl_server_wait")
                    if keep is not None and k in keep_idx:
                        keep[k] = buf
                    if sem is not None:
                        sem.release()
            except Exception as e:          # reported by the main thread
                errors.append(e)
        ths = [threading.Thread(target=waiter, args=(t,)) for t in range(args.waiters)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        if errors:
            raise errors[0]

    def closed_loop(sub):
        srv = new_server()
        tickets = [None] * len(req)
        sem = threading.Semaphore(args.window)

        def feeder():
            for k, lat in enumerate(req):
                sem.acquire()
                tickets[k] = sub(srv, lat)

        keep = {}
        t0 = time.perf_counter()
        th = threading.Thread(target=feeder)
        th.start()
        collect(srv, tickets, keep, sem)
        th.join()
        wall = time.perf_counter() - t0
        st = ccl.ccl_server_stats_get(srv)
        ccl.ccl_server_destroy(srv)
        return wall, st, keep

    clocks = ClockSampler(local)
    clocks.start()
    wall, st_closed, keep = closed_loop(submit_nocopy)
    wall_copy, st_copy, keep_copy = closed_loop(submit)
    clk = clocks.stop()
    capacity = total_sites / wall

    # one request at a time through the host-buffer entry point, same stream
    one = ccl.ccl_context_create(local)
    stream = torch.cuda.current_stream()
    for lat in pool[:16]:
        ccl.check(ccl.ccl_label_host(one, lat.n, lat.nnz, lat.row_ptr, lat.col_idx, lat.open_bits,
                                     out_bufs[id(lat)], stream), "ccl_label_host")
    lat_one, keep_one = [], {}
    t0 = time.perf_counter()
    for k, lat in enumerate(req):
        buf = np.empty(lat.n, np.int32) if k in keep_idx else out_bufs[id(lat)]
        t1 = time.perf_counter()
        ccl.check(ccl.ccl_label_host(one, lat.n, lat.nnz, lat.row_ptr, lat.col_idx, lat.open_bits, buf, stream),
                  "ccl_label_host")
        lat_one.append(time.perf_counter() - t1)
        if k in keep_idx:
            keep_one[k] = buf
    wall_one = time.perf_counter() - t0
    ccl.ccl_context_destroy(one)
    lat_one = np.array(lat_one) * 1e3

    # open loop: Poisson arrivals at load x capacity
    loads = {}
    for load in args.loads:
        rate = load * capacity / mean_sites            # requests per second
        rng = np.random.default_rng(55 + rank)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(req)))
        srv = new_server()
        tk = [None] * len(req)

        def open_feeder():
            base = time.perf_counter()
            for k, lat in enumerate(req):
                delay = base + arrivals[k] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tk[k] = submit_nocopy(srv, lat)

        t1 = time.perf_counter()
        th = threading.Thread(target=open_feeder)
        th.start()
        collect(srv, tk)
        th.join()
        el = time.perf_counter() - t1
        so = ccl.ccl_server_stats_get(srv)
        ccl.ccl_server_destroy(srv)
        # the server's percentiles cover the 16 warm-up requests too (tiny next to the stream)
        loads[str(load)] = {"offered_req_per_s": rate, "achieved_sites_per_s": total_sites / el,
                            "p50_ms": so.p50_ms, "p99_ms": so.p99_ms, "max_ms": so.max_ms,
                            "batches": int(so.batches), "arena_misses": int(so.arena_misses),
                            "phases": _phases(so)}

    ok = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:      # the CPU baseline is an N=1 figure
            import oracle
            t2, sites, done = time.perf_counter(), 0, 0
            for lat in pool:
                oracle.uf_label(lat)
                sites += lat.n
                done += 1
                if time.perf_counter() - t2 > args.cpu_seconds:
                    break
            cpu = {"value": sites / (time.perf_counter() - t2), "unit": "sites/s", "cores": 1,
                   "kind": "oracle", "sample": f"union-find oracle over {done} pool requests ({sites} sites), 1 thread"}
            # the leg's oracle also checks the kept labels of all three arms
            ok = all(np.array_equal(kp[k], oracle.uf_label(req[k]))
                     for kp in (keep, keep_copy, keep_one) for k in keep_idx)
        h2d = sum(4 * (lat.n + 1) + 4 * lat.nnz + 4 * lat.open_bits.size for lat in req) / len(req)
        line = {
            "metric": "sites labeled/s (served vs one-at-a-time)", "value": world * capacity, "unit": "sites/s",
            "n_gpus": world, "steps": len(req), "warmup": 16, "ms_per_step": 1e3 * wall / len(req),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "served", "requests": len(req), "pool": len(pool),
                       "mean_sites": mean_sites, "window": args.window, "streams": args.streams,
                       "client_waiters": args.waiters,
                       "generation_s": t_gen, "host_arrays": "pinned allocations (cudaHostAlloc)",
                       "l2": "inputs larger than L2 in aggregate (no flush)"},
            "closed_loop": {"submit": "ccl_server_submit_nocopy", "wall_s": wall,
                            "requests_per_s": len(req) / wall, "batches": int(st_closed.batches),
                            "p50_ms": st_closed.p50_ms, "p99_ms": st_closed.p99_ms,
                            "arena_misses": int(st_closed.arena_misses), "phases": _phases(st_closed)},
            "closed_loop_copying": {"submit": "ccl_server_submit", "sites_per_s": total_sites / wall_copy,
                                    "requests_per_s": len(req) / wall_copy, "batches": int(st_copy.batches),
                                    "p50_ms": st_copy.p50_ms, "p99_ms": st_copy.p99_ms,
                                    "arena_misses": int(st_copy.arena_misses), "phases": _phases(st_copy)},
            "one_at_a_time": {"entry": "ccl_label_host, one call per request, same host arrays",
                              "value": world * total_sites / wall_one, "unit": "sites/s", "wall_s": wall_one,
                              "requests_per_s": len(req) / wall_one,
                              "p50_ms": float(np.percentile(lat_one, 50)), "p99_ms": float(np.percentile(lat_one, 99)),
                              "speedup_served": wall_one / wall},
            "open_loop": loads,
            "e2e": {"value": world * capacity, "unit": "sites/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 4 * mean_sites,
                    "entry": "ccl_server_submit_nocopy / ccl_server_wait (host arrays in, labels out)"},
            "roofline": None,
            "cpu_baseline": cpu,
            "clocks": clk,
            "parity_sample": {"requests": len(keep_idx), "arms": 3, "ok": ok},
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(CONFIGS) + ["batched", "served"], default="batched")
    ap.add_argument("--instances", type=int, default=4096)
    ap.add_argument("--parity-sample", type=int, default=48, help="served: requests checked per mode")
    ap.add_argument("--reference-instances", type=int, default=512,
                    help="reference arm, batched: instances of the mix labelled per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--requests", type=int, default=20000, help="served: requests in the stream")
    ap.add_argument("--pool", type=int, default=128, help="served: distinct pre-generated requests")
    ap.add_argument("--window", type=int, default=64, help="served: requests in flight (closed loop)")
    ap.add_argument("--streams", type=int, default=2, help="served: server compute streams")
    ap.add_argument("--waiters", type=int, default=4, help="served: client threads collecting results")
    ap.add_argument("--loads", type=float, nargs="*", default=[0.5, 0.8],
                    help="served: open-loop arrival rates as fractions of the capacity")
    ap.add_argument("--input", choices=["csr", "dense", "random", "dense-random"], default="csr",
                    help="single-instance configs: CSR with bit words (default), the dense strided "
                         "neighbour list, or either with bonds drawn on the device")
    ap.add_argument("--p", type=float, default=None,
                    help="single-instance configs: bond probability in place of the config's")
    args = ap.parse_args()
    global P_OVERRIDE
    P_OVERRIDE = args.p
    rank, world, local = _env_rank()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.config == "batched":
        run_batched(args, rank, world, local)
    elif args.config == "served":
        run_served(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
