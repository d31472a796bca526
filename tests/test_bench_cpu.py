"""Host logic of bench.py that needs no GPU: the algorithmic byte counts of
each input kind, the CPU-baseline leg's timing and label check, and the
reference arm's JSON line."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import lattices as L  # noqa: E402


def test_algorithmic_bytes_by_input_kind():
    n, nnz, q, W = 1000, 6000, 300, 6
    csr = bench.algorithmic_bytes(n, nnz, q)
    assert csr["init"] == 4 * (n + 1) + 4 * nnz + 4 * ((nnz + 31) // 32) + 4 * n + 8 * q
    assert csr["analysis_ii"] == csr["analysis_iv"] == 8 * n
    assert csr["reduce"] == 16 * q
    assert csr["path"] == csr["init"] + 2 * 8 * n + 16 * q
    rnd = bench.algorithmic_bytes(n, nnz, q, "random")
    assert csr["init"] - rnd["init"] == 4 * ((nnz + 31) // 32)       # no bit words read
    dense = bench.algorithmic_bytes(n, nnz, q, "dense", W)
    assert dense["init"] == 4 * W * n + 4 * ((W * n + 31) // 32) + 4 * n + 8 * q
    assert bench.algorithmic_bytes(n, nnz, q, "dense-random", W)["init"] == 4 * W * n + 4 * n + 8 * q


def test_cpu_leg_checks_labels():
    import oracle
    lat = L.triangle(40, 0.4, 3)
    good = oracle.uf_label(lat)
    v, reps, secs, same = bench.oracle_time(lat, 0.0, check=good)
    assert v > 0 and reps >= 1 and same is True
    bad = good.copy()
    bad[5] = 5 if good[5] != 5 else 4
    assert bench.oracle_time(lat, 0.0, check=bad)[3] is False
    assert bench.oracle_time(lat, 0.0)[3] is None
    # device-drawn bonds: the leg labels the keyed realisation
    ref = bench.oracle_input(lat, 99)
    assert not np.array_equal(ref.open_bits, lat.open_bits)
    assert np.array_equal(ref.open_bits, oracle.keyed_bits(lat, 99, lat.p))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config",
                        "hc256", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "sites labeled/s" and line["unit"] == "sites/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == "hc256"


def test_committed_traffic_is_plausible():
    """Every per-launch DRAM figure in profiles/traffic.json lies within a
    small factor of the bytes its workload holds (a unit slip in turning ncu's
    Mbyte/Gbyte columns into bytes moves it by 10^3)."""
    sizes = {"tri4096": (4096 * 4096, 6 * 4096 * 4096), "tri4096/dense": (4096 * 4096, 6 * 4096 * 4096),
             "bethe24": (1 + 3 * (2 ** 24 - 1), 2 * 3 * (2 ** 24 - 1)),
             "batched": (2_127_258_178, 7_325_653_934)}
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        traffic = json.load(fh)
    assert traffic
    for key, ent in traffic.items():
        workload = key.split(":", 1)[1]
        n, nnz = sizes[workload]
        held = 4 * (n + 1) + 4 * nnz + nnz // 8 + 4 * n + 8 * nnz    # inputs, labels, a full queue
        b = ent["dram_bytes_per_launch"]
        assert 0.05 * 8 * n <= b <= 4 * held, (key, b)


def test_batched_row_pointer_bytes():
    n, nnz, q, K = 1000, 6000, 300, 7
    one = bench.algorithmic_bytes(n, nnz, q)
    many = bench.algorithmic_bytes(n, nnz, q, rows=n + K)
    assert many["init"] - one["init"] == 4 * (K - 1)


def test_reference_arm_line_batched():
    """The reference arm on the default (batched) workload: the oracle over the
    first instances of the mix, whole instances spread over the host's cores."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--instances", "64", "--reference-instances", "6", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["config"]["workload"] == "batched" and line["cpu_baseline"]["cores"] >= 1
    sb = L.make_batch(L.batched_mix_specs(64, seed=4)[:6])
    assert line["config"]["n_sites"] == sb.n_total
    assert line["value"] > 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_threaded_batched_oracle_equals_serial():
    import oracle
    b = L.make_batch(L.batched_mix_specs(40, seed=9))
    got, threads = oracle.uf_label_batched_threads(b, 3)
    assert threads == 3 and np.array_equal(got, oracle.uf_label_batched(b))
