"""Host logic of bench.py that feeds the reported rooflines and parity fields, on the CPU.

The roofline's algorithmic work is a count of in-support (sample, Lambda) pairs and of
in-support (m1 node, q node, Lambda) grid triples; both counters take shortcuts (sorted
searches, edge fix-ups) and are checked here against the support test written out directly,
including samples placed exactly on the edges.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1904_02863_gb300 import synth  # noqa: E402


def brute_pairs(theta, lam):
    m1 = theta[:, 0]
    m2 = theta[:, 1] * theta[:, 0]
    return sum(int(np.count_nonzero((m1 > L[2]) & (m1 <= L[3]) & (m2 >= L[2]))) for L in lam)


def test_in_support_pairs_matches_the_support_test():
    cat = synth.make_catalog(30, 700, 6, seed=71)
    lam = synth.make_lambdas(150, 11, seed=72)
    # Lambda rows whose edges sit exactly on sample values (ties of both edges)
    th = cat.theta
    lam[:20, 2] = th[:20, 0]
    lam[20:40, 2] = th[20:40, 0] * th[20:40, 1]
    lam[40:60, 3] = th[40:60, 0]
    lam[60:70, 2] = 5.0
    lam[70:80, 3] = 80.0
    assert bench.in_support_pairs(th, lam) == brute_pairs(th, lam)
    inj = synth.make_injections(40000, 6, seed=73)
    assert bench.in_support_pairs(inj.theta, lam) == brute_pairs(inj.theta, lam)


def test_grid_support_triples_matches_the_support_test():
    m1 = np.linspace(3.0, 100.0, 301)
    q = np.concatenate([np.linspace(0.03, 1.0, 97), [1.02, 1.05]])  # nodes past q = 1 only shape weights
    lam = synth.make_lambdas(40, 11, seed=74)
    lam[:5, 2] = m1[40:45]          # mmin on a node
    lam[5:10, 3] = m1[250:255]      # mmax on a node
    want = 0
    for L in lam:
        mm, qq = np.meshgrid(m1, q, indexing="ij")
        ok = (mm > L[2]) & (mm <= L[3]) & (qq <= 1.0) & (qq * mm >= L[2])
        want += int(np.count_nonzero(ok))
    assert bench.grid_support_triples(m1, q, lam) == want


def test_precision_report_fields():
    a = [np.array([1.0, -np.inf, 3.0]), np.log(np.array([2.0, 1.0, 4.0]))]
    b = [np.array([1.5, -np.inf, 2.0]), np.log(np.array([2.0, 1.0, 5.0]))]
    r = bench.precision_vs(a, b)
    assert r["abs_dlnL"]["rows"] == 2 and r["finite_rows_agree"]
    assert r["abs_dlnL"]["max"] == pytest.approx(1.0) and r["abs_dlnL"]["mean"] == pytest.approx(0.75)
    assert r["rel_dxi_max"] == pytest.approx(0.2)
    sub = bench.precision_vs(a, b, rows=np.array([True, True, False]))
    assert sub["abs_dlnL"]["rows"] == 1 and sub["abs_dlnL"]["max"] == pytest.approx(0.5)
    s = bench.dlnl_stats(np.arange(101.0))
    assert s["p99"] == pytest.approx(99.0) and s["max"] == 100.0 and bench.dlnl_stats(np.array([]))["rows"] == 0


def test_rounding_and_summary_of_a_line():
    line = {"value": 2529.0123456, "roofline": {"frac": 0.8412345678}, "x": [1.23456789012, np.float64(2.0)],
            "forms": {"f32": {"value": 250812.3, "roofline": {"frac": 0.63}, "vs_f64": {"abs_dlnL": {
                "max": 6.2e-4, "p99": 5e-4}}}}}
    r = bench._rounded(line)
    assert r["value"] == 2529.01 and r["x"][0] == 1.23457 and isinstance(r["x"][1], float)
    s = bench.summarise(line)
    assert s["f64"]["evals_s"] == 2529.0 and s["f32"]["dlnL_max_vs_f64"] == 6.2e-4


def test_cpu_baseline_parity_field_against_the_oracle(oracle):
    cat = synth.make_catalog(4, 300, 6, seed=75)
    inj = synth.make_injections(8000, 6, seed=76)
    lam = synth.make_lambdas(6, 11, seed=77)
    ref = oracle.loglik(cat, inj, lam)
    exact = bench.cpu_baseline(cat, inj, lam, 4, gpu_f64=[r.copy() for r in ref])
    assert exact["parity_f64_kernel"]["max_over_f64_tol"] == 0.0
    assert exact["parity_f64_kernel"]["flags_equal"] and exact["single_thread"]["cores"] == 1
    off = [r.copy() for r in ref]
    off[0] = off[0] + 1e-6
    bad = bench.cpu_baseline(cat, inj, lam, 4, gpu_f64=off)
    assert bad["parity_f64_kernel"]["max_over_f64_tol"] > 1.0


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference times the oracle on the host and prints one JSON line with the
    contract's keys (a bounded sample: 2 Lambda rows of the full catalog workload)."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--oracle-lambdas", "2"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "evals/s" and d["value"] > 0
    assert d["config"]["workload"] == bench.WORKLOAD and d["config"]["events"] == 1000
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
