"""bench.py's host logic without a GPU: argument defaults per workload, names, the oracle's
timed sample, and the reference arm's JSON line on a small instance."""
import json
import subprocess
import sys
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _args(monkeypatch, *argv):
    import bench

    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    return bench.parse_args()


@pytest.mark.parametrize("wl,m,n", [("dense", 1000, 200_000), ("sparse", 5000, 2_000_000),
                                    ("scaled", 2000, 500_000), ("serving", 512, 102_400),
                                    ("svm", 100, 20_102)])
def test_workload_defaults(monkeypatch, wl, m, n):
    a = _args(monkeypatch, "--workload", wl)
    assert (a.m, a.n) == (m, n)
    assert a.steps >= 1 and a.warmup >= 3


def test_headline_metric_name(monkeypatch):
    import bench

    a = _args(monkeypatch)
    assert bench.metric_name(a) == "IPM LPs/s (Algorithm 2 to tolerance, dense m=1000 n=200000 FP32 LP)"
    a = _args(monkeypatch, "--workload", "svm", "--svm-shape", "gene_rna")
    assert "svm m=801 n=41865" in bench.metric_name(a)
    assert "gene_rna" in bench.workload_name(a)


def test_sample_lp_shapes(monkeypatch):
    import bench

    a = _args(monkeypatch, "--m", "30", "--n", "5000", "--cpu-sample-n", "1000")
    lp, A, ns = bench.sample_lp(a)
    assert A.shape == (30, 1000) and ns == 1000
    a = _args(monkeypatch, "--workload", "sparse", "--m", "30", "--n", "5000",
              "--cpu-sample-n", "1000", "--nnz-per-col", "3")
    lp, A, ns = bench.sample_lp(a)
    assert A.shape == (30, 1000) and A.nnz == 3000


def test_reference_arm_line_on_a_small_instance():
    """The reference arm runs the oracle only and prints one JSON line with the contract's keys."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--m", "20",
                          "--n", "2000", "--cpu-sample-n", "2000", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_preconditioned_kappa():
    """The sketch study's kappa of M K with M = L L^T: the identity preconditioner gives
    cond(K), the exact K^-1/2 gives 1, and an indefinite product is reported as None."""
    import numpy as np

    import bench

    rng = np.random.default_rng(3)
    F = rng.standard_normal((30, 30))
    K = F @ F.T + 0.1 * np.eye(30)
    assert bench.preconditioned_kappa(K, np.eye(30)) == pytest.approx(np.linalg.cond(K), rel=1e-8)
    lam, V = np.linalg.eigh(K)
    assert bench.preconditioned_kappa(K, V / np.sqrt(lam)) == pytest.approx(1.0, abs=1e-10)
    assert bench.preconditioned_kappa(-K, np.eye(30)) is None


def test_traffic_figure_matches_its_profile_summary():
    """The DRAM traffic bench.py reports comes from the committed ncu summary of the same
    kernel source: the hash and the bytes per launch in bench.py and in the summary agree."""
    import re

    import bench

    text = open(os.path.join(ROOT, "profiles",
                             "k_cgprod_cg_product_dense_m1000_n200000_f32.md")).read()
    assert bench.NCU_TRAFFIC["source_sha1"] in text
    mb = float(re.search(r"traffic per launch \| \*\*([0-9.]+) MB\*\*", text).group(1))
    assert abs(bench.NCU_TRAFFIC["bytes_per_launch"] - mb * 1e6) <= 0.01e6



def test_stored_oracle_runs_are_found(monkeypatch):
    """The bench's dense, badly scaled and sparse workloads at their default sizes find the
    oracle's own stored run of the same instance (tests/golden/make_oracle_run.py)."""
    import bench

    for wl in ("dense", "scaled", "sparse"):
        rec = bench.oracle_run_record(_args(monkeypatch, "--workload", wl))
        assert rec is not None and rec["converged"] and rec["ipm_iters"] > 0, wl
        assert wl in rec["command"]
    assert bench.oracle_run_record(_args(monkeypatch, "--workload", "serving")) is None
