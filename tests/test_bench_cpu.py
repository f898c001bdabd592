"""The bench's CPU baseline: the host description and the oracle pool over the host cores
(process pool with the spawn start method; no GPU)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from workloads import load_config, make_particles  # noqa: E402


def test_host_cpu_reports_cores_and_model():
    cores, model = bench.host_cpu()
    assert cores >= 1
    assert isinstance(model, str) and "(" in model


@pytest.mark.slow
def test_oracle_pool_rate_on_a_small_sample():
    cfg = load_config("c1_box64_n129")
    parts = make_particles(cfg)
    pool = bench.OraclePool(cfg, parts)
    try:
        r, M, dt = pool.rate(0.5, seed=3)
    finally:
        pool.close()
    assert pool.cores >= 1 and M >= 64 * pool.cores and dt > 0 and r == M / dt


def test_workload_config_is_the_same_for_both_arms():
    cfg = load_config("c2_protein1000_n513")
    c = bench.workload_config(cfg, 1000)
    assert c == {"workload": "c2_protein1000_n513", "N": 1000, "n": 513, "R": 24, "R_s": 8, "eps": 1e-06,
                 "precision": "fp32_split"}


def test_assembly_roofline_counts_the_output_once():
    pk = {"hbm_gbs": 1000.0, "source": "test"}
    r = bench.assembly_roofline(513, 57, 1.0, pk)
    assert r["algorithmic_bytes"] == 4 * 513 ** 3
    assert abs(r["achieved"] - 4 * 513 ** 3 / 1e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12
    assert r["t2_read_bytes"] == 4 * 57 * 513 * 513
