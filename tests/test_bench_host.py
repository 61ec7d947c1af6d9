"""Host-side arithmetic of bench.py (no GPU): the field-operation count behind the
metric, the whole-job aggregation of replicas and the per-class roofline fractions."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_field_ops_closed_forms(bench):
    # square full rank: 2 n^3 / 3 (the metric's normalisation); rank 0: nothing
    for n in (1, 7, 1024):
        assert bench.field_ops(n, n, n) == pytest.approx(2 * n ** 3 / 3)
    assert bench.field_ops(300, 500, 0) == 0


@pytest.mark.parametrize("m,n,r", [(300, 300, 300), (400, 250, 120), (250, 400, 250), (512, 512, 64)])
def test_field_ops_counts_elimination(bench, m, n, r):
    """F(m, n, r) is the leading term of the multiply-adds (two field ops each) of
    eliminating r pivots, the k-th one updating the (m-k-1) x (n-k-1) block below
    and right of it: equal up to terms of order (m + n) r."""
    exact = 2 * sum((m - k - 1) * (n - k - 1) for k in range(r))
    assert abs(bench.field_ops(m, n, r) - exact) <= 2 * (m + n) * r


def test_whole_job_is_all_ranks_over_the_slowest(bench):
    assert bench.whole_job_gfops(1, 2e9, 1000.0) == pytest.approx(2.0)
    assert bench.whole_job_gfops(4, 1e9, 500.0) == pytest.approx(8.0)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_class_rooflines(bench):
    peaks = {"hbm_gbs": 8000.0, "bf16": 2000.0, "bf16_sustained": 1600.0, "source": "test"}
    classes = {
        "perm": {"launches": 10, "ms": 2.0, "flops": 0.0, "bytes": 4e9, "tensor_flops": 0.0},
        "fgemm": {"launches": 3, "ms": 4.0, "flops": 1e12, "bytes": 8e8, "tensor_flops": 3.2e12},
        "other": {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0, "tensor_flops": 0.0},
    }
    out = bench.class_rooflines(classes, peaks)
    # 4 GB in 2 ms = 2000 GB/s = 0.25 of 8000
    assert out["perm"]["hbm_gbs"] == pytest.approx(2000.0)
    assert out["perm"]["hbm_frac"] == pytest.approx(0.25)
    assert "tensor_tflops" not in out["perm"]
    # 3.2e12 tensor flops in 4 ms = 800 TF/s = 0.5 of the sustained 1600
    assert out["fgemm"]["tensor_tflops"] == pytest.approx(800.0)
    assert out["fgemm"]["tensor_frac"] == pytest.approx(0.5)
    assert out["other"] == {"launches": 0, "ms": 0.0}


def test_peaks_are_the_measured_ones(bench):
    peaks = bench.read_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert peaks["source"] == "measured"
    for k in ("hbm_gbs", "bf16", "bf16_sustained"):
        assert peaks[k] > 0
