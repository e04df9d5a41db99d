"""Host logic of bench.py that needs no GPU: the figures it takes from the
committed ncu summaries are used only while the kernel source they were
measured on is unchanged (its sha256 prefix), and the oracle's bounded sample
covers the workload evenly."""
import hashlib
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench(tmp_path, monkeypatch):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(mod, "ROOT", str(tmp_path))
    return mod


def _kernel(tmp_path, text):
    k = tmp_path / "kernel.cu"
    k.write_text(text)
    return str(k), hashlib.sha256(text.encode()).hexdigest()[:16]


def test_traffic_only_for_the_measured_source(bench, tmp_path):
    path, sha = _kernel(tmp_path, "// kernel v1\n")
    (tmp_path / "profiles" / "classify_kernel_s28_full_traffic.md").write_text(
        "traffic_bytes_per_launch: 123456\nkernel_source_sha256_prefix: %s\n" % sha)
    assert bench.measured_traffic(path) == 123456
    path2, _ = _kernel(tmp_path, "// kernel v2\n")
    assert bench.measured_traffic(path2) is None


def test_pipes_only_for_the_measured_source(bench, tmp_path):
    path, sha = _kernel(tmp_path, "// kernel v1\n")
    (tmp_path / "profiles" / "classify_kernel_s28_rand4M_ncu_full.md").write_text(
        "| `smsp__issue_active.avg.pct_of_peak_sustained_active` | 60.07 % |\n"
        "| `sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active` | 63.71 % |\n"
        "kernel source: x sha256 prefix " + sha + "\n")
    got = bench.measured_pipes(path)
    assert got["alu_pipe_active"] == pytest.approx(0.6371) and got["issue_active"] == pytest.approx(0.6007)
    path2, _ = _kernel(tmp_path, "// kernel v2\n")
    assert bench.measured_pipes(path2) is None


def test_missing_profiles_give_none(bench, tmp_path):
    path, _ = _kernel(tmp_path, "// kernel\n")
    assert bench.measured_traffic(path) is None and bench.measured_pipes(path) is None


def test_cpu_sample_covers_the_workload_evenly(bench):
    n, c, L, k, seed, first, count, sampled = bench.WORKLOAD_SPEC()
    plan = bench.cpu_sample_plan()
    assert len(plan) == 64
    starts = [s for s, _ in plan]
    assert starts == sorted(starts) and starts[0] == first
    assert all(first <= s and s + m <= first + count for s, m in plan)
    assert len({b - a for a, b in zip(starts, starts[1:])}) == 1  # evenly spaced
