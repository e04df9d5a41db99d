"""bench.py and __graft_entry__.py: they compile, and the reference arm (the
oracle on the host cores) prints one well-formed JSON line (on a tiny sample
here)."""
import io
import json
import os
import py_compile
import sys
import types
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_scripts_compile():
    py_compile.compile(os.path.join(ROOT, "bench.py"), doraise=True)
    py_compile.compile(os.path.join(ROOT, "__graft_entry__.py"), doraise=True)


def test_reference_arm_prints_one_json_line(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "cpu_sample_plan", lambda: [(0, 64), (1 << 23, 64)])
    args = types.SimpleNamespace(gpus=1, steps=2, warmup=3, impl="reference")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.reference_arm(args) == 0
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "genotypes/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_build_entry_point():
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_15311_gb300 import build as B
    assert os.path.exists(B.LIB_PATH)
