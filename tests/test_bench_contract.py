"""bench.py's output contract, checked on the CPU: the reference arm (the FP64
oracle timed on the host cores) prints one JSON line carrying the keys the
harness reads, and the L2 note of a workload follows its size."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "8192",
                        "--steps", "2", "--warmup", "3"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    b = _bench_module()
    assert d["impl"] == "reference" and d["metric"] == b.METRIC and d["unit"] == b.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["n"] == 8192
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_l2_note_follows_the_workload_size():
    b = _bench_module()
    assert b.l2_note(1 << 23).startswith("inputs larger than L2")
    assert b.l2_note(25 << 20).startswith("inputs larger than L2")
    assert b.l2_note(8192).startswith("inputs smaller than L2")
