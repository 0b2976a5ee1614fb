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


def test_schedule_makespan_model():
    """The list-scheduling model behind the schedule study: every order lies
    between the lower bound max(total / workers, largest group) and Graham's
    2x bound; a single worker or equal costs reach the bound exactly; the
    heap-based simulation matches a plain greedy simulation; and a large group
    left to the end of the queue costs the queue order what LPT order saves."""
    import numpy as np

    b = _bench_module()

    def greedy(cost, order, workers):
        load = [0.0] * workers
        for g in order:
            k = min(range(workers), key=lambda w: load[w])
            load[k] += cost[g]
        return max(load)

    rng = np.random.default_rng(5)
    for workers in (1, 3, 8):
        cost = rng.lognormal(0.0, 1.0, 200)
        pred = cost * rng.lognormal(0.0, 0.3, 200)
        r = b.schedule_makespans(cost, pred, workers)
        lb = max(cost.sum() / workers, cost.max())
        for key in ("morton_over_bound", "predicted_order_over_bound", "true_lpt_over_bound"):
            assert 1.0 - 1e-12 <= r[key] <= 2.0
        assert abs(r["morton_over_bound"] * lb - greedy(cost, range(cost.size), workers)) <= 1e-9 * lb
        if workers == 1:
            assert abs(r["morton_over_bound"] - 1.0) < 1e-12
    even = np.ones(64)
    assert abs(b.schedule_makespans(even, even, 8)["morton_over_bound"] - 1.0) < 1e-12
    # 4 workers, bound 12.5: in queue order the large group starts at 10 and
    # ends at 20; first, it leaves the 40 unit groups loads of 13 at most (the
    # optimum, the loads being whole numbers)
    late = np.append(np.ones(40), 10.0)
    r = b.schedule_makespans(late, late, 4)
    assert abs(r["morton_over_bound"] - 20.0 / 12.5) < 1e-12
    assert abs(r["true_lpt_over_bound"] - 13.0 / 12.5) < 1e-12
