"""bench.py's reference arm (the oracle on a bounded sample) runs on the host
alone: its JSON line carries the keys the benchmark contract names.  The
GPU arms are exercised by the GPU runs, not here."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "schlogl_n4096_T1e6_fim"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_workloads_name_their_configs():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.workload()["name"] == "schlogl_n4096_T1e6_fim"
    c3 = bench.workload("toggle_n16384")
    assert c3["name"] == "toggle_n16384_T1e5" and c3["n_replicas"] == 16384 and c3["T_burn"] == c3["T_end"] / 2
