"""bench.py's reference arm (the oracle on the host cores) runs without a GPU
and prints one JSON line with the keys of the bench line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "planted",
                          "--steps", "2", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                         timeout=300, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["unit"] == "edges/s" and d["value"] > 0
    assert d["config"]["workload"] == "planted" and d["config"]["m"] > 0
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == d["value"] and cpu["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert abs(d["ms_per_step"] * 1e-3 * d["value"] - d["config"]["m"]) < 1e-6 * d["config"]["m"]
