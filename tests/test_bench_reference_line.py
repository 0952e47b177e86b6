"""bench.py --impl reference on the CPU: one JSON line in the benchmark's
format, timing the oracle on a bounded sample of the benchmark's stream
workload (1024 channels, 640 DMs, 2^17-sample blocks)."""
import io
import json
import os
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)

    class A:
        steps, warmup, gpus = 1, 0, 1

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "DM-trial*samples/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    # the time of one full block of the workload at that rate
    assert abs(d["ms_per_step"] - 640 * 131072 / d["value"] * 1e3) <= 1e-6 * d["ms_per_step"]
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["scaling"] == "weak"
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
