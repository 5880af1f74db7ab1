"""bench.py --impl reference: the oracle timed on the host on a sample of the headline workload,
printed as one JSON line with the keys the bench contract gives that arm (impl, metric, value,
unit, higher_is_better, config, cpu_baseline with kind / cores / sample, and an e2e block whose
value is the line's own with no device copies)."""
import io
import json
from contextlib import redirect_stdout

import bench


def test_reference_line_has_the_contract_keys(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["workload"].startswith("d3q19_suspension_512")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
