"""bench.py's DRAM-traffic record (profiles/traffic.json): the per-site traffic of a sweep kernel
is reported only while the kernel sources hash to the value recorded with the ncu capture; any
change to those sources drops it (the bench then reports traffic null until it is re-taken)."""
import json
import os

import pytest

import bench

KEYS = ("sweep2_d3q19_fp32", "sweep2_d3q19_fp16", "sweep_inplace_d3q19_fp32", "sweep_batch_ensemble_fp32")


def test_committed_record_is_plausible():
    for key in KEYS:
        rec = bench.traffic_record(key)
        if rec is None:
            pytest.skip("the kernel sources changed after the traffic capture (%s): re-take it" % key)
        # the algorithmic bytes are 2 Q b per site; the record may exceed them by the owner
        # tags, IS masks and boundary-site records, never fall below them
        b = 76.0 if "fp16" in key else 152.0
        assert b <= rec["dram_bytes_per_site"] <= 1.15 * b, key


def test_record_is_dropped_when_the_sources_change(tmp_path, monkeypatch):
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    d["sweep2_d3q19_fp32"]["source_sha"] = "0" * 16
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(d))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_sha", lambda: d["sweep2_d3q19_fp16"]["source_sha"])
    assert bench.traffic_record("sweep2_d3q19_fp32") is None
    assert bench.traffic_record("sweep2_d3q19_fp16") is not None
    assert bench.traffic_record("no_such_kernel") is None
