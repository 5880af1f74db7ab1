"""Host logic of Simulation.run's JSON-lines log: one line every `every` steps and after the
last, the diagnostics and the particles' summed force and torque, and the line of a
non-finite state written before its error propagates. A stand-in context records the calls
(no GPU)."""
import io
import json

import numpy as np
import pytest

from paper_1105_2904_gb300 import lbmp


class FakeSim(lbmp.Simulation):
    def __init__(self, np_=2, nan_at=None):
        self.np = np_
        self.steps = 0
        self.nan_at = nan_at
        self.calls = []

    def step(self, n=1):
        self.calls.append(n)
        self.steps += n

    def info(self):
        return {"steps": self.steps}

    def diagnostics(self):
        d = {"mass": 100.0 + self.steps, "momentum": np.array([0.5, -0.25, 0.0]), "max_speed": 0.01,
             "mach": 0.01 * np.sqrt(3.0), "nonfinite_sites": 0}
        if self.nan_at is not None and self.steps >= self.nan_at:
            d["nonfinite_sites"] = 3
            e = lbmp.LbmError(7, "non-finite")
            e.diagnostics = d
            raise e
        return d

    def get_particles(self):
        f = np.arange(3 * self.np, dtype=float).reshape(self.np, 3)
        return {"force": f, "torque": -f}


def test_lines_every_k_steps_and_after_the_last():
    s = FakeSim()
    buf = io.StringIO()
    s.run(23, log=buf, every=10)
    assert s.calls == [10, 10, 3]
    recs = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert [r["step"] for r in recs] == [10, 20, 23]
    assert recs[0]["mass"] == 110.0 and recs[0]["momentum"] == [0.5, -0.25, 0.0]
    assert recs[0]["force_sum"] == [3.0, 5.0, 7.0] and recs[0]["torque_sum"] == [-3.0, -5.0, -7.0]


def test_no_log_steps_once():
    s = FakeSim()
    s.run(17)
    assert s.calls == [17]


def test_no_particles_no_force_keys(tmp_path):
    s = FakeSim(np_=0)
    p = tmp_path / "a.jsonl"
    s.run(4, log=str(p), every=2)
    s.run(2, log=str(p), every=5)   # appends
    recs = [json.loads(x) for x in p.read_text().splitlines()]
    assert [r["step"] for r in recs] == [2, 4, 6]
    assert all("force_sum" not in r for r in recs)


def test_non_finite_line_then_error():
    s = FakeSim(nan_at=15)
    buf = io.StringIO()
    with pytest.raises(lbmp.LbmError):
        s.run(40, log=buf, every=10)
    recs = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert [r["step"] for r in recs] == [10, 20]
    assert recs[-1]["error"] == "LBM_E_NAN" and recs[-1]["nonfinite_sites"] == 3
    assert "force_sum" not in recs[-1]


def test_every_must_be_positive():
    with pytest.raises(ValueError):
        FakeSim().run(3, log=io.StringIO(), every=0)
