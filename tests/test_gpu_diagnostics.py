"""State diagnostics (lbm_diagnostics): totals and extremes of the state, and detection of
non-finite values.

The totals must equal sums of the fields lbm_get_fields returns, in both streaming schemes and
at both in-place layouts. On a periodic suspension the total mass stays constant step after
step (every site keeps its own mass through the collision, the BS transfer and the IS
imposition, reading R5). A non-finite population set on the host through lbm_set_distributions
is reported as LBM_E_NAN with the number of affected sites, which grows as later steps spread
it; the context stays usable and a finite state clears the report. The injection runs on a
particle-free box: nothing non-finite ever reaches particle positions.
"""
import numpy as np
import pytest

from paper_1105_2904_gb300 import lbmp
from paper_1105_2904_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DIMS = (36, 30, 26)
LBM_E_NAN = 7


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()


def _suspension(streaming, precision="fp64"):
    c, rad = W.rsa_centers(DIMS, 4, 4.5, seed=71, min_gap=2.0)
    v = W.gaussian_velocities(4, 0.04, seed=72)
    g = lbmp.Simulation(1, *DIMS, 0.7, body_force=(2e-6, 0.0, 0.0), precision=precision,
                        body_force_on_particles=True, streaming=streaming)
    g.add_particles(c, rad, np.array([1.3, 2.0, 0.9, 1.6]), v)
    return g


@pytest.mark.parametrize("streaming", ["pull", "inplace"])
def test_totals_equal_sums_of_the_fields(streaming):
    g = _suspension(streaming)
    for n in (0, 7, 1):  # after 0, 7, 8 steps; in-place layouts: natural, neighbour phase, natural
        g.step(n)
        d = g.diagnostics()
        rho, u = g.get_fields()
        mass = float(rho.sum())
        mom = (rho[..., None] * u).sum(axis=(0, 1, 2))
        umax = float(np.sqrt((u * u).sum(-1)).max())
        assert abs(d["mass"] - mass) <= 1e-12 * mass
        assert np.max(np.abs(d["momentum"] - mom)) <= 1e-12 * np.max(np.abs(mom))
        assert abs(d["max_speed"] - umax) <= 1e-14
        assert abs(d["mach"] - umax * np.sqrt(3.0)) <= 1e-13
        assert d["nonfinite_sites"] == 0
    g.close()


def test_mass_is_conserved_on_a_periodic_suspension():
    g = _suspension("pull")
    m0 = g.diagnostics()["mass"]
    for _ in range(4):
        g.step(20)
        assert abs(g.diagnostics()["mass"] - m0) <= 1e-12 * m0
    g.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_non_finite_values_are_reported(precision):
    nx, ny, nz = DIMS
    g = lbmp.Simulation(1, nx, ny, nz, 0.7, body_force=(1e-6, 0.0, 0.0), precision=precision)
    g.step(5)
    f0 = g.get_f()
    f = f0.copy()
    f[4, 13, 15, 17] = np.nan          # one population of one site (f[i][z][y][x])
    g.set_f(f)
    with pytest.raises(lbmp.LbmError) as e:
        g.diagnostics()
    assert e.value.status == LBM_E_NAN
    assert e.value.diagnostics["nonfinite_sites"] == 1
    g.step(2)
    with pytest.raises(lbmp.LbmError) as e:
        g.diagnostics()
    assert e.value.diagnostics["nonfinite_sites"] > 1
    g.set_f(f0)                         # a finite state: no report, the context still works
    d = g.diagnostics()
    assert d["nonfinite_sites"] == 0
    g.step(3)
    assert g.diagnostics()["nonfinite_sites"] == 0
    g.close()


def test_json_lines_log(tmp_path):
    import json
    g = _suspension("pull", "fp32")
    path = tmp_path / "run.jsonl"
    g.run(25, log=str(path), every=10)
    lines = [json.loads(s) for s in path.read_text().splitlines()]
    assert [r["step"] for r in lines] == [10, 20, 25]
    last = lines[-1]
    d = g.diagnostics()
    p = g.get_particles()
    assert last["mass"] == d["mass"] and last["max_speed"] == d["max_speed"]
    assert last["momentum"] == [float(v) for v in d["momentum"]]
    assert last["force_sum"] == [float(v) for v in p["force"].sum(0)]
    assert last["torque_sum"] == [float(v) for v in p["torque"].sum(0)]
    assert all(r["nonfinite_sites"] == 0 and "error" not in r for r in lines)
    g.close()
    # a non-finite state (fluid only): the line is written, then the error propagates
    h = lbmp.Simulation(1, *DIMS, 0.7, body_force=(1e-6, 0.0, 0.0), precision="fp32")
    h.step(4)
    f = h.get_f()
    f[2, 5, 6, 7] = np.inf
    h.set_f(f)
    with pytest.raises(lbmp.LbmError) as e:
        h.run(3, log=str(path), every=3)
    assert e.value.status == LBM_E_NAN
    bad = json.loads(path.read_text().splitlines()[-1])
    assert bad["error"] == "LBM_E_NAN" and bad["nonfinite_sites"] > 0 and bad["step"] == 7
    assert "force_sum" not in bad
    h.close()
