"""The per-site BS records of the FP32 modes: each step's particle sums must use only the
records the sweep of that step wrote (Eqs. 8-9). A record carries the owner tag it was written
under and no step stamp; the record of a site that stops being a BS site of its particle
(another particle takes the site, or the particle's anchor moves) is cleared at that moment.
A record left over from an earlier step would add that step's momentum exchange of the site
(about 1e-3 of the total force for a sphere of ~100-900 BS sites), so the force and torque of
every particle are compared with the FP64 oracle after every single step, through contacts,
contested sites and shift changes, for both sweep kernel forms and both streaming schemes."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1105_2904_gb300 import lbmp
from paper_1105_2904_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()
    O.build()


def _cases():
    cases = []
    # head-on collision of two spheres in a channel with walls on z (contested BS shells)
    cases.append(dict(name="head_on", lattice=O.D3Q19, dims=(48, 20, 22), tau=0.8, F=(0, 0, 0),
                      walls=(0, 0, 1), gravity=(0, 0, 0), gap=0.5, bfp=False, steps=60,
                      particles=(np.array([[16.3, 10.1, 10.6], [29.7, 9.8, 10.4]]), [5.0, 5.5], [10.0, 15.0],
                                 np.array([[0.08, 0.0, 0.0], [-0.07, 0.0, 0.0]]), None)))
    # moving, spinning spheres crossing shift boundaries and the periodic faces (even nx: the
    # two-site kernel applies)
    dims = (42, 36, 30)
    c, rad = W.rsa_centers(dims, 4, 5.0, seed=41, min_gap=2.0)
    cases.append(dict(name="moving_spheres", lattice=O.D3Q19, dims=dims, tau=0.7, F=(2e-6, 0, 0),
                      walls=(0, 0, 0), gravity=(0, 0, 0), gap=0.0, bfp=True, steps=120,
                      particles=(c, rad, np.array([1.2, 2.5, 0.9, 1.5]), W.gaussian_velocities(4, 0.03, seed=42),
                                 W.gaussian_velocities(4, 0.004, seed=43))))
    # settling disks in a closed box: resting contacts between disks and with the walls
    c2, r2 = W.rsa_centers((60, 90), 6, 5.0, seed=44, min_gap=1.0, walls=(1, 1, 0))
    cases.append(dict(name="settling_disks", lattice=O.D2Q9, dims=(60, 90, 1), tau=0.7, F=(0, 0, 0),
                      walls=(1, 1, 0), gravity=(0.0, -2e-3, 0.0), gap=0.5, bfp=False, steps=200,
                      particles=(c2, r2, np.full(6, 2.0), None, None)))
    return cases


CASES = _cases()
FORMS = [("pull", 0), ("pull", 16), ("inplace", 0)]


@pytest.mark.parametrize("form", FORMS, ids=["%s_shape%d" % f for f in FORMS])
@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_force_and_torque_match_the_oracle_after_every_step(case, form):
    streaming, shape = form
    nx, ny, nz = case["dims"]
    g = lbmp.Simulation(case["lattice"], nx, ny, nz, case["tau"], body_force=case["F"], precision="fp32",
                        walls=case["walls"], gravity=case["gravity"], gap=case["gap"],
                        body_force_on_particles=case["bfp"], streaming=streaming)
    g.set_sweep_shape(shape)
    r = O.OracleSim(case["lattice"], nx, ny, nz, case["tau"], body_force=case["F"], walls=case["walls"],
                    gravity=case["gravity"], gap=case["gap"], body_force_on_particles=case["bfp"])
    c, rad, d, v, om = case["particles"]
    g.add_particles(c, rad, d, v, om)
    r.add_particles(c, rad, d, v, om)
    rad = np.asarray(rad, dtype=float)
    fscale = tscale = 0.0
    worst_f = worst_t = 0.0
    shifts = 0
    x_prev = np.floor(np.asarray(c, dtype=float))
    for s in range(case["steps"]):
        g.step(1)
        r.step(1)
        pg, pr = g.get_particles(), r.get_particles()
        # the scales: the largest force (torque, or |F| r) seen so far on the oracle side
        fscale = max(fscale, float(np.max(np.abs(pr["force"]))))
        tscale = max(tscale, float(np.max(np.abs(pr["torque"]))), fscale * rad.max())
        ef = float(np.max(np.abs(pg["force"] - pr["force"]))) / max(fscale, 1e-300)
        et = float(np.max(np.abs(pg["torque"] - pr["torque"]))) / max(tscale, 1e-300)
        worst_f, worst_t = max(worst_f, ef), max(worst_t, et)
        assert ef <= 1e-4, "force after step %d: %.3g" % (s + 1, ef)
        assert et <= 1e-4, "torque after step %d: %.3g" % (s + 1, et)
        xf = np.floor(pr["x"])
        shifts += int(np.any(xf != x_prev, axis=1).sum())
        x_prev = xf
    np.testing.assert_array_equal(g.get_tags(), r.get_tags())
    # the run did exercise shift changes (records of moved anchors)
    assert shifts > 0
    print("%s %s: worst force %.2e torque %.2e over %d steps, %d shift changes"
          % (case["name"], form, worst_f, worst_t, case["steps"], shifts))
