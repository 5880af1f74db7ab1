"""Moving walls (velocity-imposed boundaries, Secs. 3.1-3.2) on the CUDA path against the oracle.

A population that bounces off a wall moving with u_w gains -6 w_i (c_i . u_w) (halfway
bounce-back at reference density 1); a move crossing two walls takes the wall of its lowest
axis. FP64 storage must agree with the oracle to 1e-12 relative (in practice exactly), FP32
within the tolerances of the other parity tests. Cases: a lid-driven cavity (every face a
wall, corners crossing two walls), a D3Q19 duct with two moving faces, a suspension in
plane Couette flow with a sphere touching a moving wall, a wall velocity changed between
steps, and distributions set between steps.
"""
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


def make_pair(lattice, dims, tau, precision, walls, wall_velocity, F=(0.0, 0.0, 0.0), gap=0.0, bfp=False):
    nx, ny, nz = dims
    g = lbmp.Simulation(lattice, nx, ny, nz, tau, body_force=F, precision=precision, walls=walls, gap=gap,
                        body_force_on_particles=bfp, wall_velocity=wall_velocity)
    r = O.OracleSim(lattice, nx, ny, nz, tau, body_force=F, walls=walls, gap=gap, body_force_on_particles=bfp,
                    wall_velocity=wall_velocity)
    return g, r


def rel(a, b, scale=None):
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / max(s, 1e-300))


FLUID_CASES = [
    # lid-driven cavity: every face a wall, the +y lid moving along x
    ("d2q9_cavity", O.D2Q9, (133, 37, 1), (1, 1, 0), {3: (0.05, 0.0, 0.0)}),
    # duct: y and z walls, +y moving along x, -z moving along x and y (corners cross two walls)
    ("d3q19_duct", O.D3Q19, (70, 11, 9), (0, 1, 1), {3: (0.03, 0.0, 0.0), 4: (-0.01, 0.02, 0.0)}),
    # closed box, x walls moving along z (a normal axis of x is the lowest crossed axis)
    ("d3q19_box", O.D3Q19, (20, 13, 17), (1, 1, 1), {0: (0.0, 0.0, 0.02), 5: (0.0, -0.02, 0.0)}),
]


@pytest.mark.parametrize("name,lattice,dims,walls,uw", FLUID_CASES, ids=[c[0] for c in FLUID_CASES])
def test_moving_walls_fp64_match_oracle_exactly(name, lattice, dims, walls, uw):
    g, r = make_pair(lattice, dims, 0.7, "fp64", walls, uw, F=(1e-6, 0.0, 0.0))
    g.step(300)
    r.step(300)
    rg, ug = g.get_fields()
    rr, ur = r.get_fields()
    assert rel(ug, ur) <= 1e-12 and rel(rg, rr, np.max(np.abs(rr - 1.0))) <= 1e-12
    assert rel(g.get_f(), r.get_f()) <= 1e-12
    # the walls drive a flow far above the body-force flow
    assert np.max(np.abs(ur)) > 1e-3


@pytest.mark.parametrize("name,lattice,dims,walls,uw", FLUID_CASES, ids=[c[0] for c in FLUID_CASES])
def test_moving_walls_fp32_within_tolerance(name, lattice, dims, walls, uw):
    g, r = make_pair(lattice, dims, 0.7, "fp32", walls, uw, F=(1e-6, 0.0, 0.0))
    g.step(300)
    r.step(300)
    _, ug = g.get_fields()
    _, ur = r.get_fields()
    assert rel(ug, ur) <= 1e-5


def _couette_suspension():
    # Plane Couette flow between y walls moving at -U and +U along x, with four spheres, one of
    # them touching the moving +y wall plane (y = ny - 1/2).
    dims = (48, 40, 24)
    U = 0.02
    uw = {2: (-U, 0.0, 0.0), 3: (U, 0.0, 0.0)}
    c = np.array([[10.3, 20.1, 12.2], [30.6, 9.4, 6.3], [24.2, 34.5, 17.7], [40.1, 27.3, 5.6]])
    rad = np.array([5.0, 4.5, 5.0, 3.5])
    d = np.array([1.0, 1.5, 2.0, 1.2])
    v = W.gaussian_velocities(4, 1e-3, seed=71)
    om = W.gaussian_velocities(4, 1e-3, seed=72)
    return dims, uw, (c, rad, d, v, om)


def test_suspension_in_couette_flow_fp64_matches_oracle_exactly():
    dims, uw, (c, rad, d, v, om) = _couette_suspension()
    g, r = make_pair(O.D3Q19, dims, 0.8, "fp64", (0, 1, 0), uw, gap=0.5)
    g.add_particles(c, rad, d, v, om)
    r.add_particles(c, rad, d, v, om)
    g.step(400)
    r.step(400)
    assert np.array_equal(g.get_tags(), r.get_tags())
    pg, pr = g.get_particles(), r.get_particles()
    for k in ("x", "u", "omega", "force", "torque"):
        assert rel(pg[k], pr[k]) <= 1e-12, k
    rg, ug = g.get_fields()
    rr, ur = r.get_fields()
    assert rel(ug, ur) <= 1e-12 and rel(rg, rr, np.max(np.abs(rr - 1.0))) <= 1e-12
    # the sphere at the +y wall is dragged along +x by it
    assert pr["u"][2, 0] > 0.0


def test_suspension_in_couette_flow_fp32_within_tolerance():
    dims, uw, (c, rad, d, v, om) = _couette_suspension()
    g, r = make_pair(O.D3Q19, dims, 0.8, "fp32", (0, 1, 0), uw, gap=0.5)
    g.add_particles(c, rad, d, v, om)
    r.add_particles(c, rad, d, v, om)
    g.step(300)
    r.step(300)
    _, ug = g.get_fields()
    _, ur = r.get_fields()
    pg, pr = g.get_particles(), r.get_particles()
    assert rel(ug, ur) <= 1e-5
    assert rel(pg["force"], pr["force"]) <= 1e-4
    assert np.max(np.abs(pg["x"] - pr["x"]) / rad[:, None]) <= 1e-5


def test_wall_velocity_changed_and_distributions_set_between_steps():
    dims, uw, (c, rad, d, v, om) = _couette_suspension()
    g, r = make_pair(O.D3Q19, dims, 0.8, "fp64", (0, 1, 0), uw, gap=0.5)
    g.add_particles(c, rad, d, v, om)
    r.add_particles(c, rad, d, v, om)
    g.step(60)
    r.step(60)
    # reverse the top wall and set the bottom one moving along z
    for sim in (g, r):
        sim.set_wall_velocity(3, (-0.02, 0.0, 0.0))
        sim.set_wall_velocity(2, (0.0, 0.0, 0.015))
    g.step(60)
    r.step(60)
    pg, pr = g.get_particles(), r.get_particles()
    for k in ("x", "u", "force"):
        assert rel(pg[k], pr[k]) <= 1e-12, k
    # distributions set between steps are streamed as given (no wall term on the first pull)
    f = r.get_f()
    f = f * (1.0 + 1e-3 * W.perturbation(f.shape[0], f.shape[1:], 5))
    g.set_f(f)
    r.set_f(f)
    g.step(40)
    r.step(40)
    assert rel(g.get_f(), r.get_f()) <= 1e-12
    pg, pr = g.get_particles(), r.get_particles()
    for k in ("x", "u", "force"):
        assert rel(pg[k], pr[k]) <= 1e-12, k


def test_wall_velocity_is_validated():
    g = lbmp.Simulation(O.D3Q19, 8, 8, 8, 0.7, precision="fp64", walls=(0, 1, 0))
    with pytest.raises(lbmp.LbmError):
        g.set_wall_velocity(0, (0.0, 0.01, 0.0))      # x faces are periodic
    with pytest.raises(lbmp.LbmError):
        g.set_wall_velocity(3, (0.0, 0.01, 0.0))      # normal to the y wall
    with pytest.raises(lbmp.LbmError):
        g.set_wall_velocity(6, (0.01, 0.0, 0.0))      # no such face
    g.set_wall_velocity(2, (0.01, 0.0, -0.01))
    g.step(2)
    g.close()
