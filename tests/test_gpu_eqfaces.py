"""Equilibrium faces (LBM_EQUILIBRIUM) on the CUDA path against the oracle.

After the collision every fluid site on such a face takes f^eq(rho, u_face); moves out through
it bounce back without a wall-momentum term. Cases mix equilibrium faces with normal velocities
(inflow and outflow along x), tangential ones, no-slip walls and moving no-slip walls, with
particles and a body force. FP64 storage must agree with the oracle to 1e-12 relative (in
practice exactly); FP32 within the tolerances of the other parity tests, for the one-site and
two-site sweep kernels. Also the derived Couette closed form on the CUDA path."""
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


def rel(a, b, scale=None):
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / max(s, 1e-300))


CASES = [
    # flow through a 3D channel: x faces impose (0.01, 0, 0), y faces no-slip, +z moving
    # no-slip, -z equilibrium at rest; two spheres inside
    dict(name="d3q19_through_flow", lattice=O.D3Q19, dims=(40, 22, 18), walls=(1, 1, 1),
         eq={0: (0.01, 0.0, 0.0), 1: (0.01, 0.0, 0.0), 4: (0.0, 0.0, 0.0)}, uw={5: (0.02, 0.0, 0.0)},
         F=(0.0, 0.0, 0.0), n=2, r=4.0, seed=111),
    # D2Q9 shear cell: y faces impose -U / +U tangentially, x periodic, disks, body force
    dict(name="d2q9_shear", lattice=O.D2Q9, dims=(64, 46, 1), walls=(0, 1, 0),
         eq={2: (-0.02, 0.0, 0.0), 3: (0.02, 0.0, 0.0)}, uw={}, F=(1e-6, 0.0, 0.0), n=3, r=5.0, seed=112),
]


def _pair(case, precision, shape=-1):
    nx, ny, nz = case["dims"]
    g = lbmp.Simulation(case["lattice"], nx, ny, nz, 0.75, body_force=case["F"], precision=precision,
                        walls=case["walls"], gap=0.5, equilibrium_faces=case["eq"], wall_velocity=case["uw"])
    g.set_sweep_shape(shape)
    r = O.OracleSim(case["lattice"], nx, ny, nz, 0.75, body_force=case["F"], walls=case["walls"], gap=0.5,
                    equilibrium_faces=case["eq"], wall_velocity=case["uw"])
    D = 2 if case["lattice"] == O.D2Q9 else 3
    box = case["dims"][:D]
    c, rad = W.rsa_centers(box, case["n"], case["r"], seed=case["seed"], min_gap=2.0,
                           walls=tuple(int(w) for w in case["walls"]), wall_clearance=case["r"] + 3.0)
    v = W.gaussian_velocities(case["n"], 0.01, seed=case["seed"] + 1)
    if D == 2:
        v[:, 2] = 0.0
    d = np.full(case["n"], 1.8)
    g.add_particles(c, rad, d, v)
    r.add_particles(c, rad, d, v)
    return g, r


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_equilibrium_faces_fp64_match_oracle_exactly(case):
    g, r = _pair(case, "fp64")
    g.step(150)
    r.step(150)
    np.testing.assert_array_equal(g.get_tags(), r.get_tags())
    assert rel(g.get_f(), r.get_f()) <= 1e-12
    pg, pr = g.get_particles(), r.get_particles()
    for k in ("x", "u", "force"):
        assert rel(pg[k], pr[k]) <= 1e-12, k
    g.close()


@pytest.mark.parametrize("shape", [0, 16])
@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_equilibrium_faces_fp32_within_tolerance(case, shape):
    g, r = _pair(case, "fp32", shape)
    g.step(150)
    r.step(150)
    rg, ug = g.get_fields()
    rr, ur = r.get_fields()
    assert rel(ug, ur) <= 1e-5
    pg, pr = g.get_particles(), r.get_particles()
    assert rel(pg["force"], pr["force"]) <= 1e-4
    g.close()


def test_equilibrium_face_couette_closed_form_on_the_gpu():
    # as the oracle pin: interior profile u(y) = 2U (y - (ny-1)/2) / (ny - 3 + 2 tau)
    ny, U, tau = 24, 0.01, 0.8
    g = lbmp.Simulation(1, 4, ny, 4, tau, precision="fp64", walls=(0, 1, 0),
                        equilibrium_faces={2: (-U, 0.0, 0.0), 3: (U, 0.0, 0.0)})
    g.step(80000)
    rho, u = g.get_fields()
    ux = u[0, :, 0, 0]
    y = np.arange(1, ny - 1)
    want = 2.0 * U * (y - 0.5 * (ny - 1)) / (ny - 3 + 2.0 * tau)
    assert np.max(np.abs(ux[1:-1] - want)) <= 1e-10 * U
    g.close()


def test_normal_velocity_only_on_equilibrium_faces():
    g = lbmp.Simulation(1, 12, 12, 12, 0.7, walls=(1, 0, 0), equilibrium_faces={0: (0.01, 0.0, 0.0)})
    g.set_wall_velocity(0, (0.02, 0.01, 0.0))          # equilibrium face: any direction
    with pytest.raises(lbmp.LbmError):
        g.set_wall_velocity(1, (0.01, 0.0, 0.0))        # no-slip face: tangential only
    g.close()
